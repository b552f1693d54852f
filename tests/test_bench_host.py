"""Host-side checks of bench.py (no GPU): the module imports, every name its functions
read at module level is defined, and the kernel classes agree with the binding's."""
import ast
import builtins
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_bench_imports_and_kernel_classes_match_binding():
    b = _load()
    from paper_1506_06829_gb300 import gplhr as G
    assert list(b.KCLASSES) == list(G.KCLASS.keys())
    assert set(b.TENSOR_CLASSES) <= set(b.KCLASSES)
    assert set(b.TRAFFIC_64CUBED) <= set(b.TENSOR_CLASSES)


def test_bench_global_names_are_defined():
    """Every bare name a function of bench.py loads is a builtin, a module-level name, an
    import, or local to that function (a deleted constant would fail only on a GPU run)."""
    b = _load()
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    module_names = set(vars(b))
    missing = []
    # module-level functions; names bound anywhere inside one (nested closures included) count as its own
    for fn in [n for n in tree.body if isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef))]:
        local = {a.arg for a in fn.args.args + fn.args.kwonlyargs}
        if fn.args.vararg:
            local.add(fn.args.vararg.arg)
        if fn.args.kwarg:
            local.add(fn.args.kwarg.arg)
        for n in ast.walk(fn):
            if isinstance(n, ast.Name) and isinstance(n.ctx, (ast.Store, ast.Del)):
                local.add(n.id)
            elif isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
                local.add(n.name)
            elif isinstance(n, (ast.Import, ast.ImportFrom)):
                for a in n.names:
                    local.add((a.asname or a.name).split(".")[0])
            elif isinstance(n, ast.ExceptHandler) and n.name:
                local.add(n.name)
            elif isinstance(n, ast.arg):
                local.add(n.arg)
        for n in ast.walk(fn):
            if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load):
                if n.id not in local and n.id not in module_names and not hasattr(builtins, n.id):
                    missing.append((fn.name, n.id))
    assert not missing, missing
