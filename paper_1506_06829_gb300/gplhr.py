"""ctypes binding to libgplhr (``include/gplhr.h``): argument marshalling only.

Every function keeps the C name and forwards to the library; all arithmetic of the
eigensolver runs in the CUDA kernels and host C++ of ``libgplhr.so``.  PyTorch is
used only for device memory (``torch.Tensor.data_ptr()``) and streams.

Blocks are row-major complex128 (n x w); host CSR matrices come from SciPy.
If ``libgplhr.so`` has not been built, importing works but the first call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgplhr.so")

GPLHR_OK, GPLHR_EINVAL, GPLHR_ENOMEM, GPLHR_ECUDA = 0, 1, 2, 3
GPLHR_ENOTCONV, GPLHR_ESINGULAR, GPLHR_ENUMERIC, GPLHR_ETIMEOUT = 4, 5, 6, 7
GPLHR_HOST, GPLHR_DEVICE = 0, 1
GPLHR_R64, GPLHR_C128 = 0, 1
PREC = {"none": 0, "jacobi": 1, "block_jacobi": 2, "csr": 3}
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCONV", 5: "ESINGULAR",
                6: "ENUMERIC", 7: "ETIMEOUT"}

EXPORTED = ["gplhr_create", "gplhr_solve", "gplhr_start", "gplhr_iterate", "gplhr_vectors",
            "gplhr_destroy", "gplhr_last_error", "gplhr_spmm", "gplhr_precond_apply",
            "gplhr_gram", "gplhr_combine", "gplhr_orth", "gplhr_ordqz", "gplhr_ordqz_device", "gplhr_mfactors",
            "gplhr_profile",
            "gplhr_profile_read", "gplhr_gram_noalloc", "gplhr_grad", "gplhr_solve_batched",
            "gplhr_iterate_batched", "gplhr_spmm_shape", "gplhr_set_deflation", "gplhr_create_batched",
            "gplhr_iterate_persistent", "gplhr_solve_persistent"]
P_MODES = {"thick": 0, "lobpcg": 1, "none": 2}
KCLASS = {"spmm": 0, "gram": 1, "combine": 2, "precond": 3, "chol": 4, "other": 5, "gram_tc": 6,
          "combine_tc": 7}


class Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("colind", C.c_void_p), ("vals", C.c_void_p), ("dtype", C.c_int32),
                ("on_device", C.c_int32)]


class Precond(C.Structure):
    _fields_ = [("kind", C.c_int32), ("block_size", C.c_int32), ("T_csr", C.POINTER(Csr)),
                ("inner_steps", C.c_int32)]


class Opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int32), ("precision", C.c_int32),
                ("no_lock", C.c_int32), ("products", C.c_int32), ("stream", C.c_void_p),
                ("switch_tol", C.c_double), ("stall_iters", C.c_int32), ("pencil", C.c_int32),
                ("fp64_gemm", C.c_int32), ("graphs", C.c_int32), ("autotune", C.c_int32),
                ("p_mode", C.c_int32), ("no_right_proj", C.c_int32), ("variant", C.c_int32),
                ("wait_limit", C.c_int32), ("wait_probe", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("nconv", C.c_int32), ("m", C.c_int32),
                ("n_orth_fallback", C.c_int32), ("fp32_iters", C.c_int32), ("bulk", C.c_int32),
                ("n_spmm", C.c_int64), ("n_prec", C.c_int64),
                ("n_qz", C.c_int64), ("n_launch", C.c_int64), ("h2d_bytes", C.c_int64),
                ("d2h_bytes", C.c_int64), ("resid", C.c_double * 64), ("n_inner", C.c_int64)]


class PersistStats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("steps", C.c_int64), ("ops", C.c_int64), ("grid", C.c_int32),
                ("pad", C.c_int32), ("record_ms", C.c_double), ("build_ms", C.c_double),
                ("qz_ms", C.c_double), ("wait_ms", C.c_double)]


class GplhrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libgplhr.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1506_06829_gb300.build`")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    dp = C.POINTER(C.c_double)
    L.gplhr_create.argtypes = [C.POINTER(Csr), C.POINTER(Csr), dbl, dbl, i32, i32,
                               C.POINTER(Precond), C.POINTER(Opts), C.POINTER(vp)]
    L.gplhr_solve.argtypes = [vp, vp, i32, i32, u64, C.POINTER(Info)]
    L.gplhr_start.argtypes = [vp, vp, i32, i32, u64]
    L.gplhr_iterate.argtypes = [vp, i32, C.POINTER(Info)]
    L.gplhr_vectors.argtypes = [vp, dp, dp, dp, vp, vp, vp, vp, vp, dp, i32]
    L.gplhr_destroy.argtypes = [vp]
    L.gplhr_destroy.restype = None
    L.gplhr_last_error.argtypes = [vp]
    L.gplhr_last_error.restype = C.c_char_p
    L.gplhr_spmm.argtypes = [vp, vp, i32, i32, vp, i32, vp, i32]
    L.gplhr_precond_apply.argtypes = [vp, vp, i32, i32, vp, i32]
    L.gplhr_gram.argtypes = [vp, vp, i32, i32, vp, i32, i32, vp, i32]
    L.gplhr_orth.argtypes = [vp, vp, i32, i32, vp]
    L.gplhr_combine.argtypes = [vp, vp, i32, i32, vp, i32, vp, i32, i32, i32]
    L.gplhr_spmm_shape.argtypes = [vp, i32, i32, C.POINTER(i32), C.POINTER(i32), dp, dp]
    L.gplhr_set_deflation.argtypes = [vp, vp, vp, i32, i32]
    L.gplhr_ordqz.argtypes = [i32, dp, dp, dbl, dbl, dp, dp, dp, dp]
    L.gplhr_ordqz_device.argtypes = [i32, vp, vp, dbl, dbl, i32, vp, vp, vp, vp, vp, vp]
    L.gplhr_mfactors.argtypes = [i32, dp, dp, dp, dp]
    L.gplhr_profile.argtypes = [vp, i32]
    L.gplhr_gram_noalloc.argtypes = [i64, vp, i32, i32, vp, i32, i32, vp, vp]
    L.gplhr_grad.argtypes = [vp, vp, dp, vp, vp, i32]
    L.gplhr_solve_batched.argtypes = [i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(i32),
                                      C.POINTER(i32), C.POINTER(u64), C.POINTER(Info),
                                      C.POINTER(C.c_int), i32]
    L.gplhr_iterate_batched.argtypes = [i32, C.POINTER(vp), i32, C.POINTER(Info),
                                        C.POINTER(C.c_int), i32]
    L.gplhr_iterate_persistent.argtypes = [i32, C.POINTER(vp), i32, C.POINTER(Info), C.POINTER(C.c_int), i32,
                                           C.POINTER(PersistStats)]
    L.gplhr_solve_persistent.argtypes = [i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(i32), C.POINTER(i32),
                                         C.POINTER(u64), C.POINTER(Info), C.POINTER(C.c_int), i32,
                                         C.POINTER(PersistStats)]
    L.gplhr_create_batched.argtypes = [i32, C.POINTER(C.POINTER(Csr)), C.POINTER(C.POINTER(Csr)),
                                       C.POINTER(C.c_double), C.POINTER(i32), C.POINTER(i32),
                                       C.POINTER(C.POINTER(Precond)), C.POINTER(C.POINTER(Opts)),
                                       C.POINTER(vp), C.POINTER(C.c_int), i32]
    L.gplhr_profile_read.argtypes = [vp, i32, dp, C.POINTER(C.c_int64), dp, dp]
    for name in EXPORTED:
        f = getattr(L, name)
        if f.restype is C.c_int:  # default
            f.restype = C.c_int
    _lib = L
    return L


def _check(status: int, ctx=None):
    if status != GPLHR_OK:
        msg = lib().gplhr_last_error(ctx)
        raise GplhrError(status, msg.decode() if msg else "")
    return status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _HostCsr:
    """Keeps the numpy arrays of a host CSR descriptor alive."""

    def __init__(self, M):
        self.indptr = np.ascontiguousarray(M.indptr, dtype=np.int32)
        self.indices = np.ascontiguousarray(M.indices, dtype=np.int32)
        if np.iscomplexobj(M.data):
            self.data = np.ascontiguousarray(M.data, dtype=np.complex128)
            dt = GPLHR_C128
        else:
            self.data = np.ascontiguousarray(M.data, dtype=np.float64)
            dt = GPLHR_R64
        self.desc = Csr(M.shape[0], self.indices.size, self.indptr.ctypes.data,
                        self.indices.ctypes.data, self.data.ctypes.data, dt, 0)


# ------------------------------------------------------------------ C names ----

PRODUCTS = {"auto": 0, "combine": 1, "spmm": 2}


def gplhr_create(A, B, sigma: complex, k: int, m: int, precond: str = "none",
                 block_size: int = 1, T=None, tol: float = 1e-8, maxit: int = 500,
                 lock: bool = True, stream: int = 0, products: str = "auto",
                 precision: str = "fp64", switch_tol: float = 1e-5, stall_iters: int = 5,
                 pencil: str = "factored", inner_steps: int = 0, fp64_gemm: str = "tensor",
                 graphs: bool = False, autotune: bool = False, p_mode: str = "thick",
                 right_proj: bool = True, variant: str = "schur", wait_limit: int = 0,
                 wait_probe: bool = False):
    """Returns an opaque context handle (int).  A, B: SciPy CSR (B None = identity).
    inner_steps > 0: T = that many block GMRES steps on (A - sigma B) W = R,
    right-preconditioned by `precond`."""
    L = lib()
    d = _create_args(A, B, T, precond, block_size, inner_steps, tol, maxit, lock, stream, products,
                     precision, switch_tol, stall_iters, pencil, fp64_gemm, graphs, autotune, p_mode,
                     right_proj, variant, wait_limit, wait_probe)
    out = C.c_void_p()
    st = L.gplhr_create(C.byref(d["A"].desc), C.byref(d["B"].desc) if d["B"] else None, sigma.real,
                        sigma.imag, k, m, C.byref(d["T"]), C.byref(d["opts"]), C.byref(out))
    _check(st, None)
    return out.value


def _create_args(A, B, T, precond, block_size, inner_steps, tol, maxit, lock, stream, products,
                 precision, switch_tol, stall_iters, pencil, fp64_gemm, graphs, autotune, p_mode,
                 right_proj, variant, wait_limit=0, wait_probe=False):
    """Host descriptors of one context's gplhr_create arguments (kept alive together)."""
    hA = _HostCsr(A)
    hB = _HostCsr(B) if B is not None else None
    hT = _HostCsr(T.astype(np.complex128)) if T is not None else None
    pc = Precond(PREC[precond], block_size, C.pointer(hT.desc) if hT else None, inner_steps)
    opts = Opts(tol, maxit, {"fp64": 0, "mixed": 1}[precision], 0 if lock else 1,
                PRODUCTS[products], stream or None, switch_tol, stall_iters,
                {"factored": 0, "gram": 1}[pencil], {"tensor": 0, "dfma": 1}[fp64_gemm],
                1 if graphs else 0, 1 if autotune else 0, P_MODES[p_mode], 0 if right_proj else 1,
                {"schur": 0, "eig": 1}[variant], wait_limit, 1 if wait_probe else 0)
    return {"A": hA, "B": hB, "Tcsr": hT, "T": pc, "opts": opts}


_CREATE_DEFAULTS = dict(B=None, precond="none", block_size=1, T=None, tol=1e-8, maxit=500, lock=True,
                        stream=0, products="auto", precision="fp64", switch_tol=1e-5, stall_iters=5,
                        pencil="factored", inner_steps=0, fp64_gemm="tensor", graphs=False,
                        autotune=False, p_mode="thick", right_proj=True, variant="schur", wait_limit=0,
                        wait_probe=False)


def gplhr_create_batched(specs, nthreads: int = 0):
    """Creates one context per spec (a dict with the keyword arguments of gplhr_create:
    A, sigma, k, m required) in one call; returns the list of handles.  All or nothing:
    on a failure no context survives and GplhrError names the failing entry."""
    n = len(specs)
    keep, sig, ks, ms = [], [], [], []
    for spec in specs:
        a = dict(_CREATE_DEFAULTS)
        a.update(spec)
        keep.append(_create_args(a["A"], a["B"], a["T"], a["precond"], a["block_size"], a["inner_steps"],
                                 a["tol"], a["maxit"], a["lock"], a["stream"], a["products"],
                                 a["precision"], a["switch_tol"], a["stall_iters"], a["pencil"],
                                 a["fp64_gemm"], a["graphs"], a["autotune"], a["p_mode"],
                                 a["right_proj"], a["variant"], a["wait_limit"], a["wait_probe"]))
        sig += [complex(a["sigma"]).real, complex(a["sigma"]).imag]
        ks.append(int(a["k"]))
        ms.append(int(a["m"]))
    PCsr, PPre, POpt = C.POINTER(Csr), C.POINTER(Precond), C.POINTER(Opts)
    Aa = (PCsr * n)(*[C.pointer(d["A"].desc) for d in keep])
    Ba = (PCsr * n)(*[C.pointer(d["B"].desc) if d["B"] else PCsr() for d in keep])
    Ta = (PPre * n)(*[C.pointer(d["T"]) for d in keep])
    Oa = (POpt * n)(*[C.pointer(d["opts"]) for d in keep])
    out = (C.c_void_p * n)()
    sts = (C.c_int * n)()
    st = lib().gplhr_create_batched(n, Aa, Ba, (C.c_double * (2 * n))(*sig), (C.c_int32 * n)(*ks),
                                    (C.c_int32 * n)(*ms), Ta, Oa, out, sts, nthreads)
    _check(st, None)
    return [out[i] for i in range(n)]


def gplhr_destroy(ctx):
    lib().gplhr_destroy(ctx)


def gplhr_last_error(ctx=None) -> str:
    msg = lib().gplhr_last_error(ctx)
    return msg.decode() if msg else ""


def _v0_args(V0):
    if V0 is None:
        return None, GPLHR_HOST, 0, None
    if hasattr(V0, "data_ptr"):           # torch tensor
        where = GPLHR_DEVICE if V0.is_cuda else GPLHR_HOST
        return V0.data_ptr(), where, int(V0.is_complex()), V0
    arr = np.ascontiguousarray(V0)
    if np.iscomplexobj(arr):
        arr = arr.astype(np.complex128)
    else:
        arr = arr.astype(np.float64)
    return arr.ctypes.data, GPLHR_HOST, int(np.iscomplexobj(arr)), arr


def gplhr_solve(ctx, V0=None, seed: int = 0, allow_notconv: bool = False) -> Info:
    p, where, cplx, keep = _v0_args(V0)
    info = Info()
    st = lib().gplhr_solve(ctx, p, where, cplx, seed, C.byref(info))
    if not (allow_notconv and st == GPLHR_ENOTCONV):
        _check(st, ctx)
    del keep
    return info


def gplhr_start(ctx, V0=None, seed: int = 0):
    p, where, cplx, keep = _v0_args(V0)
    _check(lib().gplhr_start(ctx, p, where, cplx, seed), ctx)
    del keep


def gplhr_iterate(ctx, niter: int) -> Info:
    info = Info()
    _check(lib().gplhr_iterate(ctx, niter, C.byref(info)), ctx)
    return info


def gplhr_vectors(ctx, n: int, k: int):
    """Host copies of (alpha, beta, lambda, X, V, Q, RA, RB, resid)."""
    alpha = np.zeros(2 * k)
    beta = np.zeros(2 * k)
    lam = np.zeros(2 * k)
    X = np.zeros((n, k), dtype=np.complex128)
    V = np.zeros((n, k), dtype=np.complex128)
    Q = np.zeros((n, k), dtype=np.complex128)
    RA = np.zeros((k, k), dtype=np.complex128)
    RB = np.zeros((k, k), dtype=np.complex128)
    resid = np.zeros(k)
    _check(lib().gplhr_vectors(ctx, _dptr(alpha), _dptr(beta), _dptr(lam), X.ctypes.data,
                               V.ctypes.data, Q.ctypes.data, RA.ctypes.data, RB.ctypes.data,
                               _dptr(resid), GPLHR_HOST), ctx)
    c = lambda a: a[0::2] + 1j * a[1::2]
    return dict(alpha=c(alpha), beta=c(beta), lam=c(lam), X=X, V=V, Q=Q, RA=RA, RB=RB,
                resid=resid)


def gplhr_spmm(ctx, X, AX, BX=None):
    """Device tensors (n x w complex128, row-major, may be column slices)."""
    w = X.shape[1]
    _check(lib().gplhr_spmm(ctx, X.data_ptr(), X.stride(0), w, AX.data_ptr(), AX.stride(0),
                            BX.data_ptr() if BX is not None else None,
                            BX.stride(0) if BX is not None else 0), ctx)


def gplhr_precond_apply(ctx, X, Y):
    _check(lib().gplhr_precond_apply(ctx, X.data_ptr(), X.stride(0), X.shape[1], Y.data_ptr(),
                                     Y.stride(0)), ctx)


GRAM_ARITH = {"fp64": 0, "fp32": 1, "exact32": 2, "tensor": 3}


def gplhr_combine(ctx, X, C, Y, beta: bool = False, arith: str = "auto"):
    """Y = X C (or Y + X C); device complex128 tensors, C (w x c) row-major."""
    _check(lib().gplhr_combine(ctx, X.data_ptr(), X.stride(0), X.shape[1], C.data_ptr(), Y.shape[1],
                               Y.data_ptr(), Y.stride(0), 1 if beta else 0,
                               {"auto": 0, "dfma": 1}[arith]), ctx)


def gplhr_set_deflation(ctx, V1, Q1=None):
    """Deflate the V1 (n x k1) / Q1 Schur vectors found earlier; host arrays or device
    tensors (complex128).  V1 = None removes the deflation."""
    if V1 is None:
        _check(lib().gplhr_set_deflation(ctx, None, None, 0, GPLHR_HOST), ctx)
        return
    dev = hasattr(V1, "data_ptr")
    if dev:
        k1 = V1.shape[1]
        _check(lib().gplhr_set_deflation(ctx, V1.data_ptr(), Q1.data_ptr() if Q1 is not None else None, k1,
                                         GPLHR_DEVICE), ctx)
        return
    V = np.ascontiguousarray(V1, dtype=np.complex128)
    Q = None if Q1 is None else np.ascontiguousarray(Q1, dtype=np.complex128)
    _check(lib().gplhr_set_deflation(ctx, V.ctypes.data, None if Q is None else Q.ctypes.data, V.shape[1],
                                     GPLHR_HOST), ctx)


def gplhr_spmm_shape(ctx, w: int, fp32: bool = False):
    """(threads per CTA, grid cap per SM, measured us, default shape's us; 0 when not
    autotuned) of the sparse products on w columns."""
    t, g, us, ud = C.c_int32(), C.c_int32(), C.c_double(), C.c_double()
    _check(lib().gplhr_spmm_shape(ctx, w, 1 if fp32 else 0, C.byref(t), C.byref(g), C.byref(us), C.byref(ud)),
           ctx)
    return t.value, g.value, us.value, ud.value


def _gram_operands(X, Y, Cout):
    """Refuses, before any launch, operands that the Gram kernels would read or write
    out of bounds: the C ABI receives raw pointers and sizes only, so it cannot see a
    wrong dtype, a transposed view or a short tensor.  X (n x wx), Y (n x wy): complex128
    with unit column stride; Cout: contiguous complex128 wx x wy; all CUDA tensors on one
    device.  Returns that device."""
    import torch

    def bad(msg):
        raise GplhrError(GPLHR_EINVAL, f"Gram operands: {msg}")

    for name, T in (("X", X), ("Y", Y), ("C", Cout)):
        if not isinstance(T, torch.Tensor) or T.dim() != 2:
            bad(f"{name} must be a 2-D torch tensor")
        if T.dtype != torch.complex128:
            bad(f"{name} must be complex128, got {T.dtype}")
    if X.shape[0] != Y.shape[0]:
        bad(f"X has {X.shape[0]} rows, Y has {Y.shape[0]}")
    if X.shape[0] < 1 or X.shape[1] < 1 or Y.shape[1] < 1:
        bad("empty block")
    if X.stride(1) != 1 or Y.stride(1) != 1:
        bad("X and Y need unit column stride (row-major rows)")
    if tuple(Cout.shape) != (X.shape[1], Y.shape[1]) or not Cout.is_contiguous():
        bad(f"C must be a contiguous {X.shape[1]} x {Y.shape[1]} tensor, got {tuple(Cout.shape)}")
    if not (X.is_cuda and Y.is_cuda and Cout.is_cuda):
        bad("X, Y and C must be CUDA tensors")
    if not (X.device == Y.device == Cout.device):
        bad(f"X, Y and C on different devices ({X.device}, {Y.device}, {Cout.device})")
    return X.device


def gplhr_gram(ctx, X, Y, Cout, arith: str = "fp64"):
    _gram_operands(X, Y, Cout)
    _check(lib().gplhr_gram(ctx, X.data_ptr(), X.stride(0), X.shape[1], Y.data_ptr(),
                            Y.stride(0), Y.shape[1], Cout.data_ptr(), GRAM_ARITH[arith]), ctx)


def gplhr_gram_noalloc(X, Y, Cout, stream: int = 0):
    """C = X^* Y without any allocation (device tensors; asynchronous on `stream`).
    The call runs with the tensors' device current: the library launches on the
    current device, with that device's copy of its scratch array."""
    import torch
    dev = _gram_operands(X, Y, Cout)
    with torch.cuda.device(dev):
        _check(lib().gplhr_gram_noalloc(X.shape[0], X.data_ptr(), X.stride(0), X.shape[1],
                                        Y.data_ptr(), Y.stride(0), Y.shape[1], Cout.data_ptr(),
                                        stream or None), None)


def gplhr_grad(right, left, G, dA=None, dB=None):
    """dL/dA, dL/dB on the CSR patterns.  G: k complex (dL/dRe + i dL/dIm per eigenvalue).
    dA / dB: numpy arrays (host) or torch tensors (device), real for a real matrix."""
    g = np.ascontiguousarray(np.stack([np.real(G), np.imag(G)], axis=1).ravel(), dtype=np.float64)
    outs = [x for x in (dA, dB) if x is not None]
    on_dev = any(hasattr(x, "data_ptr") and x.is_cuda for x in outs)
    ptr = lambda x: None if x is None else (x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data)
    _check(lib().gplhr_grad(right, left, _dptr(g), ptr(dA), ptr(dB),
                            GPLHR_DEVICE if on_dev else GPLHR_HOST), right)


def gplhr_solve_batched(ctxs, V0s=None, nthreads: int = 0):
    """Solve every context concurrently.  V0s: list of host arrays (or None).
    Returns (overall status, [Info], [status])."""
    n = len(ctxs)
    cs = (C.c_void_p * n)(*ctxs)
    keep = []
    if V0s is not None:
        ptrs, where, cplx = [], [], []
        for v in V0s:
            p, w, c, k = _v0_args(v)
            keep.append(k)
            ptrs.append(p)
            where.append(w)
            cplx.append(c)
        vp_arr = (C.c_void_p * n)(*ptrs)
        w_arr = (C.c_int32 * n)(*where)
        c_arr = (C.c_int32 * n)(*cplx)
    else:
        vp_arr = w_arr = c_arr = None
    infos = (Info * n)()
    sts = (C.c_int * n)()
    st = lib().gplhr_solve_batched(n, cs, vp_arr, w_arr, c_arr, None, infos, sts, nthreads)
    del keep
    return st, list(infos), list(sts)


def gplhr_iterate_batched(ctxs, niter: int, nthreads: int = 0):
    n = len(ctxs)
    cs = (C.c_void_p * n)(*ctxs)
    infos = (Info * n)()
    sts = (C.c_int * n)()
    st = lib().gplhr_iterate_batched(n, cs, niter, infos, sts, nthreads)
    return st, list(infos), list(sts)


def gplhr_solve_persistent(ctxs, V0s=None, nthreads: int = 0):
    """Solve every context with the persistent batched iteration (each device segment of
    an iteration run for all contexts in one persistent-kernel launch).  V0s: list of host
    arrays (or None).  Returns (overall status, [Info], [status], PersistStats)."""
    n = len(ctxs)
    cs = (C.c_void_p * n)(*ctxs)
    keep = []
    if V0s is not None:
        ptrs, where, cplx = [], [], []
        for v in V0s:
            p, w, c, k = _v0_args(v)
            keep.append(k)
            ptrs.append(p)
            where.append(w)
            cplx.append(c)
        vp_arr = (C.c_void_p * n)(*ptrs)
        w_arr = (C.c_int32 * n)(*where)
        c_arr = (C.c_int32 * n)(*cplx)
    else:
        vp_arr = w_arr = c_arr = None
    infos = (Info * n)()
    sts = (C.c_int * n)()
    stats = PersistStats()
    st = lib().gplhr_solve_persistent(n, cs, vp_arr, w_arr, c_arr, None, infos, sts, nthreads, C.byref(stats))
    del keep
    return st, list(infos), list(sts), stats


def gplhr_iterate_persistent(ctxs, niter: int, nthreads: int = 0):
    """niter iterations of each started context through the persistent batched iteration.
    Returns (overall status, [Info], [status], PersistStats)."""
    n = len(ctxs)
    cs = (C.c_void_p * n)(*ctxs)
    infos = (Info * n)()
    sts = (C.c_int * n)()
    stats = PersistStats()
    st = lib().gplhr_iterate_persistent(n, cs, niter, infos, sts, nthreads, C.byref(stats))
    return st, list(infos), list(sts), stats


def gplhr_orth(ctx, X, Rinv=None):
    _check(lib().gplhr_orth(ctx, X.data_ptr(), X.stride(0), X.shape[1],
                            Rinv.data_ptr() if Rinv is not None else None), ctx)


def gplhr_ordqz(Phi: np.ndarray, Psi: np.ndarray, sigma: complex):
    """Host ordered QZ of the C library (no GPU needed)."""
    s = Phi.shape[0]
    P = np.ascontiguousarray(Phi, dtype=np.complex128)
    S = np.ascontiguousarray(Psi, dtype=np.complex128)
    out = [np.zeros((s, s), dtype=np.complex128) for _ in range(4)]
    st = lib().gplhr_ordqz(s, _dptr(P.view(np.float64)), _dptr(S.view(np.float64)),
                           sigma.real, sigma.imag, *[_dptr(o.view(np.float64)) for o in out])
    _check(st, None)
    return tuple(out)  # RA, RB, YL, YR


def gplhr_ordqz_device(Phi, Psi, sigma: complex, nsort: int = -1, stream: int = 0):
    """The ordered QZ on the device (one CTA): Phi, Psi device complex128 s x s tensors;
    returns device tensors RA, RB, YL, YR and a device int32 status (0: converged),
    asynchronously on `stream`."""
    import torch
    s = Phi.shape[0]
    for M in (Phi, Psi):
        if (M.dtype != torch.complex128 or not M.is_cuda or tuple(M.shape) != (s, s) or not M.is_contiguous()
                or M.device != Phi.device):
            raise GplhrError(GPLHR_EINVAL, "Phi, Psi: contiguous s x s complex128 tensors on one device")
    out = [torch.empty((s, s), dtype=torch.complex128, device=Phi.device) for _ in range(4)]
    status = torch.zeros(1, dtype=torch.int32, device=Phi.device)
    with torch.cuda.device(Phi.device):
        _check(lib().gplhr_ordqz_device(s, Phi.data_ptr(), Psi.data_ptr(), sigma.real, sigma.imag, nsort,
                                        *[o.data_ptr() for o in out], status.data_ptr(), stream or None), None)
    return (*out, status)


def gplhr_mfactors(RA: np.ndarray, RB: np.ndarray):
    k = RA.shape[0]
    a = np.ascontiguousarray(RA, dtype=np.complex128)
    b = np.ascontiguousarray(RB, dtype=np.complex128)
    MA = np.zeros((k, k), dtype=np.complex128)
    MB = np.zeros((k, k), dtype=np.complex128)
    _check(lib().gplhr_mfactors(k, _dptr(a.view(np.float64)), _dptr(b.view(np.float64)),
                                _dptr(MA.view(np.float64)), _dptr(MB.view(np.float64))), None)
    return MA, MB


def gplhr_profile(ctx, enable: bool):
    _check(lib().gplhr_profile(ctx, 1 if enable else 0), ctx)


def gplhr_profile_read(ctx, kclass: str):
    """(ms, launches, flops, bytes) of one kernel class."""
    ms, fl, by = C.c_double(), C.c_double(), C.c_double()
    nl = C.c_int64()
    _check(lib().gplhr_profile_read(ctx, KCLASS[kclass], C.byref(ms), C.byref(nl), C.byref(fl),
                                    C.byref(by)), ctx)
    return ms.value, nl.value, fl.value, by.value


class GPLHR:
    """Owning handle around a gplhr context (marshalling only)."""

    def __init__(self, A, B, sigma, k, m, precond="none", block_size=1, T=None, tol=1e-8,
                 maxit=500, lock=True, stream=0, products="auto", precision="fp64",
                 switch_tol=1e-5, stall_iters=5, pencil="factored", inner_steps=0,
                 fp64_gemm="tensor", graphs=False, autotune=False, p_mode="thick", right_proj=True,
                 variant="schur", wait_limit=0, wait_probe=False):
        self.n, self.k = A.shape[0], k
        self.ctx = gplhr_create(A, B, complex(sigma), k, m, precond, block_size, T, tol, maxit,
                                lock, stream, products, precision, switch_tol, stall_iters, pencil,
                                inner_steps, fp64_gemm, graphs, autotune, p_mode, right_proj, variant,
                                wait_limit, wait_probe)

    def solve(self, V0=None, seed=0, allow_notconv=False):
        return gplhr_solve(self.ctx, V0, seed, allow_notconv)

    def start(self, V0=None, seed=0):
        gplhr_start(self.ctx, V0, seed)

    def iterate(self, niter):
        return gplhr_iterate(self.ctx, niter)

    def vectors(self):
        return gplhr_vectors(self.ctx, self.n, self.k)

    def close(self):
        if self.ctx:
            gplhr_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
