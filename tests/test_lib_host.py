"""C-ABI library checks that need no GPU: every symbol declared in include/gplhr.h is
exported by libgplhr.so, and the host-side small dense algebra of the library (sorted
QZ, Q-free factors) agrees with the CPU oracle and with LAPACK."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest
import scipy.linalg as sla

from oracle.ordqz import ordqz as oracle_ordqz
from oracle.schur import m_factors as oracle_m_factors
from paper_1506_06829_gb300 import gplhr as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "gplhr.h")).read()
    return sorted(set(re.findall(r"\b(gplhr_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(G.LIB_PATH):
        from paper_1506_06829_gb300 import build
        build.build()
    return G.lib()


def test_library_exports_every_declared_symbol(built):
    declared = _declared_symbols()
    assert len(declared) >= 13
    for name in declared:
        assert hasattr(built, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", G.LIB_PATH], capture_output=True, text=True)
    exported = set(re.findall(r"\bT (gplhr_\w+)", out.stdout))
    assert set(declared) <= exported
    assert set(G.EXPORTED) == set(declared)


@pytest.mark.parametrize("seed,s,sigma", [(0, 8, 0.2 + 0.1j), (1, 16, -0.5 + 0j), (2, 24, 1.0 - 2.0j),
                                          (3, 32, 0.0 + 0.0j), (4, 1, 0.3 + 0j)])
def test_host_ordqz_matches_oracle(built, seed, s, sigma):
    rng = np.random.default_rng(100 + seed)
    Phi = rng.standard_normal((s, s)) + 1j * rng.standard_normal((s, s))
    Psi = rng.standard_normal((s, s)) + 1j * rng.standard_normal((s, s)) + 2 * np.eye(s)
    RA, RB, YL, YR = G.gplhr_ordqz(Phi, Psi, sigma)
    I = np.eye(s)
    assert np.allclose(YL.conj().T @ YL, I, atol=1e-13)
    assert np.allclose(YR.conj().T @ YR, I, atol=1e-13)
    assert np.allclose(np.tril(RA, -1), 0) and np.allclose(np.tril(RB, -1), 0)
    nP = np.linalg.norm(Phi) + np.linalg.norm(Psi)
    assert np.linalg.norm(Phi @ YR - YL @ RA) <= 1e-13 * nP
    assert np.linalg.norm(Psi @ YR - YL @ RB) <= 1e-13 * nP
    assert np.allclose(np.diag(RB).imag, 0) and np.all(np.diag(RB).real >= 0)
    oRA, oRB, oYL, oYR = oracle_ordqz(Phi, Psi, sigma)
    lam = np.diag(RA) / np.diag(RB)
    olam = np.diag(oRA) / np.diag(oRB)
    # same ordered eigenvalues (distinct with probability one), same leading subspaces
    assert np.allclose(lam, olam, rtol=1e-10, atol=1e-12)
    for j in range(1, s):
        ang = np.max(sla.subspace_angles(YR[:, :j], oYR[:, :j]))
        assert ang < 1e-9
    # same diagonal of RB (unique once ordered and phase-normalised)
    assert np.allclose(np.diag(RB), np.diag(oRB), rtol=1e-10, atol=1e-12)


def test_host_ordqz_infinite_and_zero_eigenvalues(built):
    rng = np.random.default_rng(7)
    s = 10
    Phi = rng.standard_normal((s, s)) + 0j
    Psi = rng.standard_normal((s, s)) + 0j
    Psi[:, 3] = 0.0          # an infinite eigenvalue
    Phi[:, 5] = 0.0          # a zero eigenvalue
    RA, RB, YL, YR = G.gplhr_ordqz(Phi, Psi, 0.05)
    assert np.linalg.norm(Phi @ YR - YL @ RA) <= 1e-12 * np.linalg.norm(Phi)
    assert np.linalg.norm(Psi @ YR - YL @ RB) <= 1e-12 * np.linalg.norm(Psi)
    assert abs(RB[-1, -1]) <= 1e-12 * np.linalg.norm(Psi)            # infinite one last
    lam0 = RA[0, 0] / RB[0, 0]
    assert abs(lam0) <= 1e-12 * np.linalg.norm(Phi)                   # zero eigenvalue nearest 0.05
    ref = sla.eigvals(Phi, Psi)
    fin = ref[np.isfinite(ref)]
    got = (np.diag(RA) / np.where(np.diag(RB) == 0, np.nan, np.diag(RB)))[:-1]
    for mu in fin:
        assert np.min(np.abs(got - mu)) <= 1e-9 * max(1.0, abs(mu))


def test_host_mfactors_match_oracle(built):
    rng = np.random.default_rng(9)
    k = 7
    RA = np.triu(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))
    RB = np.triu(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))
    RA[1, 1] *= 1e-3
    RB[2, 2] *= 1e-3
    MA, MB = G.gplhr_mfactors(RA, RB)
    oMA, oMB, _ = oracle_m_factors(RA, RB)
    assert np.allclose(MA, oMA, rtol=1e-13, atol=1e-13)
    assert np.allclose(MB, oMB, rtol=1e-13, atol=1e-13)


def test_create_rejects_bad_input_without_gpu_work(built):
    """Argument validation happens before any device call."""
    import scipy.sparse as sp
    A = sp.identity(10, format="csr")
    with pytest.raises(G.GplhrError) as e:
        G.gplhr_create(A, None, 0.5, 0, 1)          # k = 0
    assert e.value.status == G.GPLHR_EINVAL
    with pytest.raises(G.GplhrError):
        G.gplhr_create(A, None, float("nan"), 2, 1)  # sigma not finite
    with pytest.raises(G.GplhrError):
        G.gplhr_create(A, None, 0.5, 4, 1)           # (m+3) k > n


def test_create_batched_refuses_null_arrays_without_a_gpu(built):
    import ctypes as C
    out = (C.c_void_p * 1)()
    st = built.gplhr_create_batched(1, None, None, None, None, None, None, None, out, None, 0)
    assert st == G.GPLHR_EINVAL
    assert "non-null" in G.gplhr_last_error(None)


def test_device_qz_refuses_bad_sizes_without_a_gpu(built):
    """gplhr_ordqz_device checks s and its pointers before any device call."""
    for s in (0, 81):
        st = built.gplhr_ordqz_device(s, None, None, 0.0, 0.0, -1, None, None, None, None, None, None)
        assert st == G.GPLHR_EINVAL
    assert "s <= 80" in G.gplhr_last_error(None)


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the binding passes through the C ABI has the header's size and field
    offsets (a C program compiled against include/gplhr.h prints them)."""
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    import ctypes as C
    structs = {"gplhr_csr": G.Csr, "gplhr_precond": G.Precond, "gplhr_opts": G.Opts, "gplhr_info": G.Info,
               "gplhr_persist_stats": G.PersistStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gplhr.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
