"""The ordered QZ on the device (gplhr_ordqz_device, one CTA) against the host QZ of the
same library and against the definition of an ordered generalized Schur form (footnote to
Algorithm 2, step 2): Phi = Y_L R_A Y_R^*, Psi = Y_L R_B Y_R^*, Y_L and Y_R unitary, R_A and
R_B upper triangular with R_B's diagonal real and non-negative, and |R_A(j,j)/R_B(j,j) -
sigma| non-decreasing."""
import numpy as np
import pytest

import paper_1506_06829_gb300.gplhr as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"


def _pencil(rng, s, tri):
    Phi = rng.standard_normal((s, s)) + 1j * rng.standard_normal((s, s))
    Psi = rng.standard_normal((s, s)) + 1j * rng.standard_normal((s, s))
    if tri:  # the factored projected pencil: Phi upper triangular
        Phi = np.triu(Phi)
    return Phi, Psi


@pytest.mark.parametrize("s,tri", [(1, False), (2, False), (5, True), (16, False), (16, True), (32, False),
                                   (57, True), (80, False), (80, True)])
def test_device_qz_is_an_ordered_schur_form_equal_to_the_host_one(s, tri):
    rng = np.random.default_rng(300 + s + (1 if tri else 0))
    Phi, Psi = _pencil(rng, s, tri)
    sigma = complex(rng.standard_normal(), rng.standard_normal())
    RA, RB, YL, YR, st = G.gplhr_ordqz_device(torch.from_numpy(Phi).to(DEV), torch.from_numpy(Psi).to(DEV), sigma)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    RA, RB, YL, YR = (M.cpu().numpy() for M in (RA, RB, YL, YR))
    I = np.eye(s)
    assert np.linalg.norm(YL.conj().T @ YL - I) <= 1e-13 * s
    assert np.linalg.norm(YR.conj().T @ YR - I) <= 1e-13 * s
    assert np.all(np.tril(RA, -1) == 0) and np.all(np.tril(RB, -1) == 0)
    d = np.diag(RB)
    assert np.all(d.imag == 0) and np.all(d.real >= 0)
    nP, nS = np.linalg.norm(Phi), np.linalg.norm(Psi)
    assert np.linalg.norm(YL @ RA @ YR.conj().T - Phi) <= 1e-13 * s * nP
    assert np.linalg.norm(YL @ RB @ YR.conj().T - Psi) <= 1e-13 * s * nS
    lam = np.diag(RA) / np.diag(RB)
    dist = np.abs(lam - sigma)
    assert np.all(np.diff(dist) >= -1e-12 * np.maximum(1.0, dist[1:]))
    # the host routine: the same eigenvalues in the same order, and the same Schur vectors
    # up to a unit phase per column (well separated random eigenvalues)
    hRA, hRB, hYL, hYR = G.gplhr_ordqz(Phi, Psi, sigma)
    hlam = np.diag(hRA) / np.diag(hRB)
    assert np.max(np.abs(lam - hlam) / (1.0 + np.abs(hlam))) <= 1e-10
    for j in range(s):
        assert abs(abs(np.vdot(hYR[:, j], YR[:, j])) - 1.0) <= 1e-9
        assert abs(abs(np.vdot(hYL[:, j], YL[:, j])) - 1.0) <= 1e-9


def test_device_qz_leading_positions_only():
    """nsort = k orders the k nearest pairs into the leading positions; the rest keep the
    sweeps' order (still a Schur form)."""
    rng = np.random.default_rng(7)
    s, k = 40, 6
    Phi, Psi = _pencil(rng, s, True)
    sigma = 0.3 - 0.2j
    RA, RB, YL, YR, st = G.gplhr_ordqz_device(torch.from_numpy(Phi).to(DEV), torch.from_numpy(Psi).to(DEV), sigma,
                                              nsort=k)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    RA, RB, YL, YR = (M.cpu().numpy() for M in (RA, RB, YL, YR))
    assert np.linalg.norm(YL @ RA @ YR.conj().T - Phi) <= 1e-13 * s * np.linalg.norm(Phi)
    lam = np.diag(RA) / np.diag(RB)
    ref = np.linalg.eigvals(np.linalg.solve(Psi, Phi))
    want = np.sort(np.abs(ref - sigma))[:k]
    assert np.allclose(np.abs(lam[:k] - sigma), want, rtol=1e-10, atol=0)


def test_device_qz_bad_sizes():
    with pytest.raises(G.GplhrError):
        G.gplhr_ordqz_device(torch.zeros((81, 81), dtype=torch.complex128, device=DEV),
                             torch.zeros((81, 81), dtype=torch.complex128, device=DEV), 0.0)
