"""GPU test of gplhr_gram_noalloc, the Gram product that allocates nothing.

Some callers cannot call cudaMalloc: their device memory belongs to another
allocator or pool, or they cannot afford the synchronisation an allocation brings.
gplhr_gram_noalloc serves them with its scratch in a fixed device array inside the
library.  This file is collected last so that a run stopping at the first failure
has already run every other test; it passes alone in a fresh process and after the
rest of the suite.

The checks, through the C ABI: C = X^* Y agrees element by element with NumPy's
X^* Y and with the context-based entry point gplhr_gram, within 1e-12 of the
entry's sum |x||y| (both are DFMA dot products over at most a few ten thousand rows
per partial sum).  Two calls in a row, the second smaller than the first, so partial
sums the first call left in the shared scratch must not leak into the second result;
the two size limits the call enforces (wx + wy = 768 staged columns, wx wy = 16384
outputs); and a call on a non-default stream, read after that stream synchronises.
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from paper_1506_06829_gb300 import gplhr as G

pytestmark = pytest.mark.gpu
RTOL = 1e-12


def _rand(rng, n, w):
    return rng.standard_normal((n, w)) + 1j * rng.standard_normal((n, w))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _check(got, Xh, Yh):
    ref = Xh.conj().T @ Yh
    scale = np.abs(Xh).T @ np.abs(Yh)
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref) / scale
    assert err.max() <= RTOL, err.max()


def _via_gram(Xd, Yd, n, wx, wy):
    """The existing entry point, in column blocks of Y that its context admits."""
    C = torch.zeros((wx, wy), dtype=torch.complex128, device="cuda:0")
    ctx = G.gplhr_create(sp.identity(n, format="csr"), None, 0.5, 8, 7)   # s_max = 80
    try:
        for j0 in range(0, wy, 128):
            j1 = min(wy, j0 + 128)
            Cb = torch.zeros((wx, j1 - j0), dtype=torch.complex128, device="cuda:0")
            G.gplhr_gram(ctx, Xd, Yd[:, j0:j1], Cb)
            C[:, j0:j1] = Cb
    finally:
        G.gplhr_destroy(ctx)
    return C.cpu().numpy()


def _noalloc(Xd, Yd, wx, wy, stream=None):
    C = torch.full((wx, wy), float("nan"), dtype=torch.complex128, device="cuda:0")
    if stream is None:
        G.gplhr_gram_noalloc(Xd, Yd, C)
        torch.cuda.synchronize()
    else:
        G.gplhr_gram_noalloc(Xd, Yd, C, stream.cuda_stream)
        stream.synchronize()
    return C.cpu().numpy()


@pytest.mark.parametrize("cases", [
    [(262144, 32, 64), (70001, 8, 24)],      # second call smaller than the first
    [(50000, 16, 752), (100003, 128, 128)],  # wx + wy = 768; wx wy = 16384
])
def test_gram_noalloc_matches_gram_on_two_calls_in_a_row(cases):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(2024 + cases[0][1])
    for n, wx, wy in cases:
        Xh, Yh = _rand(rng, n, wx), _rand(rng, n, wy)
        Xd, Yd = _dev(Xh), _dev(Yh)
        got = _noalloc(Xd, Yd, wx, wy)
        _check(got, Xh, Yh)
        ref = _via_gram(Xd, Yd, n, wx, wy)
        assert np.all(np.abs(got - ref) <= RTOL * (np.abs(Xh).T @ np.abs(Yh)))


def test_gram_noalloc_on_a_side_stream():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(77)
    n, wx, wy = 123457, 24, 40
    Xh, Yh = _rand(rng, n, wx), _rand(rng, n, wy)
    Xd, Yd = _dev(Xh), _dev(Yh)
    torch.cuda.synchronize()
    s = torch.cuda.Stream(device="cuda:0")
    got = _noalloc(Xd, Yd, wx, wy, stream=s)
    _check(got, Xh, Yh)


def test_gram_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X = torch.zeros((100, 200), dtype=torch.complex128, device="cuda:0")
    Y = torch.zeros((100, 100), dtype=torch.complex128, device="cuda:0")
    C = torch.zeros((200, 100), dtype=torch.complex128, device="cuda:0")
    with pytest.raises(G.GplhrError) as e:
        G.gplhr_gram_noalloc(X, Y, C)                  # 200 * 100 > 16384 outputs
    assert e.value.status == G.GPLHR_EINVAL
    assert "16384" in G.gplhr_last_error(None)
    X = torch.zeros((100, 8), dtype=torch.complex128, device="cuda:0")
    Y = torch.zeros((100, 761), dtype=torch.complex128, device="cuda:0")
    C = torch.zeros((8, 761), dtype=torch.complex128, device="cuda:0")
    with pytest.raises(G.GplhrError) as e:
        G.gplhr_gram_noalloc(X, Y, C)                  # 8 + 761 > 768 staged columns
    assert e.value.status == G.GPLHR_EINVAL
