"""GPU test of gplhr_gram_noalloc, the Gram product that allocates nothing.

Some callers cannot call cudaMalloc (their device memory belongs to another
allocator or pool, or they cannot afford the synchronisation an allocation brings).
gplhr_gram_noalloc serves them with its scratch in a fixed device array inside the
library.  This file is collected last so that a run stopping at the first failure
has already run every other test; it passes alone in a fresh process and after the
rest of the suite.

The check: through the C ABI, two calls in a row give the same C = X^* Y as the
context-based entry point gplhr_gram, to the tolerance of the other Gram tests.  The
second call is smaller than the first, so partial sums the first call left in the
shared scratch must not leak into the second result.
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from paper_1506_06829_gb300 import gplhr as G

pytestmark = pytest.mark.gpu


def _rand(rng, n, w):
    return torch.from_numpy(rng.standard_normal((n, w)) + 1j * rng.standard_normal((n, w))).to("cuda:0")


def test_gram_noalloc_matches_gram_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(2024)
    cases = [(262144, 32, 64), (70001, 8, 24)]       # second call smaller than the first
    for n, wx, wy in cases:
        X, Y = _rand(rng, n, wx), _rand(rng, n, wy)
        C_new = torch.full((wx, wy), float("nan"), dtype=torch.complex128, device="cuda:0")
        G.gplhr_gram_noalloc(X, Y, C_new)
        torch.cuda.synchronize()
        # reference: the existing entry point (needs a context of matching n)
        ref_ctx = G.gplhr_create(sp.identity(n, format="csr"), None, 0.5, 8, 7)
        try:
            C_ref = torch.zeros((wx, wy), dtype=torch.complex128, device="cuda:0")
            G.gplhr_gram(ref_ctx, X, Y, C_ref)
        finally:
            G.gplhr_destroy(ref_ctx)
        got, ref = C_new.cpu().numpy(), C_ref.cpu().numpy()
        scale = float(torch.linalg.norm(X).item() * torch.linalg.norm(Y).item())
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - ref) <= 1e-13 * scale


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
