"""Host-side checks of the Python binding's Gram entry points (no GPU needed).

The C ABI receives raw pointers and sizes, so a wrong dtype, a transposed view, a
short Y or a small C would make the Gram kernels read or write out of bounds.  The
binding refuses each such operand with GPLHR_EINVAL before anything is launched; here
every refusal happens on CPU tensors, which also shows that no launch was attempted
(the last check, the device, comes after all the shape checks)."""
import pytest

torch = pytest.importorskip("torch")

from paper_1506_06829_gb300 import gplhr as G


def _c(*shape, dtype=torch.complex128):
    return torch.zeros(shape, dtype=dtype)


GOOD = (_c(64, 4), _c(64, 6), _c(4, 6))


def _cases():
    X, Y, C = GOOD
    yield "complex64 X", (X.to(torch.complex64), Y, C), "complex128"
    yield "float64 Y", (X, torch.zeros(64, 6, dtype=torch.float64), C), "complex128"
    yield "complex64 C", (X, Y, C.to(torch.complex64)), "complex128"
    yield "short Y", (X, _c(63, 6), C), "rows"
    yield "transposed X", (_c(4, 64).t(), Y, C), "unit column stride"
    yield "transposed Y", (X, _c(6, 64).t(), C), "unit column stride"
    yield "small C", (X, Y, _c(4, 5)), "contiguous 4 x 6"
    yield "transposed C", (X, Y, _c(6, 4).t()), "contiguous 4 x 6"
    yield "1-D X", (torch.zeros(64, dtype=torch.complex128), Y, C), "2-D"
    yield "empty X", (_c(0, 4), _c(0, 6), C), "empty"
    yield "host tensors", (X, Y, C), "CUDA"


@pytest.mark.parametrize("name,args,needle", list(_cases()), ids=[c[0] for c in _cases()])
def test_gram_operands_refused_before_launch(name, args, needle):
    for call in (lambda: G.gplhr_gram_noalloc(*args), lambda: G.gplhr_gram(None, *args)):
        with pytest.raises(G.GplhrError) as e:
            call()
        assert e.value.status == G.GPLHR_EINVAL
        assert needle in str(e.value), (name, str(e.value))
