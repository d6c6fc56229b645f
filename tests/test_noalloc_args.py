"""CPU checks of the argument validation in front of sc_all_edges_noalloc.

The entry point takes raw device pointers and trusts n, nnz and the output
length, so a wrong dtype, a non-contiguous view, a short output or a tensor on
another device would make its kernels read or write out of bounds. The binding
rejects each of these before the library is loaded or called."""
import pytest

torch = pytest.importorskip("torch")

from paper_2305_16086_gb300 import binding


@pytest.fixture
def no_library(monkeypatch):
    def fail(*a, **k):
        raise AssertionError("the library must not be reached with bad arguments")

    monkeypatch.setattr(binding, "load", fail)


def _ok():
    rp = torch.tensor([0, 1, 2], dtype=torch.int32)
    ci = torch.tensor([1, 0], dtype=torch.int32)
    out = torch.zeros(2, dtype=torch.float64)
    return rp, ci, out


@pytest.mark.parametrize("case", ["rp_dtype", "ci_dtype", "out_dtype", "rp_2d", "ci_noncontig", "out_short",
                                  "rp_short", "numpy_out", "cpu_tensors"])
def test_bad_argument_rejected_before_the_call(no_library, case):
    rp, ci, out = _ok()
    if case == "rp_dtype":
        rp = rp.to(torch.int64)
    elif case == "ci_dtype":
        ci = ci.to(torch.int64)
    elif case == "out_dtype":
        out = out.to(torch.float32)
    elif case == "rp_2d":
        rp = rp.reshape(1, 3)
    elif case == "ci_noncontig":
        ci = torch.tensor([1, 9, 0, 9], dtype=torch.int32)[::2]
    elif case == "out_short":
        out = torch.zeros(1, dtype=torch.float64)
    elif case == "rp_short":
        rp = torch.tensor([0, 2], dtype=torch.int32)
    elif case == "numpy_out":
        out = out.numpy()
    # "cpu_tensors": well-formed but not on a CUDA device
    with pytest.raises((TypeError, ValueError)):
        binding.all_edges_noalloc(rp, ci, 3, out)
