"""The no-allocation step's Python wrapper checks every buffer's shape and
device before anything reaches the C ABI (which cannot see buffer sizes, so
a wrong shape there would read or write out of bounds on the device).  These
checks run without a GPU: the wrapper raises before loading the library."""
import pytest
import torch

from paper_1606_08905_gb300 import knor


def _bufs(n=10, d=4, k=3):
    return (torch.zeros(n, d), torch.zeros(k, d), torch.zeros(n, dtype=torch.int32),
            torch.zeros(k, d, dtype=torch.float64), torch.zeros(k, dtype=torch.int64))


def test_host_tensors_are_refused_before_any_launch():
    with pytest.raises(ValueError, match="CUDA tensor"):
        knor.lloyd_step_noalloc(*_bufs())


class _FakeCuda(torch.Tensor):
    """A CPU tensor that reports itself as a CUDA tensor, so that the shape
    checks (which come after the device checks) can be exercised on a CPU."""

    @property
    def is_cuda(self):
        return True


def _fake(t):
    return t.as_subclass(_FakeCuda)


@pytest.mark.parametrize("bad", ["centroid_width", "short_assign", "short_sums", "short_counts"])
def test_wrong_shapes_are_refused(bad):
    X, C, a, S, N = _bufs()
    if bad == "centroid_width":
        C = torch.zeros(3, 5)
    elif bad == "short_assign":
        a = torch.zeros(9, dtype=torch.int32)
    elif bad == "short_sums":
        S = torch.zeros(3, 3, dtype=torch.float64)
    else:
        N = torch.zeros(2, dtype=torch.int64)
    with pytest.raises(ValueError):
        knor.lloyd_step_noalloc(*(_fake(t) for t in (X, C, a, S, N)))
