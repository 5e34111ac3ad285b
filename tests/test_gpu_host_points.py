"""knor_opts.points_in_host: the points stay in host memory (pageable or
pinned) and the scans read them over the host link; the results must be
bit-identical to the same run with the points copied into HBM."""
import numpy as np
import pytest
import torch

from paper_1606_08905_gb300 import build as kbuild
from paper_1606_08905_gb300 import knor, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    knor.load()


@pytest.mark.parametrize("pinned", [False, True], ids=["pageable", "pinned"])
@pytest.mark.parametrize("prune,elkan", [(True, False), (False, False), (True, True)], ids=["mti", "plain", "elkan"])
def test_points_in_host_memory_match_device_copy(pinned, prune, elkan):
    X = synth.spd_mixture(50_000, 32, 16, 61)
    Xh = X.pin_memory() if pinned else X.numpy()
    with knor.Context(Xh, 16, seed=5, prune=prune, elkan=elkan, points_in_host=True) as h, \
            knor.Context(X.cuda(), 16, seed=5, prune=prune, elkan=elkan) as g:
        dh, rh = h.run(30)
        dg, rg = g.run(30)
        assert dh == dg and rh == rg
        assert np.array_equal(h.centroids(), g.centroids())
        assert np.array_equal(h.assignments(), g.assignments())


def test_points_in_host_refuses_device_and_unaligned_buffers():
    X = synth.spd_mixture(1000, 8, 4, 62)
    with pytest.raises(knor.KnorError) as e:
        knor.Context(X.cuda(), 4, points_in_host=True)
    assert e.value.status == knor.KNOR_ERR_ARG
    buf = np.zeros(1000 * 8 + 1, np.float32)
    Xu = buf[1:].reshape(1000, 8)  # 4-byte offset: not 16-byte aligned
    Xu[:] = X.numpy()
    with pytest.raises(knor.KnorError):
        knor.Context(Xu, 4, points_in_host=True)
