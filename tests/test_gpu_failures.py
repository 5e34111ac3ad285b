"""Error paths of the C ABI, exercised with host-side fault injection: an
allocation that fails as if the device were out of memory, and the device
error flag that a bounded device-side wait sets when it gives up.  Nothing
here faults, traps or blocks the GPU: the failure is made on the host."""
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
    yield
    knor.test_fail_alloc(-1)


@pytest.mark.parametrize("after", [0, 1, 5, 12, 20])
def test_create_reports_out_of_memory_and_cleans_up(after):
    X = synth.spd_mixture(5000, 32, 8, 41).cuda()
    free0 = torch.cuda.mem_get_info()[0]
    knor.test_fail_alloc(after)
    try:
        with pytest.raises(knor.KnorError) as e:
            knor.Context(X, 8, seed=1)
        assert e.value.status == knor.KNOR_ERR_OOM and "injected" in str(e.value)
    finally:
        knor.test_fail_alloc(-1)
    torch.cuda.synchronize()
    # everything allocated before the failure was released again
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)
    with knor.Context(X, 8, seed=1) as c:  # and the next creation works
        c.run(5)


def test_failed_call_leaves_the_context_usable():
    X = synth.spd_mixture(5000, 16, 6, 42).cuda()
    with knor.Context(X, 6, seed=2) as c:
        c.run(3)
        knor.test_fail_alloc(0)  # knor_get_assignments into host memory allocates a staging buffer
        try:
            with pytest.raises(knor.KnorError) as e:
                c.assignments()
            assert e.value.status == knor.KNOR_ERR_OOM
        finally:
            knor.test_fail_alloc(-1)
        a = c.assignments()
        assert a.shape == (5000,) and a.min() >= 0 and a.max() < 6
        c.iterate()
    # the context was destroyed without error by the with-block


@pytest.mark.parametrize("prune", [True, False])
def test_error_flag_reports_timeout_once(prune):
    X = synth.spd_mixture(8000, 32, 10, 43).cuda()
    with knor.Context(X, 10, seed=3, prune=prune) as c, knor.Context(X, 10, seed=3, prune=prune) as ref:
        c.iterate()
        ref.iterate()
        c.test_raise_error_flag()
        with pytest.raises(knor.KnorError) as e:
            c.iterate()
        assert e.value.status == knor.KNOR_ERR_TIMEOUT
        ref.iterate()
        # the flag was cleared: the run goes on (its results match a context
        # that saw no flag, since no device wait in the FP32 path reads it)
        for _ in range(3):
            c.iterate()
            ref.iterate()
        assert np.array_equal(c.assignments(), ref.assignments())
        done, _ = c.run(5)
        assert done >= 1
