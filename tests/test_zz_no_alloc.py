"""knor_lloyd_step_noalloc: one Lloyd step that allocates no device memory.

It serves callers that cannot call cudaMalloc (device memory owned by another
allocator, or loops where cudaMalloc's device synchronisation is not
allowed).  These tests call it through the C ABI, twice in a row, and check
it against the context entry points (knor_create / knor_iterate) on the same
centroids: identical assignments and counts, and means within the parity
tolerance.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_1606_08905_gb300 import build as kbuild
from paper_1606_08905_gb300 import knor, synth
from parity import check_centroids

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    knor.load()


@pytest.mark.parametrize("n,d,k", [(50_000, 32, 20), (7_777, 3, 9), (20_000, 16, 200)])
def test_noalloc_step_matches_context_twice(n, d, k):
    X = synth.spd_mixture(n, d, min(k, 20), 31 + d).cuda()
    with knor.Context(X, k, seed=11, prune=False) as ctx:
        C32 = torch.as_tensor(ctx.centroids_f32()).cuda()
        for call in range(2):
            C_before = ctx.centroids()
            a = torch.empty(n, dtype=torch.int32, device="cuda")
            S = torch.empty((k, d), dtype=torch.float64, device="cuda")
            N = torch.empty(k, dtype=torch.int64, device="cuda")
            knor.lloyd_step_noalloc(X, C32, a, S, N)
            ctx.iterate()
            a_ref = ctx.assignments()
            assert np.array_equal(a.cpu().numpy(), a_ref), f"call {call + 1}: assignments differ"
            cnt = np.bincount(a_ref, minlength=k)
            assert np.array_equal(N.cpu().numpy(), cnt), f"call {call + 1}: counts differ"
            Nn = N.cpu().numpy()
            means = np.where(Nn[:, None] > 0, S.cpu().numpy() / np.maximum(Nn, 1)[:, None], C_before)
            check_centroids(means, ctx.centroids(), f"call {call + 1}")
            C32 = torch.as_tensor(ctx.centroids_f32()).cuda()


def test_noalloc_rejects_sizes_beyond_the_scratch_array():
    X = torch.zeros((100, 64), dtype=torch.float32, device="cuda")
    C = torch.zeros((64, 64), dtype=torch.float32, device="cuda")  # k (d + 1) = 4160 > 4096
    a = torch.empty(100, dtype=torch.int32, device="cuda")
    S = torch.empty((64, 64), dtype=torch.float64, device="cuda")
    N = torch.empty(64, dtype=torch.int64, device="cuda")
    with pytest.raises(knor.KnorError) as e:
        knor.lloyd_step_noalloc(X, C, a, S, N)
    assert e.value.status == knor.KNOR_ERR_ARG and "4096" in str(e.value)
    # host buffers are refused, not dereferenced: by the Python wrapper, and
    # by the C entry point itself when it is called directly
    with pytest.raises(ValueError):
        knor.lloyd_step_noalloc(X, C[:8].cpu(), a, S[:8], N[:8])
    Ch = C[:8].cpu().contiguous()
    st = knor.load().knor_lloyd_step_noalloc(X.data_ptr(), 100, 64, 8, Ch.data_ptr(), a.data_ptr(),
                                             S.data_ptr(), N.data_ptr(), None)
    assert st == knor.KNOR_ERR_ARG


def test_noalloc_accepts_the_largest_size():
    """k (d + 1) = 4096 exactly (d = 63, k = 64): the largest slot stride and
    shared-memory size the fixed array allows, against the context path."""
    n, d, k = 30_000, 63, 64
    X = synth.aniso_mixture(n, d, 16, 77).cuda()
    with knor.Context(X, k, seed=3, prune=False) as ctx:
        C32 = torch.as_tensor(ctx.centroids_f32()).cuda()
        C_before = ctx.centroids()
        a = torch.empty(n, dtype=torch.int32, device="cuda")
        S = torch.empty((k, d), dtype=torch.float64, device="cuda")
        N = torch.empty(k, dtype=torch.int64, device="cuda")
        knor.lloyd_step_noalloc(X, C32, a, S, N)
        ctx.iterate()
        a_ref = ctx.assignments()
        assert np.array_equal(a.cpu().numpy(), a_ref)
        Nn = N.cpu().numpy()
        assert np.array_equal(Nn, np.bincount(a_ref, minlength=k))
        means = np.where(Nn[:, None] > 0, S.cpu().numpy() / np.maximum(Nn, 1)[:, None], C_before)
        check_centroids(means, ctx.centroids(), "k (d + 1) = 4096")
