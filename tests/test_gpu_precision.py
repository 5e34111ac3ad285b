"""GPU parity of the precision forms (BF16 or FP16 tensor-core distances with
an exact FP32 recheck of the points whose top-2 gap is inside the error bound).

The form is certified to return exactly the FP32 assignment of the plain path:
at every iteration its assignments must equal, bit for bit, the oracle's FP32
restatement of the argmin on the very FP32 centroids the context scanned; they
must also meet the FP64 near-tie rule, and the new centroids must be the
oracle's means of the assignments.  Planted exact ties force rechecks.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_08905_gb300 import build as kbuild
from paper_1606_08905_gb300 import knor, synth
from parity import check_assignments, check_centroids

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    knor.load()


FORMS = ["bf16", "fp16", "fp8"]  # FP8 e4m3 needs d = 128


def _run_checked(X, k, iters, seed=42, init=None, form="bf16"):
    Xd = torch.as_tensor(X).cuda()
    rechecked = 0
    with knor.Context(Xd, k, seed=seed, precision=form, init="explicit" if init is not None else "forgy",
                      debug_invariants=True) as c:
        if init is not None:
            c.set_init_centroids(init)
        for t in range(iters):
            C_before = c.centroids()
            C32 = c.centroids_f32()
            s = c.iterate()
            a = c.assignments()
            a32 = oracle.assign_f32(X, C32)
            bad = np.flatnonzero(a != a32)
            assert bad.size == 0, f"it {t + 1}: {bad.size} assignments differ from the FP32 argmin, e.g. {bad[:5]}"
            check_assignments(X, C_before, a, f"{form} it {t + 1}")
            C_ref, cnt = oracle.means(X, a, C_before)
            check_centroids(c.centroids(), C_ref, f"{form} it {t + 1}")
            # the tensor-core scan scores every pair; a recheck scores its
            # recorded candidates (at most 14), or all k on overflow
            assert X.shape[0] * k <= s["dist_evals"] <= X.shape[0] * k + s["rechecked"] * k
            assert s["violations"] == 0
            rechecked += s["rechecked"]
            if s["changed"] == 0:
                break
    return rechecked


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("n,d,k", [(5000, 128, 64), (20011, 128, 300), (9000, 64, 256), (30000, 128, 1024),
                                   (100, 64, 3), (130, 128, 129)])
def test_precision_form_equals_fp32_assignments(n, d, k, form):
    if form == "fp8" and d != 128:
        pytest.skip("the FP8 form needs d = 128")
    X = synth.aniso_mixture(n, d, min(k, 64), 200 + k).numpy()
    _run_checked(X, k, 12, form=form)


@pytest.mark.parametrize("scale", [1e-12, 1e-3, 1e12])
def test_fp16_form_scales_any_magnitude(scale):
    """FP16 operands are scaled by powers of two into range: data many orders
    of magnitude away from 1 still gives the FP32 assignments, and few points
    need the recheck."""
    X = (synth.aniso_mixture(8000, 64, 32, 77).numpy().astype(np.float64) * scale).astype(np.float32)
    rechecked = _run_checked(X, 32, 4, form="fp16")
    assert rechecked < 0.5 * 4 * X.shape[0]


def test_fp16_form_rechecks_fewer_points_than_bf16():
    """The FP16 bound is eight times tighter (11 significand bits against 8)."""
    X = synth.aniso_mixture(30000, 128, 64, 1204).numpy()
    rb = _run_checked(X, 1024, 3, form="bf16")
    rh = _run_checked(X, 1024, 3, form="fp16")
    assert rh < rb


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("n,d,k", [(600_000, 64, 64), (300_000, 128, 256)])
def test_precision_form_many_tiles_per_cta(n, d, k, form):
    """Enough points that every CTA of the persistent kernel reuses its tile
    stages and accumulator buffers many times."""
    if form == "fp8" and d != 128:
        pytest.skip("the FP8 form needs d = 128")
    X = synth.aniso_mixture(n, d, min(k, 64), 300 + k).numpy()
    Xd = torch.as_tensor(X).cuda()
    with knor.Context(Xd, k, seed=5, precision=form) as c:
        for t in range(2):
            C32 = c.centroids_f32()
            c.iterate()
            a = c.assignments()
            a32 = oracle.assign_f32(X, C32)
            assert np.array_equal(a, a32), f"it {t + 1}: {int((a != a32).sum())} differ"


def test_plain_path_large_kd_matches_fp32_restatement():
    """The plain FP32 path when k x d is too large for shared memory
    (centroids read from global memory, cluster sums by FP64 atomics)."""
    X = synth.aniso_mixture(20000, 128, 64, 17).numpy()
    with knor.Context(torch.as_tensor(X).cuda(), 1024, seed=3, prune=False) as c:
        for t in range(3):
            C_before, C32 = c.centroids(), c.centroids_f32()
            c.iterate()
            a = c.assignments()
            a32 = oracle.assign_f32(X, C32)
            assert np.array_equal(a, a32), f"it {t + 1}: {int((a != a32).sum())} differ"
            C_ref, _ = oracle.means(X, a, C_before)
            check_centroids(c.centroids(), C_ref, f"plain large kd it {t + 1}")


@pytest.mark.parametrize("form", FORMS)
def test_planted_ties_are_rechecked(form):
    """Points exactly between two centroids have a zero top-2 gap: they must be
    re-scored in FP32 (and land on the lower index)."""
    rng = np.random.default_rng(3)
    d, k = (128 if form == "fp8" else 64), 32
    C = rng.uniform(-5, 5, (k, d)).astype(np.float32)
    mids = ((C[0:8].astype(np.float64) + C[8:16].astype(np.float64)) / 2).astype(np.float32)
    X = np.concatenate([mids, C + 0.01 * rng.standard_normal((k, d)).astype(np.float32),
                        rng.uniform(-5, 5, (3000, d)).astype(np.float32)])
    Xd = torch.as_tensor(X).cuda()
    with knor.Context(Xd, k, init="explicit", precision=form, debug_invariants=True) as c:
        c.set_init_centroids(C.astype(np.float64))
        s = c.iterate()
        assert s["rechecked"] >= 8
        assert s["violations"] == 0, s
        a, ref = c.assignments(), oracle.assign_f32(X, C)
        bad = np.flatnonzero(a != ref)
        assert bad.size == 0, (f"{bad.size} differ: points {bad[:8]}, library {a[bad[:8]]}, "
                               f"FP32 argmin {ref[bad[:8]]}, stats {s}")


@pytest.mark.parametrize("form", FORMS)
def test_stale_operand_rows_never_enter_candidate_lists(form):
    """Rows past the end of the gathered list are stale device memory.  Fill
    freed memory with 16-bit infinities first (so the context's buffers very
    likely start out holding them): those rows must record no candidates,
    in particular not into the first listed point's list."""
    # 16-bit infinities; for FP8 e4m3 (no infinity) the byte pair 0x7F7F is
    # two NaNs, the worst it can hold
    inf16 = {"fp16": 0x7C00, "bf16": 0x7F80, "fp8": 0x7F7F}[form]
    junk = torch.full((256 << 20,), inf16, dtype=torch.int16, device="cuda")
    del junk
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    rng = np.random.default_rng(11)
    d, k = (128 if form == "fp8" else 64), 48
    C = rng.uniform(-5, 5, (k, d)).astype(np.float32)
    X = rng.uniform(-5, 5, (20000, d)).astype(np.float32)
    with knor.Context(torch.as_tensor(X).cuda(), k, init="explicit", precision=form, debug_invariants=True) as c:
        c.set_init_centroids(C.astype(np.float64))
        for _ in range(3):
            C32 = c.centroids_f32()
            s = c.iterate()
            assert s["violations"] == 0, s
            a = c.assignments()
            ref = oracle.assign_f32(X, C32)
            assert np.array_equal(a, ref), f"{int((a != ref).sum())} differ"


@pytest.mark.parametrize("form", FORMS)
def test_precision_form_rejects_unsupported_shapes(form):
    for d in ((32, 64) if form == "fp8" else (32,)):
        X = torch.zeros((100, d), device="cuda")
        with pytest.raises(knor.KnorError) as e:
            knor.Context(X, 4, precision=form)
        assert e.value.status == knor.KNOR_ERR_ARG


@pytest.mark.parametrize("form", FORMS)
def test_precision_workload_full_size_teacher_forced(form):
    """The 10M x 128, k = 1024 precision workload at full size: at iterations
    1, 2 and 5 the tensor-core form assigns every point exactly as the plain
    FP32 path started from the same centroids, and the FP64 oracle agrees on
    a 20k-point sample (near-tie rule)."""
    n, d, k = 10_000_000, 128, 1024
    X = synth.make("aniso", n, d, k, 1003, device="cuda")
    rng = np.random.default_rng(1)
    sample = torch.as_tensor(np.sort(rng.choice(n, 20000, replace=False)), device="cuda")
    Xs = X[sample].cpu().numpy()
    with knor.Context(X, k, seed=42, precision=form) as c:
        for t in range(1, 6):
            C_before = c.centroids()
            s = c.iterate()
            if t not in (1, 2, 5):
                continue
            a = torch.empty(n, dtype=torch.int32, device="cuda")
            c.assignments(a)
            with knor.Context(X, k, init="explicit", prune=False) as q:
                q.set_init_centroids(C_before)
                q.iterate()
                b = torch.empty(n, dtype=torch.int32, device="cuda")
                q.assignments(b)
            check_assignments(Xs, C_before, a[sample].cpu().numpy(), f"{form} 10M it {t}")
            check_assignments(Xs, C_before, b[sample].cpu().numpy(), f"fp32 10M it {t}")
            diff = int((a != b).sum())
            assert diff == 0, f"iteration {t}: {diff} assignments differ from the FP32 path (rechecked {s['rechecked']})"
