"""GPU parity of the batched form: many independent problems in one
persistent launch per iteration.

Every instance must behave exactly as it would alone: Forgy indices from
seed + i, assignments at every iteration equal to the oracle's FP32
restatement on the very FP32 centroids the batch scanned (and to the FP64
oracle under the near-tie rule), centroids equal to the oracle's means of
the batch's assignments, and whole runs matching single-problem contexts
(assignments and iteration counts).  Converged instances stop.
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


def _instances(m, seed, n_lo=200, n_hi=30000):
    specs = synth.batched_specs(m, seed, n_lo=n_lo, n_hi=n_hi, k_hi=64)
    return [synth.batched_instance(s).numpy() for s in specs], [s.k for s in specs]


@pytest.mark.parametrize("prune", [True, False])
def test_batch_teacher_forced_against_oracle(prune):
    Xs, ks = _instances(14, 21)
    seed = 7
    with knor.Batch(Xs, ks, seed=seed, prune=prune) as b:
        for i, (X, k) in enumerate(zip(Xs, ks)):
            assert np.array_equal(b.init_indices(i), oracle.forgy_indices(X.shape[0], k, seed + i))
        for t in range(6):
            before = [(b.centroids(i), b.centroids_f32(i), b.instance(i)) for i in range(len(Xs))]
            s = b.iterate()
            assert s["violations"] == 0
            for i, X in enumerate(Xs):
                C64, C32, info = before[i]
                if info["iterations"] > 0 and info["converged"]:
                    continue  # masked: nothing may change
                a = b.assignments(i)
                a32 = oracle.assign_f32(X, C32)
                bad = np.flatnonzero(a != a32)
                assert bad.size == 0, f"it {t + 1} instance {i}: {bad.size} differ from the FP32 argmin"
                check_assignments(X, C64, a, f"batch it {t + 1} inst {i}")
                C_ref, _ = oracle.means(X, a, C64)
                check_centroids(b.centroids(i), C_ref, f"batch it {t + 1} inst {i}")


def test_batch_matches_single_problem_contexts():
    """Whole runs: each instance converges in the same number of iterations
    and to the same assignments as a knor_create context with seed + i."""
    Xs, ks = _instances(10, 33)
    seed = 100
    with knor.Batch(Xs, ks, seed=seed) as b:
        done, recs = b.run(60)
        for i, (X, k) in enumerate(zip(Xs, ks)):
            info = b.instance(i)
            with knor.Context(torch.as_tensor(X).cuda(), k, seed=seed + i) as c:
                nd, _ = c.run(60)
                assert info["iterations"] == nd, f"instance {i}: {info['iterations']} vs {nd} iterations"
                assert info["converged"] == 1
                assert np.array_equal(b.assignments(i), c.assignments()), f"instance {i}"
                check_centroids(b.centroids(i), c.centroids(), f"instance {i}")
        assert done == max(b.instance(i)["iterations"] for i in range(len(Xs)))
        assert recs[-1]["changed"] == 0
        pit, byts = b.work()
        assert pit == sum(X.shape[0] * b.instance(i)["iterations"] for i, X in enumerate(Xs))
        skipped = sum(r["clause1_skipped"] for r in recs)
        assert byts >= 8 * pit and byts <= 8 * pit + (pit - skipped) * (4 * 64 + 8)


def test_batch_pruned_equals_plain():
    Xs, ks = _instances(8, 45)
    with knor.Batch(Xs, ks, seed=3, prune=True) as bp, knor.Batch(Xs, ks, seed=3, prune=False) as bn:
        for t in range(8):
            sp, sn = bp.iterate(), bn.iterate()
            assert sp["changed"] == sn["changed"]
            for i in range(len(Xs)):
                assert np.array_equal(bp.assignments(i), bn.assignments(i)), f"it {t + 1} instance {i}"
            if t > 0:  # an instance whose Clause 1 lets most points through scans densely
                assert sp["dist_evals"] <= sn["dist_evals"]


def test_batch_explicit_init_and_reset():
    Xs, ks = _instances(5, 57)
    rng = np.random.default_rng(2)
    with knor.Batch(Xs, ks, seed=1) as b:
        C0 = [X[rng.choice(X.shape[0], k, replace=False)].astype(np.float64) for X, k in zip(Xs, ks)]
        for i, C in enumerate(C0):
            b.set_init_centroids(i, C)
        for i, C in enumerate(C0):
            assert np.array_equal(b.centroids(i), C)
        b.iterate()
        for i, X in enumerate(Xs):
            assert np.array_equal(b.assignments(i), oracle.assign_f32(X, C0[i].astype(np.float32)))
        first = [b.assignments(i) for i in range(len(Xs))]
        b.run(20)
        b.reset()
        b.iterate()
        for i in range(len(Xs)):
            assert np.array_equal(b.assignments(i), first[i])


def test_batch_device_inputs_and_edge_sizes():
    """Device tensors as input; single-point instances, k = n, k = 1."""
    rng = np.random.default_rng(4)
    Xs = [rng.standard_normal((1, 8)).astype(np.float32), rng.standard_normal((5, 16)).astype(np.float32),
          rng.standard_normal((300, 32)).astype(np.float32), rng.standard_normal((2000, 64)).astype(np.float32)]
    ks = [1, 5, 1, 200]
    with knor.Batch([torch.as_tensor(X).cuda() for X in Xs], ks, seed=9) as b:
        done, _ = b.run(30)
        for i, (X, k) in enumerate(zip(Xs, ks)):
            a = b.assignments(i)
            C = b.centroids(i)
            assert a.min() >= 0 and a.max() < k
            # a Lloyd fixed point: every point at its nearest centroid
            assert np.array_equal(a, oracle.assign_f32(X, b.centroids_f32(i)))
            if k == X.shape[0]:
                assert len(set(a.tolist())) == k


def test_batch_rejects_bad_instances():
    good = np.zeros((10, 8), np.float32)
    for X, k in [(np.zeros((10, 12), np.float32), 2), (good, 11), (good, 0), (np.zeros((300, 8), np.float32), 257)]:
        with pytest.raises(knor.KnorError) as e:
            knor.Batch([good, X], [2, k])
        assert e.value.status == knor.KNOR_ERR_ARG
    bad = good.copy()
    bad[3, 3] = np.nan
    with pytest.raises(knor.KnorError):
        knor.Batch([bad], [2])


def test_batch_autotune_describes_its_choice():
    Xs, ks = _instances(6, 71)
    with knor.Batch(Xs, ks, seed=0) as b:
        text = b.describe()
        assert "unit points" in text and "CTAs/SM" in text


def test_batch_workload_full_size_sampled():
    """The 512-instance workload at full size (n_i log-uniform in [1e3, 1e6],
    d in {8, 16, 32, 64}, k in [4, 256]): teacher-forced parity at iterations
    1, 2 and 5 on the eight smallest instances, and on 4000 sampled points of
    the eight largest (FP32 restatement, bit for bit)."""
    specs = synth.batched_specs(512, 1004)
    Xd = [synth.batched_instance(s, device="cuda") for s in specs]
    ks = [s.k for s in specs]
    order = np.argsort([s.n for s in specs])
    small, large = order[:8], order[-8:]
    rng = np.random.default_rng(0)
    samples = {int(i): np.sort(rng.choice(specs[i].n, 4000, replace=False)) for i in large}
    with knor.Batch(Xd, ks, seed=42) as b:
        for t in range(1, 6):
            watch = [int(i) for i in np.concatenate([small, large])]
            before = {i: (b.centroids(i), b.centroids_f32(i)) for i in watch}
            b.iterate()
            if t not in (1, 2, 5):
                continue
            for i in watch:
                C64, C32 = before[i]
                a = b.assignments(i)
                X = Xd[i].cpu().numpy()
                if i in samples:
                    sel = samples[i]
                    assert np.array_equal(a[sel], oracle.assign_f32(X[sel], C32)), f"it {t} instance {i}"
                    check_assignments(X[sel], C64, a[sel], f"batch512 it {t} inst {i}")
                else:
                    assert np.array_equal(a, oracle.assign_f32(X, C32)), f"it {t} instance {i}"
                    C_ref, _ = oracle.means(X, a, C64)
                    check_centroids(b.centroids(i), C_ref, f"batch512 it {t} inst {i}")
