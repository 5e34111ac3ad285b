"""Elkan's algorithm (knor_opts.elkan: MTI plus per-centroid lower bounds, the
ablation the paper leaves out) against the FP64 oracle's Elkan mode and
against the library's own MTI and plain paths."""
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


DATA = [
    ("iso_d8_k10", lambda: synth.isotropic_mixture(8000, 8, 10, 51).numpy(), 10),
    ("spd_d32_k20", lambda: synth.spd_mixture(12000, 32, 20, 52).numpy(), 20),
    ("spd_d16_k37", lambda: synth.spd_mixture(9001, 16, 37, 53).numpy(), 37),
    ("aniso_d64_k12", lambda: synth.aniso_mixture(5000, 64, 12, 54).numpy(), 12),
    ("uniform_d16_k100", lambda: synth.uniform_cube(6000, 16, 55).numpy(), 100),
]


@pytest.mark.parametrize("name,make,k", DATA, ids=[d[0] for d in DATA])
def test_elkan_matches_oracle_mti_and_plain_every_iteration(name, make, k):
    X = make()
    Xd = torch.as_tensor(X).cuda()
    with knor.Context(Xd, k, seed=42, elkan=True) as e, knor.Context(Xd, k, seed=42) as m, \
            knor.Context(Xd, k, seed=42, prune=False) as q:
        assert "elkan" in e.kernel_name("mti")
        for t in range(40):
            C_before, C32 = e.centroids(), e.centroids_f32()
            se, sm, sq = e.iterate(), m.iterate(), q.iterate()
            a = e.assignments()
            check_assignments(X, C_before, a, f"{name} it {t + 1}")
            assert np.array_equal(a, oracle.assign_f32(X, C32)), f"{name} it {t + 1}: FP32 argmin"
            assert np.array_equal(a, m.assignments()) and np.array_equal(a, q.assignments())
            assert se["changed"] == sm["changed"] == sq["changed"]
            C_ref, _ = oracle.means(X, a, C_before)
            check_centroids(e.centroids(), C_ref, f"{name} it {t + 1}")
            if t > 0:
                assert se["dist_evals"] <= sq["dist_evals"]
            if se["changed"] == 0:
                break


@pytest.mark.parametrize("name,make,k", DATA[:3], ids=[d[0] for d in DATA[:3]])
def test_elkan_counters_match_oracle(name, make, k):
    """Per-iteration changed counts equal the oracle's Elkan mode; Clause-1
    skips and distance evaluations agree up to the points in the rounding
    band between the FP32 and FP64 bounds (0.2 % of n, plus 10)."""
    X = make()
    n = X.shape[0]
    with knor.Context(torch.as_tensor(X).cuda(), k, seed=42, elkan=True) as c:
        done, recs = c.run(40)
        C0 = X[c.init_indices()].astype(np.float64)
    ref = oracle.run(X, C0, 40, prune="elkan", check_bounds=True)
    assert np.all(ref.violations == 0)
    slack = 0.002 * n + 10
    for t in range(min(done, ref.iters)):
        if recs[t]["changed"] != ref.changed[t]:
            break
        assert abs(recs[t]["clause1_skipped"] - ref.skipped[t]) <= slack, (t, recs[t], ref.skipped[t])
        assert abs(recs[t]["dist_evals"] - ref.evals[t]) <= slack + 0.002 * ref.evals[t], (t, recs[t], ref.evals[t])


def test_elkan_bounds_hold_on_the_device():
    """debug_invariants: after every iteration each upper bound is at least the
    distance to the assigned centroid and each lower bound at most the
    distance to its centroid (checked with the FP32 distance's error bound)."""
    X = torch.as_tensor(synth.spd_mixture(30000, 16, 24, 56)).cuda()
    with knor.Context(X, 24, seed=3, elkan=True, debug_invariants=True) as c:
        done, recs = c.run(40)
    assert done > 3
    assert all(r["violations"] == 0 for r in recs)


def test_elkan_checkpoint_resume_is_bit_identical():
    X = torch.as_tensor(synth.spd_mixture(20000, 32, 14, 57)).cuda()
    with knor.Context(X, 14, seed=9, elkan=True) as a:
        a.run(4)
        blob = a.get_state()
        _, tail_a = a.run(6)
        Ca, aa = a.centroids(), a.assignments()
    with knor.Context(X, 14, seed=1, elkan=True) as b:
        b.set_state(blob)
        _, tail_b = b.run(6)
        assert tail_a == tail_b
        assert np.array_equal(b.centroids(), Ca) and np.array_equal(b.assignments(), aa)
    with knor.Context(X, 14, seed=9) as m:  # an MTI context refuses an Elkan state
        with pytest.raises(knor.KnorError):
            m.set_state(blob)


@pytest.mark.parametrize("d,k,kw", [(33, 5, {}), (16, 200, {}), (16, 5, {"prune": False}),
                                    (16, 5, {"full_recompute_every": 3})])
def test_elkan_rejects_unsupported_configurations(d, k, kw):
    X = torch.zeros((1000, d), device="cuda")
    X[:, 0] = torch.arange(1000, device="cuda", dtype=torch.float32)
    with pytest.raises(knor.KnorError) as e:
        knor.Context(X, k, elkan=True, **kw)
    assert e.value.status == knor.KNOR_ERR_ARG
