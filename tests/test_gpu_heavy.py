"""GPU: the Clause-1 selection's heavy split and its warp count, pushed to
their extremes.

k_mti_sel sends a point whose bound reaches the M-th smallest 1/2 d(c_a, c)
of its cluster to the mixed bucket, where the scan scores it against every
centroid; KNOR_SEL_M sets M (0: no split).  The split changes which batch a
point is scored in, never the result: with M = 2 (nearly every surviving
point is heavy), the default, and no split, every iteration must match the
oracle (teacher forcing and the bit-exact FP32 argmin), the three runs must
give identical assignments, and the pruning counters (the evaluations the
clauses leave, whatever the scan computed) must agree with the oracle's.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1606_08905_gb300 import build as kbuild
from paper_1606_08905_gb300 import knor, synth
from test_gpu_parity import step_and_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    knor.load()


def _run(X, k, sel_m, iters, sel_mult=None):
    env = {"KNOR_SEL_M": sel_m, "KNOR_SEL_MULT": sel_mult}
    old = {name: os.environ.get(name) for name in env}
    for name, v in env.items():
        if v is None:
            os.environ.pop(name, None)
        else:
            os.environ[name] = str(v)
    try:
        with knor.Context(torch.as_tensor(X).cuda().contiguous(), k, seed=42, prune=True) as ctx:
            assert ctx.kernel_name("select") == "k_mti_sel"
            stats, ties = step_and_check(X, ctx, iters, f"KNOR_SEL_M={sel_m} KNOR_SEL_MULT={sel_mult}")
            return ctx.assignments(), stats, ties
    finally:
        for name, v in old.items():
            if v is None:
                os.environ.pop(name, None)
            else:
                os.environ[name] = v


@pytest.mark.parametrize("name,make,k", [
    ("spd_d16_k100", lambda: synth.spd_mixture(12000, 16, 100, 31, mean_lo=0.0, mean_hi=10.0).numpy(), 100),
    ("spd_d32_k20", lambda: synth.spd_mixture(12000, 32, 20, 32).numpy(), 20),
    ("iso_d8_k12", lambda: synth.isotropic_mixture(9000, 8, 12, 33).numpy(), 12),
], ids=["spd_d16_k100", "spd_d32_k20", "iso_d8_k12"])
def test_heavy_split_never_changes_the_result(name, make, k):
    X = make()
    runs = {m: _run(X, k, m, 12) for m in (2, None, 0)}
    a_ref, st_ref, _ = runs[0]
    for m, (a, st, _) in runs.items():
        assert np.array_equal(a, a_ref), f"KNOR_SEL_M={m}: assignments differ from the unsplit run"
        assert [s["changed"] for s in st] == [s["changed"] for s in st_ref], m
        # the counters count the clauses, not the work: identical in all three
        assert [s["dist_evals"] for s in st] == [s["dist_evals"] for s in st_ref], m
        assert [s["clause1_skipped"] for s in st] == [s["clause1_skipped"] for s in st_ref], m
    # and against the oracle's MTI counters, run from the same C^0
    C0 = X[oracle.forgy_indices(X.shape[0], k, 42)].astype(np.float64)
    ref = oracle.run(X, C0, 12, prune=True)
    slack = 0.002 * X.shape[0] + 10
    for t in range(min(len(st_ref), ref.iters)):
        if st_ref[t]["changed"] != ref.changed[t]:
            break
        assert abs(st_ref[t]["dist_evals"] - ref.evals[t]) <= slack + 0.002 * ref.evals[t], (t, st_ref[t], ref.evals[t])


def test_one_or_two_selection_warps_per_scan_warp_agree():
    """k_mti_sel runs two warps per scan warp where they fit (each over half
    the range, with a record list of its own, the scan taking both lists in
    order); KNOR_SEL_MULT=1 keeps one.  Only the order of the batches differs:
    assignments and counters are identical, and both match the oracle."""
    X = synth.spd_mixture(20000, 32, 20, 34).numpy()
    a1, st1, _ = _run(X, 20, None, 12, sel_mult=1)
    a2, st2, _ = _run(X, 20, None, 12, sel_mult=2)
    assert np.array_equal(a1, a2)
    for key in ("changed", "clause1_skipped", "dist_evals"):
        assert [s[key] for s in st1] == [s[key] for s in st2], key
