"""Pins for the FP64 oracle: checks against what the paper and the mathematics
fix, not against a retyped copy of the oracle's own formulas.

Each test names what pins it: a hand-worked example (tests/golden), a closed
form, a textbook property of Lloyd's algorithm, exhaustive search on tiny
inputs, or a published test vector.  A plausible mistake in the oracle (a
dropped term, a wrong sign or index, ties to the wrong centroid, a pruning
test without the factor 1/2) fails at least one of them; tests/
test_oracle_planted.py compiles such mistakes into throwaway oracle variants
and checks that these pins reject them.
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from conftest import GOLDEN, read_golden
from paper_1606_08905_gb300 import synth


# ---------------------------------------------------------------- init ----

def test_splitmix64_published_vectors():
    """Pin: SplitMix64's published first outputs for seeds 0 and 1234567."""
    g = read_golden("splitmix64.txt")
    for row in g["_rows"]:
        seed = int(row[0])
        want = [int(h, 16) for h in row[1:]]
        got = [int(v) for v in oracle.splitmix64(seed, len(want))]
        assert got == want


def test_floyd_k_equals_n_is_identity():
    """Pin: with k = n Floyd's algorithm must keep j at every step (all
    smaller indices are taken), giving 0..n-1 in order."""
    for n in (1, 2, 7, 64):
        assert list(oracle.forgy_indices(n, n, 9)) == list(range(n))


def test_floyd_distinct_in_range_and_uniform():
    """Pin: Floyd's algorithm draws k-subsets uniformly (Bentley & Floyd).
    Every one of the C(5,2) = 10 subsets should appear about 1/10 of the time."""
    counts = {}
    trials = 20000
    for s in range(trials):
        idx = oracle.forgy_indices(5, 2, s)
        assert len(set(idx.tolist())) == 2 and idx.min() >= 0 and idx.max() < 5
        key = tuple(sorted(idx.tolist()))
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 10
    expect = trials / 10
    chi2 = sum((c - expect) ** 2 / expect for c in counts.values())
    assert chi2 < 27.9  # 9 dof, p = 0.001


def test_floyd_hand_worked_indices():
    """Pin: Forgy indices worked by hand from the published SplitMix64
    outputs (tests/golden/floyd_splitmix64.txt), including a repeated draw
    that must keep j.  This fixes the multiply-shift reduction: a remainder
    reduction passes the identity and uniformity pins but not this one."""
    with open(os.path.join(GOLDEN, "floyd_splitmix64.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.startswith("case ")]
    assert len(rows) == 8
    for row in rows:
        seed, n, k = int(row[1]), int(row[2]), int(row[3])
        bars = [i for i, v in enumerate(row) if v == "|"]
        kept = [int(v) for v in row[bars[1] + 1:]]
        assert list(oracle.forgy_indices(n, k, seed)) == kept, row


def test_forgy_rejects_bad_sizes():
    with pytest.raises(ValueError):
        oracle.forgy_indices(3, 4, 1)
    with pytest.raises(ValueError):
        oracle.forgy_indices(3, 0, 1)


# ------------------------------------------------------- hand examples ----

def _frac_list(num, den):
    return [Fraction(int(a), int(b)) for a, b in zip(num, den)]


@pytest.mark.parametrize("prune", [False, True])
def test_hand_worked_1d(prune):
    """Pin: hand-computed trajectory in tests/golden/lloyd_1d_hand.txt."""
    g = read_golden("lloyd_1d_hand.txt")
    X = np.array([[float(v)] for v in g["points"]], np.float32)
    C0 = np.array([[float(v)] for v in g["init"]], np.float64)
    r = oracle.run(X, C0, 20, prune=prune, history=True)
    assert r.iters == int(g["iters"][0])
    assert list(r.changed) == [int(v) for v in g["changed"]]
    for t in range(r.iters):
        assert list(r.a_hist[t]) == [int(v) for v in g[f"assign{t + 1}"]]
    want = _frac_list(g["final_num"], g["final_den"])
    assert np.allclose(r.C[:, 0], [float(w) for w in want], rtol=0, atol=1e-14)
    obj = Fraction(int(g["objective_num"][0]), int(g["objective_den"][0]))
    assert abs(oracle.objective(X, r.C, r.a) - float(obj)) < 1e-12


@pytest.mark.parametrize("prune", [False, True])
def test_hand_worked_2d(prune):
    """Pin: hand-computed step in tests/golden/lloyd_2d_hand.txt."""
    g = read_golden("lloyd_2d_hand.txt")
    X = np.array([float(v) for v in g["points"]], np.float32).reshape(-1, 2)
    C0 = np.array([float(v) for v in g["init"]], np.float64).reshape(-1, 2)
    r = oracle.run(X, C0, 20, prune=prune, history=True)
    assert list(r.a_hist[0]) == [int(v) for v in g["assign1"]]
    want = np.array([float(f) for f in _frac_list(g["c_num"], g["c_den"])]).reshape(-1, 2)
    assert np.allclose(r.C_hist[1], want, rtol=0, atol=1e-14)
    assert list(r.changed) == [int(v) for v in g["changed"]]


# ---------------------------------------------------------- closed forms ----

@pytest.mark.parametrize("prune", [False, True])
def test_k1_global_mean_in_one_iteration(prune):
    """Pin (closed form): with k = 1 every point joins the only cluster, so
    after one iteration the centroid is the global mean and the second
    iteration changes nothing."""
    rng = np.random.default_rng(3)
    X = (rng.standard_normal((1000, 5)) * 3 + 7).astype(np.float32)
    r = oracle.run(X, X[:1].astype(np.float64), 10, prune=prune, history=True)
    exact = np.array([float(sum(Fraction(float(v)) for v in X[:, j]) / X.shape[0])
                      for j in range(X.shape[1])])
    assert r.iters == 2 and list(r.changed) == [1000, 0]
    assert np.allclose(r.C[0], exact, rtol=1e-15, atol=1e-13)


@pytest.mark.parametrize("prune", [False, True])
def test_k_equals_n_objective_zero(prune):
    """Pin (closed form): with k = n distinct points and C0 = the points, every
    point is its own centroid: objective 0, assignment i -> i."""
    rng = np.random.default_rng(4)
    X = rng.standard_normal((40, 3)).astype(np.float32)
    r = oracle.run(X, X.astype(np.float64), 10, prune=prune)
    assert list(r.a) == list(range(40))
    assert oracle.objective(X, r.C, r.a) == 0.0
    assert r.iters == 2


@pytest.mark.parametrize("prune", [False, True])
def test_two_far_clusters_exact_means(prune):
    """Pin (closed form): two groups 1e3 apart, one init point in each; after
    one step each centroid is its group's exact mean and nothing changes after."""
    rng = np.random.default_rng(5)
    A = rng.uniform(-1, 1, (300, 4)).astype(np.float32)
    B = (rng.uniform(-1, 1, (200, 4)) + 1000).astype(np.float32)
    X = np.concatenate([A, B])
    C0 = np.stack([X[7], X[400]]).astype(np.float64)
    r = oracle.run(X, C0, 10, prune=prune)
    mA = [float(sum(Fraction(float(v)) for v in A[:, j]) / 300) for j in range(4)]
    mB = [float(sum(Fraction(float(v)) for v in B[:, j]) / 200) for j in range(4)]
    assert np.allclose(r.C[0], mA, rtol=1e-15, atol=1e-13)
    assert np.allclose(r.C[1], mB, rtol=1e-15, atol=1e-12)
    assert list(r.a) == [0] * 300 + [1] * 200 and r.iters == 2


@pytest.mark.parametrize("prune", [False, True])
def test_one_dimension_fixed_point_is_midpoint_partition(prune):
    """Pin (textbook, d = 1): at a Lloyd fixed point on the line the clusters
    are contiguous intervals of the sorted data, split at the midpoints of
    consecutive centroids, and each centroid is its interval's mean."""
    rng = np.random.default_rng(6)
    X = np.sort(rng.uniform(0, 100, 500)).astype(np.float32)[:, None]
    C0 = X[[3, 100, 250, 400, 480]].astype(np.float64)
    r = oracle.run(X, C0, 200, prune=prune)
    assert r.changed[-1] == 0
    order = np.argsort(r.C[:, 0])
    cs = r.C[order, 0]
    mids = (cs[:-1] + cs[1:]) / 2
    x = X[:, 0].astype(np.float64)
    rank = np.searchsorted(mids, x)  # interval index of each point
    assert np.array_equal(order[rank], r.a)
    for j in range(len(cs)):
        members = x[rank == j]
        if members.size:
            assert abs(cs[j] - float(sum(Fraction(float(v)) for v in members) / members.size)) < 1e-12


def test_ties_go_to_lowest_index():
    """Pin (Algorithm 1 replaces the best only on a strict '<'): a point
    exactly between two centroids joins the lower-indexed one, whichever side
    that is; duplicated centroids always attract to the first copy."""
    X = np.array([[0.5], [0.5]], np.float32)
    a, _, _, _ = oracle.assign(X, np.array([[0.0], [1.0]]))
    assert list(a) == [0, 0]
    a, _, _, _ = oracle.assign(X, np.array([[1.0], [0.0]]))
    assert list(a) == [0, 0]
    Xd = np.array([[2.0, 2.0], [3.0, 1.0]], np.float32)
    a, _, _, _ = oracle.assign(Xd, np.array([[9.0, 9.0], [2.0, 2.0], [2.0, 2.0]]))
    assert list(a) == [1, 1]
    a32 = oracle.assign_f32(Xd, np.array([[9.0, 9.0], [2.0, 2.0], [2.0, 2.0]], np.float32))
    assert list(a32) == [1, 1]


@pytest.mark.parametrize("prune", [False, True])
def test_duplicate_points_and_ties_mti_matches(prune):
    """Pin: duplicated points and an exact tie survive pruning unchanged."""
    X = np.array([[0.5], [0.5], [0.5], [0.0], [1.0], [1.0]], np.float32)
    r = oracle.run(X, np.array([[0.0], [1.0]]), 10, prune=prune, history=True)
    assert list(r.a_hist[0]) == [0, 0, 0, 0, 1, 1]


@pytest.mark.parametrize("prune", [False, True])
def test_empty_cluster_keeps_centroid(prune):
    """Pin (reading R7): a centroid no point is nearest to keeps its place."""
    rng = np.random.default_rng(8)
    X = rng.uniform(0, 1, (100, 2)).astype(np.float32)
    C0 = np.array([[0.2, 0.2], [0.8, 0.8], [500.0, 500.0]])
    r = oracle.run(X, C0, 10, prune=prune, history=True)
    for t in range(r.iters + 1):
        assert np.array_equal(r.C_hist[t][2], [500.0, 500.0])


# ------------------------------------------------- textbook properties ----

def _datasets():
    out = []
    X = synth.isotropic_mixture(3000, 8, 10, 11).numpy()
    out.append(("iso", X, 10))
    X = synth.spd_mixture(3000, 16, 7, 12).numpy()
    out.append(("spd", X, 7))
    X = synth.uniform_cube(2500, 3, 13).numpy()
    out.append(("uniform", X, 12))
    rng = np.random.default_rng(14)
    base = rng.integers(-3, 4, (40, 2)).astype(np.float32)
    X = base[rng.integers(0, 40, 2000)]  # many exact duplicates, small grid
    out.append(("dups", X, 9))
    X = synth.aniso_mixture(2000, 33, 25, 15).numpy()
    out.append(("aniso_d33", X, 25))
    return out


@pytest.mark.parametrize("name,X,k", _datasets(), ids=lambda v: v if isinstance(v, str) else "")
def test_objective_never_increases(name, X, k):
    """Pin (textbook): each Phase I and Phase II step cannot raise the sum of
    squared distances when empty clusters keep their centroid."""
    C0 = oracle.forgy_centroids(X, k, 42)
    r = oracle.run(X, C0, 60, prune=False, history=True)
    objs = [oracle.objective(X, r.C_hist[t + 1], r.a_hist[t]) for t in range(r.iters)]
    prev = np.inf
    for t in range(r.iters):
        # objective with the step's assignment and the centroids before Phase II
        before = oracle.objective(X, r.C_hist[t], r.a_hist[t])
        assert before <= prev * (1 + 1e-12) + 1e-9
        assert objs[t] <= before * (1 + 1e-12) + 1e-9
        prev = objs[t]


@pytest.mark.parametrize("name,X,k", _datasets(), ids=lambda v: v if isinstance(v, str) else "")
def test_pruned_equals_unpruned_every_iteration(name, X, k):
    """Pin: MTI reaches exactly the unpruned result (identical assignments and
    bit-identical centroids at every iteration), and it does skip work."""
    C0 = oracle.forgy_centroids(X, k, 42)
    p = oracle.run(X, C0, 60, prune=True, history=True)
    u = oracle.run(X, C0, 60, prune=False, history=True)
    assert p.iters == u.iters
    assert np.array_equal(p.a_hist, u.a_hist)
    assert np.array_equal(p.C_hist, u.C_hist)
    assert np.array_equal(p.changed, u.changed)
    if p.iters > 3 and name != "uniform":
        assert p.skipped[1:].sum() > 0
        assert p.evals.sum() < u.evals.sum()


def test_mti_invariants_hold():
    """Pin (triangle inequality): after every MTI iteration u bounds the true
    distance to the assigned centroid, and s(c) <= 1/2 d(c, c') for all c'."""
    X = synth.spd_mixture(2000, 8, 6, 21).numpy()
    C = oracle.forgy_centroids(X, 6, 42)
    a = np.full(X.shape[0], -1, np.int32)
    u = np.full(X.shape[0], np.inf)
    Cprev = None
    Xd = X.astype(np.float64)
    for _ in range(15):
        halfD, s, f = oracle.mti_tables(C, Cprev)
        dcc = np.sqrt(((C[:, None, :] - C[None, :, :]) ** 2).sum(-1))
        off = ~np.eye(len(C), dtype=bool)
        assert np.all(halfD[off] <= dcc[off] / 2)
        assert np.all(s <= np.where(off, dcc / 2, np.inf).min(1))
        if Cprev is not None:
            assert np.all(f >= np.sqrt(((C - Cprev) ** 2).sum(-1)))
        oracle.mti_iter(X, C, halfD, s, f, a, u)
        true = np.sqrt(((Xd - C[a]) ** 2).sum(-1))
        assert np.all(u >= true)
        Cn, _ = oracle.means(X, a, C)
        Cprev, C = C, Cn


def test_label_recovery_well_separated():
    """Pin: on a mixture whose components are >= 10 sigma apart, started from
    one point of each component, Lloyd recovers the generating labels exactly
    (adjusted Rand index 1: the contingency table is a permutation) and each
    centroid lies within 3 sigma / sqrt(n_c) of its component's true mean."""
    k, d, sigma = 8, 6, 1.0
    rng = np.random.default_rng(22)
    means = rng.uniform(-200, 200, (k, d))
    while True:
        dm = np.sqrt(((means[:, None] - means[None]) ** 2).sum(-1)) + np.eye(k) * 1e9
        if dm.min() > 30 * sigma:
            break
        means = rng.uniform(-200, 200, (k, d))
    lab = rng.integers(0, k, 20000)
    X = (means[lab] + sigma * rng.standard_normal((20000, d))).astype(np.float32)
    first = [int(np.flatnonzero(lab == j)[0]) for j in range(k)]
    for prune in (False, True):
        r = oracle.run(X, X[first].astype(np.float64), 50, prune=prune)
        table = np.zeros((k, k), int)
        np.add.at(table, (lab, r.a), 1)
        assert np.all((table > 0).sum(0) == 1) and np.all((table > 0).sum(1) == 1)
        for j in range(k):
            c = r.a[first[j]]
            nc = (lab == j).sum()
            assert np.all(np.abs(r.C[c] - means[j]) < 3 * sigma * np.sqrt(d) / np.sqrt(nc) + 1e-9)


# ------------------------------------------------------- brute force ----

def _partitions_objective(X, k):
    """Global optimum of the k-means objective by enumerating all k^n labelings."""
    n = X.shape[0]
    best = np.inf
    Xd = X.astype(np.float64)
    for lab in itertools.product(range(k), repeat=n):
        lab = np.array(lab)
        obj = 0.0
        for j in range(k):
            m = Xd[lab == j]
            if m.size:
                obj += ((m - m.mean(0)) ** 2).sum()
        best = min(best, obj)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_tiny(seed):
    """Pin (exhaustive search, n <= 8, k <= 3, d <= 2): from every Forgy
    start Lloyd ends at a fixed point -- each point at a nearest centroid, each
    non-empty centroid at its members' mean -- with objective >= the global
    optimum over all k^n partitions, and the best start reaches it."""
    rng = np.random.default_rng(100 + seed)
    n, k, d = 7 + seed % 2, 2 + seed % 2, 1 + seed % 2
    X = rng.integers(-6, 7, (n, d)).astype(np.float32) + rng.uniform(0, 0.01, (n, d)).astype(np.float32)
    opt = _partitions_objective(X, k)
    best_seen = np.inf
    Xd = X.astype(np.float64)
    for combo in itertools.combinations(range(n), k):
        for prune in (False, True):
            r = oracle.run(X, Xd[list(combo)], 100, prune=prune)
            assert r.changed[-1] == 0
            dist = ((Xd[:, None, :] - r.C[None]) ** 2).sum(-1)
            assert np.all(dist[np.arange(n), r.a] <= dist.min(1) + 1e-12)
            for j in range(k):
                m = Xd[r.a == j]
                if m.size:
                    assert np.allclose(r.C[j], m.mean(0), atol=1e-12)
            obj = oracle.objective(X, r.C, r.a)
            assert obj >= opt - 1e-9
            best_seen = min(best_seen, obj)
    assert best_seen <= opt + 1e-9


def test_assign_matches_exhaustive_small_integers():
    """Pin: on small integer coordinates every squared distance is exact in
    both FP64 and FP32, so both argmins equal the exhaustive minimum with
    lowest-index ties."""
    rng = np.random.default_rng(31)
    X = rng.integers(-20, 21, (500, 4)).astype(np.float32)
    C = rng.integers(-20, 21, (9, 4)).astype(np.float64)
    C[5] = C[2]  # a duplicated centroid: index 2 must win
    a, d1, d2, _ = oracle.assign(X, C)
    a32 = oracle.assign_f32(X, C.astype(np.float32))
    for i in range(500):
        dd = [int(((X[i].astype(np.int64) - C[c].astype(np.int64)) ** 2).sum()) for c in range(9)]
        m = min(dd)
        assert a[i] == dd.index(m) and a32[i] == a[i]
        assert d1[i] == m and d2[i] == sorted(dd)[1]


def test_means_hand_values():
    """Pin: Phase II on a labelled example computed by hand."""
    X = np.array([[0, 0], [2, 0], [0, 2], [10, 10], [12, 10]], np.float32)
    C, cnt = oracle.means(X, np.array([0, 0, 0, 1, 1], np.int32), np.zeros((3, 2)))
    assert np.allclose(C, [[2 / 3, 2 / 3], [11, 10], [0, 0]], atol=1e-15)
    assert list(cnt) == [3, 2, 0]




# ---------------------------------------------------------------- Elkan ----

@pytest.mark.parametrize("name,seed,n,d,k", [("spd", 31, 3000, 8, 7), ("aniso", 32, 2500, 16, 12),
                                              ("uniform", 33, 2000, 4, 9)])
def test_elkan_equals_unpruned_and_prunes_more_than_mti(name, seed, n, d, k):
    """Pin: Elkan's algorithm (MTI's tests plus per-centroid lower bounds)
    reaches exactly the unpruned result at every iteration.  Also checked
    (a property of these inputs, not a theorem: Elkan's upper bound is only
    tightened when a centroid survives the tests, so its Clause 1 can skip
    fewer points than MTI's): it computes no more distances than MTI in any
    iteration, and fewer over the run."""
    X = synth.make({"spd": "spd", "aniso": "aniso", "uniform": "uniform"}[name], n, d, k, seed).numpy()
    C0 = oracle.forgy_centroids(X, k, 42)
    e = oracle.run(X, C0, 60, prune="elkan", history=True)
    m = oracle.run(X, C0, 60, prune=True, history=True)
    u = oracle.run(X, C0, 60, prune=False, history=True)
    assert e.iters == u.iters == m.iters
    assert np.array_equal(e.a_hist, u.a_hist)
    assert np.array_equal(e.C_hist, u.C_hist)
    assert np.all(e.evals <= m.evals)
    assert e.evals[1:].sum() < m.evals[1:].sum()


def test_elkan_bounds_hold_every_iteration():
    """Pin (triangle inequality): before each Elkan iteration uses them, every
    lower bound l(x, c) is at most the exact d(x, c) and every upper bound is
    at least the exact distance to the assigned centroid (the oracle checks
    them against FP64 distances over all dimensions)."""
    for seed, (n, d, k) in ((41, (3000, 8, 10)), (42, (1500, 32, 6))):
        X = synth.spd_mixture(n, d, k, seed).numpy()
        r = oracle.run(X, oracle.forgy_centroids(X, k, 42), 40, prune="elkan", check_bounds=True)
        assert r.iters > 3
        assert np.all(r.violations == 0), r.violations


# ------------------------------------------------------------ k-means++ ----

def test_kmeanspp_hand_worked_indices():
    """Pin: k-means++ indices on the points 0, 1, 3 worked by hand from the
    published SplitMix64 outputs (tests/golden/kmeanspp_hand.txt)."""
    X = np.array([[0.0], [1.0], [3.0]], np.float32)
    with open(os.path.join(GOLDEN, "kmeanspp_hand.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.startswith("case ")]
    assert len(rows) == 2
    for row in rows:
        seed = int(row[1])
        bars = [i for i, v in enumerate(row) if v == "|"]
        k2 = [int(v) for v in row[bars[0] + 1:bars[1]]]
        k3 = [int(v) for v in row[bars[1] + 1:]]
        assert list(oracle.kmeanspp_indices(X, 2, seed)) == k2
        assert list(oracle.kmeanspp_indices(X, 3, seed)) == k3


def test_kmeanspp_draws_in_proportion_to_squared_distance():
    """Pin (the definition): on the points 0, 1, 3 the first index is uniform
    and the second, given the first, is drawn with probability D^2 / sum D^2
    (the weights here are exact on the quantisation grid: squares of small
    integers).  Chi-square over 30000 seeds, 3 + 3 x 1 degrees of freedom."""
    X = np.array([[0.0], [1.0], [3.0]], np.float32)
    xs = np.array([0.0, 1.0, 3.0])
    trials = 30000
    first = np.zeros(3)
    pair = np.zeros((3, 3))
    for s in range(trials):
        i, j = oracle.kmeanspp_indices(X, 2, s + 1000)
        first[i] += 1
        pair[i, j] += 1
    chi2 = (((first - trials / 3) ** 2) / (trials / 3)).sum()
    for i in range(3):
        d2 = (xs - xs[i]) ** 2
        p = d2 / d2.sum()
        m = p > 0
        assert pair[i, ~m].sum() == 0  # the chosen point itself has weight 0
        exp = first[i] * p[m]
        chi2 += (((pair[i, m] - exp) ** 2) / exp).sum()
    assert chi2 < 24.3  # 5 dof, p = 0.0002


def test_kmeanspp_covers_every_distinct_location():
    """Pin: with exactly k distinct locations (each repeated many times) the
    seeding picks one point at each, because points on chosen centroids weigh
    nothing; with k = n distinct points it picks every point once."""
    rng = np.random.default_rng(3)
    locs = rng.normal(size=(7, 5)).astype(np.float32) * 10
    X = locs[rng.integers(0, 7, 3000)]
    for seed in range(5):
        idx = oracle.kmeanspp_indices(X, 7, seed)
        assert len({tuple(X[i]) for i in idx}) == 7
    Y = rng.normal(size=(40, 3)).astype(np.float32)
    assert sorted(oracle.kmeanspp_indices(Y, 40, 11).tolist()) == list(range(40))
