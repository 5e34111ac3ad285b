"""k-means++ seeding (KNOR_INIT_KMEANSPP) against the oracle's: the same
row indices, drawn in the same order, on every input; and a whole run from
that seeding against the oracle's run from the same rows."""
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


def _dups():
    rng = np.random.default_rng(8)
    locs = rng.normal(size=(9, 6)).astype(np.float32) * 5
    return locs[rng.integers(0, 9, 20000)]


DATA = [
    ("iso_d8_k10", lambda: synth.isotropic_mixture(20000, 8, 10, 71).numpy(), 10),
    ("spd_d32_k20", lambda: synth.spd_mixture(30001, 32, 20, 72).numpy(), 20),
    ("uniform_d16_k100", lambda: synth.uniform_cube(9000, 16, 73).numpy(), 100),
    ("aniso_d64_k30", lambda: synth.aniso_mixture(5000, 64, 30, 74).numpy(), 30),
    ("generic_d3_k7", lambda: synth.spd_mixture(7777, 3, 7, 75).numpy(), 7),
    ("generic_d33_k12", lambda: synth.aniso_mixture(4000, 33, 12, 76).numpy(), 12),
    ("nine_locations_k9", _dups, 9),
    ("tiny_k_eq_n", lambda: np.random.default_rng(9).normal(size=(17, 4)).astype(np.float32), 17),
]


@pytest.mark.parametrize("name,make,k", DATA, ids=[d[0] for d in DATA])
@pytest.mark.parametrize("seed", [42, 7])
def test_kmeanspp_indices_equal_the_oracle(name, make, k, seed):
    X = make()
    with knor.Context(torch.as_tensor(X).cuda(), k, init="kmeans++", seed=seed) as c:
        idx = c.init_indices()
        assert np.array_equal(idx, oracle.kmeanspp_indices(X, k, seed))
        assert np.array_equal(c.centroids(), X[idx].astype(np.float64))


def test_run_from_kmeanspp_matches_the_oracle():
    X = synth.spd_mixture(40000, 16, 12, 77).numpy()
    with knor.Context(torch.as_tensor(X).cuda(), 12, init="kmeans++", seed=3) as c:
        C0 = X[c.init_indices()].astype(np.float64)
        ref = oracle.run(X, C0, 40, prune=False)
        ties = 0
        for t in range(40):
            C_before = c.centroids()
            s = c.iterate()
            ties += check_assignments(X, C_before, c.assignments(), f"it {t + 1}")
            C_ref, _ = oracle.means(X, c.assignments(), C_before)
            check_centroids(c.centroids(), C_ref, f"it {t + 1}")
            if s["changed"] == 0:
                break
        if ties == 0:
            assert t + 1 == ref.iters
