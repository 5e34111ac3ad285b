"""The oracle's pins catch planted mistakes.

Each case compiles a throwaway variant of the oracle with one mistake
switched on (the ORACLE_PLANT_* switches in knor_oracle.c; a normal build
defines none), runs the pins that guard that step against it in a child
process, and requires them to fail.  Mistakes are planted on the CPU only.
"""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    # (switch, pins that must fail)
    ("ORACLE_PLANT_NO_HALF", "test_pruned_equals_unpruned_every_iteration or test_mti_invariants"),
    ("ORACLE_PLANT_TIE_HIGH", "test_ties_go_to_lowest_index or test_assign_matches_exhaustive"),
    ("ORACLE_PLANT_DROP_LAST_DIM", "test_hand_worked_2d or test_assign_matches_exhaustive"),
    ("ORACLE_PLANT_EMPTY_ZERO", "test_empty_cluster_keeps_centroid"),
    ("ORACLE_PLANT_NO_DRIFT", "test_pruned_equals_unpruned_every_iteration or test_mti_invariants"),
    ("ORACLE_PLANT_ELKAN_NO_LB_DRIFT", "test_elkan"),
    ("ORACLE_PLANT_KPP_LINEAR", "test_kmeanspp"),
]


@pytest.mark.parametrize("switch,pins", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_a_pin(tmp_path, switch, pins):
    lib = oracle.build(out=str(tmp_path / f"lib_{switch}.so"), defines=[switch])
    env = dict(os.environ, KNOR_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-k", pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"{switch} was not caught:\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout
