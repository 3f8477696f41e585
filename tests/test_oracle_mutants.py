"""The oracle's pins are sharp: each plausible mistake planted in a copy of the
oracle source (built on the CPU, in a temporary directory) fails at least one
of the pin checks that the real oracle passes."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import datagen
import oracle
from golden_io import load
import test_oracle as T

MUTANTS = {
    "split_lt": ("node = (v <= threshold[node]) ? left[node] : right[node];",
                 "node = (v < threshold[node]) ? left[node] : right[node];"),
    "children_swapped": ("node = (v <= threshold[node]) ? left[node] : right[node];",
                         "node = (v <= threshold[node]) ? right[node] : left[node];"),
    "argmax_last_on_tie": ("if (votes[c] > votes[best]) best = c;", "if (votes[c] >= votes[best]) best = c;"),
    "visits_dropped": ("++*visits;", ";"),
    "stat_tie_right": ("return f->card[b + r] > f->card[b + l];", "return f->card[b + r] >= f->card[b + l];"),
    "stat_cold_first": ("return f->card[b + r] > f->card[b + l];", "return f->card[b + r] < f->card[b + l];"),
    "layout_split_lt": ("int right = !(x[nd->feature] <= nd->threshold);", "int right = !(x[nd->feature] < nd->threshold);"),
    "bin_one_level_short": ("for (int32_t level = 0; level <= d && nf > 0; ++level)",
                            "for (int32_t level = 0; level < d && nf > 0; ++level)"),
}


def _build_mutant(tmp_path, name):
    src = open(oracle._SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", str(so),
                    str(path)], check=True)
    return str(so)


def _pin_suite(forest_tiny, rows_tiny):
    """Runs the pin checks; returns the list of the ones that failed."""
    failed = []
    checks = []
    for fx in T.FIXTURES:
        checks.append((f"fixture:{fx}", lambda fx=fx: T.test_oracle_matches_hand_fixture(fx)))
        checks.append((f"fixture_rows:{fx}", lambda fx=fx: T.test_oracle_fixture_one_row_at_a_time(fx)))
        for kind in (oracle.BF, oracle.DF, oracle.DFM, oracle.STAT):
            checks.append((f"layout:{fx}:{kind}", lambda fx=fx, k=kind: T.test_paper_layouts_match_hand_fixture(fx, k)))
        checks.append((f"stat_rules:{fx}", lambda fx=fx: T.test_stat_layout_rules(fx, forest_tiny)))
    checks.append(("leaf_boxes", lambda: T.test_leaf_boxes_tiny_workload(forest_tiny, rows_tiny)))
    checks.append(("invariants", lambda: T.test_votes_and_class_invariants(forest_tiny, rows_tiny)))
    checks.append(("stat_rules:tiny", lambda: T.test_stat_layout_rules("tiny", forest_tiny)))
    for d in (1, 2):
        checks.append((f"bin_levels:{d}", lambda d=d: T.test_bin_interleaved_levels(forest_tiny, d)))
    checks.append(("bin_roots", lambda: T.test_bin_depth0_roots_contiguous(forest_tiny)))
    for name, fn in checks:
        try:
            fn()
        except AssertionError:
            failed.append(name)
    return failed


@pytest.fixture()
def swap_oracle():
    saved = oracle._lib
    yield
    oracle._lib = saved


def _load_as_oracle(so):
    oracle._lib = None
    real_build = oracle.build
    try:
        oracle._LIB_PATH_saved = oracle._LIB_PATH
        oracle._LIB_PATH = so
        oracle.build = lambda force=False: so
        return oracle.lib()
    finally:
        oracle.build = real_build
        oracle._LIB_PATH = oracle._LIB_PATH_saved


def test_real_oracle_passes_pin_suite(tiny_forest, tiny_rows):
    assert _pin_suite(tiny_forest, tiny_rows) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, swap_oracle, tiny_forest, tiny_rows):
    so = _build_mutant(tmp_path, name)
    _load_as_oracle(so)
    failed = _pin_suite(tiny_forest, tiny_rows)
    assert failed, f"mutant {name} passed every pin"
