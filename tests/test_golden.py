"""The stored oracle results (tests/golden/oracle_ipm.json, written by make_oracle_ipm.py from
the oracle alone) still belong to the generator's grids, and record converged oracle solves."""
import json
import os

import pytest

from synth import config_grid
from tests.golden.make_oracle_ipm import CASES, OUT, grid_digest, same_grid


def test_golden_records_match_the_generator():
    d = json.load(open(OUT))
    assert set(d) == set(CASES)
    for name, rec in d.items():
        grid, kkt, gamma = CASES[name]
        assert (rec["grid"], rec["kkt"], rec["gamma"]) == (grid, kkt, gamma)
        assert rec["status"] == "converged" and rec["kkt_error"] <= 1e-6
        assert same_grid(grid_digest(config_grid(grid)), rec["grid_digest"]), name


def test_same_grid_detects_a_changed_input():
    g = config_grid("ring30")
    a = grid_digest(g)
    import dataclasses
    b = grid_digest(dataclasses.replace(g, rate=g.rate * (1 + 1e-6)))
    c = grid_digest(dataclasses.replace(g, rate=g.rate * (1 + 1e-13)))
    assert same_grid(c, a) and not same_grid(b, a)
