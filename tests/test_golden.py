"""Values the paper prints (tests/golden/, each file names its table), checked
against the oracle's grids."""
import json
import math
import os

import inputs
import oracle.boundary as Bd
import oracle.cmg_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def test_square_grids_match_table2_sizes_and_levels():
    """N_h = n^2 interior nodes; N_L grids down to n = 7 (h = 1/8)."""
    g = load("paper_grid_sizes.json")
    field = O.sine_mode_field(inputs.draw_xi(1, 2, 2), 0.5)
    for Nh, NL in g["local_control_Nh_NL"]:
        n = math.isqrt(Nh)
        assert n * n == Nh
        levels = O.make_hierarchy(n, 2, 1e-4, field, coarsest_n=7)
        assert len(levels) == NL and levels[-1].n == 7


def test_boundary_grids_match_table3_sizes_and_levels():
    """N_h = (n+1) n: the controlled edge's row counts; the same N_L."""
    g = load("paper_grid_sizes.json")
    field = O.sine_mode_field(inputs.draw_xi(1, 2, 2), 0.5)
    for Nh, NL in g["boundary_control_Nh_NL"]:
        n = next(k for k in (7, 15, 31, 63, 127) if (k + 1) * k == Nh)
        assert Bd.mass(n).size == Nh
        ns, _ = Bd.hierarchy(n, 2, 1e-4, field, coarsest_n=7)
        assert len(ns) == NL
