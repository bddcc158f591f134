"""Pins of the quadtree oracle, the list counts and the parameter rules."""
import math

import numpy as np
import pytest

from conftest import golden_lines
from oracle.fmm import make_tiling
from oracle.params import KAPPA, auto_levels, p_from_eps
from oracle.tiling_quad import Quadtree


def test_morton_containment_and_prefix():
    rng = np.random.default_rng(2)
    xy = rng.random((3000, 2))
    T = Quadtree(5)
    k = T.keys(xy[:, 0], xy[:, 1])
    for i in range(0, 3000, 29):
        assert T.contains(int(k[i]), 5, xy[i, 0], xy[i, 1])
    for l in range(6):
        assert np.array_equal(T.keys(xy[:, 0], xy[:, 1], l), k >> (2 * (5 - l)))
    # Z order: digit = xbit + 2 ybit
    assert T.keys(np.array([0.75]), np.array([0.25]), 1)[0] == 1
    assert T.keys(np.array([0.25]), np.array([0.75]), 1)[0] == 2


def _m2l_count_closed_form(l):
    # Per axis, a target coordinate i has A(i) source coordinates whose parent
    # is within one of i's parent and B(i) coordinates within one of i, so
    # the level-l list count is (sum A)^2 - (sum B)^2 with sum A = 6n - 8 and
    # sum B = 3n - 2 for n = 2^l cells per side (n >= 4).
    n = 2 ** l
    return (6 * n - 8) ** 2 - (3 * n - 2) ** 2


def test_quad_full_tree_list_counts():
    T = Quadtree(5)
    for l in (2, 3, 4, 5):
        tot = sum(len(T.far(c, l)) for c in range(4 ** l))
        assert tot == _m2l_count_closed_form(l)
        # Table 2: interior cells have P2 = 9, P4 = 27
        assert max(len(T.near(c, l)) for c in range(4 ** l)) == 9
        if l >= 3:
            assert max(len(T.far(c, l)) for c in range(4 ** l)) == 27


def test_quad_separation_ratios():
    T = Quadtree(4)
    h = 2.0 ** -4
    n = T.index(7, 7, 4)
    r = h * math.sqrt(2) / 2
    R = 1.5 * h          # inradius of the 3x3 block (tile and 8 neighbours)
    assert r / R == pytest.approx(math.sqrt(2) / 3)
    dmin = min(abs(T.center(m, 4) - T.center(n, 4)) for m in T.far(n, 4))
    assert (dmin - 2 * r) / r == pytest.approx(2 * (math.sqrt(2) - 1), abs=1e-12)


def test_table2_counts_and_cost_constants():
    """Interior P2/P4 from the oracle's own lists reproduce Table 2 and, through
    the optimised-cost expressions of App. A-C, its leading constants."""
    rows = {f[0]: f for f in (l.split() for l in golden_lines("table2.txt"))}
    measured = {}
    for name, L, l, n in (("quad", 4, 4, Quadtree.index(7, 7, 4)),
                          ("sept", 4, 4, None), ("tri", 4, 4, None)):
        T = make_tiling(name, L)
        if n is None:
            for c in range(T.b ** l):
                full = len(T.neighbors(c, l)) == {"sept": 6, "tri": 12}[name] and \
                    len(T.neighbors(c // T.b, l - 1)) == {"sept": 6, "tri": 12}[name]
                if full:
                    n = c
                    break
        measured[name] = (len(T.far(n, l)), len(T.near(n, l)))
    for name, (P4, P2) in measured.items():
        assert P4 == int(rows[name][1]) and P2 == int(rows[name][2])
        bb = 4 if name != "sept" else 7
        c = (math.sqrt(bb / (bb - 1)) + math.sqrt((bb - 1) / bb)) * math.sqrt((P4 + 2) * P2)
        assert c == pytest.approx(float(rows[name][5]), abs=0.01)


def test_p_from_eps():
    # kappa^(p+1) <= eps < kappa^p
    for t in ("quad", "sept", "tri"):
        for eps in (1e-4, 1e-6, 1e-8, 1e-10):
            p = p_from_eps(t, eps)
            assert KAPPA[t] ** (p + 1) <= eps < KAPPA[t] ** p
    assert p_from_eps("quad", 1e-6) == 22
    assert p_from_eps("sept", 1e-6) == 21
    assert p_from_eps("tri", 1e-6) == 27


def test_auto_levels():
    assert auto_levels("quad", 8192) == 4
    assert auto_levels("quad", 2 ** 20) == 7
    assert auto_levels("tri", 2 ** 20) == 8
    assert auto_levels("sept", 2 ** 20) == 6



def test_s_opt_is_table2_and_minimises_app_cost():
    """S_opt (Table 2) from P4, P2 and the branching factor reproduces the
    printed coefficients, and it is where the s-dependent cost of App. A-C
    is smallest (checked against a numeric minimisation on a fine grid)."""
    from oracle.params import app_cost, s_opt
    rows = {f[0]: (int(f[1]), int(f[2])) for f in (l.split() for l in golden_lines("table2_sopt.txt"))}
    for t, (num, den) in rows.items():
        assert s_opt(t, 1.0, 1.0, 1.0) == pytest.approx(math.sqrt(num / den), rel=1e-12)
        for p, N, M in ((12, 5120, 5120), (22, 2 ** 20, 2 ** 19), (8, 1000, 30000)):
            grid = np.exp(np.linspace(np.log(0.1), np.log(1e4), 200001))
            best = grid[np.argmin(app_cost(t, p, N, M, grid))]
            assert best == pytest.approx(s_opt(t, p, N, M), rel=1e-3)


def test_sopt_levels_balances_the_cost():
    """The S_opt level rule picks the level whose per-leaf count is nearest
    S_opt in the cost's sense: its cost is below both neighbours'."""
    from oracle.params import app_cost, leaf_area, sopt_levels
    for t in ("quad", "sept", "tri"):
        for N, M, p in ((2 ** 20, 2 ** 20, 22), (5120, 5120, 12), (10 ** 6, 3 * 10 ** 5, 14)):
            L = sopt_levels(t, N, M, p)
            c = lambda l: app_cost(t, p, N, M, N * leaf_area(t, l))
            assert c(L) <= c(L + 1) and (L == 1 or c(L) <= c(L - 1))
