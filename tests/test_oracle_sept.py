"""Pins of the septree oracle against the paper's worked examples (Sec. 5),
geometry and the Eisenstein-integer mathematics."""
import math

import numpy as np
import pytest

from conftest import golden_lines
from oracle import tiling_sept as ts
from oracle.params import sept_leaf_circumradius, sept_min_outside_norm


def eis_add_numerals(a, b):
    """a (+) b computed through the Eisenstein route only."""
    L = 12
    ea = ts.key_to_eisenstein(a, len(ts.to_digits(a)) or 1)
    eb = ts.key_to_eisenstein(b, len(ts.to_digits(b)) or 1)
    k = ts.eisenstein_to_key(np.array([ea[0] + eb[0]]), np.array([ea[1] + eb[1]]), L)[0]
    return int(k)


def b7(s):
    return int(str(s), 7)


def test_unit_sum_table_both_routes():
    rows = list(golden_lines("gbt_unit_sum.txt"))
    assert len(rows) == 6
    for line in rows:
        i, rest = line.split(":")
        i = int(i)
        for j, v in enumerate(rest.split(), start=1):
            # the Eisenstein route reproduces the printed table without using it
            assert eis_add_numerals(i, j) == b7(v), (i, j, v)
            assert ts.gbt_add(i, j) == b7(v)


def test_worked_examples():
    for line in golden_lines("sept_examples.txt"):
        lhs, rhs = line.split("=")
        f = lhs.split()
        want = [b7(v) for v in rhs.split()]
        if f[0] == "add":
            a, c = b7(f[1]), b7(f[2])
            assert ts.gbt_add(a, c) == want[0]
            assert eis_add_numerals(a, c) == want[0]
        elif f[0] in ("add3", "zext"):
            a, c, d = b7(f[1]), b7(f[2]), b7(f[3])
            assert ts.gbt_add(ts.gbt_add(a, c), d) == want[0]
        elif f[0] == "neighbors":
            n, l = b7(f[1]), int(f[2])
            T = ts.Septree(3)
            assert sorted(T.neighbors(n, l)) == sorted(want)
        elif f[0] == "centersum":
            # CellCenter of an index is the sum of the centres of its
            # zero-extended components (eq. 4), on the same level.
            n = b7(f[1])
            T = ts.Septree(4)
            l = len(f[1])
            z = T.center_frame(n, l)
            s = sum(T.center_frame(m, l) for m in want)
            assert abs(z - s) < 1e-14


def test_gbt_add_matches_eisenstein_random():
    rng = np.random.default_rng(7)
    for _ in range(300):
        a = int(rng.integers(0, 7 ** 4))
        b = int(rng.integers(0, 7 ** 4))
        assert ts.gbt_add(a, b) == eis_add_numerals(a, b)
        assert ts.gbt_add(a, b) == ts.gbt_add(b, a)


def test_zero_extension_geometry():
    # App. D: each zero extension rotates by theta = arctan(sqrt3/2) ~ 40.8934 deg
    # and scales by sqrt7 (eqs. 22-23).
    assert math.degrees(ts.THETA) == pytest.approx(40.8933946, abs=1e-6)
    T = ts.Septree(3)
    for d in range(1, 7):
        z1 = T.center_frame(d, 3)
        z10 = T.center_frame(7 * d, 3)
        assert abs(z10) == pytest.approx(math.sqrt(7) * abs(z1), rel=1e-13)
        ang = math.atan2((z10 / z1).imag, (z10 / z1).real)
        assert ang == pytest.approx(ts.THETA, abs=1e-13)
        # neighbouring leaf centres are r*sqrt3 apart (a0 = r sqrt3, App. D)
        assert abs(z1) == pytest.approx(T.r * math.sqrt(3), rel=1e-13)


def test_center_matches_eisenstein_lattice():
    T = ts.Septree(3)
    w = complex(0.5, math.sqrt(3) / 2)
    unit = T.r * math.sqrt(3) * complex(math.cos(math.pi / 6), math.sin(math.pi / 6))
    beta = 1 + 2 * w
    for l in range(1, 4):
        for n in range(7 ** l):
            a, b = ts.key_to_eisenstein(n, l)
            z = unit * beta ** (3 - l) * (a + b * w)
            assert abs(T.center_frame(n, l) - z) < 1e-12


def test_keys_paper_route_equals_eisenstein_route():
    rng = np.random.default_rng(3)
    xy = rng.random((400, 2))
    for L in (2, 3, 4):
        T = ts.Septree(L)
        assert np.array_equal(T.keys(xy[:, 0], xy[:, 1]), T.keys_literal(xy[:, 0], xy[:, 1]))


def test_round_trip_and_nearest_centre():
    L = 3
    T = ts.Septree(L)
    leaf_c = np.array([T.center_frame(n, L) for n in range(7 ** L)])
    # CellIndex(CellCenter(n)) = n for every leaf inside the domain square
    for n in range(7 ** L):
        z = T.to_world(leaf_c[n])
        if 0 <= z.real < 1 and 0 <= z.imag < 1:
            assert T.keys(np.array([z.real]), np.array([z.imag]))[0] == n
    # the key of a point is its nearest leaf centre (Voronoi reading, Sec. 5)
    rng = np.random.default_rng(11)
    xy = rng.random((500, 2))
    k = T.keys(xy[:, 0], xy[:, 1])
    X, Y = T.frame(xy[:, 0], xy[:, 1])
    d = np.abs((X + 1j * Y)[:, None] - leaf_c[None, :])
    assert np.array_equal(k, np.argmin(d, axis=1))


def test_domain_is_covered():
    for L in (2, 3, 4, 5, 6):
        T = ts.Septree(L)
        g = np.linspace(0, 1 - 1e-12, 301)
        x, y = np.meshgrid(g, g)
        T.keys(x.ravel(), y.ravel())     # raises DomainError if not covered
        # and r is as small as that allows: the smallest lattice point outside
        # the L-digit region is within sqrt(1/2) + r of the origin once r is shrunk 1%
        m = math.sqrt(sept_min_outside_norm(L))
        assert (math.sqrt(0.5) / (0.99 * T.r * math.sqrt(3)) + 1 / math.sqrt(3)) > m


def test_list_sizes_interior():
    # Table 2: P2 = 7 (cell and its 6 neighbours), P4 = 42 M2L cells, for a
    # cell whose parent neighbourhood lies inside the root.
    T = ts.Septree(4)
    for l in (2, 3, 4):
        n_interior = 0
        for n in range(7 ** l):
            nb = T.neighbors(n, l)
            assert n not in nb
            P = n // 7
            if len(T.neighbors(P, l - 1)) == 6 and len(nb) == 6:
                n_interior += 1
                assert len(T.near(n, l)) == 7
                assert len(T.far(n, l)) == 42
            else:
                assert len(T.far(n, l)) <= 42
        assert n_interior > 0
    # level 1: the M2L list of an outer cell holds the three opposite cells
    assert len(T.far(1, 1)) == 3


def test_aggregate_radius_factor():
    """Sec. 7 reading: the GBT-prefix aggregate of m levels of hexagons reaches
    at most 1.0327 times the Voronoi circumradius of its level (so that the
    M2L ratio kappa = f/(3-f) <= 0.525 used for p(eps) holds)."""
    T = ts.Septree(5)
    for m in range(1, 5):
        pts = []
        for leaf in range(7 ** m):
            pts.extend(T.leaf_vertices_frame(leaf))
        rmax = max(abs(z) for z in pts)
        vor = T.r * math.sqrt(7) ** m
        f = rmax / vor
        assert 1.0 <= f <= 1.0327
        assert f / (3 - f) <= 0.525


def test_separation_ratios():
    """Table 2 / Sec. 7: septree r/R = 1/2 and rho = r for the hexagon tiling
    (leaf level, where cells are exact hexagons)."""
    L = 3
    T = ts.Septree(L)
    n = 0
    r = T.r                                  # circumradius of the tile
    # R: inscribed radius of the tile plus its six neighbours = distance from
    # the centre to the nearest point not covered by them
    c0 = T.center_frame(n, L)
    cover = set(T.near(n, L))
    allc = np.array([T.center_frame(m, L) for m in range(7 ** L)])
    ang = np.linspace(0, 2 * math.pi, 721)          # includes multiples of 30 deg
    R = None
    for rad in np.linspace(1.9 * r, 2.1 * r, 401):
        pts = c0 + rad * np.exp(1j * ang)
        nearest = np.argmin(np.abs(pts[:, None] - allc[None, :]), axis=1)
        if not all(int(m) in cover for m in nearest):
            R = rad
            break
    assert r / R == pytest.approx(0.5, abs=2e-3)
    # rho: gap between circumscribing circles of the closest M2L pair
    dmin = min(abs(T.center_frame(m, L) - c0) for m in T.far(n, L))
    rho = dmin - 2 * r
    assert rho / r == pytest.approx(1.0, abs=1e-12)


def test_leaf_radius_table_is_monotone():
    rs = [sept_leaf_circumradius(L) for L in range(1, 8)]
    assert all(a > b for a, b in zip(rs, rs[1:]))
    for L, r in enumerate(rs, start=1):
        assert r * 2 ** 40 == int(r * 2 ** 40)


def test_deep_level_norm_bound_holds_where_enumerated():
    """Levels beyond the enumerated ones take the lower bound
    sqrt(m_{L+1}) >= sqrt7 sqrt(m_L) - 1 on the smallest norm of a lattice
    point outside the L-digit GBT region (its last base-beta digit removed,
    such a point maps to one outside the shorter region, and |beta| = sqrt7).
    Where m_L is enumerated the bound must lie below it, and a leaf radius
    computed from the bound must be at least the enumerated one (so the
    region still covers the domain square)."""
    from oracle.params import sept_root_norm_bound
    for L in range(1, 9):
        lo = math.sqrt(7.0) * math.sqrt(sept_min_outside_norm(L)) - 1.0
        assert lo < math.sqrt(sept_min_outside_norm(L + 1))
        raw = math.sqrt(0.5) / (math.sqrt(3.0) * (lo - 1e-9) - 1.0)
        assert math.ceil(raw * 2.0 ** 40) / 2.0 ** 40 >= sept_leaf_circumradius(L + 1)
    assert sept_root_norm_bound(5) == math.sqrt(sept_min_outside_norm(5))
    # beyond the enumerated levels: below sqrt7 times the previous level
    for L in (10, 11):
        assert sept_root_norm_bound(L) < math.sqrt(7.0) * sept_root_norm_bound(L - 1)
        assert sept_leaf_circumradius(L) < sept_leaf_circumradius(L - 1)


@pytest.mark.parametrize("L", [10, 11])
def test_deep_levels_cover_the_domain(L):
    """Septrees of 10 and 11 levels (keys below 7^11 < 2^32) key every point
    of the domain square: the corners (farthest from the root centre), its
    edges and random points all get an L-digit GBT key."""
    T = ts.Septree(L)
    rng = np.random.default_rng(L)
    e = 1 - 1e-12
    g = np.linspace(0, e, 2001)
    edge = np.concatenate([np.column_stack([g, np.zeros_like(g)]), np.column_stack([g, np.full_like(g, e)]),
                           np.column_stack([np.zeros_like(g), g]), np.column_stack([np.full_like(g, e), g])])
    corners = np.array([[0, 0], [e, 0], [0, e], [e, e]]) + 1e-9 * rng.random((4, 2))
    pts = np.vstack([edge, np.clip(corners, 0, e), rng.random((20000, 2))])
    k = T.keys(pts[:, 0], pts[:, 1])        # raises DomainError if a point is not covered
    assert k.min() >= 0 and k.max() < 7 ** L
