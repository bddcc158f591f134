"""Pins of the triangle-quadtree oracle against the paper's worked examples
(Sec. 6) and against plain geometry."""
import math

import numpy as np
import pytest

from conftest import golden_lines
from oracle import tiling_tri as tt


def b4(s):
    return int(str(s), 4)


def test_worked_examples():
    for line in golden_lines("tri_examples.txt"):
        lhs, rhs = line.split("=")
        f = lhs.split()
        if f[0] == "adj":
            n, l, k = b4(f[1]), int(f[2]), f[3]
            assert tt.adjacent_neighbor(n, l, k) == b4(rhs.strip())
        elif f[0] == "orient":
            n, l = b4(f[1]), int(f[2])
            want = [int(v) for v in rhs.split()]
            got = [tt.is_up(n >> (2 * (l - i)), i, i) for i in range(1, l + 1)]
            assert got == want


def _geometry(T, l):
    verts = {}
    for n in range(4 ** l):
        verts[n] = T.vertices_frame(n, l)
    return verts


def test_children_tile_parent_and_orientation():
    # Sec. 6: the four children tile the parent; only the centre child flips.
    T = tt.TriQuadtree(4)
    for l in range(0, 3):
        for n in range(4 ** l):
            up = T.orientation(n, l) if l else 1
            area_p = 3 * math.sqrt(3) * T.inradius(l) ** 2
            area_c = 0
            for d, ch in enumerate(T.children(n)):
                oc = T.orientation(ch, l + 1)
                assert oc == (-up if d == 0 else up)
                area_c += 3 * math.sqrt(3) * T.inradius(l + 1) ** 2
                # child centroid inside the parent triangle
                assert _inside(T.vertices_frame(n, l), T.center_frame(ch, l + 1))
            assert area_c == pytest.approx(area_p)


def _inside(v, z, tol=1e-12):
    def cross(a, b, c):
        return (b - a).real * (c - a).imag - (b - a).imag * (c - a).real
    s = [cross(v[i], v[(i + 1) % 3], z) for i in range(3)]
    return all(x >= -tol for x in s) or all(x <= tol for x in s)


def test_neighbors_equal_vertex_sharing_cells():
    """The 12-call recursion of Sec. 6 returns exactly the cells that share a
    vertex with n (brute force on the vertex coordinates)."""
    for l in (2, 3):
        T = tt.TriQuadtree(4)
        V = _geometry(T, l)
        for n in range(4 ** l):
            brute = set()
            for m in range(4 ** l):
                if m == n:
                    continue
                if any(abs(a - b) < 1e-9 for a in V[n] for b in V[m]):
                    brute.add(m)
            assert set(T.neighbors(n, l)) == brute, (n, l)


def test_list_sizes_interior():
    # Table 2: P2 = 13, P4 = 39 for a cell whose parent has all 12 neighbours.
    T = tt.TriQuadtree(4)
    seen = 0
    for l in (3, 4):
        for n in range(4 ** l):
            if len(T.neighbors(n // 4, l - 1)) == 12 and len(T.neighbors(n, l)) == 12:
                seen += 1
                assert len(T.near(n, l)) == 13
                assert len(T.far(n, l)) == 39
            else:
                assert len(T.far(n, l)) <= 39
    assert seen > 0


def test_keys_both_routes_and_containment():
    rng = np.random.default_rng(5)
    xy = rng.random((2000, 2))
    for L in (1, 3, 5):
        T = tt.TriQuadtree(L)
        k = T.keys(xy[:, 0], xy[:, 1])
        kl = T.keys_literal(xy[:, 0], xy[:, 1])
        assert np.array_equal(k, kl)
        X, Y = T.frame(xy[:, 0], xy[:, 1])
        for i in range(0, 2000, 37):
            assert _inside(T.vertices_frame(int(k[i]), L), complex(X[i], Y[i]))
    # prefix property: the level-l key is the leaf key div 4^(L-l)
    T5 = tt.TriQuadtree(5)
    k5 = T5.keys(xy[:, 0], xy[:, 1])
    for l in range(6):
        assert np.array_equal(T5.keys(xy[:, 0], xy[:, 1], l), k5 >> (2 * (5 - l)))


def test_round_trip():
    L = 4
    T = tt.TriQuadtree(L)
    for n in range(4 ** L):
        z = T.to_world(T.center_frame(n, L))
        if 0 <= z.real < 1 and 0 <= z.imag < 1:
            assert T.keys(np.array([z.real]), np.array([z.imag]))[0] == n


def test_root_contains_domain():
    T = tt.TriQuadtree(3)
    root = T.vertices_frame(0, 0)
    for cx in (-0.5, 0.5):
        for cy in (-0.5, 0.5):
            assert _inside(root, complex(cx, cy))


def test_separation_ratios():
    """Table 2 / Sec. 7, App. E: triangle r/R = 1/2 and rho/r = sqrt7 - 2."""
    L = 4
    T = tt.TriQuadtree(L)
    l = 4
    ratios = []
    for n in range(4 ** l):
        if len(T.neighbors(n, l)) == 12 and len(T.neighbors(n // 4, l - 1)) == 12:
            c0 = T.center_frame(n, l)
            r = 2 * T.inradius(l)               # circumradius of the tile
            dmin = min(abs(T.center_frame(m, l) - c0) for m in T.far(n, l))
            ratios.append((dmin - 2 * r) / r)
            # R: radius of the largest circle about the centroid covered by the
            # 13 cells of the neighbourhood
            tris = [T.vertices_frame(m, l) for m in T.near(n, l)]
            ang = np.linspace(0, 2 * math.pi, 1441)       # multiples of 0.25 deg
            R = None
            for rad in np.linspace(1.9 * r, 2.1 * r, 201):
                pts = c0 + rad * np.exp(1j * ang)
                if not all(any(_inside(v, z, 1e-15) for v in tris) for z in pts):
                    R = rad
                    break
            assert r / R == pytest.approx(0.5, abs=3e-3)
            if len(ratios) > 3:
                break
    assert min(ratios) == pytest.approx(math.sqrt(7) - 2, abs=1e-12)
