"""Facts about lattice positions that the list construction relies on.

The adaptive lists look cells up in a table keyed by (level, instance,
lattice position) and the uniform triangle lists read a position-indexed
slot map; both pack a position into a fixed number of bits and treat a
position outside the packing range as "no cell".  These tests pin the facts
that make that exact:

* triangle tiling (Sec. 6): the level-l cells are exactly the integer
  positions (i, j, k) in [0, 2^l)^3 with i + j + k = 2^l - 1 (up) or
  2^l - 2 (down), each cell once, and the ancestor of a cell d levels up is
  its position shifted right by d;
* septree (Sec. 5, GBT digits): the Eisenstein coordinates (a, b) of the
  level-l cells, from the oracle's key -> coordinate map, are distinct and
  bounded by |a|, |b| < 7^(l/2).
"""
import itertools

import pytest

from oracle import tiling_sept as ts


def _tri_subdivide(levels):
    """Cells of levels 0..levels by subdividing the root: a triangle splits
    into its centre triangle (opposite orientation) and three corner
    triangles (same orientation); per coordinate the child adds one bit."""
    up_codes = (0b000, 0b100, 0b010, 0b001)     # centre, then the three corners
    down_codes = (0b111, 0b011, 0b110, 0b101)
    out = [{(0, 0, 0): (True, None)}]            # position -> (up, parent position)
    for l in range(levels):
        nxt = {}
        for (i, j, k), (up, _) in out[-1].items():
            for c in (up_codes if up else down_codes):
                ch = (2 * i + (c >> 2 & 1), 2 * j + (c >> 1 & 1), 2 * k + (c & 1))
                assert ch not in nxt, "two cells at one position"
                child_up = up != (c in (0b000, 0b111))   # the centre child flips
                nxt[ch] = (child_up, (i, j, k))
        out.append(nxt)
    return out


@pytest.mark.parametrize("levels", [6])
def test_triangle_positions_are_the_cells(levels):
    cells = _tri_subdivide(levels)
    for l, lev in enumerate(cells):
        n = 1 << l
        want = {(i, j, k) for i, j, k in itertools.product(range(n), repeat=3)
                if i + j + k in (n - 1, n - 2)}
        assert set(lev) == want
        assert len(lev) == 4 ** l
        for (i, j, k), (up, par) in lev.items():
            assert up == (i + j + k == n - 1)
            if par is not None:
                assert par == (i >> 1, j >> 1, k >> 1)
            # the ancestor d levels up, by shifting
            for d in range(l + 1):
                anc = (i >> d, j >> d, k >> d)
                assert anc in cells[l - d]


@pytest.mark.parametrize("l", range(0, 7))
def test_septree_coordinates_bounded_and_distinct(l):
    seen = set()
    bound = 7 ** (l / 2)
    for key in range(7 ** l):
        a, b = ts.key_to_eisenstein(key, l)
        assert abs(a) < bound and abs(b) < bound, (key, a, b)
        seen.add((a, b))
    assert len(seen) == 7 ** l
    # the packing width per coordinate, (3l + 1) // 2 + 2 bits biased by half
    # the range, holds every cell's coordinate (a position outside it is
    # rejected before packing: it cannot be a cell)
    half = 1 << ((3 * l + 1) // 2 + 1)
    assert bound <= half
