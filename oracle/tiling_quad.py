"""Quadtree tiling with Morton Z indexing (Sec. 4, Fig. 3a).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Frame: a point (x, y) of the domain square [x0, x0+S) x [y0, y0+S) maps to
t = ((x - x0)/S, (y - y0)/S) in [0, 1)^2.  A level-l cell is the square
[i, i+1) x [j, j+1) * 2^-l; its index is the base-4 Morton number whose
digit on level m (most significant first) is xbit + 2*ybit of (i, j) on that
level, so Children(n) = 4n + {0..3} and Parent(n) = n div 4 (Sec. 4).
"""
import numpy as np

from .params import DomainError


class Quadtree:
    name = "quad"
    b = 4           # children per cell
    l_min = 2       # first level whose M2L lists are not empty

    def __init__(self, L, domain=(0.0, 0.0, 1.0)):
        self.L = int(L)
        self.x0, self.y0, self.S = (float(v) for v in domain)

    # -- frame and keys -----------------------------------------------------
    def frame(self, x, y):
        tx = (np.asarray(x, np.float64) - self.x0) / self.S
        ty = (np.asarray(y, np.float64) - self.y0) / self.S
        return tx, ty

    def keys(self, x, y, l=None):
        """CellIndex(x, y, l) for arrays of points (Sec. 4): Morton key of
        (floor(tx 2^l), floor(ty 2^l))."""
        l = self.L if l is None else l
        tx, ty = self.frame(x, y)
        if np.any((tx < 0) | (tx >= 1) | (ty < 0) | (ty >= 1)):
            raise DomainError("point outside the domain square")
        i = np.floor(tx * 2.0 ** l).astype(np.int64)
        j = np.floor(ty * 2.0 ** l).astype(np.int64)
        key = np.zeros_like(i)
        for m in range(l):                      # digit of level l-m
            key |= ((i >> m) & 1) << (2 * m)
            key |= ((j >> m) & 1) << (2 * m + 1)
        return key

    @staticmethod
    def coords(n, l):
        i = j = 0
        for m in range(l):
            i |= ((n >> (2 * m)) & 1) << m
            j |= ((n >> (2 * m + 1)) & 1) << m
        return i, j

    @staticmethod
    def index(i, j, l):
        n = 0
        for m in range(l):
            n |= ((i >> m) & 1) << (2 * m)
            n |= ((j >> m) & 1) << (2 * m + 1)
        return n

    # -- Sec. 4 auxiliary functions ------------------------------------------
    def center(self, n, l):
        """CellCenter(n, l) in original coordinates (complex)."""
        i, j = self.coords(n, l)
        h = 2.0 ** -l
        return complex(self.x0 + self.S * (i + 0.5) * h, self.y0 + self.S * (j + 0.5) * h)

    def children(self, n):
        return [4 * n + d for d in range(4)]

    def parent(self, n):
        return n // 4

    def neighbors(self, n, l):
        """Cells of level l sharing a vertex with n (Sec. 4), n excluded."""
        i, j = self.coords(n, l)
        out = []
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                if di == 0 and dj == 0:
                    continue
                a, c = i + di, j + dj
                if 0 <= a < 2 ** l and 0 <= c < 2 ** l:
                    out.append(self.index(a, c, l))
        return out

    def near(self, n, l):
        """{n} u Neighbors(n, l): the P2 cells of Table 2."""
        return [n] + self.neighbors(n, l)

    def far(self, n, l):
        """NeighborsE4(n, l) (Sec. 4, eq. 3), read as the set difference
        Children[Parent(n) u Neighbors(Parent(n), l-1)] minus Near(n)."""
        if l < 1:
            return []
        P = self.parent(n)
        cand = []
        for q in [P] + self.neighbors(P, l - 1):
            cand.extend(self.children(q))
        excl = set(self.near(n, l))
        return sorted(c for c in cand if c not in excl)

    # -- geometry used by the separation pins ---------------------------------
    def vertices(self, n, l):
        c = self.center(n, l)
        h = self.S * 2.0 ** -l / 2
        return [c + complex(sx * h, sy * h) for sx, sy in ((1, 1), (-1, 1), (-1, -1), (1, -1))]

    def contains(self, n, l, x, y):
        i, j = self.coords(n, l)
        tx, ty = self.frame(x, y)
        return (i <= tx * 2 ** l < i + 1) and (j <= ty * 2 ** l < j + 1)
