"""Triangle quadtree (Sec. 6).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Level 0 is one upright triangle centred at the origin that encloses the
domain (Sec. 6); its inradius is ``params.tri_root_inradius()`` in the frame
(X, Y) = ((x - x0)/S - 1/2, (y - y0)/S - 1/2).  Each triangle splits into four
children of types 0 = centre (orientation flipped), 1 = vertical, 2 = left,
3 = right; indices are base-4 digit strings, Children(n) = 4n + {0..3},
Parent(n) = n div 4.

Two routes give the leaf keys:

* ``keys_literal``: the CellIndex descent of Sec. 6 - at each level pick the
  nearest of the four lattice points (the current centre for type 0, or the
  three corner-child centres of eq. 13), flipping the orientation on type 0;
* ``keys``: the same descent done exactly on fixed-point barycentric
  coordinates (2^60 units): a point is in the corner child of vertex X when
  its barycentric coordinate for X exceeds 1/2, otherwise in the centre
  child; ties go to the lower child index, as the nearest-of-four search with
  a strict comparison does.  The two routes differ only within rounding of a
  triangle edge (pinned in the tests).
"""
import math

import numpy as np

from .params import DomainError, SQRT3, tri_root_inradius

# Table 1: (destination type, is-sibling) per source type and direction.
_DIRS = {"L": 0, "R": 1, "V": 2}
TABLE_D = (
    ((2, True), (3, True), (1, True)),
    ((3, False), (2, False), (0, True)),
    ((1, False), (0, True), (2, False)),
    ((0, True), (1, False), (3, False)),
)

ONE = 1 << 60
HALF = 1 << 59


def to_digits(n, l):
    return [(n >> (2 * (l - 1 - i))) & 3 for i in range(l)]


def from_digits(ds):
    n = 0
    for d in ds:
        n = 4 * n + d
    return n


def adjacent_neighbor(n, l, k):
    """adjacentNeighbor(n, k) of Sec. 6: nearest ancestor with a sibling in
    direction k (Table 1, right to left), move to it, then reflect the path
    below it through Table 1.  None if no ancestor has such a sibling (the
    neighbour would lie outside the root)."""
    t = to_digits(n, l)
    kk = _DIRS[k]
    for i in range(l - 1, -1, -1):
        dest, sib = TABLE_D[t[i]][kk]
        if sib:
            t[i] = dest
            for j in range(i + 1, l):
                t[j] = TABLE_D[t[j]][kk][0]
            return from_digits(t)
    return None


def is_up(n, ndig, l):
    """isUp(t, l) of eq. (11) for an index t with ndig digits on level l."""
    zeros = sum(1 for d in to_digits(n, ndig) if d == 0)
    return 2 * ((zeros % 2 + l - ndig + 1) % 2) - 1


class TriQuadtree:
    name = "tri"
    b = 4
    l_min = 2

    def __init__(self, L, domain=(0.0, 0.0, 1.0)):
        self.L = int(L)
        self.x0, self.y0, self.S = (float(v) for v in domain)
        self.rho0 = tri_root_inradius()
        # eq. (12): R_j = 2^(L - j) r is the distance from a level-(j-1) centre to
        # a corner-child centre, i.e. the level-(j-1) inradius rho0 2^-(j-1).
        self.r = self.rho0 * 2.0 ** (1 - self.L)

    def frame(self, x, y):
        X = (np.asarray(x, np.float64) - self.x0) / self.S - 0.5
        Y = (np.asarray(y, np.float64) - self.y0) / self.S - 0.5
        return X, Y

    def to_world(self, z):
        return complex(self.x0 + self.S * (z.real + 0.5), self.y0 + self.S * (z.imag + 0.5))

    def _check_domain(self, x, y):
        tx = (np.asarray(x, np.float64) - self.x0) / self.S
        ty = (np.asarray(y, np.float64) - self.y0) / self.S
        if np.any((tx < 0) | (tx >= 1) | (ty < 0) | (ty >= 1)):
            raise DomainError("point outside the domain square")

    # -- CellIndex -------------------------------------------------------------
    def barycentric_fixed(self, X, Y):
        """Fixed-point barycentric coordinates (vertical, left, right corners of
        the root) in units of 2^-60; the third is 1 minus the other two."""
        rho0 = self.rho0
        k3 = 3.0 * rho0
        half3 = SQRT3 * 0.5
        av = (Y + rho0) / k3
        al = ((rho0 - half3 * X) - 0.5 * Y) / k3
        AV = np.floor(av * float(ONE)).astype(np.int64)
        AL = np.floor(al * float(ONE)).astype(np.int64)
        AR = ONE - AV - AL
        return AV, AL, AR

    def keys(self, x, y, l=None):
        l = self.L if l is None else l
        self._check_domain(x, y)
        X, Y = self.frame(x, y)
        AV, AL, AR = self.barycentric_fixed(np.atleast_1d(X), np.atleast_1d(Y))
        if np.any((AV < 0) | (AL < 0) | (AR < 0)):
            raise DomainError("point outside the level-0 triangle")
        key = np.zeros(AV.shape, np.int64)
        for _ in range(l):
            tv = AV > HALF
            tl = ~tv & (AL > HALF)
            tr = ~tv & ~tl & (AR > HALF)
            tc = ~(tv | tl | tr)
            d = np.where(tv, 1, np.where(tl, 2, np.where(tr, 3, 0)))
            nAV = np.where(tv, 2 * AV - ONE, np.where(tc, ONE - 2 * AV, 2 * AV))
            nAL = np.where(tl, 2 * AL - ONE, np.where(tc, ONE - 2 * AR, 2 * AL))
            nAR = np.where(tr, 2 * AR - ONE, np.where(tc, ONE - 2 * AL, 2 * AR))
            AV, AL, AR = nAV, nAL, nAR
            key = 4 * key + d
        return key

    def keys_literal(self, x, y, l=None):
        """CellIndex(x, y, l) as the descent of Sec. 6 (eq. 13), in FP64."""
        l = self.L if l is None else l
        self._check_domain(x, y)
        X, Y = self.frame(x, y)
        out = []
        for px, py in zip(np.atleast_1d(X).tolist(), np.atleast_1d(Y).tolist()):
            u = v = 0.0
            up = 1
            t = []
            for i in range(1, l + 1):
                R = 2.0 ** (self.L - i) * self.r
                cands = [(u, v)]
                for ti in (1, 2, 3):
                    th = up * (math.pi / 2 + 2 * (ti - 1) * math.pi / 3)
                    cands.append((u + R * math.cos(th), v + R * math.sin(th)))
                best, bd = 0, None
                for ti, (cu, cv) in enumerate(cands):
                    d = (px - cu) ** 2 + (py - cv) ** 2
                    if bd is None or d < bd:
                        best, bd = ti, d
                t.append(best)
                u, v = cands[best]
                if best == 0:
                    up = -up
            out.append(from_digits(t))
        return np.array(out, np.int64)

    # -- Sec. 6 auxiliary functions ------------------------------------------
    def center_frame(self, n, l):
        """CellCenter(n, l), eq. (12): sum of R_i e^{i theta_i} over the
        non-zero digits, the orientation taken from isUp of the prefix."""
        t = to_digits(n, l)
        z = 0j
        for i, ti in enumerate(t, start=1):
            if ti == 0:
                continue
            j = l - len(t) + i
            up = is_up(n >> (2 * (l - i)), i, j)
            th = up * (math.pi / 2 + 2 * (ti - 1) * math.pi / 3)
            R = 2.0 ** (self.L - j) * self.r
            z += R * complex(math.cos(th), math.sin(th))
        return z

    def center(self, n, l):
        return self.to_world(self.center_frame(n, l))

    def orientation(self, n, l):
        return is_up(n, l, l)

    def children(self, n):
        return [4 * n + d for d in range(4)]

    def parent(self, n):
        return n // 4

    def neighbors(self, n, l):
        """Neighbors(n, l) of Sec. 6: L, R, V; VL, VR, LL, RR, LV, RV;
        VLL, VRR, LVR - each an adjacentNeighbor of an earlier one."""
        def adj(m, k):
            return None if m is None else adjacent_neighbor(m, l, k)
        L_, R_, V_ = adj(n, "L"), adj(n, "R"), adj(n, "V")
        VL, VR = adj(V_, "L"), adj(V_, "R")
        LL, RR = adj(L_, "L"), adj(R_, "R")
        LV, RV = adj(L_, "V"), adj(R_, "V")
        VLL, VRR, LVR = adj(VL, "L"), adj(VR, "R"), adj(LV, "R")
        out = []
        for m in (L_, R_, V_, VL, VR, LL, RR, LV, RV, VLL, VRR, LVR):
            if m is not None and m not in out:
                out.append(m)
        return out

    def near(self, n, l):
        return [n] + self.neighbors(n, l)

    def far(self, n, l):
        """NeighborsE4(n, l) (eq. 3) read as a set difference."""
        if l < 1:
            return []
        P = self.parent(n)
        cand = []
        for q in [P] + (self.neighbors(P, l - 1) if l - 1 >= 1 else []):
            cand.extend(self.children(q))
        excl = set(self.near(n, l))
        return sorted(c for c in cand if c not in excl)

    # -- geometry used by the pins ---------------------------------------------
    def inradius(self, l):
        return self.rho0 * 2.0 ** -l

    def vertices_frame(self, n, l):
        c = self.center_frame(n, l)
        up = self.orientation(n, l)
        R = 2.0 * self.inradius(l)
        return [c + R * complex(math.cos(up * (math.pi / 2 + 2 * k * math.pi / 3)),
                                math.sin(up * (math.pi / 2 + 2 * k * math.pi / 3)))
                for k in range(3)]
