"""Septree tiling: hexagons with base-7 Generalized Balanced Ternary indices (Sec. 5).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Indices are digit strings t_1 t_2 ... t_l (t_1 most significant), also held as
the base-7 integer n = sum t_i 7^(l-i).  Children(n) = 7n + {0..6},
Parent(n) = n div 7; the level-l cell of a leaf index is its first l digits
(Sec. 5, CellIndex).

Two independent routes are implemented:

* the paper's route, using only the GBT unit-sum table of Fig. 4(b):
  multi-digit GBT addition, Neighbors (Sec. 5.1), CellCenter (eq. 6) and
  CellIndex (eqs. 7-9, steps 1-6);
* an Eisenstein-integer route for the same keys.  Reading (checked against
  the whole table of Fig. 4(b), the example 14 (+) 35 = 32 and the neighbours of
  52 in Fig. 5a): digit d = 1..6 is the unit w^(d-1) with w = e^{i pi/3},
  and a zero-extension multiplies by beta = 1 + 2w (|beta| = sqrt7,
  arg beta = arctan(sqrt3/2), App. D).  A lattice point b*v2 + c*v3 is the
  Eisenstein integer b + c*w; its digits are its base-beta expansion.

Frame: (X, Y) = ((x - x0)/S - 1/2, (y - y0)/S - 1/2); leaf hexagon 0 is
centred at the origin with circumradius r = ``params.sept_leaf_circumradius(L)``.
"""
import math

import numpy as np

from .params import DomainError, SQRT3, sept_leaf_circumradius

# Fig. 4(b): GBT sum of unit digits (row) and (column), written in base 7.
GBT_UNIT_SUM = (
    (63, 15, 2, 0, 6, 64),
    (15, 14, 26, 3, 0, 1),
    (2, 26, 25, 31, 4, 0),
    (0, 3, 31, 36, 42, 5),
    (6, 0, 4, 42, 41, 53),
    (64, 1, 0, 5, 53, 52),
)

THETA = math.atan(math.sqrt(3.0) / 2.0)      # App. D, eq. (22)


# ---------------------------------------------------------------------------
# Paper route: GBT arithmetic from the unit-sum table
# ---------------------------------------------------------------------------
def _unit_sum(d1, d2):
    """d1 (+) d2 for single digits, as (carry digit, digit), from Fig. 4(b)."""
    if d1 == 0:
        return 0, d2
    if d2 == 0:
        return 0, d1
    v = GBT_UNIT_SUM[d1 - 1][d2 - 1]
    return v // 10, v % 10


def to_digits(n, ndig=None):
    """Base-7 digits of integer n, most significant first."""
    ds = []
    while n:
        ds.append(n % 7)
        n //= 7
    ds = ds[::-1]
    if ndig is not None:
        ds = [0] * (ndig - len(ds)) + ds
    return ds


def from_digits(ds):
    n = 0
    for d in ds:
        n = 7 * n + d
    return n


def gbt_add(a, b):
    """GBT addition a (+) b of two indices (integers holding base-7 numerals).

    Digit-wise sums from the unit-sum table give a digit and a carry for the
    next position; the carries are then added the same way until none is
    left (Sec. 5.1: summation of higher-order indices)."""
    x = to_digits(a)[::-1]
    y = to_digits(b)[::-1]
    for _ in range(200):
        n = max(len(x), len(y))
        s, c = [], [0]
        for i in range(n):
            ci, di = _unit_sum(x[i] if i < len(x) else 0, y[i] if i < len(y) else 0)
            s.append(di)
            c.append(ci)
        x, y = s, c
        if not any(y):
            return from_digits(x[::-1])
    raise RuntimeError("GBT addition did not settle")


def gbt_times(k, unit):
    """k copies of a unit digit summed with (+); negative k uses the
    opposite unit.  Double-and-add over (+) only."""
    if k < 0:
        k, unit = -k, (unit + 2) % 6 + 1
    acc, pw = 0, unit
    while k:
        if k & 1:
            acc = gbt_add(acc, pw)
        pw = gbt_add(pw, pw)
        k >>= 1
    return acc


# ---------------------------------------------------------------------------
# Eisenstein route (independent of the table)
# ---------------------------------------------------------------------------
_RES_TO_DIGIT = np.array([0, 1, 3, 2, 5, 6, 4], dtype=np.int64)   # (a+3b) mod 7 -> digit
_UNIT_A = np.array([0, 1, 0, -1, -1, 0, 1], dtype=np.int64)       # w^(d-1) = A + B w
_UNIT_B = np.array([0, 0, 1, 1, 0, -1, -1], dtype=np.int64)


def _beta_step(a, b):
    """One base-beta digit of a + b w: returns (digit, quotient a, quotient b)."""
    d = _RES_TO_DIGIT[np.mod(a + 3 * b, 7)]
    a1 = a - _UNIT_A[d]
    b1 = b - _UNIT_B[d]
    # (a1 + b1 w) / (1 + 2w) = (a1 + b1 w)(3 - 2w) / 7
    qa = 3 * a1 + 2 * b1
    qb = b1 - 2 * a1
    return d, qa // 7, qb // 7


def eisenstein_digit_count(a, b, cap):
    """Number of base-beta digits of a + b w, capped at cap + 1."""
    a = np.asarray(a, np.int64).copy()
    b = np.asarray(b, np.int64).copy()
    count = np.zeros(a.shape, np.int64)
    for _ in range(cap + 1):
        nz = (a != 0) | (b != 0)
        count += nz
        _, a, b = _beta_step(a, b)
    return count


def eisenstein_to_key(a, b, L):
    """Base-7 key (L digits) of the Eisenstein integers a + b w; -1 where
    more than L digits are needed (outside the level-0 cell)."""
    a = np.asarray(a, np.int64).copy()
    b = np.asarray(b, np.int64).copy()
    key = np.zeros(a.shape, np.int64)
    for i in range(L):
        d, a, b = _beta_step(a, b)
        key += d * 7 ** i
    key[(a != 0) | (b != 0)] = -1
    return key


def key_to_eisenstein(n, l):
    """Inverse of eisenstein_to_key for one level-l index (Horner in beta)."""
    a = b = 0
    for d in to_digits(n, l):
        # (a + b w)(1 + 2w) = a - 2b + (2a + 3b) w ; then add the unit
        a, b = a - 2 * b + int(_UNIT_A[d]), 2 * a + 3 * b + int(_UNIT_B[d])
    return a, b


class Septree:
    name = "sept"
    b = 7
    l_min = 1

    def __init__(self, L, domain=(0.0, 0.0, 1.0), r=None):
        self.L = int(L)
        self.x0, self.y0, self.S = (float(v) for v in domain)
        self.r = sept_leaf_circumradius(self.L) if r is None else float(r)

    def frame(self, x, y):
        X = (np.asarray(x, np.float64) - self.x0) / self.S - 0.5
        Y = (np.asarray(y, np.float64) - self.y0) / self.S - 0.5
        return X, Y

    def to_world(self, z):
        return complex(self.x0 + self.S * (z.real + 0.5), self.y0 + self.S * (z.imag + 0.5))

    # -- CellIndex, steps 1-4: nearest lattice point (shared by both routes) --
    def nearest_lattice(self, X, Y):
        """Steps 1-4 of CellIndex: change of basis (eq. 7), the four candidate
        lattice points (eq. 9), conversion back with eq. (8), nearest by squared
        distance, first candidate kept on ties."""
        r = self.r
        k3r = 3.0 * r
        rs3 = r * SQRT3
        b = (2.0 * X) / k3r
        c = (Y * SQRT3 - X) / k3r
        fb, cb, fc, cc = np.floor(b), np.ceil(b), np.floor(c), np.ceil(c)
        best_d = None
        for bh, ch in ((fb, fc), (cb, fc), (fb, cc), (cb, cc)):
            xh = (k3r * bh) * 0.5
            yh = (rs3 * (2.0 * ch + bh)) * 0.5
            dx = X - xh
            dy = Y - yh
            d = dx * dx + dy * dy
            if best_d is None:
                best_d, bt, ct = d, bh.copy(), ch.copy()
            else:
                take = d < best_d
                best_d = np.where(take, d, best_d)
                bt = np.where(take, bh, bt)
                ct = np.where(take, ch, ct)
        return bt.astype(np.int64), ct.astype(np.int64)

    def _check_domain(self, x, y):
        tx = (np.asarray(x, np.float64) - self.x0) / self.S
        ty = (np.asarray(y, np.float64) - self.y0) / self.S
        if np.any((tx < 0) | (tx >= 1) | (ty < 0) | (ty >= 1)):
            raise DomainError("point outside the domain square")

    def keys(self, x, y):
        """Leaf keys by the Eisenstein route (vectorised)."""
        self._check_domain(x, y)
        X, Y = self.frame(x, y)
        bt, ct = self.nearest_lattice(X, Y)
        key = eisenstein_to_key(bt, ct, self.L)
        if np.any(key < 0):
            raise DomainError("point outside the level-0 septree cell")
        return key

    def keys_literal(self, x, y):
        """Leaf keys by CellIndex steps 5-6 as the paper states them: the
        index u of b~ along axis v2 (unit digit 1) and v of c~ along v3 (unit
        digit 2), returned as u (+) v."""
        self._check_domain(x, y)
        X, Y = self.frame(x, y)
        bt, ct = self.nearest_lattice(np.atleast_1d(X), np.atleast_1d(Y))
        out = []
        for bb, cc in zip(bt.tolist(), ct.tolist()):
            k = gbt_add(gbt_times(bb, 1), gbt_times(cc, 2))
            if k >= 7 ** self.L:
                raise DomainError("point outside the level-0 septree cell")
            out.append(k)
        return np.array(out, np.int64)

    # -- Sec. 5 auxiliary functions ------------------------------------------
    def center_frame(self, n, l):
        """CellCenter(n, l) by eq. (6): sum over the non-zero digits t_i of the
        translation R_i e^{i theta_i}, j = (|t| - i) + (L - l)."""
        t = to_digits(n, l)
        z = 0j
        for i, ti in enumerate(t, start=1):
            if ti == 0:
                continue
            j = (len(t) - i) + (self.L - l)
            th = j * THETA + ti * math.pi / 3.0 - math.pi / 6.0
            R = self.r * SQRT3 * math.sqrt(7.0) ** j
            z += R * complex(math.cos(th), math.sin(th))
        return z

    def center(self, n, l):
        return self.to_world(self.center_frame(n, l))

    def children(self, n):
        return [7 * n + d for d in range(7)]

    def parent(self, n):
        return n // 7

    def neighbors(self, n, l):
        """Neighbors(n, l), Sec. 5.1: n (+) {1..6}, indices >= 7^l removed."""
        out = []
        for k in range(1, 7):
            m = gbt_add(n, k)
            if m < 7 ** l:
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
        for q in [P] + self.neighbors(P, l - 1):
            cand.extend(self.children(q))
        excl = set(self.near(n, l))
        return sorted(c for c in cand if c not in excl)

    # -- geometry used by the pins ---------------------------------------------
    def leaf_vertices_frame(self, n_leaf):
        c = self.center_frame(n_leaf, self.L)
        return [c + self.r * complex(math.cos(k * math.pi / 3), math.sin(k * math.pi / 3))
                for k in range(6)]
