"""Separation ratios, truncation order and root geometry per tiling.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Table 2 (Sec. 8) gives r/R (local separation) and rho/r (WSPD) per tiling.
  The M2L error bound (eq. 15, read in the dimensionless Greengard-Rokhlin
  form sum|u| (r/rho) (1/(1+rho/r))^(p+1)) decays like kappa^(p+1) with
  kappa = 1/(1 + rho/r).  The truncation order is the smallest p with
  kappa^(p+1) <= eps, i.e. p = ceil(ln eps / ln kappa) - 1.
* Septree reading: a level-l septree cell is the GBT-prefix aggregate of
  leaf hexagons (Sec. 5, CellIndex), whose extent is slightly larger than
  the Voronoi hexagon that Sec. 7 argues with.  Enumeration (pinned in the
  tests) gives a maximum radius factor f = 1.0327 over levels 1..8, so
  rho/r = (3 - 2f)/f and kappa = f/(3 - f) = 0.5249, which we round up to
  0.525.
* Root geometry (the paper leaves the root size free):
  - quadtree: the domain square itself;
  - septree: leaf circumradius r_L chosen so that every point of the
    frame square [-1/2, 1/2)^2 (inside the disc of radius sqrt(1/2)) has its
    nearest leaf-lattice point inside the L-digit GBT region;
  - triangle quadtree: level 0 is the upright triangle centred at the
    origin with inradius (sqrt3 + 1)/4 (1 + 2^-20), the smallest upright
    triangle centred at the origin that contains the frame square.
"""
import math

import numpy as np


class DomainError(ValueError):
    """A point lies outside the domain square or the root cell."""


SQRT3 = math.sqrt(3.0)

KAPPA = {
    "quad": 1.0 / (1.0 + 2.0 * (math.sqrt(2.0) - 1.0)),   # rho/r = 2(sqrt2-1)
    "sept": 0.525,                                         # rho/r ~ (3-2f)/f, f = 1.0327
    "tri": 1.0 / (1.0 + (math.sqrt(7.0) - 2.0)),           # rho/r = sqrt7 - 2 (App. E)
}


def p_from_eps(tiling, eps):
    """Highest expansion power p for a requested tolerance eps."""
    k = KAPPA[tiling]
    return max(1, int(math.ceil(math.log(eps) / math.log(k))) - 1)


def tri_root_inradius():
    """Inradius of the level-0 upright triangle (frame units)."""
    return (SQRT3 + 1.0) / 4.0 * (1.0 + 2.0 ** -20)


_MIN_NORM = {}


def sept_min_outside_norm(L):
    """Smallest norm a^2+ab+b^2 of an Eisenstein integer a + b*w
    (w = e^{i pi/3}) whose GBT expansion has more than L digits (brute
    force over the window |a|, |b| <= R, a block of rows at a time)."""
    from .tiling_sept import eisenstein_digit_count

    if L in _MIN_NORM:
        return _MIN_NORM[L]
    R = int(0.6 * 7.0 ** (L / 2.0)) + 4
    bs = np.arange(-R, R + 1, dtype=np.int64)
    best = None
    step = max(1, (1 << 21) // (2 * R + 1))
    for a0 in range(-R, R + 1, step):
        a, b = np.meshgrid(np.arange(a0, min(R + 1, a0 + step), dtype=np.int64), bs, indexing="ij")
        a = a.ravel()
        b = b.ravel()
        norm = a * a + a * b + b * b
        outside = eisenstein_digit_count(a, b, L) > L
        if outside.any():
            m = int(norm[outside].min())
            best = m if best is None else min(best, m)
    _MIN_NORM[L] = best
    return best


# Levels whose minimal outside norm is enumerated; deeper septree levels use
# a lower bound (below).
SEPT_ENUM_LEVELS = 9


def sept_root_norm_bound(L):
    """sqrt(m_L) for L <= SEPT_ENUM_LEVELS, else a lower bound of it.  If z
    lies outside the (L+1)-digit region and d is its last digit (z = d mod
    beta), then (z - unit_d) / beta lies outside the L-digit region, whence
    |z| >= |beta| sqrt(m_L) - 1 = sqrt7 sqrt(m_L) - 1; 1e-9 is taken off per
    step so that rounding cannot lift the bound above the true value."""
    if L <= SEPT_ENUM_LEVELS:
        return math.sqrt(float(sept_min_outside_norm(L)))
    m = math.sqrt(float(sept_min_outside_norm(SEPT_ENUM_LEVELS)))
    for _ in range(SEPT_ENUM_LEVELS, L):
        m = math.sqrt(7.0) * m - 1.0 - 1e-9
    return m


def sept_leaf_circumradius(L):
    """Leaf hexagon circumradius r_L (frame units), rounded up to 2^-40:
    every point of the disc of radius sqrt(1/2) lies within r of a lattice
    point of norm below m_L (inside the region) when
    sqrt(1/2) + r <= r sqrt3 sqrt(m_L)."""
    m = sept_root_norm_bound(L)
    raw = math.sqrt(0.5) / (SQRT3 * m - 1.0)
    return math.ceil(raw * 2.0 ** 40) / 2.0 ** 40


def leaf_area(tiling, L):
    """Area of one leaf cell in frame units (domain square has area 1)."""
    if tiling == "quad":
        return 4.0 ** -L
    if tiling == "tri":
        rho0 = tri_root_inradius()
        return 3.0 * SQRT3 * rho0 * rho0 / 4.0 ** L
    r = sept_leaf_circumradius(L)
    return 1.5 * SQRT3 * r * r


def auto_levels(tiling, n_points, leaf_target=64):
    """Smallest leaf level L whose expected mean points per occupied leaf of
    a uniform input does not exceed ``leaf_target`` (the paper fixes no
    deepest level; 15 levels serve up to 64 * 4^15 points, the septree stops
    at the 8 levels whose leaf radius the tests enumerate)."""
    top = {"quad": 15, "tri": 15, "sept": 8}[tiling]
    for L in range(1, top + 1):
        if n_points * leaf_area(tiling, L) <= leaf_target:
            return L
    return top


# Table 2: M2L cells (P4) and near cells (P2) of an interior cell, and the
# branching factor of each tiling.
P4 = {"quad": 27, "sept": 42, "tri": 39}
P2 = {"quad": 9, "sept": 7, "tri": 13}
BRANCH = {"quad": 4, "sept": 7, "tri": 4}


def app_cost(tiling, p, n_src, n_tgt, s):
    """The part of the FMM cost of App. A-C (eqs. 16, 18, 20) that depends on
    the points per cell s, for K = N / s leaves: the M2L work
    K b/(b - 1) (P4 + 2) p^2 and the direct work M P2 s."""
    b = BRANCH[tiling]
    return (n_src / s) * b / (b - 1) * (P4[tiling] + 2) * p * p + n_tgt * P2[tiling] * s


def s_opt(tiling, p, n_src, n_tgt):
    """S_opt of Table 2: the s minimising ``app_cost``,
    p sqrt(b/(b - 1) (P4 + 2) N / (P2 M))."""
    b = BRANCH[tiling]
    return p * math.sqrt(b / (b - 1) * (P4[tiling] + 2) * n_src / (P2[tiling] * n_tgt))


def sopt_levels(tiling, n_src, n_tgt, p):
    """Leaf level whose expected sources per leaf of a uniform input,
    s_L = N leaf_area(L), give the smallest ``app_cost`` (the discrete
    counterpart of S_opt), over the levels ``auto_levels`` may choose."""
    top = {"quad": 15, "tri": 15, "sept": 8}[tiling]
    n_src = max(1, n_src)
    n_tgt = max(1, n_tgt)
    best, best_l = None, 1
    for L in range(1, top + 1):
        c = app_cost(tiling, p, n_src, n_tgt, n_src * leaf_area(tiling, L))
        if best is None or c < best:
            best, best_l = c, L
    return best_l
