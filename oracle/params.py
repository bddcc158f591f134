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


def sept_min_outside_norm(L):
    """Smallest norm a^2+ab+b^2 of an Eisenstein integer a + b*w
    (w = e^{i pi/3}) whose GBT expansion has more than L digits."""
    from .tiling_sept import eisenstein_digit_count

    R = int(0.6 * 7.0 ** (L / 2.0)) + 4
    a, b = np.meshgrid(np.arange(-R, R + 1, dtype=np.int64),
                       np.arange(-R, R + 1, dtype=np.int64), indexing="ij")
    a = a.ravel()
    b = b.ravel()
    norm = a * a + a * b + b * b
    outside = eisenstein_digit_count(a, b, L) > L
    return int(norm[outside].min())


def sept_leaf_circumradius(L):
    """Leaf hexagon circumradius r_L (frame units), rounded up to 2^-40."""
    m = math.sqrt(float(sept_min_outside_norm(L)))
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
