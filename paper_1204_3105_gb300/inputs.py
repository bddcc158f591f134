"""Seeded synthetic inputs for the 2D FMM (no FMM arithmetic lives here).

Shared by the tests, the bench and the oracle-side checks; everything is drawn
with numpy's PCG64 generator so that every consumer sees the same bytes.

* ``uniform_square``: points uniform in the unit square, strengths
  uniform in [-1, 1] (the uniform workloads of the experiments, Sec. 9).
* ``gaussian_mixture``: isotropic Gaussian clusters with centres uniform in
  the unit square and sigma log-uniform, for clustered inputs.
* ``polygon_points``: a fixed number of uniform points in each of a set of
  regular polygons by the point picking of the experiments (Sec. 9): the
  polygon is cut into one isosceles triangle per edge, each triangle's two
  halves are rearranged into a rectangle, a point is drawn uniformly in the
  rectangle and a third uniform variable picks the triangle.  The polygons
  (the tiles to fill) are the caller's.
"""
import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def uniform_square(n, seed, dtype=np.float64):
    """(xy[n, 2], u[n]) with xy uniform in [0, 1)^2 and u uniform in [-1, 1]."""
    g = rng(seed)
    xy = g.random((n, 2)).astype(dtype)
    # rounding to a narrower type can turn a value just below 1 into 1.0
    xy = np.minimum(xy, np.nextafter(dtype(1.0), dtype(0.0)))
    u = g.uniform(-1.0, 1.0, n).astype(dtype)
    return xy, u


def gaussian_mixture(n, seed, k=32, sigma=(1e-3, 1e-1), dtype=np.float64, clip=True):
    """(xy[n, 2], u[n]): k equal-weight isotropic Gaussian clusters, centres
    uniform in [0, 1)^2, sigma log-uniform in ``sigma``; strengths N(0, 1).
    With ``clip`` the points are folded back into [0, 1)^2."""
    g = rng(seed)
    c = g.random((k, 2))
    s = np.exp(g.uniform(np.log(sigma[0]), np.log(sigma[1]), k))
    lab = g.integers(0, k, n)
    xy = c[lab] + s[lab, None] * g.standard_normal((n, 2))
    if clip:
        xy = np.mod(xy, 1.0)
        xy[xy >= 1.0] = np.nextafter(1.0, 0.0)
    u = g.standard_normal(n)
    xy = xy.astype(dtype)
    if clip:   # rounding to a narrower type can turn a value just below 1 into 1.0
        xy = np.minimum(xy, np.nextafter(dtype(1.0), dtype(0.0)))
    return xy, u.astype(dtype)


def sample_targets(m, count, seed):
    """Seeded sample of ``count`` distinct target indices out of m."""
    g = rng(seed + 1000)
    count = min(count, m)
    return np.sort(g.choice(m, size=count, replace=False))


def polygon_points(vertices, per_cell, seed, dtype=np.float64):
    """(xy[k * per_cell, 2], u): ``per_cell`` uniform points in each regular
    polygon (row i of ``vertices``: its corners as complex numbers, in order
    around it), strengths uniform in [-1, 1].  For the triangle (c, a, b)
    of centre c and edge ab, with m the edge midpoint, h = m - c and
    e = b - m, a point (x, y) of the unit square maps to c + t h + s e with
    (s, t) = (x, y) below the diagonal and (x - 1, 1 - y) above it: the two
    right halves of the triangle, both area preserving."""
    V = np.asarray(vertices, complex)
    k, n = V.shape
    c = V.mean(axis=1)
    g = rng(seed)
    cell = np.repeat(np.arange(k), per_cell)
    m = len(cell)
    x, y, z = g.random(m), g.random(m), g.random(m)
    edge = np.minimum((z * n).astype(np.int64), n - 1)
    a = V[cell, edge]
    b = V[cell, (edge + 1) % n]
    mid = 0.5 * (a + b)
    h = mid - c[cell]
    e = b - mid
    low = x <= y
    s = np.where(low, x, x - 1.0)
    t = np.where(low, y, 1.0 - y)
    pts = c[cell] + t * h + s * e
    xy = np.column_stack([pts.real, pts.imag]).astype(dtype)
    u = g.uniform(-1.0, 1.0, m).astype(dtype)
    return xy, u
