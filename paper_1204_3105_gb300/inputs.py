"""Seeded synthetic inputs for the 2D FMM (no FMM arithmetic lives here).

Shared by the tests, the bench and the oracle-side checks; everything is drawn
with numpy's PCG64 generator so that every consumer sees the same bytes.

* ``uniform_square``: points uniform in the unit square, strengths
  uniform in [-1, 1] (the uniform workloads of the experiments, Sec. 9).
* ``gaussian_mixture``: isotropic Gaussian clusters with centres uniform in
  the unit square and sigma log-uniform, for clustered inputs.
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
