"""The regular-polygon point picking of the experiments (Sec. 9) fills each
polygon uniformly: every point lies inside its polygon, each edge triangle
gets its share, and the mean squared distance from the centre is the closed
form R^2 (2 + cos(2 pi / n)) / 6 of a uniform regular n-gon of circumradius R
(a mapping that skipped the rectangle rearrangement, or sampled radii
uniformly, would miss it)."""
import math

import numpy as np
import pytest

from paper_1204_3105_gb300.inputs import polygon_points


def regular(n, R, rot, centre):
    k = np.arange(n)
    return centre + R * np.exp(1j * (rot + 2 * np.pi * k / n))


@pytest.mark.parametrize("n", [3, 4, 6])
def test_polygon_points_uniform(n):
    R = 0.01
    polys = np.array([regular(n, R, 0.3 * i, 0.2 + 0.05 * i + 0.3j) for i in range(4)])
    per = 40000
    xy, u = polygon_points(polys, per, seed=n)
    assert xy.shape == (4 * per, 2) and np.all(np.abs(u) <= 1)
    z = xy[:, 0] + 1j * xy[:, 1]
    for i, P in enumerate(polys):
        q = z[i * per:(i + 1) * per]
        c = P.mean()
        # inside: on the inner side of every edge (counter-clockwise corners)
        for j in range(n):
            a, b = P[j], P[(j + 1) % n]
            cross = ((b - a).conjugate() * (q - a)).imag
            assert np.all(cross >= -1e-15)
        # each edge triangle holds 1/n of the points
        ang = np.angle((q - c) * np.exp(-1j * (np.angle(P[0] - c))))
        sector = np.floor(np.mod(ang, 2 * np.pi) / (2 * np.pi / n)).astype(int)
        frac = np.bincount(sector, minlength=n) / per
        assert np.max(np.abs(frac - 1.0 / n)) < 5 * math.sqrt(1.0 / (n * per))
        # centroid and polar moment of a uniform regular polygon
        assert abs(q.mean() - c) < 5 * R / math.sqrt(per)
        j2 = np.mean(np.abs(q - c) ** 2)
        want = R * R * (2 + math.cos(2 * math.pi / n)) / 6
        assert abs(j2 - want) < 0.02 * want
