"""Brute-force evaluation of eq. (2), Sec. 2.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Phi*_j = sum_{i : x_i != y_j} u_i log|y_j - x_i|   (real part of eq. 2; a
source that coincides bitwise with the target is skipped).  Each block of
sources is summed by numpy (pairwise summation) and the block sums are
combined with Neumaier's compensated summation in FP64.
"""
import numpy as np


def direct(src_xy, u, tgt_xy, block=2048, gradient=False):
    """Return Phi*_j for every target (and, with gradient=True, also the
    complex field sum_i u_i / (y_j - x_i))."""
    xs = np.asarray(src_xy, np.float64)
    ys = np.asarray(tgt_xy, np.float64)
    u = np.asarray(u, np.float64)
    sx = xs[:, 0] + 1j * xs[:, 1]
    ty = ys[:, 0] + 1j * ys[:, 1]
    M = ty.shape[0]
    s = np.zeros(M)
    comp = np.zeros(M)
    g = np.zeros(M, complex)
    for i0 in range(0, sx.shape[0], block):
        d = ty[:, None] - sx[None, i0:i0 + block]
        same = (ys[:, 0][:, None] == xs[i0:i0 + block, 0][None, :]) & \
               (ys[:, 1][:, None] == xs[i0:i0 + block, 1][None, :])
        ad = np.abs(d)
        ad[same] = 1.0
        part = (u[None, i0:i0 + block] * np.log(ad)).sum(axis=1)
        # Neumaier step
        t = s + part
        big = np.abs(s) >= np.abs(part)
        comp += np.where(big, (s - t) + part, (part - t) + s)
        s = t
        if gradient:
            d[same] = np.inf
            g += (u[None, i0:i0 + block] / d).sum(axis=1)
    phi = s + comp
    return (phi, g) if gradient else phi


def rel_inf_error(phi, ref):
    """eps_rel_inf = max_j |phi_j - ref_j| / max_j |ref_j|."""
    phi = np.asarray(phi, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(phi - ref)) / np.max(np.abs(ref)))
