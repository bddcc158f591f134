"""Pins of the oracle's field F_j = sum_i u_i / (y_j - x_i), the derivative of
the complex potential of eq. 1 (Sec. 2), whose real-part gradient is
(Re F, -Im F).

* the direct field of ``oracle/direct.py`` against the closed form of one
  source, and against central finite differences of the direct Re Phi (a
  quantity pinned on its own), so that a conjugate, a sign or a dropped
  strength shows;
* each differentiated operator against a finite difference of the operator
  it differentiates (L2P', M2P'), with the single-source closed form;
* the whole oracle FMM field (uniform and adaptive trees, every tiling)
  against the direct field, converging geometrically in p.
"""
import numpy as np
import pytest

from oracle import adaptive as A
from oracle import fmm as F
from oracle.adaptive import adaptive_fmm
from oracle.direct import direct, rel_inf_error
from oracle.fmm import fmm, make_tiling
from paper_1204_3105_gb300.inputs import gaussian_mixture, uniform_square


def _fd_grad(src, u, y, h):
    """Fourth-order central differences of the direct Re Phi at the points y."""
    def phi(dx, dy):
        return direct(src, u, y + np.array([dx, dy]))
    gx = (-phi(2 * h, 0) + 8 * phi(h, 0) - 8 * phi(-h, 0) + phi(-2 * h, 0)) / (12 * h)
    gy = (-phi(0, 2 * h) + 8 * phi(0, h) - 8 * phi(0, -h) + phi(0, -2 * h)) / (12 * h)
    return gx, gy


def test_direct_field_single_source_closed_form():
    rng = np.random.default_rng(3)
    x = np.array([[0.3, 0.7]])
    for u in (1.0, -2.5):
        y = rng.random((50, 2))
        _, g = direct(x, [u], y, gradient=True)
        want = u / ((y[:, 0] - x[0, 0]) + 1j * (y[:, 1] - x[0, 1]))
        assert np.max(np.abs(g - want)) <= 1e-14 * np.max(np.abs(want))
    # a target on the source: the pair is skipped
    _, g = direct(x, [1.0], x, gradient=True)
    assert g[0] == 0


def test_direct_field_is_gradient_of_potential():
    """grad Re Phi = (Re F, -Im F), checked by fourth-order finite
    differences at targets at least 0.05 from every source."""
    rng = np.random.default_rng(4)
    src = rng.random((300, 2))
    u = rng.uniform(-1, 1, 300)
    y = rng.random((400, 2))
    dmin = np.min(np.hypot(y[:, None, 0] - src[None, :, 0], y[:, None, 1] - src[None, :, 1]), axis=1)
    y = y[dmin > 0.05]
    _, g = direct(src, u, y, gradient=True)
    gx, gy = _fd_grad(src, u, y, 1e-3)
    scale = np.max(np.abs(g))
    assert np.max(np.abs(gx - g.real)) <= 1e-6 * scale
    assert np.max(np.abs(gy + g.imag)) <= 1e-6 * scale


def test_l2p_field_is_derivative_of_l2p():
    """L2P' of a local expansion is the derivative of the (complex) L2P
    series: compared with central differences of the real part along x and
    y (Cauchy-Riemann gives both components)."""
    rng = np.random.default_rng(5)
    c = 0.4 + 0.6j
    for p in (1, 5, 17):
        b = rng.normal(size=p + 1) + 1j * rng.normal(size=p + 1)
        ys = c + 0.3 * (rng.random(40) - 0.5) + 0.3j * (rng.random(40) - 0.5)
        f = F.l2p_field(b, ys, c)
        h = 1e-5
        dx = (F.l2p(b, ys + h, c) - F.l2p(b, ys - h, c)) / (2 * h)
        dy = (F.l2p(b, ys + 1j * h, c) - F.l2p(b, ys - 1j * h, c)) / (2 * h)
        scale = np.max(np.abs(f)) + 1.0
        assert np.max(np.abs(dx - f.real)) <= 1e-7 * scale, p
        assert np.max(np.abs(dy + f.imag)) <= 1e-7 * scale, p


def test_m2p_field_single_source_and_derivative():
    """M2P' of the multipole of one source is the series of 1/(y - x)
    (tail bound of the derivative series), and it is the derivative of M2P."""
    rng = np.random.default_rng(6)
    c = 0.5 + 0.5j
    for p in (6, 14, 24):
        x = c + 0.08 * np.exp(2j * np.pi * rng.random())
        Q, a = F.p2m(np.array([x]), np.array([1.0]), c, p)
        zt = c + 0.3 * np.exp(2j * np.pi * rng.random(30))
        f = A.m2p_field(Q, a, c, zt)
        q = abs(x - c) / 0.3
        tail = q ** (p + 1) * (p + 2) / (1 - q) ** 2 / 0.3   # sum_{k>p} (k+1) q^k / |y - c|
        assert np.max(np.abs(f - 1.0 / (zt - x))) <= tail * (1 + 1e-6) + 1e-13, p
        h = 1e-6
        dx = (A.m2p(Q, a, c, zt + h) - A.m2p(Q, a, c, zt - h)) / (2 * h)
        dy = (A.m2p(Q, a, c, zt + 1j * h) - A.m2p(Q, a, c, zt - 1j * h)) / (2 * h)
        assert np.max(np.abs(dx - f.real)) <= 1e-6 * np.max(np.abs(f))
        assert np.max(np.abs(dy + f.imag)) <= 1e-6 * np.max(np.abs(f))


def test_p2p_field_matches_direct():
    rng = np.random.default_rng(7)
    src = rng.random((64, 2))
    tgt = np.vstack([rng.random((20, 2)), src[:5]])   # five targets on sources
    u = rng.uniform(-1, 1, 64)
    _, g = direct(src, u, tgt, gradient=True)
    assert np.max(np.abs(F.p2p_field(src, u, tgt) - g)) <= 1e-13 * np.max(np.abs(g))


@pytest.mark.parametrize("tiling,L", [("quad", 3), ("sept", 2), ("tri", 3)])
def test_fmm_field_converges_to_direct(tiling, L):
    """The oracle FMM's field approaches the direct field geometrically in p
    (the differentiated series converge at the rate of the potential's, with
    an extra factor p) and reaches round-off at p = 32."""
    xy, u = uniform_square(1500, seed=11)
    tgt = np.vstack([xy[:200], np.random.default_rng(8).random((100, 2))])
    _, g = direct(xy, u, tgt, gradient=True)
    T = make_tiling(tiling, L)
    errs = []
    for p in (8, 16, 32):
        r = fmm(T, xy, u, tgt, p, field=True)
        errs.append(float(np.max(np.abs(r.field - g)) / np.max(np.abs(g))))
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10, errs
    assert errs[2] < 1e-10, errs
    # the potential of the same run is unchanged by the field option
    r0 = fmm(T, xy, u, tgt, 16)
    r1 = fmm(T, xy, u, tgt, 16, field=True)
    assert np.array_equal(r0.phi, r1.phi)


@pytest.mark.parametrize("tiling,L", [("quad", 7), ("sept", 5), ("tri", 7)])
def test_adaptive_field_matches_direct(tiling, L):
    """Clustered input on an adaptive tree: L2P', M2P' (W lists) and P2P'
    together give the direct field."""
    xy, u = gaussian_mixture(1200, seed=12, k=4, sigma=(0.003, 0.05))
    _, g = direct(xy, u, xy, gradient=True)
    r = adaptive_fmm(make_tiling(tiling, L), xy, u, xy, 30, s=16, field=True, record=True)
    assert sum(len(v) for v in r.W.values()) > 0      # M2P' took part
    assert rel_inf_error(r.field.real, g.real) < 1e-9
    assert np.max(np.abs(r.field - g)) / np.max(np.abs(g)) < 1e-9
