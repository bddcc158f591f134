"""Pins of the oracle's expansion operators and of the whole oracle FMM
against closed forms, the error bounds of Sec. 8 and brute force."""
import math

import numpy as np
import pytest

from oracle import fmm as F
from oracle.direct import direct, rel_inf_error


def _series_tail(q, p):
    # sum_{k>p} q^k / k <= q^(p+1) / ((p+1)(1-q))
    return q ** (p + 1) / ((p + 1) * (1 - q))


def test_p2m_single_source_is_log_series():
    """The multipole of one unit source at x about c is the series of
    log(z - x) = log(z - c) + log(1 - (x-c)/(z-c)); its truncation error is the
    series tail (eq. 14, A5 reading)."""
    rng = np.random.default_rng(0)
    c = 0.3 + 0.2j
    for p in (4, 10, 20):
        for _ in range(20):
            x = c + 0.1 * np.exp(2j * np.pi * rng.random()) * rng.random()
            z = c + 0.35 * np.exp(2j * np.pi * rng.random())
            Q, a = F.p2m(np.array([x]), np.array([1.0]), c, p)
            approx = Q * np.log(z - c) + np.sum(a / (z - c) ** np.arange(1, p + 1))
            err = abs(approx.real - math.log(abs(z - x)))
            assert err <= _series_tail(abs(x - c) / abs(z - c), p) * (1 + 1e-9) + 1e-15


def _cluster(rng, c, rad, n):
    r = rad * np.sqrt(rng.random(n))
    return c + r * np.exp(2j * np.pi * rng.random(n)), rng.uniform(-1, 1, n)


def test_m2m_then_evaluate_within_bound():
    rng = np.random.default_rng(1)
    cc, cp = 0.55 + 0.45j, 0.5 + 0.5j
    xs, us = _cluster(rng, cc, 0.05, 50)
    z = cp + 0.5 * np.exp(2j * np.pi * rng.random(30))
    exact = np.array([np.sum(us * np.log(np.abs(zz - xs))) for zz in z])
    for p in (6, 12, 24):
        Q, a = F.p2m(xs, us, cc, p)
        A = F.m2m(Q, a, cc - cp, p)
        approx = (Q * np.log(z - cp) + (A[None, :] / (z[:, None] - cp) ** np.arange(1, p + 1)).sum(1)).real
        q = (abs(cc - cp) + 0.05) / 0.5
        bound = np.sum(np.abs(us)) * _series_tail(q, p)
        assert np.max(np.abs(approx - exact)) <= bound + 1e-14 * np.sum(np.abs(us))
    # at large p the shift is exact to round-off
    assert np.max(np.abs(approx - exact)) < 1e-12 * np.sum(np.abs(us))


def test_m2l_within_bound_and_l2l_exact():
    rng = np.random.default_rng(2)
    cs, ct = 0.2 + 0.2j, 0.6 + 0.35j
    rad = 0.1
    xs, us = _cluster(rng, cs, rad, 60)
    ys = ct + rad * np.sqrt(rng.random(40)) * np.exp(2j * np.pi * rng.random(40))
    exact = np.array([np.sum(us * np.log(np.abs(y - xs))) for y in ys])
    D = abs(cs - ct)
    rho_over_r = (D - 2 * rad) / rad
    errs = []
    for p in (4, 8, 16, 32):
        Q, a = F.p2m(xs, us, cs, p)
        b = F.m2l(Q, a, cs - ct, p)
        approx = F.l2p(b, ys, ct)
        err = np.max(np.abs(approx - exact))
        # eq. (15), A5 reading: sum|u| (r/rho) (1/(1+rho/r))^(p+1), with the
        # series constant of the two-expansion product
        kap = 1 / (1 + rho_over_r)
        bound = np.sum(np.abs(us)) * kap ** (p + 1) / (1 - kap) ** 2 * 4
        assert err <= bound + 1e-14 * np.sum(np.abs(us))
        errs.append(err)
    assert errs[-1] < 1e-11 * np.sum(np.abs(us))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    # L2L is exact (Sec. 8): shift b to a nearby centre and evaluate again
    c2 = ct + 0.03 - 0.02j
    b2 = F.l2l(b, c2 - ct, 32)
    y2 = c2 + 0.02 * np.exp(2j * np.pi * rng.random(20))
    assert np.max(np.abs(F.l2p(b2, y2, c2) - F.l2p(b, y2, ct))) < 1e-12 * np.max(np.abs(exact))


def test_m2l_operator_is_real_factor_times_phase():
    """The M2L operator of an offset z0 = |z0| u (the oracle's, i.e. the
    translation of Sec. 2): every entry except the log term of b_0 is a real
    number times u^-(l+k) (column 0 is the Q column, k = 0).  The float-float
    M2L applies it as a rotation of the multipole by u^-k, a real matrix and a
    rotation of the result by u^-l; a sign or index slip in the operator would
    leave a complex factor."""
    rs = np.random.default_rng(11)
    p = 24
    for _ in range(6):
        z0 = complex(rs.uniform(-5, 5), rs.uniform(-5, 5))
        if abs(z0) < 2.5:
            z0 *= 3.0 / abs(z0)
        u = z0 / abs(z0)
        M = np.zeros((p + 1, p + 1), complex)
        b = F.m2l(1.0, np.zeros(p, complex), z0, p)
        b[0] -= np.log(-z0)                       # the log term of b_0 is not translated
        M[:, 0] = b
        for k in range(1, p + 1):
            e = np.zeros(p, complex)
            e[k - 1] = 1.0
            M[:, k] = F.m2l(0.0, e, z0, p)
        lk = np.add.outer(np.arange(p + 1), np.arange(p + 1))
        A = M * u ** lk
        assert np.all(np.abs(A.imag) <= 1e-12 * np.abs(A) + 1e-300)   # entry by entry
        assert abs(M[0, 0]) == 0.0


@pytest.mark.parametrize("name,L", [("quad", 3), ("sept", 3), ("tri", 4)])
def test_fmm_converges_to_direct(name, L):
    rng = np.random.default_rng(4)
    N = 2500
    xy = rng.random((N, 2))
    u = rng.uniform(-1, 1, N)
    ref = direct(xy, u, xy)
    T = F.make_tiling(name, L)
    errs = [rel_inf_error(F.fmm(T, xy, u, xy, p).phi, ref) for p in (4, 8, 16, 32)]
    assert all(e2 < 0.2 * e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-11


def test_fmm_separate_targets_domain_and_edge_cases():
    rng = np.random.default_rng(5)
    dom = (-3.0, 2.0, 4.0)
    src = np.column_stack([dom[0] + dom[2] * rng.random(700), dom[1] + dom[2] * rng.random(700)])
    tgt = np.column_stack([dom[0] + dom[2] * rng.random(333), dom[1] + dom[2] * rng.random(333)])
    tgt[:5] = src[:5]                        # coincident pairs are skipped
    u = rng.normal(size=700)
    ref = direct(src, u, tgt)
    for name, L in (("quad", 3), ("sept", 2), ("tri", 3)):
        T = F.make_tiling(name, L, dom)
        r = F.fmm(T, src, u, tgt, 30, record=True)
        assert rel_inf_error(r.phi, ref) < 1e-11
        assert np.allclose(r.phi_near + r.phi_far, r.phi)
    # one source, one target; no targets
    T = F.make_tiling("quad", 2)
    one = np.array([[0.1, 0.2]])
    two = np.array([[0.9, 0.7]])
    r = F.fmm(T, one, np.array([2.0]), two, 10)
    assert r.phi[0] == pytest.approx(2.0 * math.log(math.hypot(0.8, 0.5)), rel=1e-12)
    r = F.fmm(T, one, np.array([2.0]), np.zeros((0, 2)), 10)
    assert r.phi.shape == (0,)


def test_max_error_grows_with_n_and_quad_is_most_accurate():
    """Qualitative trends of Sec. 9 at p = 12: the max abs error grows with N
    (Fig. 14) and the quadtree is the most accurate tiling at equal p."""
    rng = np.random.default_rng(6)
    errs = {}
    for N in (1000, 4000):
        xy = rng.random((N, 2))
        u = rng.uniform(-1, 1, N)
        ref = direct(xy, u, xy)
        for name, L in (("quad", 3), ("sept", 3), ("tri", 4)):
            ph = F.fmm(F.make_tiling(name, L), xy, u, xy, 12).phi
            errs[(name, N)] = np.max(np.abs(ph - ref))
    for name in ("quad", "sept", "tri"):
        assert errs[(name, 4000)] > errs[(name, 1000)]
    assert errs[("quad", 4000)] < errs[("tri", 4000)]
