"""Design checks, on the CPU, of the float-float arithmetic of the hybrid and
split forms, against exact rational arithmetic.

Values are unevaluated sums hi + lo of two floats.  The M2L accumulates
real x complex products with exact products (TwoProd by FMA), the cross
terms hi*lo into a compensation and every partial sum by TwoSum (the
compensated dot product of Ogita, Rump and Oishi, 2005), and turns results by
float-float complex products; the hybrid P2P forms r^2 from hi + lo
coordinates with a TwoSum difference and FMA squares.  These tests run that
arithmetic in numpy float32 (an FMA = the exact product and sum in float64,
rounded once, exact for the TwoProd residuals used here) and bound its error.
"""
from fractions import Fraction

import numpy as np

F32 = np.float32


def fmaf(a, b, c):
    return F32(np.float64(a) * np.float64(b) + np.float64(c))


def split(x):
    """float64 -> float-float (hi, lo)."""
    hi = F32(x)
    return hi, F32(np.float64(x) - np.float64(hi))


def two_sum_acc(s, comp, x):
    t = F32(s + x)
    bp = F32(t - s)
    ap = F32(t - bp)
    comp = F32(comp + F32(F32(s - ap) + F32(x - bp)))
    return t, comp


def ff_rmac(d, A, c):
    """d += A * c: A real (Ah, Al), c complex (ch.re, ch.im, cl.re, cl.im),
    d = [s.re, c.re, s.im, c.im] (the kernel's ff_rmac)."""
    Ah, Al = A
    out = list(d)
    for part, (chv, clv) in ((0, (c[0], c[2])), (2, (c[1], c[3]))):
        p = F32(Ah * chv)
        e = fmaf(Ah, chv, -p)
        cr = fmaf(Ah, clv, F32(Al * chv))
        s, comp = two_sum_acc(out[part], out[part + 1], p)
        comp = F32(comp + F32(e + cr))
        out[part], out[part + 1] = s, comp
    return out


def ff_cmul(x, y):
    """x * y for complex float-float x, y (hi.re, hi.im, lo.re, lo.im)."""
    res = []
    for sgn, (a, b, a2, b2) in ((-1, (0, 0, 1, 1)), (1, (0, 1, 1, 0))):
        p1 = F32(x[a] * y[b])
        e1 = fmaf(x[a], y[b], -p1)
        p2 = F32(sgn * x[a2] * y[b2])
        e2 = fmaf(F32(sgn * x[a2]), y[b2], -p2)
        s, c = two_sum_acc(p1, F32(0.0), p2)
        cross = fmaf(x[a], y[b + 2], fmaf(x[a + 2], y[b], fmaf(F32(sgn * x[a2]), y[b2 + 2],
                                                                F32(sgn * x[a2 + 2] * y[b2]))))
        c = F32(c + F32(F32(e1 + e2) + cross))
        hi = F32(s + c)
        lo = F32(c - F32(hi - s))
        res.append((hi, lo))
    return (res[0][0], res[1][0], res[0][1], res[1][1])


def exact(v):
    return Fraction(float(v))


def test_compensated_real_complex_dot():
    """Sum_k A_k c_k over 40 terms of mixed signs and magnitudes: within
    2^-40 of the exact sum, relative to sum |A_k c_k| (a plain FP32 sum is
    off by ~2^-24)."""
    rs = np.random.default_rng(3)
    for _ in range(20):
        n = 40
        A = rs.normal(size=n) * np.exp2(rs.integers(-12, 3, n))
        c = (rs.normal(size=n) + 1j * rs.normal(size=n)) * np.exp2(rs.integers(-12, 3, n))
        d = [F32(0.0)] * 4
        ex_re = ex_im = Fraction(0)
        scale = 0.0
        for k in range(n):
            Ah, Al = split(A[k])
            cr, crl = split(c[k].real)
            ci, cil = split(c[k].imag)
            d = ff_rmac(d, (Ah, Al), (cr, ci, crl, cil))
            a_ex = exact(Ah) + exact(Al)
            ex_re += a_ex * (exact(cr) + exact(crl))
            ex_im += a_ex * (exact(ci) + exact(cil))
            scale += abs(A[k] * c[k])
        got_re = exact(d[0]) + exact(d[1])
        got_im = exact(d[2]) + exact(d[3])
        assert abs(float(got_re - ex_re)) <= 2.0 ** -40 * scale
        assert abs(float(got_im - ex_im)) <= 2.0 ** -40 * scale


def test_float_float_complex_product():
    """x * y of two float-float complex numbers: within 2^-44 of the exact
    product of the (hi + lo) inputs, relative to |x| |y|."""
    rs = np.random.default_rng(4)
    for _ in range(200):
        x = rs.normal() + 1j * rs.normal()
        y = np.exp(1j * rs.uniform(0, 2 * np.pi))          # a phase, as in the M2L turns
        xr, xrl = split(x.real)
        xi, xil = split(x.imag)
        yr, yrl = split(y.real)
        yi, yil = split(y.imag)
        z = ff_cmul((xr, xi, xrl, xil), (yr, yi, yrl, yil))
        X = (exact(xr) + exact(xrl), exact(xi) + exact(xil))
        Y = (exact(yr) + exact(yrl), exact(yi) + exact(yil))
        ex_re = X[0] * Y[0] - X[1] * Y[1]
        ex_im = X[0] * Y[1] + X[1] * Y[0]
        mag = abs(x) * abs(y)
        assert abs(float(exact(z[0]) + exact(z[2]) - ex_re)) <= 2.0 ** -44 * mag
        assert abs(float(exact(z[1]) + exact(z[3]) - ex_im)) <= 2.0 ** -44 * mag


def _r2_case(rs, lo_exp, hi_exp):
    t = rs.uniform(-1.5, 1.5, 2)
    return t, t + rs.normal(size=2) * np.exp2(rs.uniform(lo_exp, hi_exp))


def test_float_float_r2():
    """r^2 of a target and a source given as hi + lo coordinates (relative to
    the target leaf's centre), as the hybrid P2P forms it: the accurate
    float-float difference (TwoSum of the hi parts and of the lo parts, the
    first lo error into the hi error, a TwoSum renormalisation, then the
    second lo error), FMA squares, a TwoSum of the squares and one
    renormalisation: within 2^-43 of the exact r^2 of the coordinates at every
    separation, down to points 2^-34 of the coordinate scale apart.  (Without
    the lo-part TwoSum the error grew like |coordinate| / distance and reached
    FP32 level for points ~1e-7 of a leaf apart.)"""
    rs = np.random.default_rng(5)
    for case in range(600):
        t, s = _r2_case(rs, -20, 0) if case < 300 else _r2_case(rs, -34, -20)
        th = [split(v) for v in t]
        sh = [split(-v) for v in s]        # sources are staged negated
        dh, dl = [], []
        for k in range(2):
            s1, s2 = two_sum_acc(th[k][0], F32(0.0), sh[k][0])
            t1, t2 = two_sum_acc(th[k][1], F32(0.0), sh[k][1])
            h, r = two_sum_acc(s1, F32(0.0), F32(s2 + t1))
            dh.append(h)
            dl.append(F32(r + t2))
        qx, qy = F32(dh[0] * dh[0]), F32(dh[1] * dh[1])
        qxe, qye = fmaf(dh[0], dh[0], -qx), fmaf(dh[1], dh[1], -qy)
        h, he = two_sum_acc(qx, F32(0.0), qy)
        lo = F32(F32(qxe + qye) + he)
        lo = fmaf(F32(2.0 * dh[0]), dl[0], lo)
        lo = fmaf(F32(2.0 * dh[1]), dl[1], lo)
        lo = fmaf(dl[0], dl[0], fmaf(dl[1], dl[1], lo))
        tt = F32(h + lo)
        rl = F32(lo - F32(tt - h))
        ex = sum((exact(th[k][0]) + exact(th[k][1]) + exact(sh[k][0]) + exact(sh[k][1])) ** 2
                 for k in range(2))
        if ex == 0:
            continue
        got = exact(tt) + exact(rl)
        assert abs(float(got - ex)) <= 2.0 ** -43 * float(ex)
