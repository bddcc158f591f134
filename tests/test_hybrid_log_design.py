"""Design check of the hybrid form's pair logarithm, on the CPU.

The hybrid P2P forms log2 r^2 for r^2 = rh + rl (two floats) as the exact
exponent e of rh plus a float-float log2 of its mantissa m in [1, 2): Tang's
table method with 128 reciprocals r_j ~ 1/m (f = m r_j - 1, |f| <= 2^-8),
-log2 r_j stored as hi + lo floats, a degree-4 series for ln(1 + f) and the
first-order term rl / rh.  This test runs that arithmetic in numpy float32
(FMA = exact product and one rounding) and checks the error bound the kernel
relies on, against the float64 log2 of rh + rl: below 2^-29 absolute (the
per-pair error the hybrid form's accuracy rests on), and not a plain float32
log2 (which is off by up to ~2^-23 |log2 r^2|).
"""
import numpy as np

F32 = np.float32


def fmaf(a, b, c):
    """fma in float32: the exact product and sum in float64, one rounding
    (exact here: the operands have 24-bit significands and the sums stay
    well inside 53 bits)."""
    return F32(np.float64(a) * np.float64(b) + np.float64(c))


def table():
    j = np.arange(128)
    c = (1.0 + (2.0 * j + 1.0) / 256.0).astype(np.float32)   # exactly representable
    r = (1.0 / c.astype(np.float64)).astype(np.float32)      # correctly rounded reciprocal
    lg = -np.log2(r.astype(np.float64))
    hi = lg.astype(np.float32)
    lo = (lg - hi.astype(np.float64)).astype(np.float32)
    return r, hi, lo


def log2_ff(rh, rl, tab):
    r_t, hi_t, lo_t = tab
    b = rh.view(np.int32)
    j = (b >> 16) & 127
    m = ((b & 0x007FFFFF) | 0x3F800000).astype(np.int32).view(np.float32)
    e = ((b >> 23) - 127).astype(np.float32)
    r = r_t[j]
    f = fmaf(m, r, F32(-1.0))
    q = fmaf(f, F32(-0.25), F32(1.0 / 3.0))
    q = fmaf(q, f, F32(-0.5))
    q = fmaf(q, f, F32(1.0))
    q = F32(q * f)
    corr = F32(rl / rh)
    ll = fmaf(F32(q + corr), F32(1.4426950408889634), lo_t[j])
    return e, hi_t[j], ll


def test_table_log2_error_bound():
    rs = np.random.default_rng(7)
    n = 200000
    # r^2 over 60 binades (distances from ~1e-9 to ~1e0 of a leaf), plus a lo part
    rh = np.exp2(rs.uniform(-60.0, 2.0, n)).astype(np.float32)
    ulp = np.spacing(rh).astype(np.float64)
    rl = (rs.uniform(-0.5, 0.5, n) * ulp).astype(np.float32)
    e, lh, ll = log2_ff(rh, rl, table())
    got = e.astype(np.float64) + lh.astype(np.float64) + ll.astype(np.float64)
    want = np.log2(rh.astype(np.float64) + rl.astype(np.float64))
    err = np.abs(got - want)
    assert err.max() < 2.0 ** -29
    # the parts the kernel multiplies by the strength: e exact, lh one table
    # value, |ll| small, so the products uh e and uh lh can be made exact
    assert np.all(e == np.floor(e)) and np.all(np.abs(ll) < 2.0 ** -6)
    # a plain FP32 log2 of rh is far less accurate at large |log2 r^2|
    plain = np.log2(rh).astype(np.float32).astype(np.float64)
    assert np.abs(plain - want).max() > 64 * err.max()
