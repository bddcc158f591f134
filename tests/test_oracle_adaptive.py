"""Pins of the oracle's adaptive FMM (clustered input): the cross-level
operators against closed forms, the refinement rule, exact-once coverage of
every (target, source) pair by brute force, the reduction to the uniform
oracle when every cell is split to the finest level, and the error against
the direct sum on clustered points."""
import math

import numpy as np
import pytest

from oracle import adaptive as A
from oracle import fmm as F
from oracle.direct import direct, rel_inf_error
from oracle.params import p_from_eps
from paper_1204_3105_gb300.inputs import gaussian_mixture, uniform_square


def _tail(q, p):
    return q ** (p + 1) / ((p + 1) * (1 - q))


def test_m2p_single_source_within_series_tail():
    """M2P of one unit source is the series of log(y - x) about c; the error
    is the series tail in |x - c| / |y - c|."""
    rng = np.random.default_rng(3)
    c = 0.4 - 0.1j
    for p in (3, 8, 16):
        for _ in range(20):
            x = c + 0.1 * rng.random() * np.exp(2j * np.pi * rng.random())
            y = c + (0.3 + 0.2 * rng.random()) * np.exp(2j * np.pi * rng.random())
            Q, a = F.p2m(np.array([x]), np.array([1.0]), c, p)
            v = A.m2p(Q, a, c, np.array([y]))[0]
            err = abs(v - math.log(abs(y - x)))
            assert err <= _tail(abs(x - c) / abs(y - c), p) * (1 + 1e-9) + 1e-15


def test_p2l_single_source_within_series_tail():
    """P2L of one unit source at x about c, evaluated at y near c, is the
    series of log(y - x) = log(c - x) + log(1 - (y - c)/(x - c))."""
    rng = np.random.default_rng(4)
    c = -0.2 + 0.3j
    for p in (3, 8, 16):
        for _ in range(20):
            x = c + (0.3 + 0.2 * rng.random()) * np.exp(2j * np.pi * rng.random())
            y = c + 0.1 * rng.random() * np.exp(2j * np.pi * rng.random())
            b = A.p2l(np.array([x]), np.array([1.0]), c, p)
            v = F.l2p(b, np.array([y]), c)[0]
            err = abs(v - math.log(abs(y - x)))
            assert err <= _tail(abs(y - c) / abs(x - c), p) * (1 + 1e-9) + 1e-15


def _clustered(n, seed):
    xy, u = gaussian_mixture(n, seed=seed, k=6, sigma=(3e-3, 5e-2))
    return xy, u


@pytest.mark.parametrize("name,L", [("quad", 7), ("sept", 4), ("tri", 7)])
def test_refinement_rule(name, L):
    xy, u = _clustered(1500, seed=11)
    r = A.adaptive_fmm(F.make_tiling(name, L), xy, u, xy, 4, s=20, record=True)
    depth = set()
    for l, cells in enumerate(r.cells):
        for n in cells:
            cnt = max(r.src_r[l].get(n, (0, 0))[1] - r.src_r[l].get(n, (0, 0))[0],
                      r.tgt_r[l].get(n, (0, 0))[1] - r.tgt_r[l].get(n, (0, 0))[0])
            if (l, n) in r.split:
                assert cnt > 20 and l < L
            else:
                assert cnt <= 20 or l == L
                depth.add(l)
    assert len(depth) >= 3          # clustered input: leaves on several levels


@pytest.mark.parametrize("name,L", [("quad", 6), ("sept", 4), ("tri", 6)])
def test_every_pair_covered_exactly_once(name, L):
    """Brute force over all (target, source) pairs: U, W, X and the M2L lists
    of every level together cover each pair once and only once."""
    xy, u = _clustered(700, seed=12)
    txy, _ = _clustered(500, seed=13)
    r = A.adaptive_fmm(F.make_tiling(name, L), xy, u, txy, 3, s=12, record=True)
    cnt = np.zeros((len(txy), len(xy)), np.int32)
    kinds = {"U": 0, "W": 0, "X": 0, "V": 0}
    for key, lst in (("U", r.U), ("W", r.W), ("X", r.X)):
        for (la, a), srcs in lst.items():
            t0, t1 = r.tgt_r[la][a]
            for (lc, c) in srcs:
                s0, s1 = r.src_r[lc][c]
                cnt[t0:t1, s0:s1] += 1
                kinds[key] += 1
    for (l, a), srcs in r.V.items():
        t0, t1 = r.tgt_r[l][a]
        for c in srcs:
            s0, s1 = r.src_r[l][c]
            cnt[t0:t1, s0:s1] += 1
            kinds["V"] += 1
    assert cnt.min() == 1 and cnt.max() == 1
    assert min(kinds.values()) > 0, kinds      # all four interaction kinds occur


@pytest.mark.parametrize("name,L", [("quad", 4), ("sept", 3), ("tri", 4)])
def test_split_everything_reduces_to_uniform(name, L):
    """With s = 0 every occupied cell is split down to level L: the adaptive
    tree is the uniform one and the result equals the uniform oracle."""
    xy, u = uniform_square(900, seed=14)
    T = F.make_tiling(name, L)
    a = A.adaptive_fmm(T, xy, u, xy, 8, s=0).phi
    b = F.fmm(T, xy, u, xy, 8).phi
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


@pytest.mark.parametrize("name,L", [("quad", 8), ("sept", 5), ("tri", 8)])
def test_clustered_error_vs_direct(name, L):
    xy, u = _clustered(3000, seed=15)
    p = p_from_eps(name, 1e-6)
    phi = A.adaptive_fmm(F.make_tiling(name, L), xy, u, xy, p, s=32).phi
    ref = direct(xy, u, xy)
    assert rel_inf_error(phi, ref) < 1e-6
