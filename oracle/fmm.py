"""Plain FP64 hierarchical FMM for the complex log kernel (Sec. 2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper omits the expansion and translation operators and refers to the
Greengard-Rokhlin operators for the 2D Coulomb kernel (Sec. 2; the error
bounds of Sec. 8 are stated for them).  They are restated here from the
series log(z - x) = log(z - c) - sum_k ((x - c)/(z - c))^k / k:

* P2M  about c:   Q = sum u_i,  a_k = -sum u_i (x_i - c)^k / k        (k = 1..p)
           phi(z) ~ Q log(z - c) + sum_k a_k (z - c)^-k
* M2M  child centre c -> parent centre c', z0 = c - c':
           A_l = -Q z0^l / l + sum_{k=1..l} a_k z0^(l-k) C(l-1, k-1)
* M2L  source centre c_s -> target centre c_t, z0 = c_s - c_t:
           b_0 = Q log(-z0) + sum_k a_k (-1)^k z0^-k
           b_l = -Q / (l z0^l) + z0^-l sum_k a_k z0^-k C(l+k-1, k-1) (-1)^k
           phi(z) ~ sum_{l=0..p} b_l (z - c_t)^l
* L2L  parent centre c' -> child centre c'', w = c'' - c' (exact, Sec. 8):
           b'_k = sum_{l=k..p} b_l C(l, k) w^(l-k)
* L2P      Re sum_l b_l (y - c)^l
* P2P      sum over the source points of {leaf} u Neighbors(leaf) of
           u_i log|y - x_i|, skipping a source equal to the target.

Field (optional).  The complex potential of eq. 1 is analytic in y away from
the sources and its derivative, F(y) = sum_i u_i / (y - x_i), is single
valued (the branch of the logarithm only shifts the constant b_0).  The
gradient of Re Phi is (Re F, -Im F).  The FMM gives it by differentiating the
two expansions a target meets:
* L2P'     sum_{l>=1} l b_l (y - c)^(l-1)
* P2P'     sum over the same near sources of u_i / (y - x_i), coincident
           pairs skipped.

Algorithm order (Sec. 2 / App. A cost terms): key every point with the
tiling's CellIndex, stable-sort by key, collect the occupied cells of every
level, build Near (leaf level) and NeighborsE4 lists (eq. 3), upward pass
(P2M, M2M), downward pass (M2L, L2L), L2P and P2P at the leaves, then undo
the sort.  Only occupied cells take part.  Only Re Phi is returned.
"""
import math
from functools import lru_cache

import numpy as np

from .tiling_quad import Quadtree
from .tiling_sept import Septree
from .tiling_tri import TriQuadtree


def make_tiling(name, L, domain=(0.0, 0.0, 1.0)):
    return {"quad": Quadtree, "sept": Septree, "tri": TriQuadtree}[name](L, domain)


@lru_cache(maxsize=None)
def _binom(n, k):
    return float(math.comb(n, k))


@lru_cache(maxsize=None)
def _m2l_binom(p):
    C = np.zeros((p + 1, p))
    for l in range(p + 1):
        for k in range(1, p + 1):
            C[l, k - 1] = _binom(l + k - 1, k - 1) * (-1.0) ** k
    return C


@lru_cache(maxsize=None)
def _l2l_binom(p):
    C = np.zeros((p + 1, p + 1))
    for k in range(p + 1):
        for l in range(k, p + 1):
            C[k, l] = _binom(l, k)
    return C


@lru_cache(maxsize=None)
def _m2m_binom(p):
    C = np.zeros((p, p))
    for l in range(1, p + 1):
        for k in range(1, l + 1):
            C[l - 1, k - 1] = _binom(l - 1, k - 1)
    return C


def p2m(xs, us, c, p):
    """Multipole (Q, a_1..a_p) of sources xs (complex) with strengths us about c."""
    d = xs - c
    Q = float(np.sum(us))
    a = np.zeros(p, complex)
    pw = us.astype(complex)
    for k in range(1, p + 1):
        pw = pw * d
        a[k - 1] = -np.sum(pw) / k
    return Q, a


def m2m(Q, a, z0, p):
    """Shift a multipole by z0 = (old centre) - (new centre)."""
    l = np.arange(1, p + 1)
    zp = z0 ** np.arange(0, p + 1)
    out = -Q * zp[1:] / l
    C = _m2m_binom(p)
    for li in range(1, p + 1):
        k = np.arange(1, li + 1)
        out[li - 1] += np.sum(a[k - 1] * zp[li - k] * C[li - 1, k - 1])
    return out


def m2l(Q, a, z0, p):
    """Local coefficients b_0..b_p about the target centre from a multipole
    about a source centre at offset z0 = c_s - c_t."""
    inv = 1.0 / z0
    ipw = inv ** np.arange(0, 2 * p + 1)
    l = np.arange(0, p + 1)[:, None]
    k = np.arange(1, p + 1)[None, :]
    T = _m2l_binom(p) * ipw[l + k]
    b = T @ a
    b[0] += Q * np.log(-z0)
    lv = np.arange(1, p + 1)
    b[1:] += -Q * ipw[1:p + 1] / lv
    return b


def l2l(b, w, p):
    """Shift a local expansion to a new centre at offset w."""
    wp = w ** np.arange(0, p + 1)
    C = _l2l_binom(p)
    out = np.zeros(p + 1, complex)
    for k in range(p + 1):
        out[k] = np.sum(b[k:] * C[k, k:] * wp[: p + 1 - k])
    return out


def l2p(b, ys, c):
    """Re sum_l b_l (y - c)^l at the complex points ys (Horner)."""
    d = ys - c
    acc = np.zeros(ys.shape, complex) + b[-1]
    for l in range(len(b) - 2, -1, -1):
        acc = acc * d + b[l]
    return acc.real


def l2p_field(b, ys, c):
    """d/dy of sum_l b_l (y - c)^l, i.e. sum_{l>=1} l b_l (y - c)^(l-1) (Horner)."""
    d = ys - c
    p = len(b) - 1
    acc = np.zeros(ys.shape, complex) + p * b[p]
    for l in range(p - 1, 0, -1):
        acc = acc * d + l * b[l]
    return acc


def p2p_field(src_xy, us, tgt_xy):
    """sum_i u_i / (y - x_i) over the given sources, coincident pairs skipped."""
    dz = (tgt_xy[:, 0][:, None] - src_xy[:, 0][None, :]) + \
        1j * (tgt_xy[:, 1][:, None] - src_xy[:, 1][None, :])
    same = dz == 0
    dz[same] = 1.0
    return np.where(same, 0.0, us[None, :] / dz).sum(axis=1)


def p2p(src_xy, us, tgt_xy):
    """sum_i u_i log|y - x_i| over the given sources, coincident pairs skipped."""
    dx = tgt_xy[:, 0][:, None] - src_xy[:, 0][None, :]
    dy = tgt_xy[:, 1][:, None] - src_xy[:, 1][None, :]
    same = (dx == 0) & (dy == 0)
    r = np.hypot(dx, dy)
    r[same] = 1.0
    return (us[None, :] * np.log(r)).sum(axis=1)


class FMMResult:
    pass


def fmm(tiling, src_xy, u, tgt_xy, p, record=False, field=False):
    """Evaluate Re Phi_j (eq. 2) at every target with a p-term FMM over
    ``tiling`` (a Quadtree, Septree or TriQuadtree with leaf level L).

    Returns an ``FMMResult`` with ``phi`` (original target order) and, when
    ``record`` is set, every intermediate: keys, sort permutations, cells per
    level, lists, multipoles, locals and the near / far parts of phi.  With
    ``field`` it also holds ``field``, F_j = sum_i u_i / (y_j - x_i) from the
    differentiated L2P and P2P (and, with ``record``, its near / far parts)."""
    src_xy = np.asarray(src_xy, np.float64).reshape(-1, 2)
    tgt_xy = np.asarray(tgt_xy, np.float64).reshape(-1, 2)
    u = np.asarray(u, np.float64)
    L, b = tiling.L, tiling.b
    res = FMMResult()

    # 1-2. CellIndex of every point, stable sort by key.
    skey = tiling.keys(src_xy[:, 0], src_xy[:, 1]) if len(src_xy) else np.zeros(0, np.int64)
    tkey = tiling.keys(tgt_xy[:, 0], tgt_xy[:, 1]) if len(tgt_xy) else np.zeros(0, np.int64)
    sperm = np.argsort(skey, kind="stable")
    tperm = np.argsort(tkey, kind="stable")
    skey_s, tkey_s = skey[sperm], tkey[tperm]
    xs = src_xy[sperm]
    us = u[sperm]
    ys = tgt_xy[tperm]
    zs = xs[:, 0] + 1j * xs[:, 1]
    zt = ys[:, 0] + 1j * ys[:, 1]

    # 3. Occupied cells of every level (a cell is occupied by sources or targets).
    src_leaf = {}
    for k in np.unique(skey_s):
        lo, hi = np.searchsorted(skey_s, k), np.searchsorted(skey_s, k, side="right")
        src_leaf[int(k)] = (lo, hi)
    tgt_leaf = {}
    for k in np.unique(tkey_s):
        lo, hi = np.searchsorted(tkey_s, k), np.searchsorted(tkey_s, k, side="right")
        tgt_leaf[int(k)] = (lo, hi)
    cells = {L: sorted(set(src_leaf) | set(tgt_leaf))}
    has_src = {L: set(src_leaf)}
    for l in range(L - 1, -1, -1):
        cells[l] = sorted({c // b for c in cells[l + 1]})
        has_src[l] = {c // b for c in has_src[l + 1]}
    occupied = {l: set(cells[l]) for l in cells}

    # 4. Lists: Near at the leaves, NeighborsE4 on levels >= l_min; both occupied.
    near = {n: [m for m in tiling.near(n, L) if m in src_leaf] for n in cells[L] if n in tgt_leaf}
    far = {}
    for l in range(tiling.l_min, L + 1):
        for n in cells[l]:
            far[(l, n)] = [m for m in tiling.far(n, l) if m in has_src[l]]

    centers = {}

    def C(l, n):
        key = (l, n)
        if key not in centers:
            centers[key] = tiling.center(n, l)
        return centers[key]

    # 5. P2M at the leaves.
    mult = {}
    for n, (lo, hi) in src_leaf.items():
        mult[(L, n)] = p2m(zs[lo:hi], us[lo:hi], C(L, n), p)
    # 6. M2M up to l_min.
    for l in range(L - 1, tiling.l_min - 1, -1):
        for n in has_src[l]:
            Qp, ap = 0.0, np.zeros(p, complex)
            cp = C(l, n)
            for ch in range(b * n, b * n + b):
                if (l + 1, ch) in mult:
                    Qc, ac = mult[(l + 1, ch)]
                    Qp += Qc
                    ap = ap + m2m(Qc, ac, C(l + 1, ch) - cp, p)
            mult[(l, n)] = (Qp, ap)

    # 7-8. M2L on every level, L2L from l_min down to the leaves.
    loc = {}
    for l in range(tiling.l_min, L + 1):
        for n in cells[l]:
            ct = C(l, n)
            acc = np.zeros(p + 1, complex)
            if l > tiling.l_min:
                par = n // b
                acc = acc + l2l(loc[(l - 1, par)], ct - C(l - 1, par), p)
            for m in far[(l, n)]:
                Qs, a_s = mult[(l, m)]
                acc = acc + m2l(Qs, a_s, C(l, m) - ct, p)
            loc[(l, n)] = acc

    # 9-10. L2P and P2P at the leaves.
    phi_far = np.zeros(len(zt))
    phi_near = np.zeros(len(zt))
    f_far = np.zeros(len(zt), complex)
    f_near = np.zeros(len(zt), complex)
    for n, (lo, hi) in tgt_leaf.items():
        phi_far[lo:hi] = l2p(loc[(L, n)], zt[lo:hi], C(L, n))
        if field:
            f_far[lo:hi] = l2p_field(loc[(L, n)], zt[lo:hi], C(L, n))
        parts = [np.arange(*src_leaf[m]) for m in near[n]]
        if parts:
            idx = np.concatenate(parts)
            phi_near[lo:hi] = p2p(xs[idx], us[idx], ys[lo:hi])
            if field:
                f_near[lo:hi] = p2p_field(xs[idx], us[idx], ys[lo:hi])

    # 11. Undo the sort.
    phi = np.zeros(len(zt))
    phi[tperm] = phi_far + phi_near
    res.phi = phi
    if field:
        res.field = np.zeros(len(zt), complex)
        res.field[tperm] = f_far + f_near
    if record:
        res.src_keys, res.tgt_keys = skey, tkey
        res.src_perm, res.tgt_perm = sperm, tperm
        res.cells = cells
        res.has_src = has_src
        res.near = near
        res.far = far
        res.mult = mult
        res.loc = loc
        res.centers = centers
        far_o = np.zeros(len(zt))
        near_o = np.zeros(len(zt))
        far_o[tperm] = phi_far
        near_o[tperm] = phi_near
        res.phi_far, res.phi_near = far_o, near_o
        if field:
            res.field_far = np.zeros(len(zt), complex)
            res.field_near = np.zeros(len(zt), complex)
            res.field_far[tperm] = f_far
            res.field_near[tperm] = f_near
    return res
