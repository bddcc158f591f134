"""Plain FP64 adaptive FMM over the three tilings (clustered input).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's FMM (Sec. 2, App. A-C) refines every cell to one leaf level.  For
clustered points the tilings' own hierarchy is refined locally instead: a
cell is split while it holds more than ``s`` sources or more than ``s``
targets (and is above the finest level), so leaves sit on different levels.
The interaction rule stays the paper's: two cells of one level interact by
M2L when neither is in the other's Near set (Sec. 4-6, eq. 3).  A pair of
cells of different levels appears only next to a leaf, and is resolved with
the two standard cross-level operators of the adaptive Greengard-Rokhlin
scheme:

* M2P (W list): the multipole of a small source cell c, evaluated directly at
  the targets of a larger target leaf a,
      phi(y) += Re[ Q log(y - c) + sum_k a_k (y - c)^-k ];
* P2L (X list): the sources of a larger source leaf c, expanded about the
  centre of a smaller target cell a,
      b_0 += sum u_i log(c_a - x_i),   b_l += -sum u_i (x_i - c_a)^-l / l.

Both series converge at the same rate as a same-level M2L: a level-l' cell c
is *separated* from a cell a of a coarser level l when no cell of
Near(c, l') lies inside a (ancestor test on the keys), so every target of a
sits in a level-l' cell that is well separated from c (and symmetrically for
P2L).

Traversal (per level l, starting with the root):
* Near pairs (a, m), m in Near(a, l), both existing:
  both leaves -> P2P (U list); a leaf, m split -> the children of m go to the
  W test; a split, m leaf -> the children of a go to the X test; both split ->
  their children meet again on level l + 1.
* Far pairs: the NeighborsE4 cells of a (eq. 3) that exist on level l -> M2L.
* W test for (leaf a, cell c finer than a): separated -> M2P; else c a leaf
  -> P2P; else repeat with the children of c.  The X test mirrors it.

Every (target, source) pair is covered exactly once: the tests check that by
brute force.  Re Phi is returned and, optionally, the field F = sum u / (y - x)
from the differentiated operators (L2P' and P2P' as in ``fmm``, and
M2P' = Q / (y - c) - sum_k k a_k (y - c)^-(k+1)).
"""
from collections import defaultdict

import numpy as np

from .fmm import l2l, l2p, l2p_field, m2l, m2m, p2m, p2p, p2p_field


def m2p(Q, a, c, zt):
    """Re[Q log(y - c) + sum_k a_k (y - c)^-k] at the complex targets zt."""
    d = zt - c
    inv = 1.0 / d
    acc = np.zeros(zt.shape, complex)
    for k in range(len(a), 0, -1):      # Horner in 1/d
        acc = (acc + a[k - 1]) * inv
    return Q * np.log(np.abs(d)) + acc.real


def m2p_field(Q, a, c, zt):
    """d/dy of Q log(y - c) + sum_k a_k (y - c)^-k at the complex targets zt:
    Q / (y - c) - sum_k k a_k (y - c)^-(k+1)."""
    d = zt - c
    inv = 1.0 / d
    acc = np.zeros(zt.shape, complex)
    for k in range(len(a), 0, -1):      # Horner in 1/d: sum_k k a_k d^-k
        acc = (acc + k * a[k - 1]) * inv
    return inv * (Q - acc)


def p2l(xs, us, c, p):
    """Local coefficients b_0..b_p about c of the sources xs (complex) with
    strengths us, from log(z - x) = log(c - x) - sum_l ((z - c)/(x - c))^l / l."""
    d = xs - c
    b = np.zeros(p + 1, complex)
    b[0] = np.sum(us * np.log(-d))
    inv = 1.0 / d
    pw = us.astype(complex)
    for l in range(1, p + 1):
        pw = pw * inv
        b[l] = -np.sum(pw) / l
    return b


class AdaptiveResult:
    pass


def adaptive_fmm(tiling, src_xy, u, tgt_xy, p, s=64, record=False, field=False):
    """Re Phi_j at every target with an adaptive p-term FMM over ``tiling``
    (its level L is the finest level a cell may be split to); a cell is split
    while it holds more than ``s`` sources or more than ``s`` targets."""
    src_xy = np.asarray(src_xy, np.float64).reshape(-1, 2)
    tgt_xy = np.asarray(tgt_xy, np.float64).reshape(-1, 2)
    u = np.asarray(u, np.float64)
    Lmax, b = tiling.L, tiling.b

    # keys on the finest level; a cell of level l is a key prefix (key div b^(Lmax-l))
    skey = tiling.keys(src_xy[:, 0], src_xy[:, 1]) if len(src_xy) else np.zeros(0, np.int64)
    tkey = tiling.keys(tgt_xy[:, 0], tgt_xy[:, 1]) if len(tgt_xy) else np.zeros(0, np.int64)
    sperm = np.argsort(skey, kind="stable")
    tperm = np.argsort(tkey, kind="stable")
    skey_s, tkey_s = skey[sperm], tkey[tperm]
    xs, us, ys = src_xy[sperm], u[sperm], tgt_xy[tperm]
    zs = xs[:, 0] + 1j * xs[:, 1]
    zt = ys[:, 0] + 1j * ys[:, 1]

    def ranges(keys, l):
        pre = keys // b ** (Lmax - l)
        out = {}
        for k in np.unique(pre):
            out[int(k)] = (int(np.searchsorted(pre, k)), int(np.searchsorted(pre, k, side="right")))
        return out

    src_r = [ranges(skey_s, l) for l in range(Lmax + 1)]
    tgt_r = [ranges(tkey_s, l) for l in range(Lmax + 1)]

    def ns(l, n):
        r = src_r[l].get(n)
        return 0 if r is None else r[1] - r[0]

    def nt(l, n):
        r = tgt_r[l].get(n)
        return 0 if r is None else r[1] - r[0]

    # the tree: a cell exists when its parent was split and it holds points
    cells = [[] for _ in range(Lmax + 1)]
    split = set()
    if len(zs) or len(zt):
        cells[0] = [0]
    for l in range(Lmax + 1):
        for n in cells[l]:
            if l < Lmax and max(ns(l, n), nt(l, n)) > s:
                split.add((l, n))
                for c in tiling.children(n):
                    if ns(l + 1, c) or nt(l + 1, c):
                        cells[l + 1].append(c)
    exists = [set(c) for c in cells]

    def is_leaf(l, n):
        return n in exists[l] and (l, n) not in split

    def kids(l, n):
        return [c for c in tiling.children(n) if c in exists[l + 1]]

    def separated(fine, lf, coarse, lc):
        """No cell of Near(fine, lf) lies inside the coarser cell (coarse, lc)."""
        sh = b ** (lf - lc)
        return all(m // sh != coarse for m in tiling.near(fine, lf))

    U = defaultdict(list)   # target leaf (l, a) -> source leaves (l', c)
    W = defaultdict(list)   # target leaf (l, a) -> source cells (l', c), l' > l
    X = defaultdict(list)   # target cell (l, a) -> source leaves (l', c), l' < l
    V = defaultdict(list)   # target cell (l, a) -> source cells c of level l (M2L)

    def w_test(la, a, lc, c):
        if not ns(lc, c):
            return
        if separated(c, lc, a, la):
            W[(la, a)].append((lc, c))
        elif is_leaf(lc, c):
            U[(la, a)].append((lc, c))
        else:
            for c2 in kids(lc, c):
                w_test(la, a, lc + 1, c2)

    def x_test(la, a, lc, c):
        if not nt(la, a):
            return
        if separated(a, la, c, lc):
            X[(la, a)].append((lc, c))
        elif is_leaf(la, a):
            U[(la, a)].append((lc, c))
        else:
            for a2 in kids(la, a):
                x_test(la + 1, a2, lc, c)

    for l in range(Lmax + 1):
        for a in cells[l]:
            if not nt(l, a):
                continue
            for m in tiling.near(a, l):
                if m not in exists[l] or not ns(l, m):
                    continue
                la_leaf, m_leaf = is_leaf(l, a), is_leaf(l, m)
                if la_leaf and m_leaf:
                    U[(l, a)].append((l, m))
                elif la_leaf:
                    for c2 in kids(l, m):
                        w_test(l, a, l + 1, c2)
                elif m_leaf:
                    for a2 in kids(l, a):
                        x_test(l + 1, a2, l, m)
            V[(l, a)] = [m for m in tiling.far(a, l) if m in exists[l] and ns(l, m)]

    centers = {}

    def C(l, n):
        if (l, n) not in centers:
            centers[(l, n)] = tiling.center(n, l)
        return centers[(l, n)]

    # upward pass: P2M at the source leaves, M2M into every split cell
    mult = {}
    for l in range(Lmax, -1, -1):
        for n in cells[l]:
            if not ns(l, n):
                continue
            if (l, n) not in split:
                lo, hi = src_r[l][n]
                mult[(l, n)] = p2m(zs[lo:hi], us[lo:hi], C(l, n), p)
            else:
                Qp, ap = 0.0, np.zeros(p, complex)
                for c in kids(l, n):
                    if (l + 1, c) in mult:
                        Qc, ac = mult[(l + 1, c)]
                        Qp += Qc
                        ap = ap + m2m(Qc, ac, C(l + 1, c) - C(l, n), p)
                mult[(l, n)] = (Qp, ap)

    # downward pass: L2L from the parent, M2L (V), P2L (X)
    loc = {}
    for l in range(Lmax + 1):
        for a in cells[l]:
            if not nt(l, a):
                continue
            ct = C(l, a)
            acc = np.zeros(p + 1, complex)
            if l > 0:
                acc = acc + l2l(loc[(l - 1, a // b)], ct - C(l - 1, a // b), p)
            for m in V[(l, a)]:
                Qs, a_s = mult[(l, m)]
                acc = acc + m2l(Qs, a_s, C(l, m) - ct, p)
            for (lc, c) in X[(l, a)]:
                lo, hi = src_r[lc][c]
                acc = acc + p2l(zs[lo:hi], us[lo:hi], ct, p)
            loc[(l, a)] = acc

    # target leaves: L2P + M2P (W) + P2P (U)
    phi_s = np.zeros(len(zt))
    f_s = np.zeros(len(zt), complex)
    for l in range(Lmax + 1):
        for a in cells[l]:
            if (l, a) in split or not nt(l, a):
                continue
            lo, hi = tgt_r[l][a]
            val = l2p(loc[(l, a)], zt[lo:hi], C(l, a))
            fv = l2p_field(loc[(l, a)], zt[lo:hi], C(l, a)) if field else None
            for (lc, c) in W[(l, a)]:
                Qs, a_s = mult[(lc, c)]
                val = val + m2p(Qs, a_s, C(lc, c), zt[lo:hi])
                if field:
                    fv = fv + m2p_field(Qs, a_s, C(lc, c), zt[lo:hi])
            parts = [np.arange(*src_r[lc][c]) for (lc, c) in U[(l, a)]]
            if parts:
                idx = np.concatenate(parts)
                val = val + p2p(xs[idx], us[idx], ys[lo:hi])
                if field:
                    fv = fv + p2p_field(xs[idx], us[idx], ys[lo:hi])
            phi_s[lo:hi] = val
            if field:
                f_s[lo:hi] = fv
    phi = np.zeros(len(zt))
    phi[tperm] = phi_s
    res = AdaptiveResult()
    res.phi = phi
    if field:
        res.field = np.zeros(len(zt), complex)
        res.field[tperm] = f_s
    if record:
        res.src_perm, res.tgt_perm = sperm, tperm
        res.src_keys, res.tgt_keys = skey, tkey
        res.cells, res.split = cells, split
        res.src_r, res.tgt_r = src_r, tgt_r
        res.U, res.W, res.X, res.V = dict(U), dict(W), dict(X), dict(V)
        res.mult, res.loc = mult, loc
    return res
