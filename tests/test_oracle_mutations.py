"""The oracle's pins catch plausible mistakes.

Each test plants one mistake in the oracle (on the CPU, through monkeypatch:
a wrong sign, a dropped term, a transposed or mis-indexed operand, the
intersection reading of NeighborsE4) and checks that a pin of
tests/test_oracle_*.py fails on the mutated oracle.  A pin that still passed
would not be pinning the thing it claims to.
"""
import numpy as np
import pytest

import test_oracle_fmm as pins_fmm
import test_oracle_quad_params as pins_quad
from oracle import fmm as F
from oracle.tiling_quad import Quadtree


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_p2m_without_1_over_k_is_caught(monkeypatch):
    orig = F.p2m

    def bad(xs, us, c, p):
        Q, a = orig(xs, us, c, p)
        return Q, a * np.arange(1, p + 1)           # a_k = -sum u d^k (the 1/k dropped)
    monkeypatch.setattr(F, "p2m", bad)
    _fails(pins_fmm.test_p2m_single_source_is_log_series)


def test_p2m_sign_is_caught(monkeypatch):
    orig = F.p2m

    def bad(xs, us, c, p):
        Q, a = orig(xs, us, c, p)
        return Q, -a
    monkeypatch.setattr(F, "p2m", bad)
    _fails(pins_fmm.test_p2m_single_source_is_log_series)


def test_m2m_shift_direction_is_caught(monkeypatch):
    orig = F.m2m
    monkeypatch.setattr(F, "m2m", lambda Q, a, z0, p: orig(Q, a, -z0, p))
    _fails(pins_fmm.test_m2m_then_evaluate_within_bound)


def test_m2l_dropped_q_term_is_caught(monkeypatch):
    orig = F.m2l

    def bad(Q, a, z0, p):
        b = orig(Q, a, z0, p)
        lv = np.arange(1, p + 1)
        b[1:] -= -Q * (1.0 / z0) ** lv / lv          # undo the Q (-z0^-l / l) term
        return b
    monkeypatch.setattr(F, "m2l", bad)
    _fails(pins_fmm.test_m2l_within_bound_and_l2l_exact)


def test_m2l_index_slip_is_caught(monkeypatch):
    orig = F.m2l

    def bad(Q, a, z0, p):
        # the a-part with z0^-(l+k+1) instead of z0^-(l+k)
        b0 = orig(Q, np.zeros_like(a), z0, p)
        return b0 + (orig(0.0, a, z0, p)) / z0
    monkeypatch.setattr(F, "m2l", bad)
    _fails(pins_fmm.test_m2l_within_bound_and_l2l_exact)
    _fails(pins_fmm.test_m2l_operator_is_real_factor_times_phase)


def test_l2l_shift_direction_is_caught(monkeypatch):
    orig = F.l2l
    monkeypatch.setattr(F, "l2l", lambda b, w, p: orig(b, -w, p))
    _fails(pins_fmm.test_m2l_within_bound_and_l2l_exact)


def test_l2p_conjugate_is_caught(monkeypatch):
    orig = F.l2p
    monkeypatch.setattr(F, "l2p", lambda b, ys, c: orig(np.conj(b), ys, c))
    _fails(pins_fmm.test_fmm_converges_to_direct, "quad", 3)


def test_p2p_missing_half_is_caught(monkeypatch):
    orig = F.p2p
    monkeypatch.setattr(F, "p2p", lambda s, u, t: 2.0 * orig(s, u, t))   # log r^2 for log r
    _fails(pins_fmm.test_fmm_converges_to_direct, "quad", 3)


def test_neighbors_e4_as_intersection_is_caught(monkeypatch):
    """eq. 3 printed with an intersection; the pins hold the set difference."""
    def far_intersection(self, n, l):
        if l < 1:
            return []
        P = self.parent(n)
        cand = []
        for q in [P] + self.neighbors(P, l - 1):
            cand.extend(self.children(q))
        return sorted(set(cand) & set(self.near(n, l)))
    monkeypatch.setattr(Quadtree, "far", far_intersection)
    _fails(pins_quad.test_quad_full_tree_list_counts)
    _fails(pins_quad.test_table2_counts_and_cost_constants)


def test_gbt_unit_sum_entry_is_caught(monkeypatch):
    """One entry of the unit-sum table (Fig. 4b) mis-typed: 1 (+) 2 = 15
    read as 14."""
    import test_oracle_sept as pins_sept
    from oracle import tiling_sept as ts
    table = [list(r) for r in ts.GBT_UNIT_SUM]
    table[0][1] = 14
    monkeypatch.setattr(ts, "GBT_UNIT_SUM", tuple(tuple(r) for r in table))
    _fails(pins_sept.test_unit_sum_table_both_routes)


def test_triangle_direction_table_entry_is_caught(monkeypatch):
    """One destination of the triangle direction table (Table 1) wrong."""
    import test_oracle_tri as pins_tri
    from oracle import tiling_tri as tt
    table = [list(r) for r in tt.TABLE_D]
    table[1][0] = (2, False)
    monkeypatch.setattr(tt, "TABLE_D", tuple(tuple(r) for r in table))
    _fails(pins_tri.test_neighbors_equal_vertex_sharing_cells)


def test_adaptive_near_set_missing_a_neighbour_is_caught(monkeypatch):
    """A Near set that drops one neighbour leaves (target, source) pairs of the
    adaptive traversal uncovered."""
    import test_oracle_adaptive as pins_ad
    orig = Quadtree.near
    monkeypatch.setattr(Quadtree, "near", lambda self, n, l: orig(self, n, l)[:-1])
    _fails(pins_ad.test_every_pair_covered_exactly_once, "quad", 6)


def test_m2p_conjugate_is_caught(monkeypatch):
    """M2P summing the multipole tail on the conjugate coefficients."""
    import test_oracle_adaptive as pins_ad
    from oracle import adaptive as A
    orig = A.m2p
    monkeypatch.setattr(A, "m2p", lambda Q, a, c, zt: orig(Q, np.conj(a), c, zt))
    _fails(pins_ad.test_m2p_single_source_within_series_tail)


def test_p2l_without_1_over_l_is_caught(monkeypatch):
    import test_oracle_adaptive as pins_ad
    from oracle import adaptive as A
    orig = A.p2l

    def bad(xs, us, c, p):
        b = orig(xs, us, c, p)
        b[1:] *= np.arange(1, p + 1)
        return b
    monkeypatch.setattr(A, "p2l", bad)
    _fails(pins_ad.test_p2l_single_source_within_series_tail)


def test_morton_axes_swapped_is_caught(monkeypatch):
    """The x and y bits of the Morton interleave exchanged."""
    orig = Quadtree.keys

    def bad(self, x, y, l=None):
        return orig(self, y, x, l)
    monkeypatch.setattr(Quadtree, "keys", bad)
    _fails(pins_quad.test_morton_containment_and_prefix)


# ---- the field (derivative) operators ----------------------------------------
import test_oracle_field as pins_field  # noqa: E402
from oracle import adaptive as A  # noqa: E402


def test_l2p_field_without_factor_l_is_caught(monkeypatch):
    def bad(b, ys, c):           # sum b_l (y - c)^(l-1): the factor l dropped
        d = ys - c
        acc = np.zeros(ys.shape, complex) + b[-1]
        for l in range(len(b) - 2, 0, -1):
            acc = acc * d + b[l]
        return acc
    monkeypatch.setattr(F, "l2p_field", bad)
    _fails(pins_field.test_l2p_field_is_derivative_of_l2p)
    _fails(pins_field.test_fmm_field_converges_to_direct, "quad", 3)


def test_p2p_field_conjugate_is_caught(monkeypatch):
    orig = F.p2p_field
    monkeypatch.setattr(F, "p2p_field", lambda s, u, t: np.conj(orig(s, u, t)))
    _fails(pins_field.test_p2p_field_matches_direct)
    _fails(pins_field.test_fmm_field_converges_to_direct, "tri", 3)


def test_m2p_field_sign_is_caught(monkeypatch):
    def bad(Q, a, c, zt):        # Q / (y - c) + sum k a_k (y - c)^-(k+1): wrong sign
        d = zt - c
        inv = 1.0 / d
        acc = np.zeros(zt.shape, complex)
        for k in range(len(a), 0, -1):
            acc = (acc + k * a[k - 1]) * inv
        return inv * (Q + acc)
    monkeypatch.setattr(A, "m2p_field", bad)
    _fails(pins_field.test_m2p_field_single_source_and_derivative)
    _fails(pins_field.test_adaptive_field_matches_direct, "quad", 7)


def test_direct_field_conjugate_is_caught(monkeypatch):
    orig = pins_field.direct

    def bad(src, u, tgt, block=2048, gradient=False):
        out = orig(src, u, tgt, block=block, gradient=gradient)
        return (out[0], np.conj(out[1])) if gradient else out
    monkeypatch.setattr(pins_field, "direct", bad)
    _fails(pins_field.test_direct_field_single_source_closed_form)
    _fails(pins_field.test_direct_field_is_gradient_of_potential)
