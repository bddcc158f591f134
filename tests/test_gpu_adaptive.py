"""Parity of the adaptive CUDA path (FMM2D_ADAPTIVE) with the oracle's
adaptive FMM on clustered input.

Integer work - the cells of every level with their split flags and the U
(P2P), W (M2P), X (P2L) and M2L lists - is compared bit for bit.  Potentials:
FP64 form within 1e-11 of the oracle's adaptive FMM of the same (Lmax, p,
leaf size); the mixed and tensor-core forms within the requested 1e-6; the
uniform reduction (leaf size 0) against the uniform CUDA path; and the full
clustered workload (N = M = 4,194,304, 32 clusters, eps = 1e-10) on sampled
targets against the direct sum.
"""
import numpy as np
import pytest

from gpu_util import run_gpu
from oracle.adaptive import adaptive_fmm
from oracle.direct import direct, rel_inf_error
from oracle.fmm import make_tiling
from oracle.params import p_from_eps
from paper_1204_3105_gb300.inputs import gaussian_mixture, sample_targets, uniform_square

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_3105_gb300 import build, fmm2d
    build.build()
    fmm2d.lib()


def _clustered(n, seed, sigma=(3e-3, 5e-2), k=6):
    return gaussian_mixture(n, seed=seed, k=k, sigma=sigma)


def _tuples(d, lists_of_pairs=True):
    out = []
    for (la, a), srcs in d.items():
        for e in srcs:
            lc, c = e if lists_of_pairs else (la, e)
            out.append((la, a, lc, c))
    return sorted(out)


CASES = [("quad", 8, 24), ("sept", 5, 16), ("tri", 8, 24)]


@pytest.mark.parametrize("tiling,L,cap", CASES)
@pytest.mark.parametrize("separate,prec", [(False, "fp64"), (True, "fp64"), (False, "split")])
def test_tree_and_lists_bit_exact(tiling, L, cap, separate, prec):
    xy, u = _clustered(3000, seed=31)
    txy = _clustered(2000, seed=32)[0] if separate else None
    p = 6
    phi, plan = run_gpu(tiling, xy, u, txy, levels=L, p=p, prec=prec, keep=True, leaf_size=cap)
    r = adaptive_fmm(make_tiling(tiling, L), xy, u, xy if txy is None else txy, p, s=cap, record=True)
    cells = plan.export("ad_cells")
    want = sorted((l, n, int((l, n) in r.split)) for l, cs in enumerate(r.cells) for n in cs)
    assert sorted(map(tuple, cells.tolist())) == want
    for name, d, pairs in (("ad_u", r.U, True), ("ad_w", r.W, True), ("ad_x", r.X, True),
                           ("ad_v", {k: v for k, v in r.V.items() if v}, False)):
        got = sorted(map(tuple, plan.export(name).tolist()))
        assert got == _tuples(d, pairs), name
    plan.close()
    ref = r.phi
    assert rel_inf_error(phi, ref) < 1e-11


@pytest.mark.parametrize("tiling,L,cap", CASES)
@pytest.mark.parametrize("prec", ["mixed", "tc"])
def test_mixed_forms_within_eps(tiling, L, cap, prec):
    xy, u = _clustered(6000, seed=33)
    p = p_from_eps(tiling, 1e-6)
    r = adaptive_fmm(make_tiling(tiling, L), xy, u, xy, p, s=cap)
    phi, _ = run_gpu(tiling, xy.astype(np.float32), u.astype(np.float32), levels=L, p=p, prec=prec,
                     f32=True, leaf_size=cap)
    ref = direct(xy.astype(np.float32).astype(np.float64), u.astype(np.float32).astype(np.float64),
                 xy.astype(np.float32).astype(np.float64))
    assert rel_inf_error(phi, ref) < 1e-6
    assert rel_inf_error(r.phi, direct(xy, u, xy)) < 1e-6


@pytest.mark.parametrize("tiling,L,cap", CASES)
def test_hybrid_form_adaptive(tiling, L, cap):
    """Hybrid form on an adaptive tree (float-float M2L over the class
    lists, FP64 M2P / P2L, FP32 P2P): against the FP64 oracle's adaptive FMM
    of the same tree and p, within 1e-8 (the FP32 near field's level)."""
    xy, u = _clustered(6000, seed=35)
    p = p_from_eps(tiling, 1e-8)
    r = adaptive_fmm(make_tiling(tiling, L), xy, u, xy, p, s=cap)
    phi, plan = run_gpu(tiling, xy, u, levels=L, p=p, prec="hybrid", leaf_size=cap, keep=True)
    assert plan.query()["device_error"] == 0
    plan.close()
    assert rel_inf_error(phi, r.phi) < 1e-8


@pytest.mark.parametrize("tiling,L", [("quad", 5), ("sept", 4), ("tri", 5)])
def test_leaf_size_zero_is_the_uniform_tree(tiling, L):
    xy, u = uniform_square(20000, seed=34)
    a, _ = run_gpu(tiling, xy, u, levels=L, p=14, prec="fp64", leaf_size=0)
    b, _ = run_gpu(tiling, xy, u, levels=L, p=14, prec="fp64")
    assert rel_inf_error(a, b) < 1e-12


@pytest.mark.parametrize("tiling,L", [("quad", 10), ("sept", 6), ("tri", 10)])
def test_shallow_leaf_beside_a_deep_cluster(tiling, L):
    """A leaf on level 1 (a sparse corner) next to a cluster refined many
    levels deep: the leaf's local expansion gets no M2L and must start at 0."""
    g = np.random.default_rng(35)
    sparse = 0.05 + 0.1 * g.random((12, 2))
    dense = 0.7 + 2e-3 * g.standard_normal((4000, 2))
    xy = np.concatenate([sparse, dense])
    u = g.uniform(-1, 1, len(xy))
    phi, plan = run_gpu(tiling, xy, u, levels=L, p=14, prec="fp64", leaf_size=32, keep=True)
    cells = plan.export("ad_cells")
    plan.close()
    assert any(l == 1 and not sp for l, _, sp in cells.tolist())      # a level-1 leaf exists
    ref = adaptive_fmm(make_tiling(tiling, L), xy, u, xy, 14, s=32).phi
    assert rel_inf_error(phi, ref) < 1e-11


def test_edge_cases():
    from paper_1204_3105_gb300 import fmm2d
    # a single point, all points in one cell, and fewer points than the leaf size
    for n in (1, 5, 60):
        xy = np.full((n, 2), 0.3) + 1e-9 * np.arange(n)[:, None]
        u = np.ones(n)
        phi, _ = run_gpu("quad", xy, u, levels=16, p=8, prec="fp64", leaf_size=64)
        ref = direct(xy, u, xy)
        if n == 1:
            assert phi[0] == 0.0           # no other source
        else:
            assert rel_inf_error(phi, ref) < 1e-12
    # a duplicated point cannot be split apart: it ends in a finest-level leaf
    # holding both copies, and the coincident pairs are skipped
    xy = np.array([[0.25, 0.25], [0.25, 0.25], [0.75, 0.5]])
    u = np.array([1.0, 2.0, 3.0])
    phi, _ = run_gpu("tri", xy, u, levels=6, p=8, prec="fp64", leaf_size=1)
    ref = adaptive_fmm(make_tiling("tri", 6), xy, u, xy, 8, s=1).phi
    assert rel_inf_error(phi, ref) < 1e-11
    assert rel_inf_error(phi, direct(xy, u, xy)) < 1e-5      # p = 8 truncation
    with pytest.raises(fmm2d.FMM2DError):
        fmm2d.Plan("quad", levels=17, p=8, flags=fmm2d.ADAPTIVE)
    with pytest.raises(fmm2d.FMM2DError):   # septree keys of 12 levels exceed 32 bits
        fmm2d.Plan("sept", levels=12, p=8, flags=fmm2d.ADAPTIVE)


@pytest.mark.parametrize("tiling", ["quad", "sept"])
@pytest.mark.parametrize("prec", ["fp64", "split", "hybrid"])
def test_clustered_4m_eps_1e10_sampled(tiling, prec):
    """The clustered workload at full size: N = M = 4,194,304 points from a
    32-component Gaussian mixture, strengths N(0, 1), eps = 1e-10, leaf size
    64, in the FP64, split and hybrid forms; 96 sampled targets against the
    direct sum over all sources."""
    n = 4194304
    xy, u = gaussian_mixture(n, seed=3, k=32)
    phi, plan = run_gpu(tiling, xy, u, eps=1e-10, prec=prec, leaf_size=64, keep=True)
    info = plan.query()
    plan.close()
    idx = sample_targets(n, 96, seed=5)
    ref = direct(xy, u, xy[idx])
    assert rel_inf_error(phi[idx], ref) < 1e-10
    assert info["levels"] == (16 if tiling == "quad" else 11)   # the default finest level
    # the configuration's "adaptive depth to leaf <= 64": no leaf holds more
    assert info["max_leaf_src"] <= 64 and info["max_leaf_tgt"] <= 64, info


def test_septree_eleven_levels_bit_exact():
    """Two tight clusters on an 11-level septree (the deepest with 32-bit
    keys; its leaf radius comes from the norm lower bound, not from an
    enumeration): cells and U / W / X / M2L lists bit for bit with the
    oracle, FP64 potentials within 1e-11, and the tree reaches level 11."""
    xy, u = gaussian_mixture(3000, seed=35, k=2, sigma=(2e-5, 1e-4))
    p = 6
    phi, plan = run_gpu("sept", xy, u, levels=11, p=p, prec="fp64", keep=True, leaf_size=8)
    r = adaptive_fmm(make_tiling("sept", 11), xy, u, xy, p, s=8, record=True)
    cells = plan.export("ad_cells")
    want = sorted((l, n, int((l, n) in r.split)) for l, cs in enumerate(r.cells) for n in cs)
    assert sorted(map(tuple, cells.tolist())) == want
    assert max(l for l, _, _ in want) == 11
    for name, d, pairs in (("ad_u", r.U, True), ("ad_w", r.W, True), ("ad_x", r.X, True),
                           ("ad_v", {k: v for k, v in r.V.items() if v}, False)):
        got = sorted(map(tuple, plan.export(name).tolist()))
        assert got == _tuples(d, pairs), name
    plan.close()
    assert rel_inf_error(phi, r.phi) < 1e-11
