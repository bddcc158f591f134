"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Integer work (keys, sort permutation, cells, lists) is compared bit for bit.
Potentials: the FP64 GPU form must match the FP64 oracle FMM of the same
(L, p) to 1e-11 relative (eps_rel_inf; only the summation order differs);
the mixed form (FP32 expansions and P2P, FP64 leading term) to 1e-6, the
tolerance requested of the configurations (relative eps = 1e-6).
"""
import math

import numpy as np
import pytest

from gpu_util import run_gpu
from oracle.direct import direct, rel_inf_error
from oracle.fmm import fmm, make_tiling
from paper_1204_3105_gb300.inputs import gaussian_mixture, sample_targets, uniform_square

pytestmark = pytest.mark.gpu

CASES = [("quad", 4, 12), ("sept", 3, 12), ("tri", 4, 12)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_3105_gb300 import build, fmm2d
    build.build()
    fmm2d.lib()


def _oracle(tiling, L, src, u, tgt, p, domain=(0.0, 0.0, 1.0)):
    T = make_tiling(tiling, L, domain)
    return fmm(T, src, u, src if tgt is None else tgt, p, record=True), T


@pytest.mark.parametrize("tiling,L,p", CASES)
@pytest.mark.parametrize("n", [1, 37, 4099, 20011])
def test_keys_sort_cells_lists_bitexact(tiling, L, p, n):
    xy, u = uniform_square(n, seed=100 + n)
    phi, plan = run_gpu(tiling, xy, u, levels=L, p=p, prec="fp64", keep=True)
    r, T = _oracle(tiling, L, xy, u, None, p)
    assert np.array_equal(plan.export("src_keys"), r.src_keys)
    assert np.array_equal(plan.export("src_perm"), r.src_perm)      # stable sort
    for l in range(L + 1):
        assert np.array_equal(plan.export("cells", l), np.array(r.cells[l], np.int64))
    near = {tuple(x) for x in plan.export("near").tolist()}
    want = {(t, s) for t, lst in r.near.items() for s in lst}
    assert near == want
    for l in range(T.l_min, L + 1):
        far = {tuple(x) for x in plan.export("far", l).tolist()}
        want = {(n_, m) for (ll, n_), lst in r.far.items() if ll == l for m in lst}
        assert far == want, (tiling, l)
    # cell centres agree with CellCenter of the paper (eqs. 6, 12)
    for l in (0, L):
        c = plan.export("centers", l)
        want = np.array([T.center(int(k), l) for k in r.cells[l]])
        assert np.max(np.abs(c - want), initial=0) < 1e-12
    plan.close()


@pytest.mark.parametrize("tiling,L,p", CASES)
def test_fp64_path_matches_oracle(tiling, L, p):
    n = 6007
    xy, u = uniform_square(n, seed=5)
    phi, plan = run_gpu(tiling, xy, u, levels=L, p=p, prec="fp64", keep=True)
    r, T = _oracle(tiling, L, xy, u, None, p)
    assert rel_inf_error(phi, r.phi) < 1e-11
    assert rel_inf_error(plan.export("phi_near"), r.phi_near) < 1e-11
    # multipoles and locals per level, unscaled, against the oracle's
    for l in range(T.l_min, L + 1):
        mg = plan.export("multipoles", l)
        lg = plan.export("locals", l)
        cells = r.cells[l]
        for i, key in enumerate(cells):
            if (l, key) in r.mult:
                Q, a = r.mult[(l, key)]
                assert abs(mg[i, 0].real - Q) <= 1e-12 * max(1.0, abs(Q))
                scale = np.abs(a).max() + 1e-300
                assert np.max(np.abs(mg[i, 1:] - a)) <= 1e-10 * scale
            b = r.loc[(l, key)]
            assert abs(lg[i, 0].real - b[0].real) <= 1e-10 * max(1.0, np.abs(b).max())
            assert np.max(np.abs(lg[i, 1:] - b[1:])) <= 1e-9 * (np.abs(b[1:]).max() + 1e-300)
    plan.close()


@pytest.mark.parametrize("tiling,L,p", CASES)
@pytest.mark.parametrize("f32", [False, True])
def test_mixed_path_matches_oracle(tiling, L, p, f32):
    n = 12007
    xy, u = uniform_square(n, seed=9, dtype=np.float32 if f32 else np.float64)
    phi, _ = run_gpu(tiling, xy, u, levels=L, p=p, prec="mixed", f32=f32)
    r, _ = _oracle(tiling, L, xy.astype(np.float64), u.astype(np.float64), None, p)
    assert rel_inf_error(phi, r.phi) < 1e-6


@pytest.mark.parametrize("tiling,L,p", CASES + [("quad", 5, 22), ("sept", 4, 21), ("tri", 5, 27)])
def test_tensor_core_m2l_matches_oracle(tiling, L, p):
    """Mixed form with M2L on the tensor cores (split TF32, FP32 accumulation):
    far field and total potential within 1e-6 of the FP64 oracle."""
    n = 12007
    xy, u = uniform_square(n, seed=9)
    phi, plan = run_gpu(tiling, xy, u, levels=L, p=p, prec="tc", keep=True)
    assert plan.query()["device_error"] == 0
    far = plan.export("phi_far")
    plan.close()
    r, _ = _oracle(tiling, L, xy, u, None, p)
    scale = np.max(np.abs(r.phi))
    assert np.max(np.abs(far - r.phi_far)) / scale < 1e-6
    assert rel_inf_error(phi, r.phi) < 1e-6


def test_separate_targets_domain_and_clusters():
    rng = np.random.default_rng(3)
    dom = (-2.0, 1.0, 3.0)
    src = np.column_stack([dom[0] + dom[2] * rng.random(5000), dom[1] + dom[2] * rng.random(5000)])
    tgt = np.column_stack([dom[0] + dom[2] * rng.random(3001), dom[1] + dom[2] * rng.random(3001)])
    tgt[:7] = src[:7]
    u = rng.normal(size=5000)
    ref = direct(src, u, tgt)
    for tiling, L in (("quad", 4), ("sept", 3), ("tri", 4)):
        phi, _ = run_gpu(tiling, src, u, tgt, levels=L, p=30, prec="fp64", domain=dom)
        assert rel_inf_error(phi, ref) < 1e-11
        phi, _ = run_gpu(tiling, src, u, tgt, levels=L, p=0, eps=1e-6, prec="mixed", domain=dom)
        assert rel_inf_error(phi, ref) <= 1e-6
    xy, uu = gaussian_mixture(20000, seed=3, k=8)
    ref = direct(xy, uu, xy)
    for tiling, L in (("quad", 5), ("sept", 4), ("tri", 5)):
        phi, _ = run_gpu(tiling, xy, uu, levels=L, p=24, prec="fp64")
        assert rel_inf_error(phi, ref) < 1e-9


def test_points_on_cell_edges():
    # points exactly on quadtree lines and lattice-aligned coordinates
    g = np.arange(64) / 64.0
    xy = np.array([(a, b) for a in g for b in g[::3]])
    u = np.cos(np.arange(len(xy)))
    ref = direct(xy, u, xy)
    for tiling, L in (("quad", 3), ("sept", 3), ("tri", 3)):
        phi, plan = run_gpu(tiling, xy, u, levels=L, p=30, prec="fp64", keep=True)
        r, _ = _oracle(tiling, L, xy, u, None, 30)
        assert np.array_equal(plan.export("src_keys"), r.src_keys)
        assert rel_inf_error(phi, ref) < 1e-10
        plan.close()


def test_domain_error_and_empty():
    from paper_1204_3105_gb300 import fmm2d
    xy = np.array([[0.5, 0.5], [1.5, 0.2]])
    with pytest.raises(fmm2d.FMM2DError) as e:
        run_gpu("quad", xy, np.ones(2), levels=2, p=4)
    assert e.value.status == fmm2d.EDOMAIN
    # no targets / no sources
    src, u = uniform_square(100, seed=1)
    phi, _ = run_gpu("tri", src, u, np.zeros((0, 2)), levels=3, p=8)
    assert phi.shape == (0,)
    phi, _ = run_gpu("sept", np.zeros((0, 2)), np.zeros(0), src, levels=3, p=8)
    assert np.all(phi == 0)


@pytest.mark.parametrize("prec", ["mixed", "tc"])
@pytest.mark.parametrize("tiling", ["quad", "sept", "tri"])
def test_full_size_sampled(tiling, prec):
    """N = M = 2^20 uniform points, FP32 inputs, eps = 1e-6 with the planner's
    L and p (the benchmark configuration): keys bit-exact against the oracle's
    CellIndex, potentials against direct summation on 384 sampled targets."""
    n = 2 ** 20
    xy, u = uniform_square(n, seed=2, dtype=np.float32)
    phi, plan = run_gpu(tiling, xy, u, prec=prec, f32=True, eps=1e-6, keep=True)
    info = plan.query()
    assert info["device_error"] == 0
    T = make_tiling(tiling, info["levels"])
    x64 = xy.astype(np.float64)
    assert np.array_equal(plan.export("src_keys"), T.keys(x64[:, 0], x64[:, 1]))
    plan.close()
    idx = sample_targets(n, 384, seed=2)
    ref = direct(x64, u.astype(np.float64), x64[idx])
    err = np.max(np.abs(phi[idx] - ref)) / np.max(np.abs(ref))
    assert err < 1e-6, err


@pytest.mark.parametrize("tiling", ["quad", "sept", "tri"])
def test_autotuned_benchmark_configuration(tiling):
    """The configuration bench.py times: N = M = 2^20, FP32, tensor-core M2L,
    (L, p) from fmm2d_autotune for eps = 1e-6.  The tuner's own probe error is
    <= eps/3 and the potentials of the benchmark strengths are within eps of
    the oracle's direct sum on 384 sampled targets."""
    import torch
    from paper_1204_3105_gb300 import fmm2d
    n = 2 ** 20
    xy, u = uniform_square(n, seed=2, dtype=np.float32)
    x_d = torch.from_numpy(xy).cuda()
    flags = fmm2d.PREC_MIXED_TC | fmm2d.IN_F32
    L, p, err, ms = fmm2d.fmm2d_autotune(tiling, 1e-6, flags, x_d, n, x_d, n)
    assert 0 < err <= 1e-6 / 3 and ms > 0
    phi, _ = run_gpu(tiling, xy, u, levels=L, p=p, prec="tc", f32=True)
    x64 = xy.astype(np.float64)
    idx = sample_targets(n, 384, seed=7)
    ref = direct(x64, u.astype(np.float64), x64[idx])
    assert np.max(np.abs(phi[idx] - ref)) / np.max(np.abs(ref)) < 1e-6


@pytest.mark.parametrize("tiling", ["quad", "sept", "tri"])
def test_hybrid_form_eps_1e8(tiling):
    """FMM2D_PREC_HYBRID (FP64 expansions, FP32 P2P): within 1e-8 of the
    direct sum at the a-priori p for eps = 1e-8, on uniform FP32 points (the
    P2P differences are then exact) and on a clustered set."""
    from oracle.params import p_from_eps
    p = p_from_eps(tiling, 1e-8)
    xy, u = uniform_square(30000, seed=61, dtype=np.float32)
    phi, _ = run_gpu(tiling, xy, u, p=p, eps=1e-8, prec="hybrid", f32=True)
    idx = sample_targets(len(xy), 300, seed=1)
    x64, u64 = xy.astype(np.float64), u.astype(np.float64)
    ref = direct(x64, u64, x64[idx])
    assert rel_inf_error(phi[idx], ref) < 1e-8
    cxy, cu = gaussian_mixture(20000, seed=62, k=8)
    phi, _ = run_gpu(tiling, cxy, cu, p=p, eps=1e-8, prec="hybrid", leaf_size=64)
    cidx = sample_targets(len(cxy), 300, seed=2)
    ref = direct(cxy, cu, cxy[cidx])
    assert rel_inf_error(phi[cidx], ref) < 1e-8


@pytest.mark.parametrize("tiling,L,p", CASES + [("quad", 4, 30), ("sept", 3, 28), ("tri", 4, 36)])
def test_hybrid_far_field_matches_oracle(tiling, L, p):
    """Hybrid form: multipoles (FP64 P2M, M2M) and locals (float-float M2L,
    FP64 L2L) per level against the FP64 oracle to the tolerances of the FP64
    form, and the far-field potential to 1e-11 of the potential scale; only
    the near field (FP32 P2P) is approximate."""
    n = 6007
    xy, u = uniform_square(n, seed=5)
    phi, plan = run_gpu(tiling, xy, u, levels=L, p=p, prec="hybrid", keep=True)
    r, T = _oracle(tiling, L, xy, u, None, p)
    for l in range(T.l_min, L + 1):
        mg = plan.export("multipoles", l)
        lg = plan.export("locals", l)
        for i, key in enumerate(r.cells[l]):
            if (l, key) in r.mult:
                Q, a = r.mult[(l, key)]
                assert abs(mg[i, 0].real - Q) <= 1e-12 * max(1.0, abs(Q))
                assert np.max(np.abs(mg[i, 1:] - a)) <= 1e-10 * (np.abs(a).max() + 1e-300)
            b = r.loc[(l, key)]
            assert abs(lg[i, 0].real - b[0].real) <= 1e-10 * max(1.0, np.abs(b).max())
            assert np.max(np.abs(lg[i, 1:] - b[1:])) <= 1e-9 * (np.abs(b[1:]).max() + 1e-300)
    far = plan.export("phi_far")
    plan.close()
    scale = np.max(np.abs(r.phi))
    assert np.max(np.abs(far - r.phi_far)) / scale < 1e-11
    assert rel_inf_error(phi, r.phi) < 1e-8


@pytest.mark.parametrize("tiling,L,p", CASES + [("quad", 4, 30), ("sept", 3, 28), ("tri", 4, 36)])
def test_split_form_matches_oracle(tiling, L, p):
    """FMM2D_PREC_SPLIT (FP64 with the float-float M2L): potentials, near
    field and per-level locals against the FP64 oracle to the FP64 form's
    tolerances."""
    n = 6007
    xy, u = uniform_square(n, seed=5)
    phi, plan = run_gpu(tiling, xy, u, levels=L, p=p, prec="split", keep=True)
    r, T = _oracle(tiling, L, xy, u, None, p)
    assert rel_inf_error(phi, r.phi) < 1e-11
    assert rel_inf_error(plan.export("phi_near"), r.phi_near) < 1e-11
    for l in range(T.l_min, L + 1):
        lg = plan.export("locals", l)
        for i, key in enumerate(r.cells[l]):
            b = r.loc[(l, key)]
            assert abs(lg[i, 0].real - b[0].real) <= 1e-10 * max(1.0, np.abs(b).max())
            assert np.max(np.abs(lg[i, 1:] - b[1:])) <= 1e-9 * (np.abs(b[1:]).max() + 1e-300)
    plan.close()


def test_plain_fp64_quadtree_8192():
    """The plain FP64 quadtree configuration: N = M = 8192 uniform points,
    strengths U[-1, 1], p = 16, 4 levels (leaf <= 64 on average): against the
    oracle FMM of the same (L, p) to 1e-11 and the full direct sum within the
    p = 16 truncation (reading of eq. 15: kappa^(p+1) ~ 4e-5 before the
    cancellation of the far field)."""
    xy, u = uniform_square(8192, seed=1)
    phi, _ = run_gpu("quad", xy, u, levels=4, p=16, prec="fp64")
    r, _ = _oracle("quad", 4, xy, u, None, 16)
    assert rel_inf_error(phi, r.phi) < 1e-11
    ref = direct(xy, u, xy)
    err = rel_inf_error(phi, ref)
    assert err < 1e-6
    assert abs(err - rel_inf_error(r.phi, ref)) < 1e-9


@pytest.mark.parametrize("tiling", ["quad", "sept", "tri"])
def test_separate_sets_full_size_autotuned(tiling):
    """M != N at full size: N = 2^20 sources and M = 2^19 other targets (FP32,
    uniform), (L, p) from fmm2d_autotune (levels around the S_opt level of
    Table 2 for N and M) for eps = 1e-6, tensor-core form; 512 sampled
    targets against the direct sum over all sources within eps."""
    import torch
    from paper_1204_3105_gb300 import fmm2d
    n, m = 1 << 20, 1 << 19
    src, u = uniform_square(n, seed=61, dtype=np.float32)
    tgt, _ = uniform_square(m, seed=62, dtype=np.float32)
    dev = torch.device("cuda:0")
    s_d = torch.from_numpy(src).to(dev)
    t_d = torch.from_numpy(tgt).to(dev)
    L, p, err, ms = fmm2d.fmm2d_autotune(tiling, 1e-6, fmm2d.PREC_MIXED_TC | fmm2d.IN_F32, s_d, n, t_d, m)
    assert 0 < err <= 1e-6 / 3 and ms > 0
    phi, _ = run_gpu(tiling, src, u, tgt, levels=L, p=p, eps=1e-6, prec="tc", f32=True)
    idx = sample_targets(m, 512, seed=7)
    ref = direct(src.astype(np.float64), u.astype(np.float64), tgt[idx].astype(np.float64))
    assert rel_inf_error(phi[idx], ref) <= 1e-6
