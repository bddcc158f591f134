"""Parity of the field F_j = sum_i u_i / (y_j - x_i) (fmm2d_evaluate_field,
the derivative of eq. 1's complex potential, Sec. 2) with the FP64 oracle.

Tolerances, per precision form (eps_rel_inf on the complex field, i.e.
max_j |F_j - F*_j| / max_j |F*_j|):
* FP64, split and hybrid forms (the field's sums in FP64): the oracle FMM
  of the same (L, p) to 1e-10 (summation order only);
* FP32 forms (FP32 expansions, FP32 field sums): 1e-6, the tolerance of the
  potential at the default eps.
The potentials the call returns are the ones fmm2d_evaluate returns, bit
for bit.
"""
import numpy as np
import pytest

from gpu_util import _torch
from oracle.adaptive import adaptive_fmm
from oracle.direct import direct
from oracle.fmm import fmm, make_tiling
from paper_1204_3105_gb300.inputs import gaussian_mixture, sample_targets, uniform_square

pytestmark = pytest.mark.gpu

PREC = {"fp64": 0x0, "mixed": 0x1, "tc": 0x2, "hybrid": 0x3, "split": 0x4}
TOL = {"fp64": 1e-10, "split": 1e-10, "hybrid": 1e-10, "mixed": 1e-6, "tc": 1e-6}


@pytest.fixture(scope="module")
def fm():
    torch = _torch()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_3105_gb300 import build, fmm2d
    build.build()
    fmm2d.lib()
    return fmm2d


def field_err(f, ref):
    return float(np.max(np.abs(f - ref)) / np.max(np.abs(ref)))


def run_field(fm, tiling, src, u, tgt=None, levels=0, p=0, eps=1e-6, prec="fp64", f32=False,
              leaf_size=None, check_phi=True):
    torch = _torch()
    dev = torch.device("cuda:0")
    flags = PREC[prec] | fm.FIELD | (fm.IN_F32 if f32 else 0) | (fm.ADAPTIVE if leaf_size is not None else 0)
    dt = np.float32 if f32 else np.float64
    plan = fm.Plan(tiling, levels=levels, p=p, eps=eps, flags=flags)
    if leaf_size is not None:
        plan.set_leaf_size(leaf_size)
    s_d = torch.from_numpy(np.ascontiguousarray(src, dt)).to(dev)
    t_d = s_d if tgt is None else torch.from_numpy(np.ascontiguousarray(tgt, dt)).to(dev)
    n_s, n_t = len(src), len(src) if tgt is None else len(tgt)
    u_d = torch.from_numpy(np.ascontiguousarray(u, dt)).to(dev)
    phi = torch.full((max(1, n_t),), float("nan"), dtype=torch.float64, device=dev)
    fld = torch.full((max(1, 2 * n_t),), float("nan"), dtype=torch.float64, device=dev)
    plan.build(s_d, n_s, t_d, n_t)
    plan.evaluate_field(u_d, phi, fld)
    torch.cuda.synchronize()
    out_f = fld.cpu().numpy()[: 2 * n_t].view(np.complex128)
    out_p = phi.cpu().numpy()[:n_t]
    if check_phi:   # the potentials equal fmm2d_evaluate's
        phi2 = torch.full_like(phi, float("nan"))
        plan.evaluate(u_d, phi2)
        torch.cuda.synchronize()
        assert np.array_equal(phi2.cpu().numpy()[:n_t], out_p)
    info = plan.query()
    plan.close()
    return out_f, out_p, info


@pytest.mark.parametrize("tiling,L,p", [("quad", 4, 14), ("sept", 3, 14), ("tri", 4, 14)])
@pytest.mark.parametrize("prec", ["fp64", "split", "hybrid", "mixed", "tc"])
def test_field_matches_oracle_uniform(fm, tiling, L, p, prec):
    xy, u = uniform_square(9001, seed=31)
    f, phi, _ = run_field(fm, tiling, xy, u, levels=L, p=p, prec=prec)
    r = fmm(make_tiling(tiling, L), xy, u, xy, p, field=True)
    assert field_err(f, r.field) < TOL[prec], (tiling, prec, field_err(f, r.field))


@pytest.mark.parametrize("tiling,L", [("quad", 4), ("sept", 3), ("tri", 4)])
def test_field_separate_targets_converges_to_direct(fm, tiling, L):
    """Targets apart from the sources (some on sources), shifted domain:
    the FP64 form at p = 30 gives the direct field."""
    rng = np.random.default_rng(41)
    dom = (-1.0, 2.0, 2.0)
    src = np.column_stack([dom[0] + dom[2] * rng.random(4000), dom[1] + dom[2] * rng.random(4000)])
    tgt = np.column_stack([dom[0] + dom[2] * rng.random(2501), dom[1] + dom[2] * rng.random(2501)])
    tgt[:9] = src[:9]
    u = rng.normal(size=4000)
    torch = _torch()
    dev = torch.device("cuda:0")
    plan = fm.Plan(tiling, levels=L, p=30, flags=PREC["fp64"])
    plan.set_domain(*dom)
    s_d = torch.from_numpy(src).to(dev)
    t_d = torch.from_numpy(tgt).to(dev)
    u_d = torch.from_numpy(u).to(dev)
    phi = torch.empty(len(tgt), dtype=torch.float64, device=dev)
    fld = torch.empty(2 * len(tgt), dtype=torch.float64, device=dev)
    plan.build(s_d, len(src), t_d, len(tgt))
    plan.evaluate_field(u_d, phi, fld)
    f = fld.cpu().numpy().view(np.complex128)
    plan.close()
    _, g = direct(src, u, tgt, gradient=True)
    assert field_err(f, g) < 1e-9


@pytest.mark.parametrize("tiling,L", [("quad", 8), ("sept", 6), ("tri", 8)])
@pytest.mark.parametrize("prec", ["fp64", "hybrid", "tc"])
def test_field_adaptive_matches_oracle(fm, tiling, L, prec):
    """Clustered points on an adaptive tree (W lists, M2P')."""
    xy, u = gaussian_mixture(6000, seed=43, k=6, sigma=(0.002, 0.05))
    p = 14
    f, _, info = run_field(fm, tiling, xy, u, levels=L, p=p, prec=prec, leaf_size=24)
    r = adaptive_fmm(make_tiling(tiling, L), xy, u, xy, p, s=24, field=True)
    assert field_err(f, r.field) < TOL[prec], (tiling, prec, field_err(f, r.field))


@pytest.mark.parametrize("tiling", ["quad", "sept", "tri"])
def test_field_full_size_sampled(fm, tiling):
    """N = M = 2^20 uniform FP32 points, tensor-core form at the planner's
    (L, p) for eps = 1e-6: the field on 2048 sampled targets against the
    direct field."""
    n = 1 << 20
    xy, u = uniform_square(n, seed=2, dtype=np.float32)
    f, _, _ = run_field(fm, tiling, xy, u, prec="tc", f32=True, check_phi=False)
    idx = sample_targets(n, 2048, seed=5)
    x64, u64 = xy.astype(np.float64), u.astype(np.float64)
    _, g = direct(x64, u64, x64[idx], gradient=True)
    assert field_err(f[idx], g) < 1e-6


def test_field_edge_cases(fm):
    torch = _torch()
    dev = torch.device("cuda:0")
    xy, u = uniform_square(100, seed=3)
    plan = fm.Plan("quad", levels=2, p=8, flags=PREC["fp64"])
    x_d = torch.from_numpy(xy).to(dev)
    u_d = torch.from_numpy(u).to(dev)
    phi = torch.empty(100, dtype=torch.float64, device=dev)
    plan.build(x_d, 100, x_d, 100)
    with pytest.raises(fm.FMM2DError) as e:
        plan.evaluate_field(u_d, phi, None)
    assert e.value.status == fm.EINVAL
    # one point: nothing to sum, the field is zero
    one = torch.from_numpy(np.array([[0.25, 0.5]])).to(dev)
    plan.build(one, 1, one, 1)
    fld = torch.full((2,), 7.0, dtype=torch.float64, device=dev)
    plan.evaluate_field(u_d[:1], phi[:1], fld)
    torch.cuda.synchronize()
    assert fld.cpu().numpy().tolist() == [0.0, 0.0]
    plan.close()
    # an FP32-form plan made without FMM2D_FIELD refuses the field
    p32 = fm.Plan("quad", levels=2, p=8, flags=PREC["mixed"])
    p32.build(x_d, 100, x_d, 100)
    with pytest.raises(fm.FMM2DError) as e:
        p32.evaluate_field(u_d, phi, torch.empty(200, dtype=torch.float64, device=dev))
    assert e.value.status == fm.EINVAL
    p32.close()
