"""Batched solves (fmm2d_build_forest): many independent instances in one
adaptive tree.  Each instance's result must equal the same instance solved
alone bit for bit (same finest level and leaf size), its tree and lists must
equal the oracle's adaptive FMM of that instance alone, and the potentials must
match the oracle within 1e-11 (FP64) or the requested 1e-6 (mixed forms)."""
import numpy as np
import pytest

from gpu_util import _torch, run_gpu
from oracle.adaptive import adaptive_fmm
from oracle.direct import direct, rel_inf_error
from oracle.fmm import make_tiling
from paper_1204_3105_gb300.inputs import rng, uniform_square

pytestmark = pytest.mark.gpu

B = {"quad": 4, "sept": 7, "tri": 4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_3105_gb300 import build, fmm2d
    build.build()
    fmm2d.lib()


def _batch(n_inst, seed, lo=20, hi=3000):
    g = rng(seed)
    sizes = np.exp(g.uniform(np.log(lo), np.log(hi), n_inst)).astype(np.int64)
    sizes[3] = 0                      # an empty instance
    sizes[5] = 1                      # a single point
    pts = [uniform_square(int(n), seed=seed * 100 + i) for i, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    xy = np.concatenate([p[0] for p in pts]) if off[-1] else np.zeros((0, 2))
    u = np.concatenate([p[1] for p in pts]) if off[-1] else np.zeros(0)
    return xy, u, off


def _forest(tiling, xy, u, off, p, prec="fp64", cap=32, f32=False):
    from paper_1204_3105_gb300 import fmm2d
    t = _torch()
    dev = t.device("cuda:0")
    flags = {"fp64": fmm2d.PREC_FP64, "mixed": fmm2d.PREC_MIXED, "tc": fmm2d.PREC_MIXED_TC}[prec]
    flags |= fmm2d.ADAPTIVE | (fmm2d.IN_F32 if f32 else 0)
    dt = np.float32 if f32 else np.float64
    plan = fmm2d.Plan(tiling, levels=0, p=p, flags=flags)
    plan.set_leaf_size(cap)
    xd = t.from_numpy(np.ascontiguousarray(xy, dt)).to(dev)
    ud = t.from_numpy(np.ascontiguousarray(u, dt)).to(dev)
    out = t.full((max(1, len(xy)),), float("nan"), dtype=t.float64, device=dev)
    plan.build_forest(xd, off)
    plan.evaluate(ud, out)
    t.cuda.synchronize()
    return out.cpu().numpy()[: len(xy)], plan


@pytest.mark.parametrize("tiling", ["quad", "sept", "tri"])
def test_forest_equals_instances_alone_and_oracle(tiling):
    xy, u, off = _batch(25, seed=41, hi=1500)
    p = 10
    phi, plan = _forest(tiling, xy, u, off, p)
    L = plan.query()["levels"]
    b = B[tiling]
    cells = plan.export("ad_cells")
    lists = {k: plan.export(k) for k in ("ad_u", "ad_w", "ad_x", "ad_v")}
    plan.close()
    for i in range(len(off) - 1):
        a, e = int(off[i]), int(off[i + 1])
        if e == a:
            continue
        alone, _ = run_gpu(tiling, xy[a:e], u[a:e], levels=L, p=p, prec="fp64", leaf_size=32)
        assert np.array_equal(phi[a:e], alone), i                      # bit for bit
        if e - a < 2:
            assert phi[a] == 0.0
            continue
        if i % 3:                     # the oracle on every third instance
            continue
        r = adaptive_fmm(make_tiling(tiling, L), xy[a:e], u[a:e], xy[a:e], p, s=32, record=True)
        assert rel_inf_error(phi[a:e], r.phi) < 1e-11, i
        # this instance's cells and lists, instance prefix removed
        mine = sorted((l, k % b ** l, sp) for l, k, sp in cells.tolist() if k // b ** l == i)
        want = sorted((l, n, int((l, n) in r.split)) for l, cs in enumerate(r.cells) for n in cs)
        assert mine == want, i
        for name, d, pairs in (("ad_u", r.U, True), ("ad_w", r.W, True), ("ad_x", r.X, True),
                               ("ad_v", {k: v for k, v in r.V.items() if v}, False)):
            got = sorted((lt, kt % b ** lt, ls, ks % b ** ls) for lt, kt, ls, ks in lists[name].tolist()
                         if kt // b ** lt == i)
            exp = sorted((la, aa, *(e2 if pairs else (la, e2))) for (la, aa), v in d.items() for e2 in v)
            assert got == exp, (i, name)


@pytest.mark.parametrize("tiling", ["quad", "sept", "tri"])
@pytest.mark.parametrize("prec", ["mixed", "tc"])
def test_forest_mixed_forms_within_eps(tiling, prec):
    xy, u, off = _batch(60, seed=42, lo=100, hi=6000)
    phi, plan = _forest(tiling, xy.astype(np.float32), u.astype(np.float32), off,
                        {"quad": 12, "sept": 13, "tri": 13}[tiling], prec=prec, cap=64, f32=True)
    plan.close()
    x64 = xy.astype(np.float32).astype(np.float64)
    u64 = u.astype(np.float32).astype(np.float64)
    for i in range(0, len(off) - 1, 7):
        a, e = int(off[i]), int(off[i + 1])
        if e - a < 2:
            continue
        ref = direct(x64[a:e], u64[a:e], x64[a:e])
        assert rel_inf_error(phi[a:e], ref) < 1e-6, (i, e - a)


@pytest.mark.parametrize("tiling", ["quad", "tri"])
def test_forest_fp32_forms_equal_instances_alone(tiling):
    """In the FP32 forms too, an instance in the forest gives bit for bit its
    result alone (every per-leaf and per-cell sum depends on that leaf or
    cell only)."""
    xy, u, off = _batch(12, seed=43, lo=200, hi=4000)
    x32, u32 = xy.astype(np.float32), u.astype(np.float32)
    for prec in ("mixed", "tc"):
        phi, plan = _forest(tiling, x32, u32, off, 12, prec=prec, cap=64, f32=True)
        L = plan.query()["levels"]
        plan.close()
        for i in (0, 4, 9):
            a, e = int(off[i]), int(off[i + 1])
            alone, _ = run_gpu(tiling, x32[a:e], u32[a:e], levels=L, p=12, prec=prec, f32=True,
                               leaf_size=64)
            assert np.array_equal(phi[a:e], alone), (prec, i)


def test_batch_workload_full_size_sampled():
    """The 4096-instance batch exactly as bench.py runs it (same instance
    sizes, tilings, seeds, leaf size 64, tensor-core form), on sampled
    instances and targets against the direct sum over each instance."""
    from paper_1204_3105_gb300.inputs import rng, uniform_square as us
    g = rng(2 + 40)
    count = 4096
    sizes = np.exp(g.uniform(np.log(256), np.log(65536), count)).astype(np.int64)
    tilings = g.integers(0, 3, count)
    for ti, name in enumerate(("quad", "sept", "tri")):
        idx = np.nonzero(tilings == ti)[0]
        pts = [us(int(sizes[i]), seed=1000 + int(i), dtype=np.float32) for i in idx]
        off = np.concatenate([[0], np.cumsum(sizes[idx])]).astype(np.int64)
        xy = np.concatenate([q[0] for q in pts])
        u = np.concatenate([q[1] for q in pts])
        phi, plan = _forest(name, xy, u, off, {"quad": 12, "sept": 14, "tri": 14}[name], prec="tc",
                            cap=64, f32=True)
        plan.close()
        sel = np.random.default_rng(ti).choice(len(idx), 6, replace=False)
        for k in sel:
            a, e = int(off[k]), int(off[k + 1])
            x64, u64 = xy[a:e].astype(np.float64), u[a:e].astype(np.float64)
            t = np.random.default_rng(int(k)).choice(e - a, min(64, e - a), replace=False)
            ref = direct(x64, u64, x64[t])
            assert rel_inf_error(phi[a:e][t], ref) < 1e-6, (name, int(k), e - a)


def test_forest_argument_errors():
    from paper_1204_3105_gb300 import fmm2d
    t = _torch()
    xd = t.zeros((10, 2), dtype=t.float64, device="cuda:0")
    uniform = fmm2d.Plan("quad", p=8, flags=fmm2d.PREC_FP64)
    with pytest.raises(fmm2d.FMM2DError):
        uniform.build_forest(xd, np.array([0, 10]))
    ad = fmm2d.Plan("quad", p=8, flags=fmm2d.PREC_FP64 | fmm2d.ADAPTIVE)
    with pytest.raises(fmm2d.FMM2DError):
        ad.build_forest(xd, np.array([0, 6, 4, 10]))
    with pytest.raises(fmm2d.FMM2DError):
        ad.build_forest(xd, np.array([1, 10]))
