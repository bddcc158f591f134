"""fmm2d_evaluate_graph: the evaluation recorded into a CUDA graph and
replayed.  Each replay must equal fmm2d_evaluate on the same plan bit for bit,
after the strengths change in place, and after a rebuild (which re-records);
the replayed potentials also meet eps against the direct sum (oracle) on
sampled targets."""
import numpy as np
import pytest

from gpu_util import _torch
from oracle.direct import direct, rel_inf_error
from paper_1204_3105_gb300.inputs import rng, uniform_square

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_3105_gb300 import build, fmm2d
    build.build()
    fmm2d.lib()


CASES = [("quad", "tc", None, 1e-6), ("tri", "tc", None, 1e-6), ("sept", "tc", None, 1e-6),
         ("quad", "fp64", 64, 1e-10), ("tri", "tc", 64, 1e-6)]


@pytest.mark.parametrize("tiling,prec,leaf,eps", CASES)
def test_graph_replay_equals_evaluate(tiling, prec, leaf, eps):
    from paper_1204_3105_gb300 import fmm2d
    t = _torch()
    dev = t.device("cuda:0")
    flags = {"tc": fmm2d.PREC_MIXED_TC | fmm2d.IN_F32, "fp64": fmm2d.PREC_FP64}[prec]
    dt = np.float32 if prec == "tc" else np.float64
    if leaf is not None:
        flags |= fmm2d.ADAPTIVE
    plan = fmm2d.Plan(tiling, levels=0, p=0, eps=eps, flags=flags)
    if leaf is not None:
        plan.set_leaf_size(leaf)
    s = t.cuda.Stream(device=dev)
    g = rng(71)
    try:
        for rebuild in range(2):
            n = 20000 + 3001 * rebuild
            xy, u = uniform_square(n, seed=300 + rebuild, dtype=dt)
            xy_d = t.from_numpy(xy).to(dev)
            u_d = t.from_numpy(u).to(dev)
            t.cuda.synchronize()
            plan.build(xy_d, n, xy_d, n, s)
            out_g = t.full((n,), float("nan"), dtype=t.float64, device=dev)
            out_e = t.full((n,), float("nan"), dtype=t.float64, device=dev)
            for rep in range(3):
                if rep > 0:   # new strengths in the same buffer
                    u_d.copy_(t.from_numpy(g.uniform(-1, 1, n).astype(dt)).to(dev))
                    t.cuda.synchronize()
                plan.evaluate_graph(u_d, out_g, s)
                s.synchronize()
                plan.evaluate(u_d, out_e, s)
                s.synchronize()
                a, b = out_g.cpu().numpy(), out_e.cpu().numpy()
                assert np.isfinite(a).all()
                assert np.array_equal(a, b), (tiling, prec, leaf, rebuild, rep)
            # the replayed potentials against the direct sum on sampled targets
            idx = np.random.default_rng(5).choice(n, 200, replace=False)
            uu = u_d.cpu().numpy().astype(np.float64)
            xx = xy.astype(np.float64)
            ref = direct(xx, uu, xx[idx])
            assert rel_inf_error(out_g.cpu().numpy()[idx], ref) <= eps
    finally:
        plan.close()
