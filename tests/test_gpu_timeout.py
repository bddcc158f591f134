"""The bounded device waits give up cleanly.

A test switch (fmm2d_plan_set_debug_stall) makes the first operator wait of
every tensor-core M2L CTA wait on an mbarrier that nothing arrives on, before
any MMA is issued.  The wait runs out after about a second, the CTA lets its
operator copies land, frees its tensor memory and returns; the plan reports
device_error.  The same plan then evaluates normally and matches the oracle:
the context and the plan stay usable.  No GPU fault is involved.
"""
import numpy as np
import pytest

from gpu_util import _torch
from oracle.direct import rel_inf_error
from oracle.fmm import fmm, make_tiling
from paper_1204_3105_gb300.inputs import uniform_square

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_plan_recovers():
    torch = _torch()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_3105_gb300 import build, fmm2d
    build.build()
    dev = torch.device("cuda:0")
    n, L, p = 12007, 4, 12
    xy, u = uniform_square(n, seed=9)
    plan = fmm2d.Plan("quad", levels=L, p=p, flags=fmm2d.PREC_MIXED_TC)
    x_d = torch.from_numpy(xy).to(dev)
    u_d = torch.from_numpy(u).to(dev)
    out = torch.empty(n, dtype=torch.float64, device=dev)
    plan.build(x_d, n, x_d, n)
    plan.set_debug_stall(True)
    plan.evaluate(u_d, out)
    torch.cuda.synchronize()
    assert plan.query()["device_error"] != 0
    plan.set_debug_stall(False)
    out.fill_(float("nan"))
    plan.evaluate(u_d, out)
    torch.cuda.synchronize()
    assert plan.query()["device_error"] == 0
    ref = fmm(make_tiling("quad", L), xy, u, xy, p).phi
    assert rel_inf_error(out.cpu().numpy(), ref) < 1e-6
    plan.close()
