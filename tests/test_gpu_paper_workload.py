"""The experiments of Sec. 9 on the GPU, on the paper's own workload: S_opt
(Table 2) uniform points in each occupied leaf, picked by the regular-polygon
method of Fig. 10; the number of points changes with the number of occupied
leaves.  The paper ran double precision, so these runs use the FP64 form.

* N-sweep at p = 12 (N = M = 1152 ... 9216): every run matches the oracle
  FMM element by element (1e-11), and the trends of Sec. 9 hold: the maximum
  absolute error grows with N, the quadtree has the smallest error and the
  septree a larger one than the triangle quadtree.
* p-sweep at N = M = 5120 (p = 8 ... 24; at smaller p, S_opt points per
  leaf would need more leaves than these levels hold in the square): the
  error falls geometrically with p.
* runtime at fixed p grows linearly with N (measured with CUDA events).
The leaf levels give the three tilings leaves of about equal area (~1e-3 for
the sweeps); only leaves lying inside the domain square are filled.
"""
import math
import statistics

import numpy as np
import pytest

from gpu_util import _torch
from oracle.direct import direct, rel_inf_error
from oracle.fmm import fmm, make_tiling
from oracle.params import s_opt
from paper_1204_3105_gb300.inputs import polygon_points, rng

pytestmark = pytest.mark.gpu

TILINGS = ("quad", "sept", "tri")
LV = {"quad": 5, "sept": 4, "tri": 5}        # leaf area ~1e-3 in all three
LV_BIG = {"quad": 8, "sept": 7, "tri": 9}    # room for 2^19 points at S_opt


@pytest.fixture(scope="module")
def fm():
    torch = _torch()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_3105_gb300 import build, fmm2d
    build.build()
    fmm2d.lib()
    return fmm2d


def leaf_polygons(name, L, count, seed):
    """``count`` distinct leaves of the tiling (a seeded random subset, by
    keying random points of the square) that lie inside the unit square, as
    corner lists in world coordinates (oracle geometry)."""
    T = make_tiling(name, L)
    g = rng(seed)
    pts = g.random((count * 32 + 1024, 2))
    keys = T.keys(pts[:, 0], pts[:, 1])
    _, first = np.unique(keys, return_index=True)
    out = []
    for k in keys[np.sort(first)]:
        k = int(k)
        if name == "quad":
            V = T.vertices(k, L)
        elif name == "sept":
            V = [T.to_world(v) for v in T.leaf_vertices_frame(k)]
        else:
            V = [T.to_world(v) for v in T.vertices_frame(k, L)]
        V = np.array(V)
        if np.all((V.real >= 0) & (V.real < 1) & (V.imag >= 0) & (V.imag < 1)):
            out.append(V)
            if len(out) == count:
                break
    assert len(out) == count, (name, L, count, len(out))
    return np.array(out)


def paper_input(name, L, p, n, seed):
    per = int(round(s_opt(name, p, 1, 1)))          # S_opt for N = M
    V = leaf_polygons(name, L, max(1, n // per), seed)
    return polygon_points(V, per, seed + 1)


def gpu_fp64(fm, name, L, p, xy, u, reps=3):
    """FP64 form: potentials and the best build + evaluate time (ms)."""
    torch = _torch()
    dev = torch.device("cuda:0")
    st = torch.cuda.Stream(device=dev)
    plan = fm.Plan(name, levels=L, p=p, flags=fm.PREC_FP64)
    x_d = torch.from_numpy(xy).to(dev)
    u_d = torch.from_numpy(u).to(dev)
    out = torch.empty(len(xy), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(reps + 1):                       # the first run is a warm-up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        plan.build(x_d, len(xy), x_d, len(xy), st)
        plan.evaluate(u_d, out, st)
        e1.record(st)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    phi = out.cpu().numpy()
    plan.close()
    return phi, best


def test_n_sweep_p12(fm):
    p = 12
    sizes = (1152, 2304, 4608, 9216)
    err = {t: [] for t in TILINGS}
    for n in sizes:
        for t in TILINGS:
            e = []
            for sd in range(3):
                xy, u = paper_input(t, LV[t], p, n, seed=10 * n + sd)
                phi, _ = gpu_fp64(fm, t, LV[t], p, xy, u, reps=0)
                if sd == 0:     # parity with the oracle FMM of the same (L, p)
                    r = fmm(make_tiling(t, LV[t]), xy, u, xy, p)
                    assert rel_inf_error(phi, r.phi) < 1e-11, (t, n)
                e.append(float(np.max(np.abs(phi - direct(xy, u, xy)))))
            err[t].append(statistics.mean(e))
    print("\nN-sweep, p = 12, mean over 3 seeds of the max abs error:")
    for i, n in enumerate(sizes):
        print("  N=%5d  " % n + "  ".join("%s %.3g" % (t, err[t][i]) for t in TILINGS))
    for t in TILINGS:                                   # grows with N
        assert err[t][-1] > err[t][0], (t, err[t])
    for i in range(len(sizes)):                         # quadtree least, septree above triangle
        assert err["quad"][i] < err["sept"][i] and err["quad"][i] < err["tri"][i], i
        assert err["sept"][i] > err["tri"][i], i


def test_p_sweep_n5120(fm):
    ps = (8, 12, 16, 20, 24)
    err = {t: [] for t in TILINGS}
    for t in TILINGS:
        for p in ps:
            xy, u = paper_input(t, LV[t], p, 5120, seed=7000 + p)
            phi, _ = gpu_fp64(fm, t, LV[t], p, xy, u, reps=0)
            err[t].append(float(np.max(np.abs(phi - direct(xy, u, xy)))))
    print("\np-sweep, N = M = 5120, max abs error:")
    for i, p in enumerate(ps):
        print("  p=%2d  " % p + "  ".join("%s %.3g" % (t, err[t][i]) for t in TILINGS))
    for t in TILINGS:
        # geometric decay: every 4 more terms gain at least a factor 3, and the
        # fitted log-slope is below log 0.6 per term
        for a, b in zip(err[t], err[t][1:]):
            assert b < a / 3, (t, err[t])
        slope = np.polyfit(ps, np.log(err[t]), 1)[0]
        assert slope < math.log(0.6), (t, slope)
    for i, p in enumerate(ps):
        assert err["quad"][i] < min(err["sept"][i], err["tri"][i]), p


def test_runtime_linear_in_n(fm):
    """At fixed p = 12 the build + evaluate time grows linearly with N: from
    2^16 to 2^19 points (8x) the time grows between 2x and 12x."""
    p = 12
    sizes = (1 << 16, 1 << 17, 1 << 18, 1 << 19)
    ms = {t: [] for t in TILINGS}
    for t in TILINGS:
        for n in sizes:
            xy, u = paper_input(t, LV_BIG[t], p, n, seed=9000 + n)
            ms[t].append(gpu_fp64(fm, t, LV_BIG[t], p, xy, u)[1])
    print("\nruntime (ms, FP64 form, p = 12):")
    for i, n in enumerate(sizes):
        print("  N=%7d  " % n + "  ".join("%s %.3f" % (t, ms[t][i]) for t in TILINGS))
    for t in TILINGS:
        growth = ms[t][-1] / ms[t][0]
        assert 2.0 < growth < 12.0, (t, ms[t])
