"""The continuous-batching server (fmm2d_serve_*): a request gives the same
result alone and mixed with concurrent requests, results match the oracle's
direct sum within the requested eps, and admission respects the HBM budget."""
import time

import numpy as np
import pytest

from oracle.direct import direct, rel_inf_error
from paper_1204_3105_gb300.inputs import gaussian_mixture, rng, sample_targets, uniform_square

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_3105_gb300 import build, fmm2d
    build.build()
    fmm2d.lib()
    return fmm2d


def _mix(count, seed):
    g = rng(seed)
    reqs = []
    for i in range(count):
        n = int(np.exp(g.uniform(np.log(1e3), np.log(1.5e5))))
        tiling = ("quad", "sept", "tri")[int(g.integers(0, 3))]
        eps = (1e-4, 1e-8)[int(g.integers(0, 2))]
        if g.random() < 0.5:
            xy, u = uniform_square(n, seed=seed * 1000 + i)
        else:
            xy, u = gaussian_mixture(n, seed=seed * 1000 + i, k=8)
        reqs.append((tiling, xy, u, eps))
    return reqs


def test_alone_equals_in_the_mix(fm):
    sv = fm.Server(8 << 30, max_slots=6)
    xy, u = uniform_square(60000, seed=21, dtype=np.float32)
    alone = np.zeros(len(xy))
    t = sv.submit("sept", xy, u, alone, eps=1e-6)
    r = sv.wait(t)
    assert r["status"] == 0
    others = _mix(24, seed=5)
    outs, tickets = [], []
    for k, (tiling, pxy, pu, eps) in enumerate(others):
        o = np.zeros(len(pxy))
        outs.append(o)
        tickets.append(sv.submit(tiling, pxy, pu, o, eps=eps))
        if k == 12:
            mixed = np.zeros(len(xy))
            tm = sv.submit("sept", xy, u, mixed, eps=1e-6)
    results = [sv.wait(t) for t in tickets]
    rm = sv.wait(tm)
    assert rm["status"] == 0 and all(r["status"] == 0 for r in results)
    assert len({r["slot"] for r in results}) > 1          # the work was spread over slots
    assert np.array_equal(alone, mixed)                   # bit for bit
    # every mixed request against the oracle's direct sum, at its own eps
    for k, (tiling, pxy, pu, eps) in enumerate(others):
        idx = sample_targets(len(pxy), 200, seed=k)
        ref = direct(pxy, pu, pxy[idx])
        assert rel_inf_error(outs[k][idx], ref) <= eps, (k, tiling, eps, len(pxy))
    sv.close()


SIZES = (1000, 10000, 100000)


@pytest.mark.parametrize("tiling", ["quad", "sept", "tri"])
@pytest.mark.parametrize("tree", ["adaptive", "uniform"])
def test_served_results_meet_their_eps(fm, tiling, tree):
    """Served requests of the serving workload's two tolerances (1e-4 and
    1e-8), at N = 1e3, 1e4 and 1e5, uniform and 8-cluster points, each meet
    their own eps: eps_rel_inf against the direct sum of eq. (2) on 256
    sampled targets (the server picks the precision form from eps and N)."""
    sv = fm.Server(16 << 30, max_slots=4)
    flags = fm.ADAPTIVE if tree == "adaptive" else 0
    reqs = []
    for eps in (1e-8, 1e-4):
        for n in SIZES:
            for cl in (False, True):
                seed = 7000 + n // 100 + (1 if cl else 0) + (2 if eps < 1e-6 else 0)
                if cl:
                    xy, u = gaussian_mixture(n, seed=seed, k=8)
                else:
                    xy, u = uniform_square(n, seed=seed)
                o = np.full(n, np.nan)
                reqs.append((eps, n, cl, xy, u, o, sv.submit(tiling, xy, u, o, eps=eps, flags=flags)))
    bad = []
    for eps, n, cl, xy, u, o, t in reqs:
        r = sv.wait(t, 600000.0)
        assert r["status"] == 0
        idx = sample_targets(n, 256, seed=n)
        err = rel_inf_error(o[idx], direct(xy, u, xy[idx]))
        if not err <= eps:
            bad.append((eps, n, "cluster" if cl else "uniform", r["flags"] & 7, r["p"], err))
    sv.close()
    assert not bad, bad


def test_small_requests_merge_into_one_forest(fm):
    """Small adaptive requests that wait together with equal tiling, eps and
    flags are solved as one forest; each result equals the same request
    solved alone within eps, and the direct sum on samples."""
    sv = fm.Server(8 << 30, max_slots=1)
    bxy, bu = uniform_square(400000, seed=40, dtype=np.float32)
    big = np.zeros(len(bxy))
    tb = sv.submit("quad", bxy, bu, big, eps=1e-6, flags=fm.ADAPTIVE)   # holds the only slot
    reqs = []
    for i in range(20):
        n = 500 + 173 * i
        if i % 2:
            xy, u = uniform_square(n, seed=300 + i, dtype=np.float32)
        else:
            xy, u = gaussian_mixture(n, seed=300 + i, k=8, dtype=np.float32)
            u = u.astype(np.float32)
        o = np.zeros(n)
        reqs.append((xy, u, o, sv.submit("tri", xy, u, o, eps=1e-6, flags=fm.ADAPTIVE)))
    res = [sv.wait(t) for (_, _, _, t) in reqs]
    assert sv.wait(tb)["status"] == 0
    assert all(r["status"] == 0 for r in res)
    assert max(r["batched"] for r in res) > 1                       # merged into a forest
    for (xy, u, o, _), r in zip(reqs, res):
        a = np.zeros(len(xy))
        ra = sv.wait(sv.submit("tri", xy, u, a, eps=1e-6, flags=fm.ADAPTIVE))
        assert ra["status"] == 0 and ra["batched"] == 1             # alone
        assert np.max(np.abs(a - o)) <= 1e-6 * np.max(np.abs(a))
    for k in (3, 8):
        xy, u, o, _ = reqs[k]
        x64, u64 = xy.astype(np.float64), u.astype(np.float64)
        idx = sample_targets(len(xy), 200, seed=k)
        ref = direct(x64, u64, x64[idx])
        assert rel_inf_error(o[idx], ref) <= 1e-6
    sv.close()


def test_budget_admission_and_busy(fm):
    xy, u = uniform_square(200000, seed=3, dtype=np.float32)
    est_one = 200000 * (3 * 4 + 2 * 0 + 8) + 200000 * 96 + 200000 * 1024 // 16 + (32 << 20)
    sv = fm.Server(int(2.5 * est_one), max_slots=8)     # at most two of these at once
    outs, tickets = [], []
    for i in range(6):
        o = np.zeros(len(xy))
        outs.append(o)
        tickets.append(sv.submit("quad", xy, u, o, eps=1e-6))
    peak_running, peak_bytes = 0, 0
    t0 = time.time()
    while time.time() - t0 < 60:
        st = sv.stats()
        peak_running = max(peak_running, st["running"])
        peak_bytes = max(peak_bytes, st["bytes_in_use"])
        assert st["bytes_in_use"] <= st["budget_bytes"]
        if st["completed"] == 6:
            break
        time.sleep(0.001)
    assert peak_running <= 2
    res = [sv.wait(t) for t in tickets]
    assert all(r["status"] == 0 for r in res)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    big, bu = uniform_square(4_000_000, seed=4, dtype=np.float32)
    with pytest.raises(fm.FMM2DError) as e:
        sv.submit("quad", big, bu, np.zeros(len(big)), eps=1e-6)
    assert e.value.status == fm.EBUSY
    sv.close()


def test_concurrent_requests_of_different_p(fm):
    """Requests of the float-float (hybrid) form with different expansion
    orders p run at once on several slots.  The kernel's shared-memory size
    depends on p and its limit is one setting for the whole process; every
    request must still launch and succeed (a slot lowering the limit while
    another launched used to fail that launch)."""
    sv = fm.Server(16 << 30, max_slots=8)
    reqs = []
    for i in range(48):
        n = 20000 + 997 * i
        xy, u = gaussian_mixture(n, seed=900 + i, k=8)
        o = np.zeros(n)
        t = sv.submit(("quad", "sept", "tri")[i % 3], xy, u, o, eps=1e-8, p=14 + (i % 24),
                      flags=fm.ADAPTIVE)
        reqs.append(t)
    res = [sv.wait(t, 600000.0) for t in reqs]
    sv.close()
    assert all(r["status"] == 0 for r in res), [(r["status"], r["error"]) for r in res if r["status"]]
