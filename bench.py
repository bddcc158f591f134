"""Benchmark: FMM evaluation points/s at eps = 1e-6 for the three tilings.

Workload (one step): for each tiling (quadtree, septree, triangle quadtree)
one full FMM - fmm2d_build (keys, sort, cells, lists) + fmm2d_evaluate
(P2M, M2M, M2L, L2L, L2P, P2P) - over N = M = 2^20 seeded points uniform in
the unit square (sources = targets), FP32 points and strengths uniform in
[-1, 1], p and L from the planner for eps = 1e-6, mixed precision.
The three FMMs of a step are independent and run on three streams (one
tiling's build overlaps the evaluation of the one before it); --serial runs
them one after another on one stream.  value = 3 * M / (device time of one
step), all ranks summed.

--impl reference times the FP64 CPU oracle (the reference arm of this
build) on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_POINTS = 2 ** 20
EPS = 1e-6
TILINGS = ("quad", "sept", "tri")
SEED = 2
MUFU_PER_CLK_SM = 16      # lg2 results per clock per SM (MUFU pipe)
# DRAM bytes (read + write) of one P2P launch per tiling on the 2^20-point
# workload, from an ncu capture of the current kernel (dram__bytes_read.sum +
# dram__bytes_write.sum; summarised in profiles/p2p_x2_traffic_2p20.md)
P2P_TRAFFIC = {"quad": 18322688 + 0, "sept": 17506048 + 0, "tri": 19338240 + 0}
FP32_LANES_SM = 128       # FP32 FMA lanes per SM


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def eps_label(eps):
    """eps as the metric strings print it: 1e-06 -> '1e-6' (one formatter for
    both arms, so that their metric names are identical)."""
    m, e = ("%.0e" % eps).split("e")
    return "%se%d" % (m, int(e))


def metric_name(eps):
    return "FMM eval points/s at eps=%s (3 tilings)" % eps_label(eps)


# Clock sampler: a separate process polls NVML (read-only queries) every
# 2 ms and appends "monotonic_time sm_mhz max_mhz power_mw reasons" lines to a
# file, so that even a timed region of a few tens of milliseconds holds
# samples and the benchmark process itself is not disturbed.
_SAMPLER = r"""
import ctypes, sys, time
bus, out, period = sys.argv[1], sys.argv[2], float(sys.argv[3])
f = open(out, "w", buffering=1)
try:
    nv = ctypes.CDLL("libnvidia-ml.so.1")
    if nv.nvmlInit_v2() != 0:
        raise OSError("nvmlInit")
    h = ctypes.c_void_p()
    if bus.startswith("pci:"):
        r = nv.nvmlDeviceGetHandleByPciBusId_v2(bus[4:].encode(), ctypes.byref(h))
    else:
        r = nv.nvmlDeviceGetHandleByIndex_v2(int(bus[4:]), ctypes.byref(h))
    if r != 0:
        raise OSError("handle %d" % r)
    get_reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or         nv.nvmlDeviceGetCurrentClocksThrottleReasons
    sm, mx, pw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
    nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))
    while True:
        nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(sm))
        nv.nvmlDeviceGetPowerUsage(h, ctypes.byref(pw))
        get_reasons(h, ctypes.byref(rs))
        f.write("%.6f %d %d %d %d\n" % (time.monotonic(), sm.value, mx.value, pw.value, rs.value))
        time.sleep(period)
except Exception as e:
    f.write("error %s\n" % e)
"""
_REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
            0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}


class Clocks:
    """SM clocks and throttle reasons of the benchmarked GPU, sampled by NVML
    in a separate process; mark() the start and end of the timed region and
    summary() reports the samples taken inside it."""

    def __init__(self, device_index=0, period_s=0.002):
        self.index = device_index
        self.period = period_s
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def _bus(self):
        try:
            import torch
            pr = torch.cuda.get_device_properties(self.index)
            if hasattr(pr, "pci_bus_id"):
                return "pci:%08x:%02x:%02x.0" % (getattr(pr, "pci_domain_id", 0), pr.pci_bus_id,
                                                 pr.pci_device_id)
        except Exception:
            pass
        return "idx:%d" % self.index

    def __enter__(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".txt")
        os.close(fd)
        try:
            self.proc = subprocess.Popen([sys.executable, "-c", _SAMPLER, self._bus(), self.path,
                                          str(self.period)], stdout=subprocess.DEVNULL,
                                         stderr=subprocess.DEVNULL)
            t = time.time()   # wait for the first sample (NVML initialised)
            while time.time() - t < 10.0 and self.proc.poll() is None:
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.01)
        except OSError:
            self.proc = None
        self.t0 = time.monotonic()
        return self

    def start(self):
        self.t0 = time.monotonic()

    def stop(self):
        self.t1 = time.monotonic()

    def __exit__(self, *a):
        if self.t1 is None:
            self.t1 = time.monotonic()
        time.sleep(2 * self.period)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows, err = [], None
        try:
            with open(self.path) as f:
                for line in f:
                    if line.startswith("error"):
                        err = line.strip()
                        continue
                    v = line.split()
                    if len(v) == 5:
                        rows.append((float(v[0]), int(v[1]), int(v[2]), int(v[3]), int(v[4])))
            os.unlink(self.path)
        except OSError:
            pass
        inside = [r for r in rows if self.t0 <= r[0] <= self.t1]
        if not inside:   # a region shorter than the period: the next sample after its start
            inside = [r for r in rows if r[0] >= self.t0][:1]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                    "note": err or "no NVML sample"}
        reasons = sorted({name for r in inside for bit, name in _REASONS.items() if r[4] & bit})
        return {"sm_mhz": statistics.median(r[1] for r in inside),
                "sm_max_mhz": max(r[2] for r in inside), "reasons": reasons,
                "power_w_median": statistics.median(r[3] for r in inside) / 1e3,
                "samples": len(inside), "window_ms": 1e3 * (self.t1 - self.t0),
                "source": "NVML, every %g ms" % (1e3 * self.period)}


def oracle_sample(tilings=TILINGS, n=16384, seed=SEED, eps=EPS):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload:
    N = M = n uniform points per tiling, the planner's L and p for eps."""
    t0 = time.perf_counter()
    for t in tilings:
        _oracle_task((t, n, seed, eps))
    dt = time.perf_counter() - t0
    return len(tilings) * n / dt, dt


def _oracle_task(args):
    """One oracle FMM (one tiling, N = M = n uniform points); returns seconds."""
    from oracle.fmm import fmm, make_tiling
    from oracle.params import auto_levels, p_from_eps
    from paper_1204_3105_gb300.inputs import uniform_square
    tiling, n, seed, eps = args
    xy, u = uniform_square(n, seed=seed, dtype=np.float32)
    xy = xy.astype(np.float64)
    u = u.astype(np.float64)
    t0 = time.perf_counter()
    fmm(make_tiling(tiling, auto_levels(tiling, n)), xy, u, xy, p_from_eps(tiling, eps))
    return time.perf_counter() - t0


def _oracle_warm(_):
    import oracle.fmm  # noqa: F401  (imports paid before the timed maps)
    return os.getpid()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The oracle on every host core: one single-threaded process per core
    (spawned, so that it holds no CUDA state), each running whole oracle
    FMMs; throughput = points of all tasks / wall time of the batch."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        self.cores = cores or host_cores()
        keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                              "MKL_NUM_THREADS")}
        for k in keep:
            os.environ[k] = "1"   # one thread per process: the pool supplies the parallelism
        try:
            self.pool = mp.get_context("spawn").Pool(self.cores)
        finally:
            for k, v in keep.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.pool.map(_oracle_warm, range(self.cores), chunksize=1)

    def run(self, n, eps=EPS, tasks=None, seed0=SEED + 100):
        tasks = tasks or self.cores * len(TILINGS)
        work = [(TILINGS[i % len(TILINGS)], n, seed0 + i, eps) for i in range(tasks)]
        t0 = time.perf_counter()
        self.pool.map(_oracle_task, work, chunksize=1)
        dt = time.perf_counter() - t0
        return tasks * n / dt, dt, tasks

    def close(self):
        self.pool.close()
        self.pool.join()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        return dist, rank, ws
    return None, rank, ws


def replica_aggregate(dist, ms_local, units_per_rank, ws, device=None):
    """Whole-job throughput of N replicas: the slowest rank's time (max over
    ranks, one all_reduce) and units = every rank's units."""
    ms = float(ms_local)
    if dist is not None and ws > 1:
        import torch
        tm = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        ms = float(tm.item())
    return ms, ws * units_per_rank / (ms / 1e3)


def run_reference(args):
    dist, rank, ws = dist_setup(args)
    if rank != 0:
        return
    pool = OraclePool()
    # bounded sample: the whole run takes about --ref-seconds on the host; a
    # step is 3 oracle FMMs (one per tiling) on each core, N = M = n each
    _, dt_cal, _ = pool.run(2048, tasks=pool.cores)
    per_step = args.ref_seconds / max(1, args.steps + args.warmup)
    n = int(min(args.ref_points, max(512, 2048 * (per_step / 3) / max(dt_cal, 1e-3))))
    for _ in range(args.warmup):
        pool.run(n)
    times, tasks = [], 0
    for _ in range(args.steps):
        _, dt, tasks = pool.run(n)
        times.append(dt)
    pool.close()
    ms = 1e3 * statistics.mean(times)
    value = tasks * n / (ms / 1e3)
    sample = ("N=M=%d uniform points per FMM, %d FP64 oracle FMMs per step (the 3 tilings on each "
              "of %d host cores, one process per core)" % (n, tasks, pool.cores))
    line = {"impl": "reference", "metric": metric_name(EPS),
            "value": value, "unit": "points/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "N=M=%d uniform unit square, quad+sept+tri, eps=%s (oracle sample "
                                   "of the N=M=2^20 workload)" % (n, eps_label(EPS))},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": pool.cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_ours(args):
    import torch
    from paper_1204_3105_gb300 import fmm2d
    from paper_1204_3105_gb300.inputs import uniform_square

    dist, rank, ws = dist_setup(args)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    fmm2d.lib()

    xy, u = uniform_square(N_POINTS, seed=SEED, dtype=np.float32)
    xy_d = torch.from_numpy(xy).to(dev)
    u_d = torch.from_numpy(u).to(dev)
    outs = {t: torch.empty(N_POINTS, dtype=torch.float64, device=dev) for t in args.tilings}
    prec = {"tc": fmm2d.PREC_MIXED_TC, "mixed": fmm2d.PREC_MIXED, "fp64": fmm2d.PREC_FP64,
            "hybrid": fmm2d.PREC_HYBRID, "split": fmm2d.PREC_SPLIT}[args.prec]
    tuned = {}
    fixed = {}
    for item in filter(None, args.params.split(",")):
        t, L, p = item.split(":")
        fixed[t] = (int(L), int(p), None, None)
    for t in args.tilings:
        if t in fixed:
            tuned[t] = fixed[t]
        elif args.no_tune:
            tuned[t] = (0, 0, None, None)
        else:   # measured (L, p) for eps on this point set (seeded probe strengths)
            tuned[t] = fmm2d.fmm2d_autotune(t, args.eps, prec | fmm2d.IN_F32, xy_d, N_POINTS, xy_d,
                                            N_POINTS, stream=stream)
    plans = {t: fmm2d.Plan(t, tuned[t][0], tuned[t][1], args.eps, prec | fmm2d.IN_F32)
             for t in args.tilings}
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device=dev)   # 256 MB > L2

    def step(per):
        for t in args.tilings:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plans[t].build(xy_d, N_POINTS, xy_d, N_POINTS, stream)
            plans[t].evaluate(u_d, outs[t], stream)
            e1.record(stream)
            per[t].append((e0, e1))
            flush.zero_()

    # the three tilings are independent problems: each runs on a stream of
    # its own, so one tiling's build (latency-bound small kernels and one
    # host read-back) overlaps the evaluation of the one before it
    tstreams = {t: torch.cuda.Stream(device=dev) for t in args.tilings}

    # ... and each is issued from a host thread of its own: fmm2d_build waits
    # for its own level counts, so from one thread the three builds (chains of
    # small latency-bound kernels) would follow one another
    from concurrent.futures import ThreadPoolExecutor
    issuers = ThreadPoolExecutor(len(args.tilings), initializer=torch.cuda.set_device,
                                 initargs=(local,))

    def solve_on(t, start, xs, us):   # one tiling's build + evaluate on its stream
        ts = tstreams[t]
        ts.wait_event(start)
        plans[t].build(xs, N_POINTS, xs, N_POINTS, ts)
        plans[t].evaluate(us, outs[t], ts)
        d = torch.cuda.Event()
        d.record(ts)
        return d

    def step_concurrent(evs):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for d in issuers.map(lambda t: solve_on(t, e0, xy_d, u_d), args.tilings):
            stream.wait_event(d)
        e1.record(stream)
        evs.append((e0, e1))
        flush.zero_()

    warm = {t: [] for t in args.tilings}
    for _ in range(args.warmup):
        step(warm)
        step_concurrent([])
    torch.cuda.synchronize()
    per = {t: [] for t in args.tilings}
    whole = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        clk.start()
        for _ in range(args.steps):
            if args.serial:
                step(per)
            else:
                step_concurrent(whole)
        torch.cuda.synchronize()
        clk.stop()
    if dist:
        dist.barrier()
    if not args.serial:   # per-tiling times: the same steps, one tiling after another
        for _ in range(min(args.steps, 20)):
            step(per)
        torch.cuda.synchronize()
    tt = {t: [a.elapsed_time(b) for a, b in per[t]] for t in args.tilings}
    # stage split: a few more steps with per-stage CUDA events on the stream of
    # each stage (far-field stages concurrent with P2P, as in the timed steps;
    # kept out of the timed steps, whose host enqueue they would slow)
    n_prof = 0 if args.no_profile else 5
    for t in args.tilings:
        plans[t].set_profiling(0 if args.no_profile else 1)
    for _ in range(n_prof):
        step({t: [] for t in args.tilings})
    torch.cuda.synchronize()
    stage = {t: {k: (v[0] / max(1, n_prof), v[1] / max(1, n_prof))
                 for k, v in plans[t].stage_times().items()} for t in args.tilings}
    # one more step with the stages serialised: each stage's own time
    for t in args.tilings:
        plans[t].set_profiling(0 if args.no_profile else 2)
    step({t: [] for t in args.tilings})
    torch.cuda.synchronize()
    stage_iso = {t: plans[t].stage_times() for t in args.tilings}
    for t in args.tilings:
        plans[t].set_profiling(0)
    info = {t: plans[t].query() for t in args.tilings}
    ms_serial = sum(statistics.mean(tt[t]) for t in args.tilings)
    ms_step = ms_serial if args.serial else statistics.mean(a.elapsed_time(b) for a, b in whole)
    ms_step, value = replica_aggregate(dist, ms_step, len(args.tilings) * N_POINTS, ws, dev)

    # the plain FP64 GPU form on the same points, (L, p) tuned for the same eps
    fp64_form = None
    if not args.no_fp64_form and args.prec != "fp64":
        f64 = {}
        for t in args.tilings:
            L64, p64, e64, _ = fmm2d.fmm2d_autotune(t, args.eps, fmm2d.PREC_FP64 | fmm2d.IN_F32, xy_d, N_POINTS,
                                                    xy_d, N_POINTS, stream=stream)
            pl64 = fmm2d.Plan(t, L64, p64, args.eps, fmm2d.PREC_FP64 | fmm2d.IN_F32)
            ts64 = []
            for it in range(1 + args.fp64_steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pl64.build(xy_d, N_POINTS, xy_d, N_POINTS, stream)
                pl64.evaluate(u_d, outs[t], stream)
                e1.record(stream)
                e1.synchronize()
                if it > 0:
                    ts64.append(e0.elapsed_time(e1))
                flush.zero_()
            pl64.close()
            ms64 = statistics.mean(ts64)
            f64[t] = {"points_per_s": N_POINTS / (ms64 / 1e3), "ms": ms64, "L": L64, "p": p64,
                      "tune_probe_err": e64}
        ms64_step = sum(v["ms"] for v in f64.values())
        fp64_form = {"value": ws * len(args.tilings) * N_POINTS / (ms64_step / 1e3), "unit": "points/s",
                     "ms_per_step": ms64_step, "steps": args.fp64_steps, "per_tiling": f64,
                     "speedup_of_mixed": ms64_step / ms_step}

    # e2e: host buffers, copies inside the timed region, through the same ABI
    xy_h = torch.from_numpy(xy).pin_memory()
    u_h = torch.from_numpy(u).pin_memory()
    res_h = {t: torch.empty(N_POINTS, dtype=torch.float64).pin_memory() for t in args.tilings}
    e2e = []
    copy_stream = torch.cuda.Stream(device=dev)   # device->host copies overlap the next tiling
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xd = xy_h.to(dev, non_blocking=True)
        ud = u_h.to(dev, non_blocking=True)
        ready = torch.cuda.Event()
        ready.record(stream)
        if args.serial:
            dones = []
            for t in args.tilings:
                stream.wait_event(ready)
                plans[t].build(xd, N_POINTS, xd, N_POINTS, stream)
                plans[t].evaluate(ud, outs[t], stream)
                done = torch.cuda.Event()
                done.record(stream)
                dones.append(done)
        else:
            dones = list(issuers.map(lambda t: solve_on(t, ready, xd, ud), args.tilings))
        for t, done in zip(args.tilings, dones):
            copy_stream.wait_event(done)
            with torch.cuda.stream(copy_stream):
                res_h[t].copy_(outs[t], non_blocking=True)
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e.append(time.perf_counter() - t0)
    e2e_v = ws * len(args.tilings) * N_POINTS / statistics.mean(e2e)

    # roofline of the dominant kernel (ALU peaks measured on this device)
    peaks, src = _peaks()
    alu = fmm2d.fmm2d_measure_alu_peaks()
    sm_count = alu["sms"]
    clk_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    tot = {}
    for t in args.tilings:
        for k, (ms, n) in stage[t].items():
            tot.setdefault(k, [0.0, 0])
            tot[k][0] += ms
            tot[k][1] += n
    tot_iso = {}
    for t in args.tilings:
        for k, (ms, n) in stage_iso[t].items():
            tot_iso.setdefault(k, [0.0, 0])
            tot_iso[k][0] += ms
            tot_iso[k][1] += n

    def roofline(tt_, note):
        dom = max(tt_, key=lambda k: tt_[k][0])
        if tt_[dom][0] <= 0.0:
            return None
        if dom == "p2p":
            # one MUFU log2 per pair; peak = measured lg2 throughput
            pairs = sum(info[t]["n_p2p_pairs"] for t in args.tilings)
            peak = alu["lg2_gops"]
            ach = pairs / (tt_[dom][0] / 1e3) / 1e9
            traffic = None
            if all(t in P2P_TRAFFIC for t in args.tilings):
                traffic = sum(P2P_TRAFFIC[t] for t in args.tilings) / len(args.tilings)
            return {"kernel": "k_p2p_x2 (P2P)", "bound": "alu", "achieved": ach, "peak": peak,
                    "unit": "Gpair/s", "frac": ach / peak, "traffic": traffic,
                    "traffic_note": "bytes per launch, mean of the tilings' launches (ncu): "
                                    "the sorted sources read once (16 B each); algorithmic "
                                    "16.8 MB per launch",
                    "peak_source": "measured MUFU lg2 rate (fmm2d_measure_alu_peaks), one lg2 per pair",
                    "timing": note}
        fl = 0.0
        for t in args.tilings:
            p = info[t]["p"]
            fl += info[t]["n_m2l"] * 8.0 * p * (p + 1)
        peak = alu["fp32_tflops"]
        ach = fl / (tt_[dom][0] / 1e3) / 1e12
        return {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None,
                "peak_source": "measured FP32 FMA rate (fmm2d_measure_alu_peaks)", "timing": note}

    def roofline_m2l(tt_, note):
        """The tensor-core M2L against the measured TF32 tensor rate: useful
        flops 8 p (p + 1) per translation (a complex (p+1) x p product); the
        split form issues five TF32 products for each."""
        ms_ = tt_.get("m2l", (0.0, 0))[0]
        if args.prec != "tc" or ms_ <= 0.0 or not alu.get("tf32_tflops"):
            return None
        fl = sum(info[t]["n_m2l"] * 8.0 * info[t]["p"] * (info[t]["p"] + 1) for t in args.tilings)
        ach = fl / (ms_ / 1e3) / 1e12
        return {"kernel": "k_m2l_tc (M2L, tcgen05 kind::tf32)", "bound": "tensor", "achieved": ach,
                "issued": 5 * ach, "peak": alu["tf32_tflops"], "unit": "TFLOP/s",
                "frac": ach / alu["tf32_tflops"], "frac_issued": 5 * ach / alu["tf32_tflops"],
                "peak_source": "measured TF32 tcgen05 rate (fmm2d_measure_alu_peaks)", "timing": note}

    lg2_p2p = args.prec in ("tc", "mixed")   # the P2P roofline counts one MUFU lg2 per pair
    roof = roofline(tot, "CUDA events around the stage, 5 steps after the timed ones (far field concurrent)") \
        if lg2_p2p else None
    roof_iso = roofline(tot_iso, "CUDA events, one extra step with the stages serialised") if lg2_p2p else None

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v1, dt1 = oracle_sample(n=args.ref_points, eps=args.eps)
        pool = OraclePool()
        vc, dtc, ntask = pool.run(args.ref_points, eps=args.eps)
        pool.close()
        cpu = {"value": vc, "unit": "points/s", "cores": pool.cores, "kind": "oracle",
               "sample": "N=M=%d uniform points per FMM, eps=%s: %d FP64 oracle FMMs (the 3 tilings "
                         "on each of %d host cores, one process per core) in %.1f s"
                         % (args.ref_points, eps_label(args.eps), ntask, pool.cores, dtc),
               "single_core": {"value": v1, "unit": "points/s", "cores": 1,
                               "sample": "the 3 tilings one after another, %.1f s" % dt1}}
    launches = int(sum(tot_iso[k][1] for k in tot_iso))
    if rank == 0:
        line = {
            "metric": metric_name(args.eps), "value": value, "unit": "points/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "hybrid": "f64 + float-float M2L + f32 pairs P2P",
                      "split": "f64 + float-float M2L"}.get(
                args.prec, "tf32x3+f32+f64"), "data": "synthetic",
            "config": {"workload": "N=M=2^20 uniform unit square (sources=targets), FP32 points and "
                                   "strengths, quad+sept+tri, eps=%s, %s L/p, %s form" % (eps_label(args.eps),
                                   "fixed" if args.params else "planner" if args.no_tune else "autotuned",
                                   args.prec),
                       "global_batch": N_POINTS,
                       "l2": "flushed between tilings (256 MB write)" if args.serial else
                             "flushed between steps (256 MB write)",
                       "streams": "one tiling after another on one stream" if args.serial else
                                  "the three tilings on three streams, issued from three host "
                                  "threads, joined at the end of the step",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "ms_per_step_serial": ms_serial,
            "per_tiling": {t: {"points_per_s": N_POINTS / (statistics.mean(tt[t]) / 1e3),
                               "ms": statistics.mean(tt[t]), "L": info[t]["levels"], "p": info[t]["p"],
                               "m2l": info[t]["n_m2l"], "p2p_pairs": info[t]["n_p2p_pairs"],
                               "leaf_points": {"mean": N_POINTS / max(1, info[t]["n_leaves"]),
                                               "max": info[t]["max_leaf_src"],
                                               "occupied_leaves": info[t]["n_leaves"]},
                               "tune_probe_err": tuned[t][2],
                               "stages_ms": {k: v[0] for k, v in stage[t].items()},
                               "stages_ms_isolated": {k: v[0] for k, v in stage_iso[t].items()}}
                           for t in args.tilings},
            "fp64_form": fp64_form,
            "roofline": roof,
            "roofline_isolated": roof_iso,
            "roofline_m2l": roofline_m2l(tot_iso, "CUDA events, one extra step with the stages serialised"),
            "peaks_source": src,
            "alu_peaks": alu,
            "stage_ms_total": {k: v[0] for k, v in tot.items()},
            "stage_ms_total_isolated": {k: v[0] for k, v in tot_iso.items()},
            "stage_note": "stage_ms: mean of 5 steps after the timed ones, far field concurrent "
                          "with P2P; isolated: one extra step with the stages serialised",
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_v, "unit": "points/s",
                    "h2d_bytes_per_step": int(xy.nbytes + u.nbytes),
                    "d2h_bytes_per_step": int(8 * N_POINTS * len(args.tilings))},
            "gpu_launches": launches * args.steps,
            "clocks": clk.summary(),
        }
        print(json.dumps(line))
    issuers.shutdown()
    for p_ in plans.values():
        p_.close()
    if dist:
        dist.destroy_process_group()


def _pool(n_max, seed):
    """Two seeded point sets (uniform, 8-cluster mixture) of n_max FP32 points;
    a request of size n uses the first n points of one of them."""
    from paper_1204_3105_gb300.inputs import gaussian_mixture, uniform_square
    uxy, uu = uniform_square(n_max, seed=seed, dtype=np.float32)
    gxy, gu = gaussian_mixture(n_max, seed=seed + 1, k=8, dtype=np.float32)
    return (uxy, uu), (gxy, gu.astype(np.float32))


def run_clustered(args):
    """The clustered workload: N = M = 4,194,304 points from a 32-component
    Gaussian mixture, strengths N(0, 1), FP64, eps = 1e-10, quadtree and
    septree on adaptive trees (leaf size 64), FP64 leading terms with the
    split-precision M2L (the plain FP64 form timed beside it).  One step =
    build + evaluate of both tilings; device time with CUDA events, inputs
    resident."""
    import torch
    from paper_1204_3105_gb300 import fmm2d
    from paper_1204_3105_gb300.inputs import gaussian_mixture
    fmm2d.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    n = 4194304
    xy, u = gaussian_mixture(n, seed=3, k=32)
    xy_d = torch.from_numpy(xy).to(dev)
    u_d = torch.from_numpy(u).to(dev)
    out = torch.empty(n, dtype=torch.float64, device=dev)
    names = ("quad", "sept")
    # FP64 leading terms with the split-precision (float-float) M2L; --prec
    # fp64 runs the plain FP64 form
    form = {"fp64": fmm2d.PREC_FP64, "hybrid": fmm2d.PREC_HYBRID}.get(args.prec, fmm2d.PREC_SPLIT)
    plans = {}
    for t in names:
        plans[t] = fmm2d.Plan(t, 0, 0, 1e-10, form | fmm2d.ADAPTIVE)
        plans[t].set_leaf_size(args.leaf_size)
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device=dev)

    def step(times):
        for t in names:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plans[t].build(xy_d, n, xy_d, n, stream)
            plans[t].evaluate(u_d, out, stream)
            e1.record(stream)
            times.append((t, e0, e1))
            flush.zero_()

    for _ in range(args.warmup):
        step([])
    torch.cuda.synchronize()
    times = []
    with Clocks(0) as clk:
        for _ in range(args.steps):
            step(times)
        torch.cuda.synchronize()
    per = {t: [] for t in names}
    for t, a, b in times:
        per[t].append(a.elapsed_time(b))
    for t in names:
        plans[t].set_profiling(2)
    step([])
    torch.cuda.synchronize()
    info = {t: plans[t].query() for t in names}
    stages = {t: {k: v[0] for k, v in plans[t].stage_times().items()} for t in names}
    ms = sum(statistics.mean(v) for v in per.values())
    def leg(lform, steps=2):   # another precision form on the same points
        ms_t = {}
        for t in names:
            pl = fmm2d.Plan(t, 0, 0, 1e-10, lform | fmm2d.ADAPTIVE)
            pl.set_leaf_size(args.leaf_size)
            ts = []
            for it in range(1 + steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pl.build(xy_d, n, xy_d, n, stream)
                pl.evaluate(u_d, out, stream)
                e1.record(stream)
                e1.synchronize()
                if it > 0:
                    ts.append(e0.elapsed_time(e1))
                flush.zero_()
            pl.close()
            ms_t[t] = statistics.mean(ts)
        tot = sum(ms_t.values())
        return {"value": len(names) * n / (tot / 1e3), "unit": "points/s", "ms_per_step": tot,
                "per_tiling_ms": ms_t, "time_vs_headline": tot / ms}

    fp64_form = hybrid_form = None
    if not args.no_fp64_form:
        if form != fmm2d.PREC_FP64:
            fp64_form = leg(fmm2d.PREC_FP64)
        if form != fmm2d.PREC_HYBRID:   # FP32-pair P2P: within 1e-10 here (sampled test)
            hybrid_form = leg(fmm2d.PREC_HYBRID)
    line = {
        "metric": "clustered FMM points/s (4,194,304 points, 32-cluster mixture, eps=1e-10, %s)" % (
            {fmm2d.PREC_FP64: "FP64", fmm2d.PREC_HYBRID: "hybrid form"}.get(
                form, "FP64 leading terms, split-precision M2L")),
        "value": len(names) * n / (ms / 1e3), "unit": "points/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {fmm2d.PREC_FP64: "f64", fmm2d.PREC_HYBRID: "f64 + float-float M2L + f32 pairs P2P"}.get(
            form, "f64 + float-float M2L"),
        "data": "synthetic", "fp64_form": fp64_form, "hybrid_form": hybrid_form,
        "config": {"workload": "N=M=4194304 Gaussian mixture (32 components, sigma log-uniform "
                               "[1e-3, 1e-1]), strengths N(0,1) FP64, quad + sept, eps=1e-10, adaptive "
                               "trees, leaf size %d" % args.leaf_size, "l2": "flushed between tilings"},
        "per_tiling": {t: {"points_per_s": n / (statistics.mean(per[t]) / 1e3), "ms": statistics.mean(per[t]),
                           "levels": info[t]["levels"], "p": info[t]["p"], "m2l": info[t]["n_m2l"],
                           "p2p_pairs": info[t]["n_p2p_pairs"], "stages_ms_isolated": stages[t]}
                       for t in names},
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    for pl in plans.values():
        pl.close()


def run_forest_batch(args):
    """The 4096-instance batch as three forests (one per tiling): each forest is
    one fmm2d_build_forest + fmm2d_evaluate over all its instances.  Device
    time with CUDA events (inputs resident), and end to end from pinned host
    buffers with the copies inside the timed region."""
    import torch
    from paper_1204_3105_gb300 import fmm2d
    from paper_1204_3105_gb300.inputs import rng, uniform_square
    fmm2d.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    g = rng(SEED + 40)
    count = args.instances
    sizes = np.exp(g.uniform(np.log(256), np.log(65536), count)).astype(np.int64)
    tilings = g.integers(0, 3, count)
    names = ("quad", "sept", "tri")
    forests = {}
    for ti, name in enumerate(names):
        idx = np.nonzero(tilings == ti)[0]
        pts = [uniform_square(int(sizes[i]), seed=1000 + int(i), dtype=np.float32) for i in idx]
        off = np.concatenate([[0], np.cumsum(sizes[idx])]).astype(np.int64)
        xy = np.concatenate([q[0] for q in pts])
        u = np.concatenate([q[1] for q in pts])
        # p from fmm2d_autotune on the forest's largest instance (eps, seeded probe)
        big = int(np.argmax(sizes[idx]))
        bxy = torch.from_numpy(pts[big][0]).to(dev)
        _, p_t, e_t, _ = fmm2d.fmm2d_autotune(name, 1e-6, fmm2d.PREC_MIXED_TC | fmm2d.IN_F32, bxy,
                                             len(pts[big][0]), bxy, len(pts[big][0]), stream=stream)
        plan = fmm2d.Plan(name, 0, p_t, 1e-6, fmm2d.PREC_MIXED_TC | fmm2d.IN_F32 | fmm2d.ADAPTIVE)
        plan.set_leaf_size(args.leaf_size)
        forests[name] = dict(off=off, xy=xy, u=u, plan=plan, p=p_t, tune_err=e_t, n=len(idx),
                             xy_d=torch.from_numpy(xy).to(dev), u_d=torch.from_numpy(u).to(dev),
                             out=torch.empty(len(xy), dtype=torch.float64, device=dev),
                             xy_h=torch.from_numpy(xy).pin_memory(), u_h=torch.from_numpy(u).pin_memory(),
                             res_h=torch.empty(len(xy), dtype=torch.float64).pin_memory())
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device=dev)
    total = int(sizes.sum())

    def step(times):
        for name in names:
            f = forests[name]
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f["plan"].build_forest(f["xy_d"], f["off"], stream)
            f["plan"].evaluate(f["u_d"], f["out"], stream)
            e1.record(stream)
            times.append((name, e0, e1))
            flush.zero_()

    # the three forests are independent: one stream and one issuing host
    # thread each (a forest build waits for its level counts), joined per step
    fstreams = {nm: torch.cuda.Stream(device=dev) for nm in names}
    from concurrent.futures import ThreadPoolExecutor
    issuers = ThreadPoolExecutor(len(names), initializer=torch.cuda.set_device, initargs=(0,))

    def forest_on(name, start):
        f, fs = forests[name], fstreams[name]
        fs.wait_event(start)
        f["plan"].build_forest(f["xy_d"], f["off"], fs)
        f["plan"].evaluate(f["u_d"], f["out"], fs)
        d = torch.cuda.Event()
        d.record(fs)
        return d

    def step_concurrent(whole):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for d in issuers.map(lambda nm: forest_on(nm, e0), names):
            stream.wait_event(d)
        e1.record(stream)
        whole.append((e0, e1))
        flush.zero_()

    for _ in range(args.warmup):
        step([])
        step_concurrent([])
    torch.cuda.synchronize()
    times, whole = [], []
    with Clocks(0) as clk:
        for _ in range(args.steps):
            if args.serial:
                step(times)
            else:
                step_concurrent(whole)
        torch.cuda.synchronize()
    if not args.serial:   # per-forest times: the same steps, one forest after another
        for _ in range(min(args.steps, 10)):
            step(times)
        torch.cuda.synchronize()
    per = {n: [] for n in names}
    for name, a, b in times:
        per[name].append(a.elapsed_time(b))
    ms_serial = sum(statistics.mean(v) for v in per.values())
    ms = ms_serial if args.serial else statistics.mean(a.elapsed_time(b) for a, b in whole)
    for name in names:   # one more step with the stages serialised: each stage's own time
        forests[name]["plan"].set_profiling(2)
    step([])
    torch.cuda.synchronize()
    stages = {}
    for name in names:
        stages[name] = {k: v[0] for k, v in forests[name]["plan"].stage_times().items()}
        forests[name]["plan"].set_profiling(0)
    e2e = []
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        def forest_e2e(name):
            f = forests[name]
            fs = stream if args.serial else fstreams[name]
            with torch.cuda.stream(fs):   # copies, build and evaluation on the forest's stream
                xd = f["xy_h"].to(dev, non_blocking=True)
                ud = f["u_h"].to(dev, non_blocking=True)
                f["plan"].build_forest(xd, f["off"], fs)
                f["plan"].evaluate(ud, f["out"], fs)
                f["res_h"].copy_(f["out"], non_blocking=True)
        if args.serial:
            for name in names:
                forest_e2e(name)
        else:
            list(issuers.map(forest_e2e, names))
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e.append(time.perf_counter() - t0)
    # the plain FP64 GPU form on the same forests, p tuned for the same eps
    fp64_form = None
    if not args.no_fp64_form:
        ms64 = 0.0
        per64 = {}
        for name in names:
            f = forests[name]
            idx = np.nonzero(tilings == names.index(name))[0]
            big = int(np.argmax(sizes[idx]))
            bxy = torch.from_numpy(uniform_square(int(sizes[idx][big]), seed=1000 + int(idx[big]),
                                                  dtype=np.float32)[0]).to(dev)
            _, p64, e64, _ = fmm2d.fmm2d_autotune(name, 1e-6, fmm2d.PREC_FP64 | fmm2d.IN_F32, bxy,
                                                  len(bxy), bxy, len(bxy), stream=stream)
            pl = fmm2d.Plan(name, 0, p64, 1e-6, fmm2d.PREC_FP64 | fmm2d.IN_F32 | fmm2d.ADAPTIVE)
            pl.set_leaf_size(args.leaf_size)
            ts = []
            for it in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pl.build_forest(f["xy_d"], f["off"], stream)
                pl.evaluate(f["u_d"], f["out"], stream)
                e1.record(stream)
                e1.synchronize()
                if it > 0:
                    ts.append(e0.elapsed_time(e1))
                flush.zero_()
            pl.close()
            per64[name] = {"ms": statistics.mean(ts), "p": p64, "tune_probe_err": e64}
            ms64 += per64[name]["ms"]
        fp64_form = {"value": total / (ms64 / 1e3), "unit": "points/s", "ms_per_step": ms64,
                     "per_tiling": per64, "speedup_of_mixed": ms64 / ms,
                     "note": "forests one after another, 2 timed steps each"}
    line = {
        "metric": "batched FMM points/s (4096 instances, eps=1e-6)", "value": total / (ms / 1e3),
        "unit": "points/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "ms_per_step_serial": ms_serial, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "tf32x3+f32+f64", "data": "synthetic",
        "config": {"workload": "4096 instances, N log-uniform [256, 65536], uniform unit square, tiling "
                               "uniform over 3, eps=1e-6, FP32; one forest per tiling "
                               "(fmm2d_build_forest + fmm2d_evaluate), leaf size %d" % args.leaf_size,
                   "instances": count, "points": total,
                   "l2": "flushed between forests (256 MB write)" if args.serial else
                         "flushed between steps (256 MB write)",
                   "streams": "one forest after another" if args.serial else
                              "the three forests on three streams, issued from three host "
                              "threads, joined at the end of the step"},
        "per_tiling": {n: {"instances": forests[n]["n"], "points": int(forests[n]["off"][-1]),
                           "stages_ms_isolated": stages[n],
                           "ms": statistics.mean(per[n]), "p": forests[n]["p"],
                           "levels": forests[n]["plan"].query()["levels"],
                           "tune_probe_err": forests[n]["tune_err"]} for n in names},
        "e2e": {"value": total / statistics.mean(e2e), "unit": "points/s",
                "h2d_bytes_per_step": int(sum(f["xy"].nbytes + f["u"].nbytes for f in forests.values())),
                "d2h_bytes_per_step": int(8 * total)},
        "fp64_form": fp64_form,
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    issuers.shutdown()
    for f in forests.values():
        f["plan"].close()


def run_server_workload(args):
    """Batched instances (--workload batch) or a Poisson request stream
    (--workload serve) through fmm2d_serve_*, host buffers in and out."""
    from paper_1204_3105_gb300 import fmm2d
    from paper_1204_3105_gb300.inputs import rng
    fmm2d.lib()
    g = rng(SEED + 40)
    if args.workload == "batch":
        count = args.instances
        sizes = np.exp(g.uniform(np.log(256), np.log(65536), count)).astype(np.int64)
        tilings = g.integers(0, 3, count)
        eps = np.full(count, 1e-6)
        cluster = np.zeros(count, bool)
        arrivals = np.zeros(count)
        n_max = int(sizes.max())
    else:
        lam = args.rate
        count = max(1, int(lam * args.duration))
        arrivals = np.cumsum(g.exponential(1.0 / lam, count))
        sizes = np.exp(g.uniform(np.log(1e3), np.log(2e6), count)).astype(np.int64)
        tilings = g.integers(0, 3, count)
        eps = np.where(g.random(count) < 0.5, 1e-4, 1e-8)
        cluster = g.random(count) < 0.5
        n_max = int(sizes.max())
    (uxy, uu), (gxy, gu) = _pool(n_max, SEED + 41)
    tree = args.tree if args.tree != "auto" else ("adaptive" if args.workload == "serve" else "uniform")
    tree_flag = fmm2d.ADAPTIVE if tree == "adaptive" else 0
    if args.serve_prec == "fp64":   # the plain FP64 GPU form for every request
        tree_flag |= fmm2d.SERVE_PREC_AS_GIVEN | fmm2d.PREC_FP64
    names = ("quad", "sept", "tri")
    sv = fmm2d.Server(int(args.budget_gb * (1 << 30)), max_slots=args.slots)
    # untimed warm-up: every (tiling, eps) once per slot, so that module
    # loading and each slot's plans (operator tables) precede the timed stream
    warm = []
    for ti in range(3):
        for e in sorted(set(eps.tolist())):
            for _ in range(args.slots):
                o = np.empty(2000)
                warm.append((sv.submit(names[ti], uxy[:2000], uu[:2000], o, eps=float(e),
                                       flags=tree_flag), o))
    for t, _ in warm:
        sv.wait(t, 600000.0)
    outs, tickets, t_sub = [], [], []
    t0 = time.perf_counter()
    for i in range(count):
        wait = t0 + arrivals[i] - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        xy, u = (gxy, gu) if cluster[i] else (uxy, uu)
        n = int(sizes[i])
        o = np.empty(n)
        outs.append(o)
        tickets.append(sv.submit(names[tilings[i]], xy[:n], u[:n], o, eps=float(eps[i]), flags=tree_flag))
    res = [sv.wait(t, 600000.0) for t in tickets]
    t1 = time.perf_counter()
    sv.close()
    lat = np.array([r["latency_ms"] for r in res])
    ok = sum(r["status"] == 0 for r in res)
    failed = [{"i": i, "status": int(r["status"]), "tiling": names[tilings[i]], "n": int(sizes[i]),
               "eps": float(eps[i]), "cluster": bool(cluster[i]), "batched": int(r["batched"]),
               "slot": int(r["slot"]), "error": r.get("error", "")}
              for i, r in enumerate(res) if r["status"] != 0]
    if args.dump:   # one line per request: what it was and how long it took
        with open(args.dump, "w") as f:
            for i, r in enumerate(res):
                f.write(json.dumps({"i": i, "tiling": names[tilings[i]], "n": int(sizes[i]),
                                    "eps": float(eps[i]), "cluster": bool(cluster[i]),
                                    "slot": r["slot"], "batched": r["batched"], "queue_ms": r["queue_ms"],
                                    "run_ms": r["run_ms"], "p": r["p"], "levels": r["levels"]}) + "\n")
    by_eps = {}
    for e in sorted(set(eps.tolist())):
        m = eps == e
        run = np.array([r["run_ms"] for r, k in zip(res, m) if k])
        by_eps["%g" % e] = {"requests": int(m.sum()), "points": int(sizes[m].sum()),
                            "run_ms_mean": float(run.mean()), "run_ms_sum": float(run.sum()),
                            "latency_p50_ms": float(np.percentile(lat[m], 50)),
                            "latency_p99_ms": float(np.percentile(lat[m], 99))}
    points = int(sizes.sum())
    # steady state or not: latency of the first, middle and last third of the
    # requests in arrival order (a queue that grows shows rising thirds), and
    # how long after the last arrival the last result came
    thirds = []
    for part in np.array_split(np.arange(count), 3):
        if len(part):
            thirds.append({"p50": float(np.percentile(lat[part], 50)),
                           "p99": float(np.percentile(lat[part], 99))})
    drain_s = (t1 - t0) - float(arrivals[-1])
    line = {
        "metric": ("batched FMM points/s (4096-instance config)" if args.workload == "batch"
                   else "served FMM requests: p50/p99 latency and points/s"),
        "value": points / (t1 - t0), "unit": "points/s", "n_gpus": 1,
        "higher_is_better": True, "data": "synthetic", "workload": args.workload,
        "requests": count, "completed_ok": int(ok), "failed": failed[:20], "wall_s": t1 - t0,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(lat.max())},
        "run_ms_mean": float(np.mean([r["run_ms"] for r in res])),
        "latency_by_third_ms": thirds, "drain_after_last_arrival_s": drain_s,
        "offered_points_per_s": points / max(1e-9, float(arrivals[-1])) if count > 1 else None,
        "by_eps": by_eps,
        "config": {"slots": args.slots, "hbm_budget_gb": args.budget_gb,
                   "sizes": "log-uniform [256, 65536]" if args.workload == "batch"
                   else "log-uniform [1e3, 2e6]",
                   "eps": "1e-6" if args.workload == "batch" else (
                       "1e-4 / 1e-8, plain FP64 form for both" if args.serve_prec == "fp64" else
                       "1e-4 (mixed form) / 1e-8 (hybrid form)"),
                   "arrival_rate_per_s": None if args.workload == "batch" else args.rate,
                   "points": "uniform" if args.workload == "batch" else "uniform / 8-cluster mixture",
                   "tree": tree + (" (leaf size chosen by the server: quad 64, sept and tri 128)"
                                   if tree == "adaptive" else ""),
                   "io": "host numpy buffers, copies inside each request",
                   "warmup": "untimed: one 2000-point request per (tiling, eps) per slot"},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="tc", choices=["tc", "mixed", "fp64", "hybrid", "split"],
                    help="fmm workload: precision form (clustered: split unless fp64)")
    ap.add_argument("--eps", type=float, default=EPS, help="fmm workload: requested tolerance")
    ap.add_argument("--tilings", default=",".join(TILINGS))
    ap.add_argument("--ref-points", type=int, default=16384)
    ap.add_argument("--ref-seconds", type=float, default=150.0, help="reference arm: host time budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="a-priori L and p instead of fmm2d_autotune")
    ap.add_argument("--no-profile", action="store_true", help="no per-stage event pass")
    ap.add_argument("--no-fp64-form", action="store_true", help="skip the plain FP64 GPU form")
    ap.add_argument("--serial", action="store_true",
                    help="time the tilings one after another on one stream")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed steps of the FP64 form")
    ap.add_argument("--params", default="", help="fixed L and p per tiling, e.g. quad:7:12,sept:5:13")
    ap.add_argument("--workload", default="fmm", choices=["fmm", "batch", "serve", "clustered"])
    ap.add_argument("--instances", type=int, default=4096, help="batch: number of instances")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: arrivals per second")
    ap.add_argument("--duration", type=float, default=1.0, help="serve: seconds of arrivals")
    ap.add_argument("--slots", type=int, default=16, help="batch/serve: server slots")
    ap.add_argument("--budget-gb", type=float, default=80.0, help="batch/serve: HBM budget")
    ap.add_argument("--batch-mode", default="forest", choices=["forest", "server"],
                    help="batch: one forest per tiling, or one server request per instance")
    ap.add_argument("--leaf-size", type=int, default=64, help="batch/serve: adaptive leaf size")
    ap.add_argument("--dump", default="", help="batch/serve: write one JSON line per request here")
    ap.add_argument("--serve-prec", default="auto", choices=["auto", "fp64"],
                    help="serve: precision form chosen by the server, or the plain FP64 form")
    ap.add_argument("--tree", default="auto", choices=["auto", "uniform", "adaptive"],
                    help="batch/serve: tree of each request (auto: adaptive for serve)")
    args = ap.parse_args()
    args.tilings = tuple(args.tilings.split(","))
    if args.workload == "clustered" and args.impl != "reference":
        run_clustered(args)
        return
    if args.workload == "batch" and args.batch_mode == "forest" and args.impl != "reference":
        run_forest_batch(args)
        return
    if args.workload != "fmm" and args.impl != "reference":
        run_server_workload(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
