"""Benchmark of the event-manifold reconstruction hot path on GB300.

A step is one event packet through the whole hot path: event validation and
scatter, packet prologue (time surface, metric, data image) and K primal-dual
iterations.  Default workload: 346x260 sensor, seeded scene of 200 Gaussian blobs
(1 rad/s rotation + 100 px/s), 1M events, 1000-event packets, 50 iterations per
packet, FP32.  With more steps than packets the stream is replayed with its
timestamps shifted forward, so every packet stays valid.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Rank 0 prints one JSON line.  Under torchrun each rank solves its own independent
stream (seed + rank): weak scaling, no data-path collective; the timed region is
bracketed by a barrier and the time is the maximum over ranks.
"""
from __future__ import annotations

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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "events/s and Gpixel-iter/s per GB300 at stated error vs FP64; batched vs plain"
B_ALG = 40  # algorithmic bytes per pixel-iteration, FP32 state (read u,p1,p2,p3,f,t; write u,p)
B_ALG_16 = 28  # the same with p stored in FP16/BF16 (2 B per component)


def b_alg(storage):
    return B_ALG if storage == 0 else B_ALG_16
# algorithmic bytes per pixel of the packet's front launches, timed with the iteration
# kernels: the prologue reads t_last (8), n+, n-, u (4 each) and writes L_x t, L_y t,
# 1/G, sqrt(G), f (4 each) and the cleared counts (4 each); one TV-L1 iteration of the
# time surface reads t0, s, q1, q2 and writes s, sbar (primal), reads sbar, q1, q2 and
# writes q1, q2 (dual)
B_PROLOGUE = 48
B_TVL1_ITER = 44
# the push, per event: reads x, y, t, pol (13 B) and updates t_last (8 B read + write) and
# one count (4 B read + write) of its pixel
B_PUSH_EVENT = 37
# the differentiation's reverse pass (the adjoint state stays on chip within a launch):
# per reversed pixel-iteration the tape's p (12 B), v and ubar (4 B each); per pixel and
# launch the adjoint state in and out (5 planes each), dL/df read and written, the metric
# (L_x t, L_y t, 1/G, sqrt(G)) and f: 17 planes of 4 B
B_REV_ITER = 20
B_REV_LAUNCH = 68
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=980)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="blobs346")
    ap.add_argument("--every", type=int, default=10,
                    help="diff64: checkpoint spacing of the unrolled solve (>= 30: whole tape "
                         "kept from the forward, no recomputation)")
    ap.add_argument("--cpu-budget-s", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solver", type=int, default=0, help="evr_params.solver")
    ap.add_argument("--tile", type=int, default=0, help="evr_params.tile_config")
    ap.add_argument("--storage", type=int, default=0, help="evr_params.storage (0 FP32, 1 FP16, "
                    "2 BF16)")
    ap.add_argument("--tvl1", type=int, default=0, help="evr_params.tvl1_iters")
    ap.add_argument("--schedule", default="auto", choices=["auto", "graph", "persistent"],
                    help="batch256: evr_batch_set_schedule (default: autotuned)")
    ap.add_argument("--grouping", default=None,
                    help="batch256: BYTES[,BRANCHES] for evr_batch_set_grouping (default: "
                         "autotuned; 0 = one group)")
    ap.add_argument("--check-error", action="store_true",
                    help="also state the max-abs error vs the FP64 oracle on one packet")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def workload(name, rank, max_packets=None):
    from evsim import CONFIGS, make_stream
    from paper_1607_06283_gb300.shard import stream_seed
    cfg = CONFIGS[name]
    if max_packets is not None and cfg.n_packets > max_packets:
        cfg = cfg.with_events(max_packets * cfg.packet)  # only the packets the run uses
    if rank:
        d = dict(cfg.__dict__)
        d["seed"] = stream_seed(cfg.seed, rank)
        cfg = type(cfg)(**d)
    return cfg, make_stream(cfg)


def packet_slices(stream, cfg, n_steps):
    """(start, stop, time shift) of each step; replays the stream shifted in time."""
    n_pk = cfg.n_packets
    span = int(stream.t[-1] - stream.t[0]) + 1
    for k in range(n_steps):
        rep, j = divmod(k, n_pk)
        a = j * cfg.packet
        yield a, min(a + cfg.packet, len(stream)), rep * span


def describe(cfg):
    return (f"{cfg.name}: {cfg.W}x{cfg.H} sensor, {cfg.kind} scene ({cfg.n_objects} objects), "
            f"{cfg.n_events} events, {cfg.packet}-event packets, {cfg.iters} iterations")


# ----------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def wait_first(self, timeout=5.0):
        """Block until nvidia-smi has produced its first sample (its start-up runs before
        the timed region, not inside it)."""
        t_end = time.perf_counter() + timeout
        while self.proc and not self.rows and time.perf_counter() < t_end:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": len(self.rows)}
        mhz = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        if mhz:
            out["sm_mhz"] = statistics.median(mhz)
        if mx:
            out["sm_max_mhz"] = max(mx)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower() == "active":
                    seen.add(nm)
        out["reasons"] = sorted(seen)
        return out


# ----------------------------------------------------------------------- helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profiled(workload, solver_name):
    """ncu counters of the dominant kernel for this workload and solver configuration
    (profiles/counters.json, written by paper_1607_06283_gb300/profiling.py from the
    captures its summaries describe), if they were taken on the current kernel source;
    else None."""
    from paper_1607_06283_gb300.profiling import source_hash, sources_for
    source_sha = source_hash(sources_for(solver_name))
    p = os.path.join(ROOT, "profiles", "counters.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        entries = json.load(fh)
    for e in entries:
        if (e.get("workload") == workload and e.get("solver") == solver_name and
                e.get("source_sha") == source_sha):
            return e
    return None


def cpu_info():
    """Host core count and CPU model (lscpu's "Model name", which Arm hosts report there
    and not in /proc/cpuinfo)."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(),
            "cpu_model": f"{model or platform.processor() or 'unknown'} ({platform.machine()})"}


def _oracle_rate(cfg, stream, budget_s, omp, shift_steps=None):
    from oracle import oracle as O
    o = O.OracleStream(cfg.W, cfg.H, omp=omp)
    t0 = time.perf_counter()
    done = ev = 0
    while True:
        a = done * cfg.packet
        if a >= len(stream):
            break
        b = min(a + cfg.packet, len(stream))
        o.push(stream.x[a:b], stream.y[a:b], stream.t[a:b], stream.pol[a:b])
        o.solve(cfg.iters)
        done += 1
        ev += b - a
        if time.perf_counter() - t0 > budget_s and done >= 3:
            break
    dt = time.perf_counter() - t0
    return ev / dt, done, ev, dt


def cpu_baseline(cfg, stream, budget_s):
    """The FP64 oracle, as it stands, on this host's cores: packets of the same stream
    until the time budget is spent, once on one thread and once with its per-pixel loops
    spread over every core by OpenMP (the same source and results)."""
    info = cpu_info()
    v1, d1, e1, t1 = _oracle_rate(cfg, stream, budget_s / 2, omp=False)
    vn, dn, en, tn = _oracle_rate(cfg, stream, budget_s / 2, omp=True)
    threads = int(os.environ.get("OMP_NUM_THREADS", info["nproc"]))
    return {"value": vn, "unit": "events/s", "cores": threads, "kind": "oracle",
            "gpix_iter_per_s": dn * cfg.W * cfg.H * cfg.iters / tn / 1e9,
            "sample": f"first {dn} packets ({en} events) of the same stream, FP64, OpenMP "
                      f"over pixels on {threads} threads, {tn:.1f} s",
            "nproc": info["nproc"], "cpu_model": info["cpu_model"],
            "single_thread": {"value": v1, "unit": "events/s", "cores": 1,
                              "gpix_iter_per_s": d1 * cfg.W * cfg.H * cfg.iters / t1 / 1e9,
                              "sample": f"first {d1} packets ({e1} events), FP64, one "
                                        f"thread, {t1:.1f} s"}}


def error_vs_oracle(E, cfg, stream, p):
    """Max |u_gpu - u_oracle| on the third packet, teacher-forced (the oracle starts
    from the GPU's state), with the run's parameters."""
    from oracle import oracle as O
    g = E.Stream(cfg.W, cfg.H, p)
    o = O.OracleStream(cfg.W, cfg.H, O.OracleParams(
        lam=float(p.lambda_), delta_pos=float(p.delta_pos), delta_neg=float(p.delta_neg),
        u_min=float(p.u_min), u_max=float(p.u_max), u_init=float(p.u_init), tau=float(p.tau),
        sigma=float(p.sigma), time_scale=float(np.float32(p.time_scale)),
        t_max_us=int(p.t_max_us), data_term=int(p.data_term), tvl1_iters=int(p.tvl1_iters),
        tvl1_lambda=float(np.float32(p.tvl1_lambda))))
    for k in range(2):
        a = k * cfg.packet
        g.push(stream.x[a:a + cfg.packet], stream.y[a:a + cfg.packet],
               stream.t[a:a + cfg.packet], stream.pol[a:a + cfg.packet])
        g.solve(cfg.iters)
    o.set_up(g.state(E.EVR_STATE_U).astype(np.float64), g.p().astype(np.float64))
    o.set(O.TLAST, g.state(E.EVR_STATE_TLAST))
    o.set(O.TREF, int(g.state(E.EVR_STATE_CLOCK)))
    o.set(O.TINIT, int(g.state(E.EVR_STATE_TINIT)))
    a = 2 * cfg.packet
    sl = slice(a, a + cfg.packet)
    g.push(stream.x[sl], stream.y[sl], stream.t[sl], stream.pol[sl])
    o.push(stream.x[sl], stream.y[sl], stream.t[sl], stream.pol[sl])
    g.solve(cfg.iters)
    o.solve(cfg.iters)
    d = np.abs(g.image().astype(np.float64) - o.u)
    g.close()
    return {"max_abs": float(d.max()), "p99_9": float(np.percentile(d, 99.9)),
            "sample": "packet 3, teacher-forced, FP64 oracle"}


# ----------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    big = args.config != "blobs346"
    cfg, stream = workload(args.config, 0,
                           max_packets=args.warmup + args.steps if big else None)
    from oracle import oracle as O
    o = O.OracleStream(cfg.W, cfg.H, omp=True)  # per-pixel loops on every host core
    info = cpu_info()
    threads = int(os.environ.get("OMP_NUM_THREADS", info["nproc"]))
    steps = list(packet_slices(stream, cfg, args.warmup + args.steps))
    for a, b, sh in steps[:args.warmup]:
        o.push(stream.x[a:b], stream.y[a:b], stream.t[a:b] + sh, stream.pol[a:b])
        o.solve(cfg.iters)
    budget = 150.0
    t0 = time.perf_counter()
    done = ev = 0
    for a, b, sh in steps[args.warmup:]:
        o.push(stream.x[a:b], stream.y[a:b], stream.t[a:b] + sh, stream.pol[a:b])
        o.solve(cfg.iters)
        done += 1
        ev += b - a
        if time.perf_counter() - t0 > budget:
            break
    dt = time.perf_counter() - t0
    v = ev / dt
    sample = (f"{done} of {args.steps} timed packets (time budget {budget:.0f} s), "
              f"after {args.warmup} warm-up packets; FP64 oracle, OpenMP over pixels on "
              f"{threads} threads")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "events/s",
            "n_gpus": 1, "steps": done, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / max(1, done), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "gpix_iter_per_s": done * cfg.W * cfg.H * cfg.iters / dt / 1e9,
            "config": {"workload": describe(cfg), "sensor": f"{cfg.W}x{cfg.H}",
                       "packet": cfg.packet, "iters": cfg.iters},
            "cpu_baseline": {"value": v, "unit": "events/s", "cores": threads,
                             "kind": "oracle", "sample": sample, "nproc": info["nproc"],
                             "cpu_model": info["cpu_model"]},
            "e2e": {"value": v, "unit": "events/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------- our arm
SETTLE_MAX = 12  # untimed packets at most before the solver configuration is settled


def roofline_level(solver_name, n_sms, l2_gbs, smem_gbs):
    """The memory level that holds the iterated state between the iterations of a packet,
    and its measured peak.  A cluster over the whole sensor (R0) keeps u, p and the packet
    constants in registers and shared memory for all iterations: its bound is the
    shared-memory bandwidth of the SMs it occupies.  The multi-launch solvers keep the state
    on chip within a launch and in L2 between launches: their bound is L2."""
    import re
    m = re.search(r"R(\d+) \((\d+) threads, (\d+) CTAs\)", solver_name)
    if solver_name.startswith("cluster") and m and int(m.group(1)) == 0:
        ctas = int(m.group(3))
        return "smem", smem_gbs * min(ctas, n_sms) / n_sms, (
            f"shared memory of the {min(ctas, n_sms)} SMs the cluster occupies: "
            f"{min(ctas, n_sms)}/{n_sms} of the aggregate measured in this run")
    return "l2", l2_gbs, "L2, measured in this run (evr_measure_peak level 0)"


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}), flush=True)
        return 1
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    from paper_1607_06283_gb300 import build
    if rank == 0:
        build.build()
    if pg:
        pg.barrier()
    from paper_1607_06283_gb300 import evr as E

    big = args.config != "blobs346"
    # packets: up to SETTLE_MAX to settle the solver, the warm-up, the timed steps and as
    # many again for the kernel-timing pass
    n_all = SETTLE_MAX + args.warmup + 2 * args.steps
    cfg, stream = workload(args.config, rank, max_packets=n_all if big else None)
    cur = torch.cuda.Stream()  # one non-default stream for the library and the timing events
    torch.cuda.set_stream(cur)
    p = E.evr_default_params()
    p.solver = args.solver
    p.tile_config = args.tile
    p.storage = args.storage
    p.tvl1_iters = args.tvl1
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    l2_gbs = E.evr_measure_peak(0, cur.cuda_stream)
    smem_gbs = E.evr_measure_peak(1, cur.cuda_stream)

    steps = list(packet_slices(stream, cfg, n_all))
    # device-resident inputs: the whole (time-shifted) event sequence of the run
    t_all = np.concatenate([stream.t[a:b] + sh for a, b, sh in steps])
    idx = np.concatenate([np.arange(a, b) for a, b, _ in steps])
    dx = torch.from_numpy(stream.x[idx].view(np.int16)).cuda()
    dy = torch.from_numpy(stream.y[idx].view(np.int16)).cuda()
    dt_ = torch.from_numpy(t_all).cuda()
    dp = torch.from_numpy(stream.pol[idx]).cuda()
    offs = np.concatenate([[0], np.cumsum([b - a for a, b, _ in steps])])
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    g = E.Stream(cfg.W, cfg.H, p)
    E.evr_set_cuda_stream(g.h, cur.cuda_stream)

    def step(k):  # push (device arrays) and solve: one graph per packet once settled
        s, e = int(offs[k]), int(offs[k + 1])
        rc = E.evr_step_device(g.h, dx[s:e], dy[s:e], dt_[s:e], dp[s:e], cfg.iters)
        if rc:
            raise RuntimeError(f"step failed: {rc}")

    # the first packet of a new stream tunes the solver (autotuner): its latency to the
    # image, then untimed packets until the online refinement has decided
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step(0)
    assert g.synchronize() == 0
    first_ms = (time.perf_counter() - t0) * 1e3
    k = 1
    while not E.evr_solver_settled(g.h) and k < SETTLE_MAX:
        step(k)
        k += 1
    settled = E.evr_solver_settled(g.h)
    # the clock sampler starts before the warm-up packets, so that its start-up is over
    # and the GPU busy when the timed region begins
    clk = ClockSampler(local)
    if rank == 0:
        clk.start()
        clk.wait_first()
    # warm-up steps exactly as the timed ones: L2 flush, events, the library's own kernel
    # timing (its events around each graph launch sit inside ours)
    k0 = SETTLE_MAX  # first warm-up packet
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(max(args.steps, args.warmup))]
    E.evr_enable_kernel_timing(g.h, True)
    for j in range(args.warmup):
        flush.fill_(float(j))
        evs[j][0].record(cur)
        step(k0 + j)
        evs[j][1].record(cur)
    assert g.synchronize() == 0
    torch.cuda.synchronize()
    k1 = k0 + args.warmup  # first timed packet
    evs = evs[:args.steps]
    if pg:
        pg.barrier()
    E.evr_enable_kernel_timing(g.h, True)  # counts from here
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for j in range(args.steps):
        flush.fill_(float(j))  # L2 flush between timed steps (outside the events)
        evs[j][0].record(cur)
        step(k1 + j)
        evs[j][1].record(cur)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if pg:
        pg.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms_steps = sum(step_ms)
    _, step_launches, _ = E.evr_kernel_time(g.h)
    E.evr_enable_kernel_timing(g.h, False)

    # the dominant kernels alone: the same packets' solves (front fused into the iteration
    # kernels) bracketed by the library's CUDA events on this stream, each push queued
    # before them and outside the events
    k2 = k1 + args.steps
    E.evr_enable_kernel_timing(g.h, True)
    for j in range(args.steps):
        flush.fill_(float(j))
        s_, e_ = int(offs[k2 + j]), int(offs[k2 + j + 1])
        if E.evr_push_events_device(g.h, dx[s_:e_], dy[s_:e_], dt_[s_:e_], dp[s_:e_]):
            raise RuntimeError("push failed")
        g.solve(cfg.iters)
    torch.cuda.synchronize()
    k_ms, k_launches, k_pixiters = E.evr_kernel_time(g.h)
    E.evr_enable_kernel_timing(g.h, False)
    clocks = clk.stop() if rank == 0 else None
    status = g.synchronize()
    if status:
        raise RuntimeError(f"device-side rejection during the run: {status}")
    ev_timed = int(offs[k1 + args.steps] - offs[k1])
    from paper_1607_06283_gb300.shard import reduce_timing
    t_max, ev_total = reduce_timing(ms_steps, ev_timed, pg, "cuda")
    value = ev_total / (t_max * 1e-3)
    gpix = world * args.steps * cfg.W * cfg.H * cfg.iters / (t_max * 1e-3) / 1e9
    # this rank's timed steps as five consecutive runs: events/s of each, and the median
    runs = []
    if args.steps >= 5:
        bounds = np.linspace(0, args.steps, 6).astype(int)
        for r in range(5):
            a_, b_ = int(bounds[r]), int(bounds[r + 1])
            ev_r = int(offs[k1 + b_] - offs[k1 + a_])
            runs.append(ev_r / (sum(step_ms[a_:b_]) * 1e-3))

    # ---- end to end through the C ABI with host buffers (same number of steps): every
    # step pushes its packet from host arrays (the library stages it in pinned memory and
    # copies it to the device), solves, and reads the image back into pinned host memory.
    # Readbacks are asynchronous with three steps in flight: step k is queued before the
    # image of step k - 2 is waited for, as a real-time consumer with a short queue would
    # drive the stream.
    g2 = E.Stream(cfg.W, cfg.H, p)
    E.evr_set_cuda_stream(g2.h, cur.cuda_stream)
    depth = 3  # steps in flight: the image of step j - depth + 1 is waited for after step j
    imgs = [torch.empty((cfg.H, cfg.W), dtype=torch.float32).pin_memory().numpy()
            for _ in range(depth)]
    hx = stream.x[idx]
    hy = stream.y[idx]
    hp = stream.pol[idx]

    def step_host(k, slot):
        s, e = int(offs[k]), int(offs[k + 1])
        rc = E.evr_step(g2.h, hx[s:e], hy[s:e], t_all[s:e], hp[s:e], cfg.iters)
        if rc:
            raise RuntimeError(f"step failed: {rc}")
        return E.evr_get_image_async(g2.h, imgs[slot])

    def wait(ticket):
        rc = E.evr_wait_image(g2.h, ticket)
        if rc:
            raise RuntimeError(f"wait_image: {rc}")

    k = 0
    while k < SETTLE_MAX and (k == 0 or not E.evr_solver_settled(g2.h)):
        wait(step_host(k, k % depth))
        k += 1
    for j in range(args.warmup):
        wait(step_host(k0 + j, j % depth))
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    pending = []
    for j in range(args.steps):
        pending.append(step_host(k1 + j, j % depth))
        if len(pending) == depth:
            wait(pending.pop(0))
    for t in pending:
        wait(t)
    e2e_s = time.perf_counter() - e0
    e2e_s, _ = reduce_timing(e2e_s, 0.0, pg, "cuda")
    e2e_val = ev_total / e2e_s

    if rank == 0:
        hbm, hbm_kind = measured_peaks()
        # the solve graphs: the iteration kernels, the first of them computing the packet's
        # metric and data image (the fused front; a separate prologue launch where it is
        # not fused is counted with them)
        avg_launch_ms = k_ms / max(1, k_launches)
        alg_bytes = (b_alg(args.storage) * k_pixiters +
                     (B_PROLOGUE + B_TVL1_ITER * args.tvl1) * cfg.W * cfg.H * args.steps)
        bytes_per_launch = alg_bytes / max(1, k_launches)
        achieved = bytes_per_launch / (avg_launch_ms * 1e-3) / 1e9
        bound, peak, peak_src = roofline_level(g.solver_name, n_sms, l2_gbs, smem_gbs)
        prof = profiled(cfg.name, g.solver_name)
        kernel = ("k_cluster" if g.solver_name.startswith("cluster") else
                  "k_tiled" if g.solver_name.startswith("tiled") else "iteration kernels")
        line = {
            "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": ["f32", "f32 (p, ubar stored f16)",
                                           "f32 (p, ubar stored bf16)"][args.storage],
            "data": "synthetic",
            "gpix_iter_per_s": gpix,
            "median_of_5_runs": ({"value": float(np.median(runs)), "unit": "events/s",
                                  "runs": runs, "rank": 0} if runs else None),
            "config": {"workload": describe(cfg), "sensor": f"{cfg.W}x{cfg.H}",
                       "events_per_step": cfg.packet, "iters": cfg.iters,
                       "solver": g.solver_name, "parallelism": f"{world} independent streams",
                       "tvl1_iters": args.tvl1,
                       "l2": "flushed between timed steps (256 MiB write, outside the events)",
                       "inputs": "device-resident event arrays (evr_step_device: push "
                                 "and solve)",
                       "settled": bool(settled),
                       "untimed_before_warmup": "first packet (autotuner) + packets until "
                                                "the solver configuration is settled"},
            "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": (prof["dram_bytes_per_launch"] if prof else None),
                         "kernel": f"{kernel}: the solve's iteration launches "
                                   f"({g.solver_name}), prologue fused",
                         "peak_source": peak_src,
                         "frac_hbm": achieved / hbm, "hbm_peak": hbm,
                         "hbm_peak_source": f"{hbm_kind} hbm_gbs (MEASURED_PEAKS.json)",
                         "l2_gbs": l2_gbs, "smem_gbs_all_sms": smem_gbs,
                         "issue_active": (prof.get("issue_active") if prof else None),
                         "avg_launch_us": avg_launch_ms * 1e3,
                         "launches_per_solve": k_launches / args.steps,
                         "bytes_per_launch": bytes_per_launch,
                         "timing": "CUDA events around each solve graph on the launching "
                                   "stream, a second pass over as many packets as the "
                                   "timed steps (pushes outside the events)"},
            "e2e": {"value": e2e_val, "unit": "events/s",
                    "h2d_bytes_per_step": cfg.packet * (2 + 2 + 8 + 1),
                    "d2h_bytes_per_step": cfg.W * cfg.H * 4 + 4,  # image + status word
                    "calls": "evr_step (host arrays: push and solve) + "
                             "evr_get_image_async into pinned memory, three steps in flight"},
            # the timed steps' graphs, as the library counted them: the solve's launches,
            # plus the push kernel unless the solver's first launch integrates the packet
            "gpu_launches": int(step_launches),
            "launches_per_step": step_launches / args.steps,
            "first_image_ms": first_ms,
            "clocks": clocks,
            "wall_s_timed": wall,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(cfg, stream, args.cpu_budget_s)
        if args.check_error:
            line["error_vs_fp64"] = error_vs_oracle(E, cfg, stream, p)
        print(json.dumps(line), flush=True)
    g.close()
    g2.close()
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


# ----------------------------------------------------------------------- batched streams
def run_batch_bench(args):
    """256 independent streams of mixed sizes, one packet per active stream per step.
    Under torchrun the streams are split over the ranks by their work (shard.batch_share):
    strong scaling of the one batched workload, no data-path collective."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    from paper_1607_06283_gb300 import build
    if rank == 0:
        build.build()
    if pg:
        pg.barrier()
    from paper_1607_06283_gb300 import evr as E
    from paper_1607_06283_gb300.shard import batch_share, reduce_timing
    from evsim.configs import batch_configs, batch_step_arrays, make_batch
    all_cfgs = batch_configs()
    mine = batch_share(all_cfgs, world, rank)
    cfgs = [all_cfgs[i] for i in mine]
    # every stream holds at least 20 packets and at most 400: past step 400 the batch
    # would be idle, so the timed steps are capped (the line reports the count used)
    args.steps = min(args.steps, 60)
    args.warmup = min(args.warmup, 20)
    n_steps = args.warmup + args.steps
    streams = make_batch(cfgs, max_packets=n_steps)
    packet, iters = cfgs[0].packet, cfgs[0].iters
    sizes = [(c.W, c.H) for c in cfgs]
    cur = torch.cuda.Stream()
    torch.cuda.set_stream(cur)
    b = E.Batch(sizes, storage=args.storage, tile_config=args.tile)
    b.set_cuda_stream(cur.cuda_stream)
    grouping = None
    if args.grouping is not None:
        parts = [int(v) for v in args.grouping.split(",")]
        grouping = (parts[0], parts[1] if len(parts) > 1 else 1)
        b.set_grouping(*grouping)
    schedule = {"auto": E.EVR_BATCH_SCHEDULE_AUTO, "graph": E.EVR_BATCH_SCHEDULE_GRAPH,
                "persistent": E.EVR_BATCH_SCHEDULE_PERSISTENT}[args.schedule]
    b.set_schedule(schedule)
    l2_gbs = E.evr_measure_peak(0, cur.cuda_stream)
    steps = [batch_step_arrays(streams, packet, k) for k in range(n_steps)]
    dev = []
    for x, y, t, p, off in steps:
        dev.append(tuple(torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).cuda()
                         for a in (x, y, t, p, off)))
    clk = ClockSampler(local)  # started (and running) before the warm-up steps
    if rank == 0:
        clk.start()
        clk.wait_first()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(max(args.steps, args.warmup))]
    b.enable_kernel_timing(True)
    for k in range(args.warmup):  # as the timed steps: flush, events, kernel timing
        flush.fill_(float(k))
        evs[k][0].record(cur)
        b.step_device(*dev[k], iters)
        evs[k][1].record(cur)
    assert b.synchronize() == (0, -1)
    evs = evs[:args.steps]
    b.enable_kernel_timing(True)  # counts from here
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    for j in range(args.steps):
        flush.fill_(float(j))
        evs[j][0].record(cur)
        b.step_device(*dev[args.warmup + j], iters)
        evs[j][1].record(cur)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = clk.stop() if rank == 0 else None
    ms = sum(a.elapsed_time(c) for a, c in evs)
    k_ms, k_launches, _ = b.kernel_time()
    assert b.synchronize() == (0, -1)
    ev = 0
    pxit = 0
    for j in range(args.steps):
        off = steps[args.warmup + j][4]
        cnt = np.diff(off)
        ev += int(cnt.sum())
        pxit += sum(w * h for (w, h), c in zip(sizes, cnt) if c > 0) * iters
    ms_local, ev_local, pxit_local = ms, ev, pxit
    ms, ev = reduce_timing(ms_local, ev_local, pg, "cuda")
    _, pxit = reduce_timing(ms_local, pxit_local, pg, "cuda")
    value = ev / (ms * 1e-3)
    # end to end: host arrays in, all images out into pinned memory, every step; two
    # steps in flight (the next step is queued before the previous images are waited for)
    b2 = E.Batch(sizes, storage=args.storage, tile_config=args.tile)
    b2.set_cuda_stream(cur.cuda_stream)
    if grouping is not None:
        b2.set_grouping(*grouping)
    b2.set_schedule(schedule)
    n_img = sum(w * h for w, h in sizes)
    imgs = [torch.empty(n_img, dtype=torch.float32).pin_memory().numpy() for _ in range(2)]
    for k in range(args.warmup):
        b2.step(*steps[k], iters)
        b2.wait_images(b2.images_async(imgs[k % 2]))
    t0 = time.perf_counter()
    prev = None
    for j in range(args.steps):
        b2.step(*steps[args.warmup + j], iters)
        t = b2.images_async(imgs[j % 2])
        if prev is not None:
            b2.wait_images(prev)
        prev = t
    b2.wait_images(prev)
    e2e_s = time.perf_counter() - t0
    e2e_s, _ = reduce_timing(e2e_s, 0.0, pg, "cuda")
    peak, peak_kind = measured_peaks()
    # the step graph: prologue (B_PROLOGUE per pixel of an active stream) + passes, this
    # rank's kernels on this rank's launching stream
    achieved = ((b_alg(args.storage) * pxit_local + B_PROLOGUE * pxit_local / iters) /
                (k_ms * 1e-3) / 1e9)
    # cut into groups that fit L2, a group's state stays in L2 across its passes (the
    # level that bounds them); one group sweeps the whole batch through HBM every pass
    persistent = b.schedule == E.EVR_BATCH_SCHEDULE_PERSISTENT
    grouped = "L2 groups" in b.solver_name or "windows of" in b.solver_name
    # ncu counters of the persistent launch (one per step), keyed by its configuration
    prof = None
    if persistent and args.storage == 0 and world == 1:
        key = b.solver_name.split(": ", 1)[-1].split(", windows")[0]
        prof = profiled("batch256", key)
    if grouped:
        level = {"bound": "l2", "peak": l2_gbs, "frac": achieved / l2_gbs,
                 "peak_source": "L2, measured in this run (evr_measure_peak level 0)"}
    else:
        level = {"bound": "hbm", "peak": peak, "frac": achieved / peak,
                 "peak_source": f"{peak_kind} hbm_gbs"}
    if rank != 0:
        b.close()
        b2.close()
        pg.barrier()
        pg.destroy_process_group()
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
        "dtype": ["f32", "f32 (p, ubar stored f16)", "f32 (p, ubar stored bf16)"][args.storage],
        "data": "synthetic",
        "gpix_iter_per_s": pxit / (ms * 1e-3) / 1e9,
        "config": {"workload": "batch256: 256 streams (96 x 128x128, 96 x 240x180, "
                               "64 x 346x260), rects/blobs scenes, packets U[20,400], "
                               "500-event packets, 50 iterations",
                   "solver": b.solver_name, "schedule": args.schedule,
                   "steps_timed": "one packet per active stream",
                   "parallelism": (f"streams split over {world} ranks by work "
                                   f"(rank 0: {len(mine)} streams)" if world > 1 else
                                   "one GPU"),
                   "l2": "flushed between timed steps (256 MiB write, outside the events)"},
        "roofline": {"bound": level["bound"], "achieved": achieved, "peak": level["peak"],
                     "unit": "GB/s", "frac": level["frac"],
                     "traffic": prof["dram_bytes_per_launch"] if prof else None,
                     "issue_active": prof["issue_active"] if prof else None,
                     "frac_hbm": achieved / peak,
                     "kernel": ("k_batch_persist: the whole step (pushes, prologue, "
                                "iteration passes) in one persistent launch" if persistent
                                else "batched prologue + iteration passes (graph)"),
                     "peak_source": level["peak_source"],
                     "launches_per_step": (k_launches if persistent
                                           else k_launches + args.steps) / args.steps},
        "e2e": {"value": ev / e2e_s, "unit": "events/s",
                "h2d_bytes_per_step": int(13 * ev / args.steps) + 8 * (len(sizes) + 1),
                "d2h_bytes_per_step": int(4 * n_img),
                "calls": "evr_batch_step (host arrays) + evr_batch_get_images_async into "
                         "pinned memory, two steps in flight"},
        "clocks": clocks,
        # per step: the persistent launch, or the push kernel and then the graph (per L2
        # group the prologue and the passes; the buffer flip); the library counts the
        # launches it times (all but the graph schedule's push)
        "gpu_launches": int(k_launches) + (0 if persistent else args.steps),
    }
    print(json.dumps(line), flush=True)
    b.close()
    b2.close()
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


# ----------------------------------------------------------------------- differentiation
def run_diff_bench(args):
    """64 streams of 240x180: per step and stream, f = data_image(u_prev, n+-, C),
    u = packet_solve(f, lambda) with 30 unrolled iterations (checkpoints every 10), an L2
    loss against the ground-truth frame, and the backward pass to lambda, C and f."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_1607_06283_gb300 import build
    build.build()
    from paper_1607_06283_gb300 import autograd as AG
    from paper_1607_06283_gb300 import evr as E
    from evsim.configs import StreamConfig, make_batch
    n_streams, W, H, packet, K = 64, 240, 180, 2000, 30
    every = args.every
    cfgs = [StreamConfig(f"diff{s}", W, H, "rects", 40, 5000 + s, 2 * packet, packet, K,
                         speed=120.0, noise=0.01, dt_us=250.0) for s in range(n_streams)]
    streams = make_batch(cfgs)
    dev = torch.device("cuda")
    items = []
    for st in streams:
        # one fixed solver configuration: the set-up states do not depend on it, and the
        # autotuner's trial solves of 64 new streams are skipped
        g = E.Stream(W, H, tile_config=45)
        a = st.slice(0, packet)
        g.push(a.x, a.y, a.t, a.pol)
        g.solve(K)
        b = st.slice(packet, 2 * packet)
        u_prev = g.state(E.EVR_STATE_U)
        p0 = g.p()
        g.push(b.x, b.y, b.t, b.pol)
        npos, nneg = g.state(E.EVR_STATE_NPOS), g.state(E.EVR_STATE_NNEG)
        g.solve(0)  # metric of this packet
        tx, ty = g.state(E.EVR_STATE_TX), g.state(E.EVR_STATE_TY)
        target = np.exp(st.log_frame(float(b.t[-1])) - st.log_frame(float(st.t[0]))).astype(
            np.float32)
        g.close()
        items.append((u_prev, p0, npos, nneg, tx, ty, target))
    # the 64 packets as one batch: images (64, H, W), dual variables (64, 3, H, W)
    u_prev, p0, npos, nneg, tx, ty, target = [
        torch.from_numpy(np.ascontiguousarray(np.stack([it[k] for it in items]))).to(dev)
        for k in range(7)]
    lam = torch.tensor(90.0, device=dev, requires_grad=True)
    C = torch.tensor(0.15, device=dev, requires_grad=True)

    def step():
        f = AG.data_image(u_prev, npos, nneg, C, C)
        u, _ = AG.packet_solve(f, lam, u_prev, p0, tx, ty, K, every)
        # sum of the 64 per-stream mean-square losses
        loss = ((u - target) ** 2).mean(dim=(1, 2)).sum()
        loss.backward()

    clk = ClockSampler(local)  # started (and running) before the warm-up steps
    clk.start()
    clk.wait_first()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    E.evr_unrolled_timing_start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    rev_ms, rev_n, rev_pi, rev_pl, launches = E.evr_unrolled_timing_stop()
    ms = e0.elapsed_time(e1)
    solves = n_streams * args.steps
    peak, peak_kind = measured_peaks()
    rev_bytes = B_REV_ITER * rev_pi + B_REV_LAUNCH * rev_pl
    achieved = rev_bytes / (rev_ms * 1e-3) / 1e9 if rev_ms > 0 else None
    # the captured launch's DRAM bytes, scaled to the average launch by algorithmic bytes
    # (traffic grows with the reversed pixel-iterations)
    prof = profiled("diff64", "k_rev_tiled")
    traffic = None
    if prof and prof.get("alg_bytes_per_launch"):
        traffic = (prof["dram_bytes_per_launch"] * (rev_bytes / max(rev_n, 1)) /
                   prof["alg_bytes_per_launch"])
    roofline = {
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": achieved / peak if achieved else None,
        "traffic": traffic,
        "issue_active": prof.get("issue_active") if prof else None,
        "kernel": "k_rev_tiled (reverse pass: 4 reversed iterations per launch, 32x32 tiles, "
                  "4-pixel halo)",
        "peak_source": f"{peak_kind} hbm_gbs", "avg_launch_us": rev_ms * 1e3 / max(rev_n, 1),
        "launches_timed": rev_n, "bytes_per_launch": rev_bytes / max(rev_n, 1)}
    line = {
        "metric": METRIC, "value": solves / (ms * 1e-3), "unit": "differentiated packet solves/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "gpix_iter_per_s_fwd_bwd": solves * W * H * K / (ms * 1e-3) / 1e9,
        "events_per_s": solves * packet / (ms * 1e-3),
        "config": {"workload": "diff64: 64 streams of 240x180 rectangles scenes, 2000-event "
                               f"packets, 30 unrolled iterations, checkpoints every {every}, L2 "
                               "loss vs ground-truth frames, gradients w.r.t. lambda, C and f",
                   "timing": "CUDA events around the whole step (one batched forward + "
                             "backward of the 64 packets per step, autograd on the host)",
                   "l2": "no flush: the working set is larger than L2 (the tape of one "
                         f"checkpoint segment alone is {min(every, K)} x 5 planes x 11 MB = "
                         f"{min(every, K) * 5 * 11e6 / 1e9:.2f} GB)"},
        "wall_s": wall,
        "roofline": roofline,
        "clocks": clocks,
        "gpu_launches": launches,
        "grad": {"lambda": float(lam.grad), "C": float(C.grad)},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "batch256":
        return run_batch_bench(args)
    if args.config == "diff64":
        return run_diff_bench(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
