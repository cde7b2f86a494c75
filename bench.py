"""Benchmark of the on-line back projection (Eq. (BP)) on the paper-shaped frame.

Workload (the paper's 0.39 mm case, Sec. III): 256x256 grid at 0.1 mm, skull
ring 2200-3000 m/s, 512 sensors on a ring, 2048 FP32 samples, 21 323
reconstructed pixels; synthetic signals (see paper_1501_03869_gb300/synth.py).
One step = one frame through the whole on-line path: the preprocessing kernel
(b = 2p - 2t dp/dt) and the gather kernel.  The table (off-line fast marching)
is built before timing, as in the paper.

Output: one JSON line (rank 0).  `value` is pixel*sensor updates per second
(G/s) of the single-frame FP32 path with inputs resident in HBM, L2 flushed
before every step; `e2e` is the same metric through pat_bp_reconstruct_host
(pinned host buffers, copies inside the timed region); `forms` adds the
batched FP32 / BF16 forms, the constant-speed (conventional) back projection
of the same frame, many instances in one launch and 3-D serving;
`cpu_baseline` is the FP64 oracle on this host.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G pixel·sensor updates/s & frames/s; p50/p99 frame latency vs plain FP32 kernel"
UNIT = "G pixel*sensor updates/s"
WORKLOAD = ("paper-shaped frame: 2D 256x256 dx 0.1 mm, skull ring 2200-3000 m/s, 512 sensors "
            "on a ring, 2048 FP32 samples, 21323-pixel disc mask, plain FP32 kernel")
L2_FLUSH_BYTES = 512 << 20
C_CONSTANT_BP = 1560.0  # m/s: the conventional back projection's speed in Sec. III


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch-frames", type=int, default=64)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-multi", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-constant", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=300)
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def max_over_ranks(value, world, dist=None, device=None):
    """The largest of the ranks' values, returned on every rank (the replicas'
    timed region ends when the slowest one does); one rank: unchanged."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.first = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            # wait for the first sample so the sampler runs before timing starts
            self.first = self.proc.stdout.readline()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in ([self.first or ""] + out.splitlines()) if l.strip()]

    def summary(self):
        if not getattr(self, "lines", None):
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash():
    """Hash of the sources of the single-frame gather (the kernel the roofline
    line is about); a committed traffic record is used only while it matches."""
    h = hashlib.sha256()
    for fn in ("gather_direct.cu", "gather.cuh", "kernels.cuh"):
        with open(os.path.join(ROOT, "paper_1501_03869_gb300", "csrc", fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(per_update_units):
    """DRAM bytes per launch of the gather kernel from the committed ncu summary,
    scaled to this launch; None if the kernel changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "gather_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    if d.get("kernel_hash") != kernel_source_hash():
        return None
    return float(d["dram_bytes_per_update"]) * per_update_units


def oracle_cpu_rate(w, n_sensors, seconds, frames=1):
    """FP64 oracle back projection on this host: updates/s over a bounded run."""
    import oracle
    pix = np.flatnonzero(w.mask.ravel())
    sens = w.sensors[:n_sensors]
    T = oracle.travel_table(w.speed, w.dx, w.origin, sens, pix)
    p = w.signals[0, :n_sensors].astype(np.float64)
    n = 0
    t0 = time.perf_counter()
    while True:
        oracle.bp(T, p, w.dt)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return n * n_sensors * pix.size / el, el, n


def _oracle_chunk(args):
    """One worker of the all-cores oracle timing: the oracle's back projection
    over a chunk of the pixels, repeated for about `seconds`."""
    T, p, dt, seconds = args
    import oracle
    n = 0
    t0 = time.perf_counter()
    while True:
        oracle.bp(T, p, dt)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return n * T.shape[0] * T.shape[1], time.perf_counter() - t0


def oracle_cpu_rate_all_cores(w, n_sensors, seconds):
    """The same oracle back projection, unmodified, run over pixel chunks by one
    process per host core (a spawn-started pool: this runs after CUDA work).
    Returns (updates/s summed over the workers' rates, workers)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import oracle
    pix = np.flatnonzero(w.mask.ravel())
    T = oracle.travel_table(w.speed, w.dx, w.origin, w.sensors[:n_sensors], pix)
    p = w.signals[0, :n_sensors].astype(np.float64)
    n_w = max(1, os.cpu_count() or 1)
    chunks = np.array_split(np.arange(pix.size), n_w)
    jobs = [(np.ascontiguousarray(T[:, c]), p, w.dt, seconds) for c in chunks if c.size]
    with cf.ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_chunk, jobs))
    return sum(u / t for u, t in res), len(jobs)


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    from paper_1501_03869_gb300 import synth
    import oracle
    w = synth.config2(n_frames=1)
    pix = np.flatnonzero(w.mask.ravel())
    n_s = 32  # a bounded sample of the frame per step: 32 sensors x all pixels
    T = oracle.travel_table(w.speed, w.dx, w.origin, w.sensors[:n_s], pix)
    p = w.signals[0, :n_s].astype(np.float64)
    for _ in range(args.warmup):
        oracle.bp(T, p, w.dt)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.bp(T, p, w.dt)
        times.append(time.perf_counter() - t0)
    upd = n_s * pix.size
    tot = sum(times)
    val = upd * args.steps / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "frames_per_s": args.steps / tot * n_s / w.n_sensors,
        "config": {"workload": WORKLOAD, "global_batch": 1, "n_sensors": w.n_sensors,
                   "n_pix": int(pix.size), "n_samples": w.nt, "l2": "host run"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"per step the first {n_s} sensors x {pix.size} pixels of the "
                                   "frame, FP64 oracle back projection (table built before timing)"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def multi_form(args, flush, stream):
    """Uneven instances in one persistent launch: the 32-instance workload
    (grids 96^2-384^2, 128-1024 sensors, 1024-4096 samples, 1-16 frames),
    autotuned, replayed as a CUDA graph; L2 flushed before every execution."""
    import torch
    from paper_1501_03869_gb300 import BP, Plan, synth
    ws = [synth.config4_instance(i) for i in range(32)]
    bps = [BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) for w in ws]
    sig = [torch.from_numpy(w.signals).cuda() for w in ws]
    outs = [torch.empty(bp.out_shape(w.n_frames), device="cuda") for bp, w in zip(bps, ws)]
    plan = Plan(bps, [w.n_frames for w in ws], autotune=True, graph=True)
    plan.execute(sig, outs)
    plan.sync()
    Ev = torch.cuda.Event
    recs = []
    for i in range(max(5, min(args.steps // 100, 40)) + 3):
        flush.zero_()
        e0, e1 = Ev(enable_timing=True), Ev(enable_timing=True)
        e0.record(stream)
        plan.execute(sig, outs, stream=stream)
        e1.record(stream)
        recs.append((e0, e1))
    plan.sync(stream)
    ms = statistics.mean(a.elapsed_time(b) for a, b in recs[3:])
    frames = sum(w.n_frames for w in ws)
    upd = sum(w.n_frames * w.n_sensors * w.n_pix for w in ws)
    info = plan.info
    plan.close()
    for bp in bps:
        bp.close()
    return {"workload": "32 uneven instances, one persistent launch, CUDA graph", "frames": frames,
            "ms_per_execution": ms, "frames_per_s": frames / (ms / 1e3),
            "value": upd / (ms / 1e3) / 1e9, "unit": UNIT, "launch_shape": info,
            "gpu_launches_per_execution": 2}


def serving_form(args):
    """Request loop over several 3-D subjects (hemisphere of sensors around a
    spherical-shell skull, BF16 signals of 2048 samples): Poisson arrivals at
    several rates, frames/s and p50/p99 submit-to-done latency."""
    import torch  # noqa: F401  (CUDA context)
    from paper_1501_03869_gb300 import Server, synth
    shape, n_s, n_sub = (48, 80, 80), 256, 4
    subs = [synth.config5_subject(k, n_frames=4, n_sensors=n_s, shape=shape, dx=0.5e-3)
            for k in range(n_sub)]
    srv = Server(hbm_budget=120 << 30, n_streams=4, max_batch_frames=16)
    ids = [srv.register(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) for w in subs]
    q = [synth.quantise(w.signals, "bf16") for w in subs]
    rng = np.random.default_rng(5)
    out = {"workload": f"{n_sub} 3-D subjects {shape[::-1]} at 0.5 mm, {n_s} sensors on a hemisphere, "
                       "BF16 signals of 2048 samples, HBM budget 120 GB", "rates": []}
    for rate in (200.0, 800.0, 3200.0):
        n = args.serving_requests
        gaps = rng.exponential(1.0 / rate, n)
        pending = []
        t0 = time.perf_counter()
        t_next = t0
        for i in range(n):
            t_next += gaps[i]
            while time.perf_counter() < t_next:
                pass
            k = int(rng.integers(n_sub))
            f = int(rng.integers(subs[k].n_frames))
            codes, sc, _ = q[k]
            o = np.empty(subs[k].speed.shape, np.float32)
            pending.append(srv.submit(ids[k], codes[f], o, dtype="bf16", scales=sc[f]))
        lat = [srv.wait(t) for t in pending]
        el = time.perf_counter() - t0
        out["rates"].append({"offered_fps": rate, "requests": n, "frames_per_s": n / el,
                             "p50_ms": float(np.percentile(lat, 50) * 1e3),
                             "p99_ms": float(np.percentile(lat, 99) * 1e3)})
    st = srv.stats()
    out["mean_batch_frames"] = st["mean_batch_frames"]
    out["batches"] = st["batches"]
    srv.close()
    return out


def constant_form(args, w, flush, stream):
    """The conventional back projection of the same frame (Sec. III's
    comparison method, 1560 m/s): delays computed in the gather kernel, no
    table stream.  Single frame as a replayed CUDA graph, and 64 frames."""
    import torch
    from paper_1501_03869_gb300 import BP
    Ev = torch.cuda.Event
    dev = torch.device("cuda", torch.cuda.current_device())
    bpc = BP.constant(C_CONSTANT_BP, w.speed.shape, w.dx, w.origin, w.sensors, w.dt, w.nt,
                      mask=w.mask)
    updates = bpc.info["n_pix"] * w.n_sensors
    sig = torch.from_numpy(w.signals).to(dev)
    out = torch.empty(bpc.out_shape(1), device=dev)
    bpc.reserve(64)
    bpc.autotune(sig, out=out)

    def kern():
        e0, e1 = Ev(enable_timing=True), Ev(enable_timing=True)
        e0.record(stream)
        bpc.reconstruct(sig, out=out, stream=stream)
        e1.record(stream)
        return e0, e1

    kr = time_steps(kern, max(20, min(args.steps, 200)), args.warmup, stream, flush)
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        bpc.reconstruct(sig, out=out, stream=side)
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bpc.reconstruct(sig, out=out, stream=torch.cuda.current_stream())

    def step():
        e0, e1 = Ev(enable_timing=True), Ev(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        return e0, e1

    rr = time_steps(step, max(50, min(args.steps, 1000)), args.warmup, stream, flush)
    ms = statistics.mean(a.elapsed_time(b) for a, b in rr)
    form = {"c0": C_CONSTANT_BP, "ms_per_step": ms, "frames_per_s": 1e3 / ms,
            "value": updates / (ms / 1e3) / 1e9, "unit": UNIT,
            "path_us": statistics.mean(a.elapsed_time(b) for a, b in kr) * 1e3,
            "delay_bytes": bpc.info["table_bytes"]}
    F = 64
    rng = np.random.default_rng(9)
    sigF = torch.from_numpy(
        (w.signals[0][None] * rng.uniform(0.5, 1.5, (F, 1, 1))).astype(np.float32)).to(dev)
    outF = torch.empty(bpc.out_shape(F), device=dev)
    bpc.autotune(sigF, out=outF)

    def fstep():
        e0, e1 = Ev(enable_timing=True), Ev(enable_timing=True)
        e0.record(stream)
        bpc.reconstruct(sigF, out=outF, stream=stream)
        e1.record(stream)
        return e0, e1

    rr = time_steps(fstep, max(3, args.steps // 5), 2, stream, flush)
    msF = statistics.mean(a.elapsed_time(b) for a, b in rr)
    form["batched_f32"] = {"frames": F, "ms_per_batch": msF, "frames_per_s": F / (msF / 1e3),
                           "value": F * updates / (msF / 1e3) / 1e9, "unit": UNIT}
    bpc.sync()
    bpc.close()
    return form


def time_steps(fn, steps, warmup, stream, flush):
    """Per-step device times (ms) of fn(); L2 flushed before every step, events
    on `stream`.  fn returns a list of (name, start_evt, end_evt) spans."""
    import torch
    for _ in range(warmup):
        flush.zero_()
        fn()
    torch.cuda.synchronize()
    recs = []
    for _ in range(steps):
        flush.zero_()
        recs.append(fn())
    torch.cuda.synchronize()
    return recs


def main():
    args = parse()
    rank, local_rank, world = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import torch.distributed as dist

    from paper_1501_03869_gb300 import BP, synth

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    w = synth.config2(n_frames=1)
    bp = BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask)
    info = bp.info
    n_pix, ns, nt = info["n_pix"], w.n_sensors, w.nt
    updates = n_pix * ns
    sig = torch.from_numpy(w.signals).to(dev)
    out = torch.empty(bp.out_shape(1), device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    bp.reserve(max(args.batch_frames, 1))
    # (one frame takes the unstaged gather, which has no launch shape to tune)
    Ev = torch.cuda.Event

    def path_kernels():
        # the user call: preprocessing, gather and reduction of one FP32 frame
        e0, e1 = Ev(enable_timing=True), Ev(enable_timing=True)
        e0.record(stream)
        bp.reconstruct(sig, out=out, stream=stream)
        e1.record(stream)
        return e0, e1

    def split_kernels():
        # the same frame through the two-call API: preprocessing, then gather + reduction
        e0, e1, e2 = Ev(enable_timing=True), Ev(enable_timing=True), Ev(enable_timing=True)
        e0.record(stream)
        bp.preprocess(sig, stream=stream)
        e1.record(stream)
        bp.gather(1, out, stream=stream)
        e2.record(stream)
        return e0, e1, e2

    # per-kernel device times (events on the launching stream, L2 flushed)
    n_k = max(20, min(args.steps, 200))
    path_ms = [a.elapsed_time(b) for a, b in time_steps(path_kernels, n_k, args.warmup, stream, flush)]
    kr = time_steps(split_kernels, n_k, args.warmup, stream, flush)
    pre_ms = [a.elapsed_time(b) for a, b, c in kr]
    gat_ms = [b.elapsed_time(c) for a, b, c in kr]

    # one step = the on-line path (the user call) captured once as a CUDA graph, replayed
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        bp.reconstruct(sig, out=out, stream=side)
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bp.reconstruct(sig, out=out, stream=torch.cuda.current_stream())

    def step():
        e0, e1 = Ev(enable_timing=True), Ev(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        return e0, e1

    # ---------------------------------------------------- timed single frame --
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    gid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    gid = f"GPU-{gid}" if gid is not None and not str(gid).startswith("GPU-") else (gid or local_rank)
    with ClockSampler(gid) as clk:
        wall0 = time.perf_counter()
        recs = []
        for _ in range(args.steps):
            flush.zero_()
            recs.append(step())
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    bp.sync()
    step_ms = [a.elapsed_time(b) for a, b in recs]
    tot_ms = sum(step_ms)
    tot_ms = max_over_ranks(tot_ms, world, dist, dev)
    ms_per_step = tot_ms / args.steps
    value = world * updates * args.steps / (tot_ms / 1e3) / 1e9
    clocks = clk.summary()

    # ------------------------------------------------------------ roofline --
    hbm_peak, peak_kind = peaks()
    alg_bytes = 4.0 * ns * n_pix + 4.0 * ns * nt + 4.0 * n_pix
    gat_avg_s = statistics.mean(gat_ms) / 1e3
    achieved = alg_bytes / gat_avg_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_source": peak_kind,
                "traffic": ncu_traffic(updates),
                "kernel": "gather_direct_kernel<128,4,f32,table> + direct_reduce_kernel<128,4>",
                "timed": "the gather and its reduction (split-call API), by events on the launching stream",
                "algorithmic_bytes_per_launch": alg_bytes,
                "path_us": statistics.mean(path_ms) * 1e3,
                "split_call_us": {"preprocess": statistics.mean(pre_ms) * 1e3,
                                  "gather_and_reduction": statistics.mean(gat_ms) * 1e3}}

    # ------------------------------------------------------------------ e2e --
    pin_sig = torch.empty(w.signals.shape, dtype=torch.float32, pin_memory=True)
    pin_sig.copy_(torch.from_numpy(w.signals))
    pin_out = torch.empty(bp.out_shape(1), dtype=torch.float32, pin_memory=True)
    sig_np, out_np = pin_sig.numpy(), pin_out.numpy()
    for _ in range(args.warmup):
        bp.reconstruct_host(sig_np, out=out_np)
    e2e_t = []
    for _ in range(min(args.steps, 500)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bp.reconstruct_host(sig_np, out=out_np)
        e2e_t.append(time.perf_counter() - t0)
    e2e = {"value": world * updates * len(e2e_t) / sum(e2e_t) / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": int(w.signals.nbytes), "d2h_bytes_per_step": int(out_np.nbytes),
           "path": "pat_bp_reconstruct_host on page-locked buffers: the kernels read the signals and "
                   "write the image in host memory over the host link, L2 flushed before every call",
           "ms_per_step": sum(e2e_t) / len(e2e_t) * 1e3,
           "p50_ms": float(np.percentile(e2e_t, 50) * 1e3),
           "p99_ms": float(np.percentile(e2e_t, 99) * 1e3)}

    # --------------------------------------------------------------- forms --
    forms = {}
    if not args.no_forms and args.batch_frames > 1:
        F = args.batch_frames
        from paper_1501_03869_gb300 import _lib
        bpb = BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask,
                 flags=_lib.PAT_FLAG_TILE_256)
        rng = np.random.default_rng(7)
        sigF = torch.from_numpy(
            (w.signals[0][None] * rng.uniform(0.5, 1.5, (F, 1, 1))).astype(np.float32)).to(dev)
        outF = torch.empty(bpb.out_shape(F), device=dev)
        codes, sc, _ = synth.quantise(sigF.cpu().numpy(), "bf16")
        sig16 = torch.from_numpy(codes.astype(np.int16)).to(dev).view(torch.bfloat16)
        sc16 = torch.from_numpy(sc).to(dev)
        for name, s, scl in (("batched_f32", sigF, None), ("batched_bf16", sig16, sc16)):
            bpb.autotune(s, scales=scl, out=outF)
            def fstep(s=s, scl=scl):
                e0, e1 = Ev(enable_timing=True), Ev(enable_timing=True)
                e0.record(stream)
                bpb.reconstruct(s, scales=scl, out=outF, stream=stream)
                e1.record(stream)
                return e0, e1
            n_rep = max(3, args.steps // 5)
            rr = time_steps(fstep, n_rep, 2, stream, flush)
            ms = statistics.mean(a.elapsed_time(b) for a, b in rr)
            forms[name] = {"frames": F, "ms_per_batch": ms, "frames_per_s": F / (ms / 1e3),
                           "value": F * updates / (ms / 1e3) / 1e9, "unit": UNIT, "tile_pix": 256}
        bpb.sync()
        bpb.close()

    if not args.no_forms:
        # the off-line step on this frame: the table built by the host march
        # (all host cores) and by the GPU solver (same first-order scheme)
        from paper_1501_03869_gb300 import _lib
        with BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask,
                flags=_lib.PAT_FLAG_GPU_TABLE) as bpg:
            gpu_s = float(bpg.info["build_seconds"])
        forms["table_build_c2"] = {"sensors": int(w.sensors.shape[0]),
                                   "host_march_s": float(bp.info["build_seconds"]),
                                   "host_threads": os.cpu_count(),
                                   "gpu_solver_s": gpu_s}
    if not args.no_constant:
        forms["constant_speed_c2"] = constant_form(args, w, flush, stream)
    if not args.no_multi and world == 1:
        forms["multi_instance_c4"] = multi_form(args, flush, stream)
    if not args.no_serving and world == 1:
        forms["serving_3d"] = serving_form(args)

    # -------------------------------------------------------- cpu baseline --
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        n_s = 128
        rate, el, n = oracle_cpu_rate(w, n_s, args.cpu_seconds)
        cpu = {"value": rate / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} runs of the FP64 oracle back projection over the first {n_s} "
                         f"sensors x {n_pix} pixels ({el:.1f} s, table built before timing)"}
        if not args.no_forms:
            rate_all, n_w = oracle_cpu_rate_all_cores(w, n_s, min(args.cpu_seconds, 5.0))
            forms["cpu_oracle_all_cores"] = {
                "value": rate_all / 1e9, "unit": UNIT, "cores": n_w, "kind": "oracle",
                "sample": f"the same back projection over pixel chunks, one process per host core"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "frames_per_s": world * args.steps / (tot_ms / 1e3),
            "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
            "config": {"workload": WORKLOAD, "global_batch": world, "n_sensors": ns,
                       "n_pix": n_pix, "n_samples": nt, "tile_pix": info["tile_pix"],
                       "split": info["split"], "parallelism": f"replicas x{world}",
                       "l2": "flushed before every step (512 MB write)"},
            "gpu_launches": 3 * args.steps,
            "step": "CUDA graph of pat_bp_reconstruct (preprocessing + gather + segment reduction), "
                    "replayed",
            "roofline": roofline, "e2e": e2e, "forms": forms,
            "clocks": clocks, "cpu_baseline": cpu, "wall_s": wall,
            "paper_context": {"ms": 123.79, "hardware": "Tesla C2075, incl. transfers",
                              "note": "sample count not stated in the paper"},
        }
        print(json.dumps(line), flush=True)
    bp.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
