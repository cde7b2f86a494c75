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
    ap.add_argument("--serving-requests", type=int, default=200)
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


def peaks_sm_mhz():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return float(json.load(fh).get("sm_max_mhz", 2070.0))
    return 2070.0


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
    for fn in ("gather_direct.cu", "gather.cuh", "kernels.cuh", "device.cuh"):
        with open(os.path.join(ROOT, "paper_1501_03869_gb300", "csrc", fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def single_frame_kernels(info):
    """Names of the two kernels one FP32 frame of a stored table takes: the
    windowed gather when every window fits its largest slot (288 rows)."""
    P = info["tile_pix"]
    sw = 4 if P == 128 else 2
    W = info["window"]
    if W <= 288:
        wb = 128 if W <= 128 else (192 if W <= 192 else 288)
        return f"gather_window_kernel<{P},{sw},f32,{wb}> + direct_reduce_kernel<{P},1>"
    return f"gather_direct_kernel<{P},{sw},f32,table> + direct_reduce_kernel<{P},{sw}>"


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


def _oracle_table_chunk(args):
    speed, dx, origin, sensors, pix = args
    import oracle
    return oracle.travel_table(speed, dx, origin, sensors, pix)


def oracle_tables_all_cores(speed, dx, origin, sensors, pix):
    """The oracle's fast-marching table T[ns, npix], sensors split over one
    spawn-started process per host core; returns (T, seconds, workers)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    n_w = max(1, os.cpu_count() or 1)
    sensors = np.asarray(sensors, dtype=np.float64)
    bounds = np.linspace(0, sensors.shape[0], min(4 * n_w, sensors.shape[0]) + 1).astype(int)
    jobs = [(np.asarray(speed, dtype=np.float64), dx, np.asarray(origin), sensors[a:b], np.asarray(pix))
            for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
    t0 = time.perf_counter()
    with cf.ProcessPoolExecutor(max_workers=n_w, mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_oracle_table_chunk, jobs))
    return np.concatenate(parts, axis=0), time.perf_counter() - t0, n_w


def accuracy(got, ref, p0max):
    """rel-L2 and max-abs / max|p0| of one image against the oracle's."""
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    return {"rel_l2": float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)),
            "max_abs_over_p0": float(np.abs(got - ref).max() / p0max)}


def oracle_leg(w, checks):
    """Host leg after the timed region: the oracle's own table build (one core
    and all cores) and every form's accuracy against the oracle on the same
    seeded inputs (FP32 gate rel-L2 1e-5, max-abs 1e-4 max|p0|; 16-bit gate
    rel-L2 5e-3 against the oracle on the original FP32 signals)."""
    import oracle
    from paper_1501_03869_gb300 import synth
    pix = np.flatnonzero(w.mask.ravel())
    out = {}
    n1 = 16
    t0 = time.perf_counter()
    oracle.travel_table(w.speed, w.dx, w.origin, w.sensors[:n1], pix)
    one = (time.perf_counter() - t0) / n1
    T, t_all, n_w = oracle_tables_all_cores(w.speed, w.dx, w.origin, w.sensors, pix)
    out["oracle_table_build_c2"] = {
        "sensors": int(w.n_sensors), "one_core_s_per_sensor": one,
        "one_core_s_extrapolated": one * w.n_sensors, "all_cores_s": t_all, "cores": n_w,
        "sample": f"one core: the first {n1} sensors' fast marching, timed and scaled to "
                  f"{w.n_sensors}; all cores: every sensor, one spawn-started process per core"}
    acc = {}
    p0 = float(np.abs(w.p0).max())
    ref1 = oracle.bp(T, w.signals[0].astype(np.float64), w.dt)
    if "single_f32" in checks:
        acc["single_f32"] = accuracy(checks["single_f32"].ravel()[pix], ref1, p0)
    for name in ("batched_f32", "batched_bf16"):
        if name not in checks:
            continue
        sigF, imgs, frames = checks[name]
        worst = None
        for f in frames:
            ref = oracle.bp(T, sigF[f].astype(np.float64), w.dt)
            a = accuracy(imgs[f].ravel()[pix], ref, p0 * float(np.abs(sigF[f]).max() /
                                                               np.abs(w.signals[0]).max()))
            if worst is None or a["rel_l2"] > worst["rel_l2"]:
                worst = a
        worst["frames_checked"] = list(frames)
        acc[name] = worst
    if "constant_f32" in checks:
        c0, img = checks["constant_f32"]
        Tc = oracle.constant_table(w.speed.shape, w.dx, w.origin, w.sensors, pix, c0)
        acc["constant_speed_f32"] = accuracy(img.ravel()[pix],
                                             oracle.bp(Tc, w.signals[0].astype(np.float64), w.dt), p0)
    if "c1" in checks:
        w1, img = checks["c1"]
        pix1 = np.flatnonzero(w1.mask.ravel())
        T1 = oracle.travel_table(w1.speed, w1.dx, w1.origin, w1.sensors, pix1)
        acc["latency_c1_f32"] = accuracy(img.ravel()[pix1],
                                         oracle.bp(T1, w1.signals[0].astype(np.float64), w1.dt),
                                         float(np.abs(w1.p0).max()))
    for key, (wi, img) in checks.get("c4", {}).items():
        pixi = np.flatnonzero(wi.mask.ravel())
        Ti, _, _ = oracle_tables_all_cores(wi.speed, wi.dx, wi.origin, wi.sensors, pixi)
        worst = None
        for f in range(wi.n_frames):
            a = accuracy(img[f].ravel()[pixi], oracle.bp(Ti, wi.signals[f].astype(np.float64), wi.dt),
                         float(np.abs(wi.p0).max()))
            if worst is None or a["rel_l2"] > worst["rel_l2"]:
                worst = a
        worst["frames"] = int(wi.n_frames)
        acc[key] = worst
    if "c3" in checks:
        # every frame of the precision form against the oracle on the original
        # FP32 signals (the 5e-3 gate) and on the dequantised input (the kernel's
        # own arithmetic)
        w3, imgs = checks["c3"]
        pix3 = np.flatnonzero(w3.mask.ravel())
        T3 = oracle.travel_table(w3.speed, w3.dx, w3.origin, w3.sensors, pix3)
        refs = [oracle.bp(T3, w3.signals[f].astype(np.float64), w3.dt) for f in range(w3.n_frames)]
        for dtype, img in imgs.items():
            _, _, deq = synth.quantise(w3.signals, dtype)
            e = [accuracy(img[f].ravel()[pix3], refs[f], float(np.abs(w3.p0).max()))["rel_l2"]
                 for f in range(w3.n_frames)]
            eq = [accuracy(img[f].ravel()[pix3], oracle.bp(T3, deq[f].astype(np.float64), w3.dt),
                           float(np.abs(w3.p0).max()))["rel_l2"] for f in range(w3.n_frames)]
            acc[f"precision_c3_{dtype}"] = {"frames": int(w3.n_frames),
                                            "rel_l2_max": float(max(e)), "rel_l2_mean": float(np.mean(e)),
                                            "rel_l2_vs_dequantised_max": float(max(eq)),
                                            "gate": 5e-3}
    out["accuracy_vs_oracle"] = acc
    return out


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


def multi_form(args, flush, stream, checks):
    """Uneven instances in one persistent launch: the 32-instance workload
    (grids 96^2-384^2, 128-1024 sensors, 1024-4096 samples, 1-16 frames),
    autotuned, replayed as a CUDA graph; L2 flushed before every execution."""
    import torch
    from paper_1501_03869_gb300 import BP, Plan, _lib, synth
    ws = [synth.config4_instance(i) for i in range(32)]
    # 256-pixel tiles, as in the batched form: fewer window rows per pixel and
    # sensor (measured 2.95 against 3.43 ms per execution with 128-pixel tiles)
    bps = [BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask,
              flags=_lib.PAT_FLAG_TILE_256) for w in ws]
    sig = [torch.from_numpy(w.signals).cuda() for w in ws]
    outs = [torch.empty(bp.out_shape(w.n_frames), device="cuda") for bp, w in zip(bps, ws)]
    plan = Plan(bps, [w.n_frames for w in ws], autotune=True, graph=True)
    plan.execute(sig, outs)
    plan.sync()
    Ev = torch.cuda.Event
    recs = []
    for i in range(max(5, min(args.steps // 100, 40)) + 3):
        flush()
        e0, e1 = Ev(enable_timing=True), Ev(enable_timing=True)
        e0.record(stream)
        plan.execute(sig, outs, stream=stream)
        e1.record(stream)
        recs.append((e0, e1))
    plan.sync(stream)
    ms = statistics.mean(a.elapsed_time(b) for a, b in recs[3:])
    cost = sorted((w.n_frames * w.n_sensors * w.n_pix, i) for i, w in enumerate(ws))
    checks["c4"] = {f"multi_c4_inst{i}": (ws[i], outs[i].cpu().numpy())
                    for i in (cost[0][1], cost[-1][1])}
    frames = sum(w.n_frames for w in ws)
    upd = sum(w.n_frames * w.n_sensors * w.n_pix for w in ws)
    info = plan.info
    # HBM bytes one execution must move: every instance's table once per
    # frame group (frames per unit FB_i), its signals, and its image
    hbm = 0.0
    for bp, w in zip(bps, ws):
        fb = min(8, 1 << (w.n_frames.bit_length() - 1))
        passes = -(-w.n_frames // fb)
        hbm += passes * bp.info["table_bytes"] + 4.0 * w.n_frames * w.n_sensors * w.nt \
            + 4.0 * w.n_frames * w.n_pix
    hbm_peak, kind = peaks()
    plan.close()
    for bp in bps:
        bp.close()
    return {"workload": "32 uneven instances (grids 96^2-384^2, 128-1024 sensors, 1024-4096 samples, "
                        "1-16 frames), 256-pixel tiles, instances grouped by frames per unit, CUDA graph",
            "frames": frames, "ms_per_execution": ms, "frames_per_s": frames / (ms / 1e3),
            "value": upd / (ms / 1e3) / 1e9, "unit": UNIT, "launch_shape": info,
            "gpu_launches_per_execution": 2 * info["n_classes"],
            "roofline": {"bound": "hbm", "algorithmic_bytes": hbm,
                         "achieved": hbm / (ms / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                         "frac": hbm / (ms / 1e3) / 1e9 / hbm_peak, "peak_source": kind,
                         "note": "tables once per frame group, signals and images; the HBM floor, "
                                 "not the binding resource (shared-memory window traffic is)"}}


def serving_form(args):
    """The 3-D serving workload at full size: 8 subjects (160x160x96 voxels at
    0.25 mm, all 2 457 600 reconstructed, 1024 sensors on a hemisphere,
    spherical-shell skull 2200-3000 m/s), tables solved on the GPU, BF16
    signals of 2048 samples submitted from page-locked buffers, results into
    page-locked buffers.  Poisson arrivals (subjects uniform) at 50, 100, 200
    and 400 frames/s and a saturating burst under a 120 GB HBM budget, then a
    40 GB budget that holds three subjects, so admissions evict the least
    recently used table and reload it from its host copy inside the latency."""
    import torch
    from paper_1501_03869_gb300 import Server, _lib, synth
    n_sub = 8
    subs = [synth.config5_subject(k, n_frames=2) for k in range(n_sub)]
    srv = Server(hbm_budget=120 << 30, n_streams=4, max_batch_frames=16)
    t0 = time.perf_counter()
    ids = [srv.register(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask,
                        flags=_lib.PAT_FLAG_GPU_TABLE) for w in subs]
    reg_s = (time.perf_counter() - t0) / n_sub
    inp = []
    for w in subs:
        codes, sc, _ = synth.quantise(w.signals, "bf16")
        c = torch.empty(codes.shape, dtype=torch.int16, pin_memory=True).numpy().view(np.uint16)
        c[:] = codes
        scl = torch.empty(sc.shape, dtype=torch.float32, pin_memory=True).numpy()
        scl[:] = sc
        inp.append((c, scl))
    # results go to a ring of 256 page-locked images (9.8 MB each): a request
    # waits for the ring slot's previous request, so at most 256 are queued
    ring = [torch.empty(subs[0].speed.shape, dtype=torch.float32, pin_memory=True).numpy()
            for _ in range(256)]
    ring_t = [None] * len(ring)
    rng = np.random.default_rng(5)

    def run(rate, n):
        st0 = srv.stats()
        lat = []
        t_start = time.perf_counter()
        t_next = t_start
        for i in range(n):
            if rate:
                t_next += rng.exponential(1.0 / rate)
                while time.perf_counter() < t_next:
                    pass
            j = i % len(ring)
            if ring_t[j] is not None:  # the ring slot's earlier request must be done
                lat.append(srv.wait(ring_t[j], timeout_s=300.0))
            k, f = int(rng.integers(n_sub)), int(rng.integers(2))
            ring_t[j] = srv.submit(ids[k], inp[k][0][f], ring[j], dtype="bf16", scales=inp[k][1][f])
        for j in range(len(ring)):
            if ring_t[j] is not None:
                lat.append(srv.wait(ring_t[j], timeout_s=300.0))
                ring_t[j] = None
        el = time.perf_counter() - t_start
        st1 = srv.stats()
        nb = st1["batches"] - st0["batches"]
        nf = st1["mean_batch_frames"] * st1["batches"] - st0["mean_batch_frames"] * st0["batches"]
        return {"offered_fps": rate if rate else "burst", "requests": n, "frames_per_s": n / el,
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_batch_frames": nf / max(nb, 1), "batches": nb,
                "evictions": st1["evictions"] - st0["evictions"],
                "uploads": st1["uploads"] - st0["uploads"]}

    n = args.serving_requests
    run(None, 16)  # warm-up: every subject's working buffers allocated
    # warm-up of every batch shape (unstaged 2-3 frames, 4- and 8-frame units):
    # first uses of a kernel and its launch shape happen outside the timed runs
    for nb in (2, 3, 4, 8, 16):
        ts = [srv.submit(ids[0], inp[0][0][f % 2], ring[f], dtype="bf16", scales=inp[0][1][f % 2])
              for f in range(nb)]
        for t in ts:
            srv.wait(t, timeout_s=300.0)
    out = {"workload": "8 subjects 160x160x96 at 0.25 mm (2 457 600 voxels each), 1024 sensors on "
                       "a hemisphere, BF16 signals of 2048 samples, page-locked host buffers",
           "updates_per_frame": int(subs[0].n_pix) * 1024,
           "register_s_per_subject": reg_s, "budget_gb": 120, "rates": []}
    for rate in (50.0, 100.0, 200.0, 400.0):
        out["rates"].append(run(rate, n))
    out["rates"].append(run(None, 4 * n))
    st = srv.stats()
    out["resident_gb_at_120"] = st["resident_bytes"] / 2**30
    srv.set_budget(40 << 30)
    out["evict_40gb"] = run(50.0, max(n // 4, 20))
    out["evict_40gb"]["resident_gb"] = srv.stats()["resident_bytes"] / 2**30
    srv.close()
    return out


def serving_batching_form(args, w):
    """Continuous batching against no batching on the paper-shaped frame: a
    burst of requests (64 distinct FP32 frames, page-locked buffers) through a
    server that batches up to 16 frames of a subject and through one that runs
    every frame alone; frames/s of both and whether every result has the same
    bits in both."""
    import torch
    from paper_1501_03869_gb300 import Server
    F = 64
    rng = np.random.default_rng(11)
    frames = torch.empty((F,) + w.signals.shape[1:], dtype=torch.float32, pin_memory=True).numpy()
    frames[:] = (w.signals[0][None] * rng.uniform(0.5, 1.5, (F, 1, 1))).astype(np.float32)
    res, outs = {}, {}
    for name, mb in (("batched", 16), ("unbatched", 1)):
        srv = Server(hbm_budget=8 << 30, n_streams=4, max_batch_frames=mb)
        sid = srv.register(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask)
        out = torch.empty((F,) + w.speed.shape, dtype=torch.float32, pin_memory=True).numpy()
        for f in range(8):  # warm-up: working buffers and streams
            srv.wait(srv.submit(sid, frames[f], out[f]))
        reps = max(2, args.serving_requests // F)
        t0 = time.perf_counter()
        lat = []
        for _ in range(reps):
            ts = [srv.submit(sid, frames[f], out[f]) for f in range(F)]
            lat += [srv.wait(t) for t in ts]
        el = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        res[name] = {"frames_per_s": reps * F / el, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                     "p99_ms": float(np.percentile(lat, 99) * 1e3),
                     "mean_batch_frames": st["mean_batch_frames"], "max_batch_frames": mb}
        outs[name] = out
    res["gain"] = res["batched"]["frames_per_s"] / res["unbatched"]["frames_per_s"]
    res["same_bits"] = bool(np.array_equal(outs["batched"], outs["unbatched"]))
    res["workload"] = ("paper-shaped frame, bursts of 64 distinct FP32 frames from page-locked "
                       "buffers, results into page-locked buffers")
    return res


def constant_form(args, w, flush, stream, checks):
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
    checks["constant_f32"] = (C_CONSTANT_BP, out.cpu().numpy()[0])
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


def batched_roofline(w, tile_flags, F, FB, shared_read_bytes, gather_ms, sm_mhz, n_sm, l2_smem_gbs):
    """Roofline of the staged gather on F frames: the larger of the
    shared-memory time (gather reads plus the bulk copies' writes, 128 B per
    clock per SM) and the L2 -> shared stream time (window and table-block
    copies against the measured bulk-copy bandwidth), against the measured
    gather time.  Window rows per (tile, sensor) are the library's: from the
    first integer sample of the tile's arrivals to two past the last, in
    multiples of 8."""
    from paper_1501_03869_gb300 import table_host
    info, u, base, slot = table_host(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask,
                                     flags=tile_flags)
    P, nt_, ns = info["tile_pix"], info["n_tiles"], w.n_sensors
    uu = np.where(u < 1e29, u, np.nan).reshape(nt_, ns, P)
    mx = np.nan_to_num(np.nanmax(uu, axis=2), nan=0.0)
    rows = np.ceil((np.floor(mx) + 3) / 8) * 8
    n_fg = -(-F // FB)
    n_pix = int(info["n_pix"])
    win = float(rows.sum()) * FB * 4 * n_fg                  # window copies
    tab = float(nt_ * ns * P * 4) * n_fg                     # table blocks
    upd = F * ns * n_pix
    smem_bytes = shared_read_bytes * upd + win + tab
    xbar_bytes = win + tab
    smem_peak = 128.0 * n_sm * sm_mhz * 1e6 / 1e9
    t_smem = smem_bytes / (smem_peak * 1e9)
    t_xbar = xbar_bytes / (l2_smem_gbs * 1e9)
    bound = "smem" if t_smem >= t_xbar else "l2_to_smem"
    t = max(t_smem, t_xbar)
    return {"bound": bound, "frac": t / (gather_ms / 1e3), "gather_ms": gather_ms,
            "smem_bytes": smem_bytes, "smem_peak_GBps": smem_peak,
            "smem_achieved_GBps": smem_bytes / (gather_ms / 1e3) / 1e9,
            "l2_to_smem_bytes": xbar_bytes, "l2_to_smem_peak_GBps": l2_smem_gbs,
            "l2_to_smem_achieved_GBps": xbar_bytes / (gather_ms / 1e3) / 1e9,
            "shared_read_bytes_per_update": shared_read_bytes,
            "window_rows_per_pixel_sensor": float(rows.sum()) / (ns * n_pix),
            "frames_per_unit": FB, "peak_source": "smem: 128 B/clk/SM x SMs x max SM clock; "
                                                  "l2_to_smem: bulk-copy bandwidth measured in this "
                                                  "run (pat_probe_l2_to_smem)"}


def time_steps_warm(fn, steps, warmup):
    """Per-step spans of fn() with nothing between the steps (warm L2)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    recs = [fn() for _ in range(steps)]
    torch.cuda.synchronize()
    return recs


def c3_form(args, flush, stream, checks):
    """The precision form: the 128x128 geometry (64 sensors, 1024 samples, 6 092
    pixels), 64 frames sharing one table, BF16 and FP16 signals with per-row
    FP32 scales, FP32 accumulation; each batch is the whole user call
    (preprocessing + gather) replayed as a CUDA graph, L2 flushed before it.
    The per-frame error against the FP64 oracle is added in the host leg."""
    import torch
    from paper_1501_03869_gb300 import BP, synth
    Ev = torch.cuda.Event
    w = synth.config3(n_frames=64)
    bp = BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask)
    res = {"workload": "128x128 at 0.2 mm, 64 sensors, 1024 samples, 6092-pixel mask, 64 frames, "
                       "16-bit signals with per-row FP32 scales", "frames": 64}
    imgs = {}
    for dtype, tdt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        codes, sc, _ = synth.quantise(w.signals, dtype)
        s16 = torch.from_numpy(codes.astype(np.int16)).cuda().view(tdt)
        scl = torch.from_numpy(sc).cuda()
        out = torch.empty(bp.out_shape(64), device="cuda")
        bp.autotune(s16, scales=scl, out=out)
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            bp.reconstruct(s16, scales=scl, out=out, stream=side)
        stream.wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            bp.reconstruct(s16, scales=scl, out=out, stream=torch.cuda.current_stream())

        def step():
            e0, e1 = Ev(enable_timing=True), Ev(enable_timing=True)
            e0.record(stream)
            graph.replay()
            e1.record(stream)
            return e0, e1

        n = max(20, min(args.steps // 10, 200))
        ms = statistics.mean(a.elapsed_time(b) for a, b in time_steps(step, n, args.warmup, stream, flush))
        upd = 64 * int(w.n_pix) * w.n_sensors
        res[dtype] = {"ms_per_batch": ms, "frames_per_s": 64 / (ms / 1e3),
                      "value": upd / (ms / 1e3) / 1e9, "unit": UNIT}
        imgs[dtype] = out.cpu().numpy()
    bp.close()
    checks["c3"] = (w, imgs)
    return res


def c5_frame_form(args, flush, stream):
    """One full-size 3-D frame (160x160x96 at 0.25 mm, every voxel, 1024 sensors,
    a 10 GB GPU-solved table), FP32 and BF16 signals: the whole user call by
    events, L2 flushed before it, with its HBM roofline (table + signals +
    image bytes over the call time)."""
    import torch
    from paper_1501_03869_gb300 import BP, _lib, synth
    Ev = torch.cuda.Event
    w = synth.config5_subject(0, n_frames=1)
    bp = BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask, flags=_lib.PAT_FLAG_GPU_TABLE)
    codes, sc, _ = synth.quantise(w.signals, "bf16")
    inputs = {"f32": (torch.from_numpy(w.signals).cuda(), None, 4),
              "bf16": (torch.from_numpy(codes.astype(np.int16)).cuda().view(torch.bfloat16),
                       torch.from_numpy(sc).cuda(), 2)}
    hbm_peak, kind = peaks()
    upd = int(w.n_pix) * w.n_sensors
    res = {"workload": "160x160x96 at 0.25 mm, 2 457 600 voxels, 1024 hemisphere sensors, 2048 samples, "
                       "GPU-solved table", "table_gb": bp.info["table_bytes"] / 1e9,
           "window": bp.info["window"]}
    for dt, (sig, scl, esz) in inputs.items():
        out = torch.empty(bp.out_shape(1), device="cuda")

        def step():
            e0, e1 = Ev(enable_timing=True), Ev(enable_timing=True)
            e0.record(stream)
            bp.reconstruct(sig, scales=scl, out=out, stream=stream)
            e1.record(stream)
            return e0, e1

        ms = statistics.median(a.elapsed_time(b) for a, b in time_steps(step, 30, args.warmup, stream, flush))
        alg = bp.info["table_bytes"] + esz * w.n_sensors * w.nt + 4.0 * w.n_pix
        res[dt] = {"ms_per_frame": ms, "value": upd / (ms / 1e3) / 1e9, "unit": UNIT,
                   "roofline": {"bound": "hbm", "algorithmic_bytes": alg,
                                "achieved": alg / (ms / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                                "frac": alg / (ms / 1e3) / 1e9 / hbm_peak, "peak_source": kind,
                                "timed": "the whole call (preprocessing, gather, reduction) by events"}}
    bp.close()
    return res


def c1_form(args, flush, stream, checks):
    """Latency of the small single-frame workload (128x128 grid, 64 sensors,
    1024 samples, 6 092 pixels): the user call replayed as a CUDA graph, L2
    flushed (cold) and not (warm), by events; and through the host round trip
    (page-locked buffers, wall clock)."""
    import torch
    from paper_1501_03869_gb300 import BP, synth
    Ev = torch.cuda.Event
    w1 = synth.config1(n_frames=1)
    bp1 = BP(w1.speed, w1.dx, w1.origin, w1.sensors, w1.dt, w1.nt, mask=w1.mask)
    sig = torch.from_numpy(w1.signals).cuda()
    out = torch.empty(bp1.out_shape(1), device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        bp1.reconstruct(sig, out=out, stream=side)
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bp1.reconstruct(sig, out=out, stream=torch.cuda.current_stream())

    def step():
        e0, e1 = Ev(enable_timing=True), Ev(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        return e0, e1

    n = max(50, min(args.steps, 1000))
    cold = [a.elapsed_time(b) for a, b in time_steps(step, n, args.warmup, stream, flush)]
    warm = [a.elapsed_time(b) for a, b in time_steps_warm(step, n, args.warmup)]
    checks["c1"] = (w1, out.cpu().numpy()[0])
    pin_sig = torch.empty(w1.signals.shape, dtype=torch.float32, pin_memory=True).numpy()
    pin_sig[:] = w1.signals
    pin_out = torch.empty(bp1.out_shape(1), dtype=torch.float32, pin_memory=True).numpy()
    for _ in range(args.warmup):
        bp1.reconstruct_host(pin_sig, out=pin_out)
    host = []
    for _ in range(min(n, 300)):
        t0 = time.perf_counter()
        bp1.reconstruct_host(pin_sig, out=pin_out)
        host.append(time.perf_counter() - t0)
    bp1.close()
    upd = int(w1.n_pix) * w1.n_sensors
    return {"workload": "128x128 at 0.2 mm, 64 sensors, 1024 FP32 samples, 6092-pixel mask",
            "device_cold_p50_us": float(np.percentile(cold, 50) * 1e3),
            "device_cold_p99_us": float(np.percentile(cold, 99) * 1e3),
            "device_warm_p50_us": float(np.percentile(warm, 50) * 1e3),
            "host_round_trip_p50_us": float(np.percentile(host, 50) * 1e6),
            "host_round_trip_p99_us": float(np.percentile(host, 99) * 1e6),
            "value_cold": upd / (statistics.mean(cold) / 1e3) / 1e9, "unit": UNIT}


class L2Flush:
    """Empties the L2 (129 MB) before a timed step: a 512 MB write, then a
    256 MB read of another buffer.  The read evicts the write's dirty lines
    (writing them back) before the step starts, so the step's DRAM traffic is
    its own, not the flush's write-back, while nothing the step reads is left
    in L2."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        self.r = torch.zeros(L2_FLUSH_BYTES // 8, dtype=torch.float32, device=dev)
        self.sink = None

    def __call__(self):
        self.w.zero_()
        self.sink = self.r.sum()


def time_steps(fn, steps, warmup, stream, flush):
    """Per-step device times (ms) of fn(); L2 flushed before every step, events
    on `stream`.  fn returns a list of (name, start_evt, end_evt) spans."""
    import torch
    for _ in range(warmup):
        flush()
        fn()
    torch.cuda.synchronize()
    recs = []
    for _ in range(steps):
        flush()
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
    flush = L2Flush(dev)
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

    def gather_only():
        # the gather kernel alone (measurement hook: no reduction into the image)
        import ctypes
        e0, e1, e2 = Ev(enable_timing=True), Ev(enable_timing=True), Ev(enable_timing=True)
        e0.record(stream)
        bp.preprocess(sig, stream=stream)
        e1.record(stream)
        rc = bp._lib.pat_test_gather_only(bp._h, ctypes.c_void_p(stream.cuda_stream))
        e2.record(stream)
        if rc != 0:
            raise RuntimeError(f"pat_test_gather_only: status {rc}")
        return e0, e1, e2

    # per-kernel device times (events on the launching stream, L2 flushed)
    n_k = max(20, min(args.steps, 200))
    path_ms = [a.elapsed_time(b) for a, b in time_steps(path_kernels, n_k, args.warmup, stream, flush)]
    kr = time_steps(split_kernels, n_k, args.warmup, stream, flush)
    pre_ms = [a.elapsed_time(b) for a, b, c in kr]
    gat_ms = [b.elapsed_time(c) for a, b, c in kr]
    go_ms = [b.elapsed_time(c) for a, b, c in time_steps(gather_only, n_k, args.warmup, stream, flush)]

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
        flush()
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
            flush()
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
    # the gather kernel reads the table and the integrand; its reduction reads
    # the segment sums and writes the image (4 bytes per pixel)
    alg_bytes = 4.0 * ns * n_pix + 4.0 * ns * nt
    alg_bytes_red = alg_bytes + 4.0 * n_pix
    go_avg_s = statistics.mean(go_ms) / 1e3
    achieved = alg_bytes / go_avg_s / 1e9
    gat_avg_s = statistics.mean(gat_ms) / 1e3
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_source": peak_kind,
                "traffic": ncu_traffic(updates),
                "kernel": single_frame_kernels(info).split(" + ")[0],
                "timed": "the gather kernel alone (pat_test_gather_only after the preprocessing), by events "
                         "on the launching stream, L2 flushed before every step",
                "algorithmic_bytes_per_launch": alg_bytes,
                "with_reduction": {"kernels": single_frame_kernels(info),
                                   "timed": "the gather and its reduction (split-call API), by events",
                                   "us": gat_avg_s * 1e6, "algorithmic_bytes": alg_bytes_red,
                                   "frac": alg_bytes_red / gat_avg_s / 1e9 / hbm_peak},
                "path_us": statistics.mean(path_ms) * 1e3,
                "split_call_us": {"preprocess": statistics.mean(pre_ms) * 1e3,
                                  "gather_alone": statistics.mean(go_ms) * 1e3,
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
        flush()
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
    checks = {"single_f32": out.cpu().numpy()[0]}
    # warm L2: the same replayed step without the flush (table and integrand
    # stay in the 129 MB L2 between steps)
    warm = time_steps_warm(step, max(50, min(args.steps, 1000)), args.warmup)
    warm_ms = statistics.mean(a.elapsed_time(b) for a, b in warm)
    forms["single_f32_warm_l2"] = {"ms_per_step": warm_ms, "value": updates / (warm_ms / 1e3) / 1e9,
                                   "unit": UNIT, "frames_per_s": 1e3 / warm_ms}
    if not args.no_forms:
        forms["latency_c1"] = c1_form(args, flush, stream, checks)
        forms["precision_c3"] = c3_form(args, flush, stream, checks)
        forms["single_frame_c5"] = c5_frame_form(args, flush, stream)
    if not args.no_forms and args.batch_frames > 1:
        F = args.batch_frames
        from paper_1501_03869_gb300 import _lib
        from paper_1501_03869_gb300 import probe_l2_to_smem
        l2s = probe_l2_to_smem()
        forms["l2_to_smem_bulk_GBps"] = l2s
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

            def gstep(s=s, scl=scl):
                e0, e1, e2 = Ev(enable_timing=True), Ev(enable_timing=True), Ev(enable_timing=True)
                e0.record(stream)
                bpb.preprocess(s, scales=scl, stream=stream)
                e1.record(stream)
                bpb.gather(F, outF, stream=stream)
                e2.record(stream)
                return e0, e1, e2
            rg = time_steps(gstep, n_rep, 2, stream, flush)
            g_ms = statistics.mean(b.elapsed_time(c) for a, b, c in rg)
            FB = min(8, 1 << (F.bit_length() - 1))
            forms[name] = {"frames": F, "ms_per_batch": ms, "frames_per_s": F / (ms / 1e3),
                           "value": F * updates / (ms / 1e3) / 1e9, "unit": UNIT, "tile_pix": 256,
                           "gather_ms": g_ms,
                           "roofline": batched_roofline(
                               w, _lib.PAT_FLAG_TILE_256, F, FB, 8.0 if scl is None else 4.0, g_ms,
                               peaks_sm_mhz(), torch.cuda.get_device_properties(dev).multi_processor_count,
                               l2s)}
            picks = sorted({0, F // 3, (2 * F) // 3, F - 1})
            imgs = outF.cpu().numpy()
            checks[name] = (sigF.cpu().numpy(), {f: imgs[f] for f in picks}, picks)
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
        forms["constant_speed_c2"] = constant_form(args, w, flush, stream, checks)
    if not args.no_multi and world == 1:
        forms["multi_instance_c4"] = multi_form(args, flush, stream, checks)
    if not args.no_serving and world == 1:
        forms["serving_batching_c2"] = serving_batching_form(args, w)
        forms["serving_c5_full"] = serving_form(args)

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
            forms.update(oracle_leg(w, checks))

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
                       "l2": "flushed before every step: 512 MB write, then a 256 MB read of "
                             "another buffer (no dirty flush lines left to write back in the step)"},
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
