"""GB300 fast-marching back projection for photoacoustic tomography.

Wang & Jing, "A fast marching method based back projection algorithm for
photoacoustic tomography in heterogeneous media":
  * Sec. II-B: fast-marching travel times from each sensor (off line, once per
    speed map) -- built inside :class:`BP` creation by the host march or, with
    PAT_FLAG_GPU_TABLE, by the GPU solver (:func:`fmm_gpu` solves whole grids);
  * Sec. II-C, Eq. (BP): per-frame back projection of 2p - 2t dp/dt at those
    travel times -- CUDA kernels for sm_103a behind the C ABI of
    ``include/pat_bp.h``; :meth:`BP.constant` for the constant-speed
    comparison, :meth:`BP.set_solid_angle` for the exact back projection.

PyTorch is used for device memory and streams only.  The CUDA library is
loaded lazily; any call fails loudly when it has not been built.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import PatError

__all__ = ["BP", "Plan", "Server", "PatError", "fmm_host", "fmm_gpu", "table_host", "reconstruct_multi",
           "wait_timeout_probe", "probe_l2_to_smem", "DTYPES"]

DTYPES = {"f32": _lib.PAT_F32, "bf16": _lib.PAT_BF16, "f16": _lib.PAT_F16}


def _torch():
    import torch
    return torch


def _dtype_code(t):
    torch = _torch()
    m = {torch.float32: _lib.PAT_F32, torch.bfloat16: _lib.PAT_BF16, torch.float16: _lib.PAT_F16}
    if t.dtype not in m:
        raise TypeError(f"signals must be float32, bfloat16 or float16, not {t.dtype}")
    return m[t.dtype]


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class BP:
    """One speed map, sensor layout and mask with its device travel-time table.

    speed      ([nz,] ny, nx) sound speed (m/s) at the nodes
    dx         node spacing (m); origin: position of node 0 (x first, m)
    sensors    [ns, 3] sensor positions (m)
    dt, n_samples   sampling of every signal (t_k = k dt)
    mask       grid-shaped, nonzero = reconstruct (None = all nodes)
    weights    [ns] w_s of Eq. (BP) (None = 1/ns)
    flags      PAT_FLAG_* (tile size, compact output, host mirror, second-order
               or GPU-solved table, ...)
    """

    def __init__(self, speed, dx, origin, sensors, dt, n_samples, mask=None, weights=None,
                 flags=0, compact=False):
        speed = np.ascontiguousarray(speed, dtype=np.float32)
        self._create(speed.shape, dx, origin, sensors, dt, n_samples, mask, weights, flags,
                     compact, lambda lib, *args: lib.pat_bp_create(speed.ctypes.data, *args),
                     "pat_bp_create")

    @classmethod
    def constant(cls, c0, shape, dx, origin, sensors, dt, n_samples, mask=None, weights=None,
                 flags=0, compact=False):
        """The conventional back projection (Sec. III's comparison method):
        delays |r - r_s| / c0 for a constant sound speed c0 (m/s), computed in
        the gather kernel; no travel-time table.  shape is the grid's
        ([nz,] ny, nx); sensors may lie outside the grid."""
        self = cls.__new__(cls)
        self._create(tuple(shape), dx, origin, sensors, dt, n_samples, mask, weights, flags,
                     compact, lambda lib, *args: lib.pat_bp_create_constant(float(c0), *args),
                     "pat_bp_create_constant")
        return self

    def _create(self, shape, dx, origin, sensors, dt, n_samples, mask, weights, flags, compact,
                create, what):
        lib = _lib.load()
        self.shape = tuple(shape)
        self.grid = _lib.make_grid(self.shape, dx, origin)
        sensors = np.ascontiguousarray(sensors, dtype=np.float64)
        if sensors.ndim != 2 or sensors.shape[1] != 3:
            raise ValueError("sensors must be [ns, 3]")
        self.n_sensors = sensors.shape[0]
        self.n_samples = int(n_samples)
        self.dt = float(dt)
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        if m is not None and m.shape != self.shape:
            raise ValueError("mask must have the grid's shape")
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
        if compact:
            flags |= _lib.PAT_FLAG_COMPACT_OUT
        self.compact = bool(flags & _lib.PAT_FLAG_COMPACT_OUT)
        h = ctypes.c_void_p()
        _lib.check(create(lib, ctypes.byref(self.grid), sensors.ctypes.data, self.n_sensors,
                          None if m is None else m.ctypes.data,
                          None if w is None else w.ctypes.data, self.dt, self.n_samples, flags,
                          ctypes.byref(h)), what)
        self._h = h
        self._lib = lib
        self._refresh_info()

    def _refresh_info(self):
        inf = _lib.PatInfo()
        _lib.check(self._lib.pat_bp_info(self._h, ctypes.byref(inf)), "pat_bp_info")
        self.info = {k: getattr(inf, k) for k, _ in _lib.PatInfo._fields_}

    def set_solid_angle(self, normals, elem, omega0):
        """Exact back projection (Sec. II-C): weight every term by the share of
        the full angle omega0 that the sensor's element subtends at the pixel,
        elem_s (n_s . (r - r_s)) / |r - r_s|^d / omega0 (d = grid dimension).
        normals [ns, 3] point into the imaged region; elem [ns] are element
        lengths (2-D) or areas (3-D).  Replaces the per-sensor weights; plans
        take the handle together with other weighted handles only."""
        nrm = np.ascontiguousarray(normals, dtype=np.float64)
        el = np.ascontiguousarray(elem, dtype=np.float64)
        if nrm.shape != (self.n_sensors, 3) or el.shape != (self.n_sensors,):
            raise ValueError("normals must be [ns, 3] and elem [ns]")
        _lib.check(self._lib.pat_bp_set_solid_angle(self._h, nrm.ctypes.data, el.ctypes.data,
                                                    float(omega0)), "pat_bp_set_solid_angle")
        self._refresh_info()
        return self

    # ------------------------------------------------------------ lifecycle --
    def close(self):
        if getattr(self, "_h", None):
            self._lib.pat_bp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    @property
    def n_pix(self):
        return int(self.info["n_pix"])

    def out_shape(self, n_frames):
        return (n_frames, self.n_pix) if self.compact else (n_frames,) + tuple(self.shape)

    # -------------------------------------------------------------- compute --
    def reconstruct(self, signals, scales=None, out=None, stream=None):
        """Eq. (BP) for signals [F, ns, nt] (CUDA tensor).  Asynchronous on
        `stream` (default: torch's current stream).  Returns `out`."""
        torch = _torch()
        if signals.dim() == 2:
            signals = signals.unsqueeze(0)
        if not signals.is_cuda or not signals.is_contiguous():
            raise ValueError("signals must be a contiguous CUDA tensor")
        F, ns, nt = signals.shape
        if ns != self.n_sensors or nt != self.n_samples:
            raise ValueError(f"signals shape {tuple(signals.shape)} does not match the handle")
        code = _dtype_code(signals)
        if scales is not None:
            if not scales.is_cuda or scales.dtype != torch.float32 or not scales.is_contiguous():
                raise ValueError("scales must be a contiguous float32 CUDA tensor")
            if tuple(scales.shape) != (F, ns):
                raise ValueError("scales must be [F, ns]")
        if out is None:
            out = torch.empty(self.out_shape(F), dtype=torch.float32, device=signals.device)
        elif not out.is_contiguous() or out.dtype != torch.float32 or out.numel() != int(
                np.prod(self.out_shape(F))):
            raise ValueError("out must be a contiguous float32 tensor of the output shape")
        _lib.check(self._lib.pat_bp_reconstruct(
            self._h, ctypes.c_void_p(signals.data_ptr()), code,
            None if scales is None else ctypes.c_void_p(scales.data_ptr()), F,
            ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)), "pat_bp_reconstruct")
        return out

    def preprocess(self, signals, scales=None, stream=None):
        """First kernel only: Eq. (BP) integrand of signals [F, ns, nt] into the
        handle's buffer (asynchronous)."""
        if signals.dim() == 2:
            signals = signals.unsqueeze(0)
        if not signals.is_cuda or not signals.is_contiguous():
            raise ValueError("signals must be a contiguous CUDA tensor")
        F = signals.shape[0]
        _lib.check(self._lib.pat_bp_preprocess(
            self._h, ctypes.c_void_p(signals.data_ptr()), _dtype_code(signals),
            None if scales is None else ctypes.c_void_p(scales.data_ptr()), F,
            _stream_ptr(stream)), "pat_bp_preprocess")
        return F

    def gather(self, n_frames, out, stream=None):
        """Second kernel only: back projection of the last preprocessed frames."""
        if not out.is_contiguous() or out.dtype != _torch().float32 or out.numel() != int(
                np.prod(self.out_shape(n_frames))):
            raise ValueError("out must be a contiguous float32 tensor of the output shape")
        _lib.check(self._lib.pat_bp_gather(self._h, int(n_frames), ctypes.c_void_p(out.data_ptr()),
                                           _stream_ptr(stream)), "pat_bp_gather")
        return out

    def reconstruct_host(self, signals, dtype="f32", scales=None, out=None):
        """Host-to-host path: numpy signals [F, ns, nt] (float32, or uint16 codes
        for 'bf16'/'f16' with float32 scales [F, ns]); returns the image."""
        code = DTYPES[dtype]
        sig = np.ascontiguousarray(signals)
        if sig.ndim == 2:
            sig = sig[None]
        want = np.float32 if code == _lib.PAT_F32 else np.uint16
        if sig.dtype != want:
            raise TypeError(f"{dtype} signals must be {np.dtype(want).name}")
        F = sig.shape[0]
        sc = None if scales is None else np.ascontiguousarray(scales, dtype=np.float32)
        if out is None:
            out = np.empty(self.out_shape(F), dtype=np.float32)
        _lib.check(self._lib.pat_bp_reconstruct_host(
            self._h, sig.ctypes.data, code, None if sc is None else sc.ctypes.data, F,
            out.ctypes.data), "pat_bp_reconstruct_host")
        return out

    def autotune(self, signals, scales=None, out=None, stream=None):
        """Time launch shapes for this frame count on these inputs; later calls
        with the same frames-per-unit grouping use the fastest."""
        if signals.dim() == 2:
            signals = signals.unsqueeze(0)
        F = signals.shape[0]
        if out is None:
            out = _torch().empty(self.out_shape(F), dtype=_torch().float32, device=signals.device)
        _lib.check(self._lib.pat_bp_autotune(
            self._h, ctypes.c_void_p(signals.data_ptr()), _dtype_code(signals),
            None if scales is None else ctypes.c_void_p(scales.data_ptr()), F,
            ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)), "pat_bp_autotune")
        return out

    def reconstruct_noalloc(self, signals, out, scales=None, stream=None):
        """pat_bp_reconstruct_noalloc: the library allocates no device memory
        for this call (scratch comes from a fixed 16 MiB device array; calls
        must not overlap on the GPU).  `out` must be given."""
        if signals.dim() == 2:
            signals = signals.unsqueeze(0)
        F = signals.shape[0]
        if not out.is_contiguous() or out.dtype != _torch().float32 or out.numel() != int(
                np.prod(self.out_shape(F))):
            raise ValueError("out must be a contiguous float32 tensor of the output shape")
        _lib.check(self._lib.pat_bp_reconstruct_noalloc(
            self._h, ctypes.c_void_p(signals.data_ptr()), _dtype_code(signals),
            None if scales is None else ctypes.c_void_p(scales.data_ptr()), F,
            ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)), "pat_bp_reconstruct_noalloc")
        return out

    def evict(self):
        """Free the device table (needs flags |= PAT_FLAG_HOST_MIRROR at creation)."""
        _lib.check(self._lib.pat_bp_evict(self._h), "pat_bp_evict")

    def restore(self, stream=None):
        _lib.check(self._lib.pat_bp_restore(self._h, _stream_ptr(stream)), "pat_bp_restore")

    def reserve(self, max_frames, dtype="f32"):
        _lib.check(self._lib.pat_bp_reserve(self._h, int(max_frames), DTYPES[dtype]),
                   "pat_bp_reserve")

    def sync(self, stream=None):
        _lib.check(self._lib.pat_bp_sync(self._h, _stream_ptr(stream)), "pat_bp_sync")

    def table(self):
        """(u [tiles, ns, P] float32, base [tiles, ns] int32, slot [tiles*P] int32);
        u is None for a constant-speed handle (it stores no offsets)."""
        nt, ns, P = self.info["n_tiles"], self.n_sensors, self.info["tile_pix"]
        u = None if self.info["delays"] else np.empty((nt, ns, P), dtype=np.float32)
        b = np.empty((nt, ns), dtype=np.int32)
        s = np.empty(nt * P, dtype=np.int32)
        _lib.check(self._lib.pat_bp_table(self._h, None if u is None else u.ctypes.data,
                                          b.ctypes.data, s.ctypes.data), "pat_bp_table")
        return u, b, s


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p
    return arr


def _tensor_ptrs(ts):
    return _ptr_array([None if t is None else t.data_ptr() for t in ts])


class Plan:
    """Several handles reconstructed by one persistent launch (uneven grids,
    sensor, sample and frame counts); optionally autotuned and replayed as a
    CUDA graph.  frames[i] frames of handle bps[i] per execution."""

    def __init__(self, bps, frames, dtype="f32", autotune=False, graph=False):
        lib = _lib.load()
        self._lib = lib
        self.bps = list(bps)
        self.frames = [int(f) for f in frames]
        if len(self.frames) != len(self.bps):
            raise ValueError("one frame count per handle")
        self.dtype = dtype
        flags = (_lib.PAT_PLAN_AUTOTUNE if autotune else 0) | (_lib.PAT_PLAN_GRAPH if graph else 0)
        hs = _ptr_array([b.handle.value for b in self.bps])
        fr = (ctypes.c_int * len(self.frames))(*self.frames)
        h = ctypes.c_void_p()
        _lib.check(lib.pat_plan_create(hs, fr, len(self.bps), DTYPES[dtype], flags, ctypes.byref(h)),
                   "pat_plan_create")
        self._h = h

    def out_shapes(self):
        return [b.out_shape(f) for b, f in zip(self.bps, self.frames)]

    def execute(self, signals, outs, scales=None, stream=None):
        if len(signals) != len(self.bps) or len(outs) != len(self.bps):
            raise ValueError("one signal tensor and one output per handle")
        for b, f, s, o in zip(self.bps, self.frames, signals, outs):
            if not s.is_cuda or not s.is_contiguous() or tuple(s.shape) != (f, b.n_sensors, b.n_samples):
                raise ValueError("signals must be contiguous CUDA tensors [F, ns, nt]")
            if not o.is_contiguous() or o.numel() != int(np.prod(b.out_shape(f))):
                raise ValueError("outs must be contiguous float32 tensors of the output shapes")
        sc = None if scales is None else _tensor_ptrs(scales)
        _lib.check(self._lib.pat_plan_execute(self._h, _tensor_ptrs(signals), sc, _tensor_ptrs(outs),
                                              _stream_ptr(stream)), "pat_plan_execute")
        return outs

    def sync(self, stream=None):
        _lib.check(self._lib.pat_plan_sync(self._h, _stream_ptr(stream)), "pat_plan_sync")

    @property
    def info(self):
        inf = _lib.PatPlanInfo()
        _lib.check(self._lib.pat_plan_info(self._h, ctypes.byref(inf)), "pat_plan_info")
        return {k: getattr(inf, k) for k, _ in _lib.PatPlanInfo._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pat_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop over several subjects (speed maps)
    within an HBM budget.  submit() takes one frame [ns, nt] (float32, or
    uint16 codes with float32 scales [ns] for 'bf16'/'f16') and a float32
    output array; both are kept alive here until the ticket is polled done."""

    def __init__(self, hbm_budget, n_streams=4, max_batch_frames=16, max_queue=4096, stall_us=0):
        lib = _lib.load()
        self._lib = lib
        cfg = _lib.PatSrvCfg(n_streams, max_batch_frames, max_queue, stall_us)
        h = ctypes.c_void_p()
        _lib.check(lib.pat_srv_create(int(hbm_budget), ctypes.byref(cfg), ctypes.byref(h)),
                   "pat_srv_create")
        self._h = h
        self._keep = {}
        self.shapes = []

    def register(self, speed, dx, origin, sensors, dt, n_samples, mask=None, weights=None,
                 flags=0, compact=False):
        speed = np.ascontiguousarray(speed, dtype=np.float32)
        g = _lib.make_grid(speed.shape, dx, origin)
        sensors = np.ascontiguousarray(sensors, dtype=np.float64)
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
        if compact:
            flags |= _lib.PAT_FLAG_COMPACT_OUT
        sid = ctypes.c_int()
        _lib.check(self._lib.pat_srv_register(
            self._h, speed.ctypes.data, ctypes.byref(g), sensors.ctypes.data, sensors.shape[0],
            None if m is None else m.ctypes.data, None if w is None else w.ctypes.data, float(dt),
            int(n_samples), int(flags), ctypes.byref(sid)), "pat_srv_register")
        npix = int(np.count_nonzero(m)) if m is not None else speed.size
        self.shapes.append((npix,) if compact else tuple(speed.shape))
        return sid.value

    def submit(self, subject, signals, out, dtype="f32", scales=None):
        sig = np.ascontiguousarray(signals)
        sc = None if scales is None else np.ascontiguousarray(scales, dtype=np.float32)
        if out.dtype != np.float32 or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a contiguous float32 array")
        t = ctypes.c_uint64()
        _lib.check(self._lib.pat_srv_submit(self._h, int(subject), sig.ctypes.data, DTYPES[dtype],
                                            None if sc is None else sc.ctypes.data,
                                            out.ctypes.data, ctypes.byref(t)), "pat_srv_submit")
        self._keep[t.value] = (sig, sc, out)
        return t.value

    def poll(self, ticket, timeout_us=0):
        """(status, latency_s); status PAT_PENDING (7) while in flight."""
        lat = ctypes.c_double()
        st = self._lib.pat_srv_poll(self._h, int(ticket), int(timeout_us), ctypes.byref(lat))
        if st != _lib.PAT_PENDING:
            self._keep.pop(ticket, None)
        return st, lat.value

    def wait(self, ticket, timeout_s=30.0):
        st, lat = self.poll(ticket, int(timeout_s * 1e6))
        _lib.check(st, "pat_srv_poll")
        return lat

    def set_budget(self, hbm_budget):
        """pat_srv_set_budget: new HBM budget (bytes); idle subjects beyond it are
        evicted to their host copies, least recently used first."""
        _lib.check(self._lib.pat_srv_set_budget(self._h, int(hbm_budget)), "pat_srv_set_budget")

    def stats(self):
        st = _lib.PatSrvStats()
        _lib.check(self._lib.pat_srv_stats(self._h, ctypes.byref(st)), "pat_srv_stats")
        return {k: getattr(st, k) for k, _ in _lib.PatSrvStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pat_srv_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reconstruct_multi(bps, signals, outs, scales=None, stream=None):
    """One-shot multi-instance launch (no tuning, no graph)."""
    lib = _lib.load()
    code = _dtype_code(signals[0])
    hs = _ptr_array([b.handle.value for b in bps])
    fr = (ctypes.c_int * len(bps))(*[int(s.shape[0]) for s in signals])
    sc = None if scales is None else _tensor_ptrs(scales)
    _lib.check(lib.pat_bp_reconstruct_multi(hs, _tensor_ptrs(signals), code, sc, fr,
                                            _tensor_ptrs(outs), len(bps), _stream_ptr(stream)),
               "pat_bp_reconstruct_multi")
    return outs


def fmm_host(speed, dx, origin, src, order=1):
    """The library's host fast marching (FP64) from one point source; order 1
    (first-order upwind) or 2 (the second-order stencil of Sec. II-B)."""
    lib = _lib.load()
    speed = np.ascontiguousarray(speed, dtype=np.float32)
    g = _lib.make_grid(speed.shape, dx, origin)
    src = np.ascontiguousarray(np.resize(np.asarray(src, dtype=np.float64), 3))
    T = np.empty(speed.shape, dtype=np.float64)
    _lib.check(lib.pat_fmm_host(speed.ctypes.data, ctypes.byref(g), src.ctypes.data, int(order),
                                T.ctypes.data), "pat_fmm_host")
    return T


def fmm_gpu(speed, dx, origin, sources):
    """First-order arrival times of point sources ([n, 3] or one xyz) solved on
    the current CUDA device; equal to fmm_host(order=1) of each source.
    Returns [n, *speed.shape] FP64 (or speed.shape for one source)."""
    lib = _lib.load()
    speed = np.ascontiguousarray(speed, dtype=np.float32)
    g = _lib.make_grid(speed.shape, dx, origin)
    src = np.asarray(sources, dtype=np.float64)
    one = src.ndim == 1
    src = np.atleast_2d(src)
    src = np.ascontiguousarray(np.concatenate(
        [src, np.zeros((src.shape[0], 3 - src.shape[1]))], axis=1) if src.shape[1] < 3 else src)
    T = np.empty((src.shape[0],) + speed.shape, dtype=np.float64)
    _lib.check(lib.pat_fmm_gpu(speed.ctypes.data, ctypes.byref(g), src.ctypes.data, src.shape[0],
                               T.ctypes.data), "pat_fmm_gpu")
    return T[0] if one else T


def probe_l2_to_smem():
    """pat_probe_l2_to_smem: aggregate L2 -> shared-memory bulk-copy bandwidth
    of the current device in GB/s (a roofline of the staged gather)."""
    lib = _lib.load()
    v = ctypes.c_double()
    _lib.check(lib.pat_probe_l2_to_smem(ctypes.byref(v)), "pat_probe_l2_to_smem")
    return v.value


def table_host(speed, dx, origin, sensors, dt, n_samples, mask=None, flags=0):
    """The table pat_bp_create would upload, returned to the host: (info, u,
    base, slot).  Built by the host march, or by the GPU solver with
    flags |= PAT_FLAG_GPU_TABLE."""
    lib = _lib.load()
    speed = np.ascontiguousarray(speed, dtype=np.float32)
    g = _lib.make_grid(speed.shape, dx, origin)
    sensors = np.ascontiguousarray(sensors, dtype=np.float64)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    inf = _lib.PatInfo()
    args = (speed.ctypes.data, ctypes.byref(g), sensors.ctypes.data, sensors.shape[0],
            None if m is None else m.ctypes.data, float(dt), int(n_samples), int(flags),
            ctypes.byref(inf))
    _lib.check(lib.pat_table_host(*args, None, None, None), "pat_table_host")
    nt, ns, P = inf.n_tiles, sensors.shape[0], inf.tile_pix
    u = np.empty((nt, ns, P), dtype=np.float32)
    b = np.empty((nt, ns), dtype=np.int32)
    s = np.empty(nt * P, dtype=np.int32)
    _lib.check(lib.pat_table_host(*args, u.ctypes.data, b.ctypes.data, s.ctypes.data),
               "pat_table_host")
    info = {k: getattr(inf, k) for k, _ in _lib.PatInfo._fields_}
    return info, u, b, s


def wait_timeout_probe(timeout_ns=1_000_000):
    """Run the bounded-wait probe kernel; returns the library status code."""
    return _lib.load().pat_test_wait_timeout(int(timeout_ns))
