"""FP64 CPU oracle of the FMM-corrected back projection (Wang & Jing).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark may use this package; the product library never does.
It shares no code with the CUDA library.

The arithmetic lives in ``oracle.c`` (plain C, double precision); this module
only compiles it with gcc on first use and marshals numpy arrays:

* :func:`fmm_point`, :func:`fmm_sources` -- Sec. II-B, first-order Godunov fast
  marching (or, with ``order=2``, the printed second-order stencil) from a
  point source (corners of the enclosing cell accepted with exact distance
  times local slowness) or from an arbitrary accepted set.
* :func:`travel_table` -- one fast-marching run per sensor (Sec. II-B: each
  sensor is used as the source since ray paths are reversible), values read
  at the requested pixels.
* :func:`constant_table` -- the conventional back projection's time of flight
  for a constant sound speed (Sec. II-C; Sec. III compares at 1560 m/s):
  straight-line distance over c0.
* :func:`solid_angle_weights` -- the weight of the exact back projection that
  Eq. (BP) approximates (Sec. II-C): the share of the total solid angle (2-D:
  plane angle) that a sensor's element subtends at a pixel, written out in
  numpy from its definition.
* :func:`preprocess` -- Sec. II-C, Eq. (BP) integrand b = 2p - 2t dp/dt.
* :func:`sample` / :func:`bp` -- Sec. II-C, Eq. (BP), P_j = sum_s w_s b_s(T_sj/dt)
  with linear interpolation, zero after the last sample; the weights may be
  per sensor or per (sensor, pixel) pair.
* :func:`reconstruct` -- the whole chain on a grid with a mask, dense output.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_fmm_sources.argtypes = [ctypes.c_int, _i64p, ctypes.c_double, _dp,
                                               _i64p, _dp, ctypes.c_int64, _dp, _i64p, _i64p,
                                               ctypes.c_int]
            lib.oracle_fmm_point.argtypes = [ctypes.c_int, _i64p, ctypes.c_double, _dp, _dp,
                                             _dp, _dp, _i64p, _i64p, ctypes.c_int]
            lib.oracle_preprocess.argtypes = [_dp, ctypes.c_int64, ctypes.c_double, _dp]
            lib.oracle_sample.argtypes = [_dp, ctypes.c_int64, ctypes.c_double]
            lib.oracle_sample.restype = ctypes.c_double
            lib.oracle_bp.argtypes = [ctypes.c_int64, ctypes.c_int64, _dp, ctypes.c_double,
                                      ctypes.c_int64, _dp, _dp, _dp]
            lib.oracle_bp_pairs.argtypes = [ctypes.c_int64, ctypes.c_int64, _dp, ctypes.c_double,
                                            ctypes.c_int64, _dp, _dp, _dp]
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_i64p)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def _shape_n(shape):
    """numpy shape ([nz,] ny, nx) -> n per axis with x first."""
    return np.ascontiguousarray(shape[::-1], dtype=np.int64)


def fmm_sources(speed, h, src_idx, src_T, return_order=False, order=1):
    """Fast marching from accepted nodes src_idx (linear indices) with values src_T;
    order 1 (first-order upwind) or 2 (the second-order stencil of Sec. II-B)."""
    lib = _load()
    speed = np.ascontiguousarray(speed, dtype=np.float64)
    n = _shape_n(speed.shape)
    src_idx = np.ascontiguousarray(src_idx, dtype=np.int64).ravel()
    src_T = np.ascontiguousarray(src_T, dtype=np.float64).ravel()
    T = np.empty(speed.shape, dtype=np.float64)
    pops = np.empty(speed.size, dtype=np.int64) if return_order else None
    npop = np.zeros(1, dtype=np.int64)
    rc = lib.oracle_fmm_sources(speed.ndim, _i(n), float(h), _d(speed), _i(src_idx), _d(src_T),
                                src_idx.size, _d(T), _i(pops) if return_order else None, _i(npop),
                                int(order))
    _check(rc, "fmm_sources")
    if return_order:
        return T, pops[: int(npop[0])]
    return T


def fmm_point(speed, h, origin, src, return_order=False, order=1):
    """Fast marching from a point source at src (metres, x first); order 1 or 2."""
    lib = _load()
    speed = np.ascontiguousarray(speed, dtype=np.float64)
    n = _shape_n(speed.shape)
    origin = np.ascontiguousarray(origin, dtype=np.float64)
    src = np.ascontiguousarray(src, dtype=np.float64)
    T = np.empty(speed.shape, dtype=np.float64)
    pops = np.empty(speed.size, dtype=np.int64) if return_order else None
    npop = np.zeros(1, dtype=np.int64)
    rc = lib.oracle_fmm_point(speed.ndim, _i(n), float(h), _d(origin), _d(speed), _d(src), _d(T),
                              _i(pops) if return_order else None, _i(npop), int(order))
    _check(rc, "fmm_point")
    if return_order:
        return T, pops[: int(npop[0])]
    return T


def travel_table(speed, h, origin, sensors, pix, order=1):
    """T[s, j]: arrival time from sensor s at pixel linear index pix[j]."""
    sensors = np.asarray(sensors, dtype=np.float64)
    pix = np.asarray(pix, dtype=np.int64)
    out = np.empty((sensors.shape[0], pix.size), dtype=np.float64)
    for s in range(sensors.shape[0]):
        out[s] = fmm_point(speed, h, origin, sensors[s], order=order).ravel()[pix]
    return out


def node_positions(shape, h, origin, pix):
    """[len(pix), 3] positions (m) of the nodes with linear indices pix (x
    fastest) of a grid of numpy shape ([nz,] ny, nx); z = 0 in 2-D."""
    idx = np.unravel_index(np.asarray(pix, dtype=np.int64), tuple(shape))[::-1]  # x, y[, z]
    pos = np.zeros((len(pix), 3), dtype=np.float64)
    for d, i in enumerate(idx):
        pos[:, d] = float(origin[d]) + i.astype(np.float64) * float(h)
    return pos


def constant_table(shape, h, origin, sensors, pix, c0):
    """T[s, j] = |x_j - r_s| / c0 for the nodes pix[j]; in 2-D only the
    sensors' x and y count (the image plane)."""
    sensors = np.asarray(sensors, dtype=np.float64)
    nd = len(shape)
    pos = node_positions(shape, h, origin, pix)[:, :nd]
    out = np.empty((sensors.shape[0], len(pix)), dtype=np.float64)
    for s in range(sensors.shape[0]):
        diff = pos - sensors[s, :nd]
        out[s] = np.sqrt(np.sum(diff * diff, axis=1)) / float(c0)
    return out


def solid_angle_weights(shape, h, origin, sensors, normals, elem, omega0, pix):
    """W[s, j] = elem_s (n_s . (x_j - r_s)) / |x_j - r_s|^d / omega0: the share
    of the solid angle omega0 (2-D: plane angle) that sensor s's element
    subtends at node pix[j] -- the weight of the exact back projection that
    Eq. (BP) approximates (Sec. II-C).  d = len(shape); n_s is the element's
    normal towards the imaged region (normalised here), elem_s its length
    (2-D) or area (3-D).  In 2-D only x and y of sensors and normals count."""
    sensors = np.asarray(sensors, dtype=np.float64)
    normals = np.asarray(normals, dtype=np.float64)
    elem = np.asarray(elem, dtype=np.float64)
    nd = len(shape)
    pos = node_positions(shape, h, origin, pix)[:, :nd]
    out = np.empty((sensors.shape[0], len(pix)), dtype=np.float64)
    for s in range(sensors.shape[0]):
        n = normals[s, :nd] / np.sqrt(np.sum(normals[s, :nd] ** 2))
        v = pos - sensors[s, :nd]
        r = np.sqrt(np.sum(v * v, axis=1))
        out[s] = elem[s] * (v @ n) / r ** nd / float(omega0)
    return out


def preprocess(p, dt):
    """b = 2p - 2t dp/dt along the last axis (Eq. (BP) integrand)."""
    lib = _load()
    p = np.ascontiguousarray(p, dtype=np.float64)
    nt = p.shape[-1]
    flat = p.reshape(-1, nt)
    b = np.empty_like(flat)
    for r in range(flat.shape[0]):
        _check(lib.oracle_preprocess(_d(flat[r]), nt, float(dt), _d(b[r])), "preprocess")
    return b.reshape(p.shape)


def sample(b, u):
    """Linear interpolation of one integrand row b at fractional sample u."""
    lib = _load()
    b = np.ascontiguousarray(b, dtype=np.float64)
    return lib.oracle_sample(_d(b), b.size, float(u))


def bp(T, p, dt, weights=None):
    """P_j = sum_s w_s b_s(T[s, j] / dt); T [ns, npix], p [ns, nt].  weights
    is None (1/ns), [ns] per sensor, or [ns, npix] per (sensor, pixel) pair
    (the exact back projection's solid-angle weights)."""
    lib = _load()
    T = np.ascontiguousarray(T, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    ns, npix = T.shape
    assert p.shape[0] == ns
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    out = np.empty(npix, dtype=np.float64)
    if w is not None and w.ndim == 2:
        assert w.shape == T.shape
        rc = lib.oracle_bp_pairs(ns, npix, _d(T), float(dt), p.shape[1], _d(p), _d(w), _d(out))
    else:
        rc = lib.oracle_bp(ns, npix, _d(T), float(dt), p.shape[1], _d(p),
                           _d(w) if w is not None else None, _d(out))
    _check(rc, "bp")
    return out


def reconstruct(speed, h, origin, sensors, p, dt, mask=None, weights=None, T=None, order=1):
    """Whole chain on a grid: fast-marching table, then back projection of each
    frame.  p is [ns, nt] or [F, ns, nt]; the output is dense ([F,] grid shape)
    with zeros outside the mask.  A precomputed table T[ns, npix] may be passed.
    """
    speed = np.asarray(speed)
    if mask is None:
        pix = np.arange(speed.size, dtype=np.int64)
    else:
        pix = np.flatnonzero(np.asarray(mask).ravel())
    if T is None:
        T = travel_table(speed, h, origin, sensors, pix, order=order)
    p = np.asarray(p, dtype=np.float64)
    single = p.ndim == 2
    frames = p[None] if single else p
    out = np.zeros((frames.shape[0], speed.size), dtype=np.float64)
    for f in range(frames.shape[0]):
        out[f, pix] = bp(T, frames[f], dt, weights)
    out = out.reshape((frames.shape[0],) + speed.shape)
    return out[0] if single else out
