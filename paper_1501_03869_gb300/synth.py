"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds none of the reconstruction's arithmetic (no fast marching,
no back projection).  It builds speed maps, sensor layouts, masks, absorber
phantoms and sensor signals, and is shared by the CUDA path, the oracle tests
and the benchmark.

The paper's own data (a CT-derived macaque skull, Sec. III, and k-Wave
simulations, Sec. II-A) are not available; the stand-ins keep their shapes:
a ring of 512 sensors around a skull of 2200-3000 m/s with brain at
1540 m/s and water around it (Sec. I, Sec. III), 21 323 reconstructed pixels
(Sec. III, 0.39 mm case).

Forward model for the signals (a stand-in for the k-space simulation): every
absorber is a small disc/ball of radius R and initial pressure A; its signal at
a sensor is the N-shaped pulse of a uniform sphere in 3-D,

    p(t) = A (T0 - t) / (2 T0)       for |t - T0| <= R / c_a,

centred on the straight-ray travel time T0 = integral of 1/c along the segment
from the absorber to the sensor (slowness sampled bilinearly), with c_a the
local speed.  For this pulse 2p - 2t dp/dt = A on its support, so a
reconstruction has the scale of the initial pressure.  Noise is white Gaussian
with sigma a fraction of the clean peak.  Straight rays ignore refraction, so
the data is not produced by the method under test.

Seeds: every random draw comes from ``np.random.default_rng([cfg, inst, frame,
purpose])`` so configs, instances, frames and purposes never share a stream.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C_WATER = 1500.0
C_BRAIN = 1540.0  # Sec. III
C_SKULL_LO, C_SKULL_HI = 2200.0, 3000.0  # Sec. I


def rng_for(cfg: int, inst: int = 0, frame: int = 0, purpose: int = 0) -> np.random.Generator:
    return np.random.default_rng([cfg, inst, frame, purpose])


@dataclasses.dataclass
class Workload:
    """One speed map with its sensors, mask and F frames of signals."""
    name: str
    speed: np.ndarray            # float32, shape ([nz,] ny, nx), m/s at nodes
    dx: float                    # node spacing (m)
    origin: np.ndarray           # coordinates of node 0 (m), (x, y[, z])
    sensors: np.ndarray          # float64 [ns, 3] (m); z = 0 in 2-D
    mask: np.ndarray             # uint8, grid shape; nonzero = reconstruct
    dt: float                    # sample interval (s)
    nt: int                      # samples per signal
    signals: np.ndarray          # float32 [F, ns, nt]
    p0: np.ndarray               # float32 [F, grid] initial-pressure phantom

    @property
    def ndim(self) -> int:
        return self.speed.ndim

    @property
    def n_sensors(self) -> int:
        return self.sensors.shape[0]

    @property
    def n_frames(self) -> int:
        return self.signals.shape[0]

    @property
    def n_pix(self) -> int:
        return int(np.count_nonzero(self.mask))


# ------------------------------------------------------------------ grids --
def centred_origin(shape, dx):
    """Origin (x first) of a grid whose centre sits at 0."""
    return np.array([-(n - 1) / 2.0 * dx for n in shape[::-1]], dtype=np.float64)


def node_radius_px(shape, centre_px=None):
    """Distance (in node units) of every node from centre_px (x first)."""
    axes = [np.arange(n, dtype=np.float64) for n in shape]
    mesh = np.meshgrid(*axes, indexing="ij")  # mesh[0] is the slowest axis
    if centre_px is None:
        centre_px = [(n - 1) / 2.0 for n in shape[::-1]]
    r2 = np.zeros(shape, dtype=np.float64)
    for d in range(len(shape)):
        c = centre_px[d]
        r2 += (mesh[len(shape) - 1 - d] - c) ** 2
    return np.sqrt(r2)


def ring_sensors(n, radius):
    """n sensors on a circle of radius (m) around 0; sensor s at angle 2 pi s/n from +x."""
    a = 2.0 * np.pi * np.arange(n) / n
    return np.stack([radius * np.cos(a), radius * np.sin(a), np.zeros(n)], axis=1)


def fibonacci_hemisphere(n, radius, centre):
    """n near-uniform points on the upper hemisphere (z >= centre z)."""
    k = np.arange(n) + 0.5
    z = k / n                                  # cos(polar angle) uniform in (0, 1]
    phi = np.pi * (3.0 - math.sqrt(5.0)) * np.arange(n)
    rxy = np.sqrt(1.0 - z * z)
    pts = np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=1) * radius
    return pts + np.asarray(centre, dtype=np.float64)[None, :]


def smooth_field(shape, sigma_px, rng):
    """Gaussian-smoothed white noise mapped to [0, 1] (periodic FFT filter)."""
    noise = rng.standard_normal(shape)
    freqs = np.meshgrid(*[np.fft.fftfreq(n) for n in shape], indexing="ij")
    k2 = sum(f * f for f in freqs)
    filt = np.exp(-2.0 * (np.pi ** 2) * (sigma_px ** 2) * k2)
    f = np.real(np.fft.ifftn(np.fft.fftn(noise) * filt))
    lo, hi = f.min(), f.max()
    return (f - lo) / (hi - lo) if hi > lo else np.zeros(shape)


def fourier_curve(theta, n_modes, rng):
    """Seeded low-order Fourier series in [-1, 1]."""
    acc = np.zeros_like(theta)
    for m in range(1, n_modes + 1):
        acc += rng.uniform(-1, 1) / m * np.cos(m * theta + rng.uniform(0, 2 * np.pi))
    peak = np.max(np.abs(acc)) if np.max(np.abs(acc)) > 0 else 1.0
    return acc / peak


def skull_ring_2d(shape, r_in_px, thick_px, rng, r_in_var=0.0, thick_var=0.0,
                  skull_speed=None, smooth_px=6.0):
    """Water / skull annulus / brain speed map on a 2-D grid centred on 0.

    r_in(theta) = r_in_px + r_in_var * g1(theta); thickness = thick_px +
    thick_var * g2(theta) with g1, g2 seeded Fourier curves in [-1, 1].  The
    skull speed is a fixed value or, if None, a smoothed random field mapped to
    [2200, 3000] m/s.
    """
    ny, nx = shape
    yy, xx = np.meshgrid(np.arange(ny) - (ny - 1) / 2.0, np.arange(nx) - (nx - 1) / 2.0,
                         indexing="ij")
    r = np.hypot(xx, yy)
    th = np.arctan2(yy, xx)
    rin = r_in_px + (r_in_var * fourier_curve(th, 4, rng) if r_in_var else 0.0)
    thick = thick_px + (thick_var * fourier_curve(th, 3, rng) if thick_var else 0.0)
    speed = np.full(shape, C_WATER, dtype=np.float64)
    speed[r < rin] = C_BRAIN
    skull = (r >= rin) & (r < rin + thick)
    if skull_speed is None:
        field = smooth_field(shape, smooth_px, rng)
        vals = field[skull]
        lo, hi = vals.min(), vals.max()
        vals = (vals - lo) / (hi - lo) if hi > lo else np.zeros_like(vals)
        speed[skull] = C_SKULL_LO + (C_SKULL_HI - C_SKULL_LO) * vals
    else:
        speed[skull] = skull_speed
    return speed.astype(np.float32)


def speed_error(speed, rng, frac=0.017, region=None):
    """The speed-of-sound error of Sec. III's robustness study: uncorrelated
    Gaussian noise whose mean and standard deviation are both frac times the
    map's maximum, added independently at every node of `region` (default: the
    skull, i.e. the nodes whose speed is neither water's nor brain's)."""
    speed = np.asarray(speed, dtype=np.float64)
    if region is None:
        region = (np.abs(speed - C_WATER) > 1e-3) & (np.abs(speed - C_BRAIN) > 1e-3)
    top = float(speed.max())
    out = speed.copy()
    n = int(np.count_nonzero(region))
    out[region] += rng.normal(frac * top, frac * top, n)
    return out.astype(np.float32)


def nearest_nodes_mask(shape, count):
    """The `count` nodes nearest the grid centre; equal radii ordered by linear index."""
    r = node_radius_px(shape).ravel()
    order = np.lexsort((np.arange(r.size), r))
    mask = np.zeros(r.size, dtype=np.uint8)
    mask[order[:count]] = 1
    return mask.reshape(shape)


# ------------------------------------------------------------- forward model --
def _interp_slowness(slow, dx, origin, pts):
    """Multilinear interpolation of the slowness grid at pts [..., ndim] (x first)."""
    nd = slow.ndim
    g = (pts - origin[:nd]) / dx
    shape_x = slow.shape[::-1]
    i0 = []
    fr = []
    for d in range(nd):
        x = np.clip(g[..., d], 0.0, shape_x[d] - 1.000001)
        i = np.floor(x).astype(np.int64)
        i0.append(i)
        fr.append(x - i)
    flat = slow.ravel()
    strides = [1]
    for d in range(1, nd):
        strides.append(strides[-1] * shape_x[d - 1])
    out = np.zeros(pts.shape[:-1])
    for corner in range(1 << nd):
        w = np.ones(pts.shape[:-1])
        idx = np.zeros(pts.shape[:-1], dtype=np.int64)
        for d in range(nd):
            bit = (corner >> d) & 1
            w = w * (fr[d] if bit else (1.0 - fr[d]))
            idx += (i0[d] + bit) * strides[d]
        out += w * flat[idx]
    return out


def straight_ray_times(speed, dx, origin, starts, ends, step_frac=1.0, chunk=2048):
    """Line integral of 1/c along straight segments (midpoint rule, step dx*step_frac)."""
    slow = 1.0 / np.asarray(speed, dtype=np.float64)
    nd = slow.ndim
    starts = np.asarray(starts, dtype=np.float64)[:, :nd]
    ends = np.asarray(ends, dtype=np.float64)[:, :nd]
    out = np.empty(starts.shape[0])
    for c0 in range(0, starts.shape[0], chunk):
        a = starts[c0:c0 + chunk]
        b = ends[c0:c0 + chunk]
        seg = b - a
        length = np.sqrt(np.sum(seg * seg, axis=1))
        k = max(1, int(math.ceil(length.max() / (dx * step_frac))))
        t = (np.arange(k) + 0.5) / k
        pts = a[:, None, :] + t[None, :, None] * seg[:, None, :]
        s = _interp_slowness(slow, dx, origin, pts)
        out[c0:c0 + chunk] = s.mean(axis=1) * length
    return out


def local_speed(speed, dx, origin, pts):
    return 1.0 / _interp_slowness(1.0 / np.asarray(speed, dtype=np.float64), dx, origin,
                                  np.asarray(pts, dtype=np.float64)[:, :speed.ndim])


def straight_ray_arrivals(speed, dx, origin, centres, sensors):
    """Arrival times [na, ns] from every absorber centre to every sensor along
    straight rays (the default forward model; ignores refraction)."""
    centres = np.asarray(centres, dtype=np.float64)
    sensors = np.asarray(sensors, dtype=np.float64)
    na, ns = centres.shape[0], sensors.shape[0]
    st = np.repeat(centres, ns, axis=0)
    en = np.tile(sensors, (na, 1))
    return straight_ray_times(speed, dx, origin, st, en).reshape(na, ns)


def render_signals(speed, dx, origin, sensors, centres, radii, amps, dt, nt,
                   noise_frac, rng, arrivals=None):
    """Sum of spherical N-pulses (see module docstring) plus white noise.

    centres [na, 3] (m), radii [na] (m), amps [na].  `arrivals(speed, dx,
    origin, centres, sensors) -> [na, ns]` gives the pulse arrival times; the
    default is :func:`straight_ray_arrivals`.
    """
    arrivals = arrivals or straight_ray_arrivals
    centres = np.asarray(centres, dtype=np.float64)
    T0 = arrivals(speed, dx, origin, centres, sensors)
    ca = local_speed(speed, dx, origin, centres)
    return _pulses(T0, ca, radii, amps, dt, nt, noise_frac, rng)


def _pulses(T0, ca, radii, amps, dt, nt, noise_frac, rng, chunk=256):
    """Render the N-pulses of T0 [na, ns] into p [ns, nt] and add noise."""
    T0 = np.asarray(T0, dtype=np.float64)
    na, ns = T0.shape
    tau = (np.asarray(radii, dtype=np.float64) / np.asarray(ca, dtype=np.float64))[:, None]
    k0 = np.maximum(0, np.ceil((T0 - tau) / dt)).astype(np.int64)
    k1 = np.minimum(nt - 1, np.floor((T0 + tau) / dt)).astype(np.int64)
    span = int(max(0, (k1 - k0 + 1).max())) if na else 0
    p = np.zeros(ns * nt, dtype=np.float64)
    amps = np.asarray(amps, dtype=np.float64)
    off = np.arange(span)
    for a0 in range(0, na, chunk):
        sl = slice(a0, a0 + chunk)
        k = k0[sl][..., None] + off[None, None, :]
        valid = k <= k1[sl][..., None]
        t0 = T0[sl][..., None]
        val = amps[sl][:, None, None] * (t0 - k * dt) / (2.0 * t0)
        idx = np.arange(ns)[None, :, None] * nt + k
        p += np.bincount(idx[valid], weights=val[valid], minlength=ns * nt)
    p = p.reshape(ns, nt)
    peak = np.max(np.abs(p)) if p.size else 0.0
    if noise_frac > 0 and peak > 0:
        p += rng.standard_normal(p.shape) * noise_frac * peak
    return p.astype(np.float32)


def _render_lines(speed, dx, origin, sensors, segs, amps, dt, nt, noise_frac, rng,
                  disc_px=1.0, spacing_px=0.5, anchor_px=2.0, arrivals=None):
    """Line absorbers: discs of radius disc_px every spacing_px along each segment.

    Travel times are traced at anchors every anchor_px along each segment and
    interpolated linearly in between (the straight-ray time is smooth along a
    segment)."""
    arrivals = arrivals or straight_ray_arrivals
    sensors = np.asarray(sensors, dtype=np.float64)
    all_T0, all_ca, all_r, all_a = [], [], [], []
    for (a, b), amp in zip(segs, amps):
        a = np.asarray(a, dtype=np.float64)
        b = np.asarray(b, dtype=np.float64)
        L = np.linalg.norm(b - a) / dx
        nd_disc = max(2, int(math.floor(L / spacing_px)) + 1)
        n_anchor = max(2, int(math.ceil(L / anchor_px)) + 1)
        ta = np.linspace(0.0, 1.0, n_anchor)
        anchors = a[None, :] + ta[:, None] * (b - a)[None, :]
        Ta = arrivals(speed, dx, origin, anchors, sensors)
        td = np.linspace(0.0, 1.0, nd_disc)
        pos = td * (n_anchor - 1)
        i0 = np.minimum(np.floor(pos).astype(int), n_anchor - 2)
        fr = pos - i0
        Td = Ta[i0] * (1.0 - fr)[:, None] + Ta[i0 + 1] * fr[:, None]
        discs = a[None, :] + td[:, None] * (b - a)[None, :]
        all_T0.append(Td)
        all_ca.append(local_speed(speed, dx, origin, discs))
        all_r.append(np.full(nd_disc, disc_px * dx))
        all_a.append(np.full(nd_disc, amp))
    return _pulses(np.concatenate(all_T0), np.concatenate(all_ca), np.concatenate(all_r),
                   np.concatenate(all_a), dt, nt, noise_frac, rng)


def phantom_discs(shape, dx, origin, centres, radii, amps):
    """Dense initial-pressure image of disc/ball absorbers (max of overlapping amps)."""
    axes = [origin[d] + dx * np.arange(n) for d, n in enumerate(shape[::-1])]
    mesh = np.meshgrid(*axes[::-1], indexing="ij")  # slowest axis first
    nd = len(shape)
    img = np.zeros(shape, dtype=np.float64)
    for c, r, a in zip(centres, radii, amps):
        d2 = np.zeros(shape)
        for d in range(nd):
            d2 += (mesh[nd - 1 - d] - c[d]) ** 2
        img = np.where(d2 <= r * r, np.maximum(img, a), img)
    return img.astype(np.float32)


def _random_points_in_disc(rng, n, radius):
    r = radius * np.sqrt(rng.uniform(0, 1, n))
    a = rng.uniform(0, 2 * np.pi, n)
    return np.stack([r * np.cos(a), r * np.sin(a), np.zeros(n)], axis=1)


# ---------------------------------------------------------------- configs --
def config1(n_frames=1, inst=0, cfg_id=1, noise=0.01, arrivals=None):
    """128x128, dx 0.2 mm; water 1500, skull annulus [44, 50) px at 2800 m/s,
    brain 1540; 64 sensors at r = 60 px; 1024 samples at 25 ns; 5 disc
    absorbers (radius 1-3 px, amplitude 0.5-1) inside r < 40 px; mask r < 44 px."""
    shape, dx = (128, 128), 0.2e-3
    origin = centred_origin(shape, dx)
    speed = skull_ring_2d(shape, 44.0, 6.0, rng_for(cfg_id, inst, 0, 1), skull_speed=2800.0)
    sensors = ring_sensors(64, 60.0 * dx)
    mask = (node_radius_px(shape) < 44.0).astype(np.uint8)
    dt, nt = 25e-9, 1024
    sig, p0 = [], []
    for f in range(n_frames):
        rng = rng_for(cfg_id, inst, f, 2)
        c = _random_points_in_disc(rng, 5, 40.0 * dx)
        r = rng.uniform(1.0, 3.0, 5) * dx
        a = rng.uniform(0.5, 1.0, 5)
        sig.append(render_signals(speed, dx, origin, sensors, c, r, a, dt, nt, noise, rng,
                                  arrivals))
        p0.append(phantom_discs(shape, dx, origin, c, r, a))
    return Workload("c1", speed, dx, origin, sensors, mask, dt, nt, np.stack(sig), np.stack(p0))


def config2(n_frames=1, inst=0, noise=0.01, n_lines=20, arrivals=None, n_sensors=512,
            nt=2048, dt=12.5e-9):
    """Paper-shaped frame: 256x256, dx 0.1 mm, skull ring (inner radius 86 +- 2 px,
    thickness 25 +- 5 px, speed field 2200-3000 m/s), 512 sensors at r = 120 px,
    2048 samples at 12.5 ns, the 21 323 nodes nearest the centre, 20 line
    absorbers of 10-60 px rendered as 1-px discs every 0.5 px.  Tests may ask
    for more sensors on the same ring and a finer sampling of the record."""
    shape, dx = (256, 256), 0.1e-3
    origin = centred_origin(shape, dx)
    speed = skull_ring_2d(shape, 86.0, 25.0, rng_for(2, inst, 0, 1), r_in_var=2.0,
                          thick_var=5.0, skull_speed=None)
    sensors = ring_sensors(n_sensors, 120.0 * dx)
    mask = nearest_nodes_mask(shape, 21323)
    sig, p0 = [], []
    for f in range(n_frames):
        rng = rng_for(2, inst, f, 2)
        segs, amps = [], []
        while len(segs) < n_lines:
            a = _random_points_in_disc(rng, 1, 80.0 * dx)[0]
            L = rng.uniform(10.0, 60.0) * dx
            th = rng.uniform(0, 2 * np.pi)
            b = a + L * np.array([math.cos(th), math.sin(th), 0.0])
            if math.hypot(b[0], b[1]) < 80.0 * dx:
                segs.append((a, b))
                amps.append(rng.uniform(0.5, 1.0))
        sig.append(_render_lines(speed, dx, origin, sensors, segs, amps, dt, nt, noise, rng,
                                 arrivals=arrivals))
        centres, radii, aa = [], [], []
        for (a, b), amp in zip(segs, amps):
            k = int(math.floor(np.linalg.norm(b - a) / dx / 0.5)) + 1
            for t in np.linspace(0, 1, max(2, k)):
                centres.append(a + t * (b - a))
                radii.append(dx)
                aa.append(amp)
        p0.append(phantom_discs(shape, dx, origin, centres, radii, aa))
    return Workload("c2", speed, dx, origin, sensors, mask, dt, nt, np.stack(sig), np.stack(p0))


def quantise(signals, dtype):
    """Per-(frame, sensor) scale sigma = max|p| and 16-bit codes of p / sigma.

    Returns (codes as a numpy uint16 view, scales float32 [F, ns], dequantised
    float64 signals).  dtype is 'bf16' or 'f16'.  Rounding is to nearest even.
    """
    sig = np.asarray(signals, dtype=np.float32)
    sc = np.max(np.abs(sig), axis=-1).astype(np.float32)
    sc[sc == 0] = 1.0
    x = (sig / sc[..., None]).astype(np.float32)
    if dtype == "f16":
        h = x.astype(np.float16)
        codes = h.view(np.uint16)
        deq = h.astype(np.float64) * sc[..., None].astype(np.float64)
    elif dtype == "bf16":
        u = x.view(np.uint32).astype(np.uint64)
        lsb = (u >> 16) & 1
        r = ((u + 0x7FFF + lsb) >> 16).astype(np.uint16)
        codes = r
        back = (r.astype(np.uint32) << 16).view(np.float32)
        deq = back.astype(np.float64) * sc[..., None].astype(np.float64)
    else:
        raise ValueError(dtype)
    return codes, sc, deq


def config3(n_frames=64, arrivals=None):
    """Config-1 geometry with 64 frames of different absorbers (precision form)."""
    return config1(n_frames=n_frames, cfg_id=3, arrivals=arrivals)


def config4_instance(inst, noise=0.01, arrivals=None, n_frames=None):
    """One uneven instance: N ~ U{96..384}, dx ~ U[0.1, 0.2] mm, ns ~ U{128..1024},
    nt ~ U{1024..4096}, F ~ U{1..16}; skull like config 2 scaled to N, ring at
    0.47 N, dt such that nt dt >= 1.5 d / c0; mask r < 0.32 N; 5 disc absorbers
    shared by the frames, amplitudes and noise drawn per frame."""
    rng = rng_for(4, inst, 0, 0)
    N = int(rng.integers(96, 385))
    dx = float(rng.uniform(0.1e-3, 0.2e-3))
    ns = int(rng.integers(128, 1025))
    nt = int(rng.integers(1024, 4097))
    F = int(rng.integers(1, 17))
    shape = (N, N)
    origin = centred_origin(shape, dx)
    s = N / 256.0
    speed = skull_ring_2d(shape, 86.0 * s, 25.0 * s, rng_for(4, inst, 0, 1), r_in_var=2.0 * s,
                          thick_var=5.0 * s, skull_speed=None, smooth_px=6.0 * s)
    rr = 0.47 * N
    sensors = ring_sensors(ns, rr * dx)
    d = 2 * rr * dx
    dt = 1.5 * d / C_WATER / nt * 1.02
    mask = (node_radius_px(shape) < 0.32 * N).astype(np.uint8)
    if n_frames is not None:
        F = n_frames
    # the frames of one instance share the absorber positions (one set of
    # arrival times) and differ in amplitudes and noise
    r2 = rng_for(4, inst, 0, 2)
    c = _random_points_in_disc(r2, 5, 0.3 * N * dx)
    r = r2.uniform(1.0, 3.0, 5) * dx
    T0 = (arrivals or straight_ray_arrivals)(speed, dx, origin, c, sensors)
    ca = local_speed(speed, dx, origin, c)
    sig, p0 = [], []
    for f in range(F):
        rf = rng_for(4, inst, f, 3)
        a = rf.uniform(0.5, 1.0, 5)
        sig.append(_pulses(T0, ca, r, a, dt, nt, noise, rf))
        p0.append(phantom_discs(shape, dx, origin, c, r, a))
    return Workload(f"c4_{inst}", speed, dx, origin, sensors, mask, dt, nt, np.stack(sig),
                    np.stack(p0))


def config4_shapes(n_inst=32):
    """(N, dx, ns, nt, F) of the uneven instances without rendering signals."""
    out = []
    for inst in range(n_inst):
        rng = rng_for(4, inst, 0, 0)
        out.append((int(rng.integers(96, 385)), float(rng.uniform(0.1e-3, 0.2e-3)),
                    int(rng.integers(128, 1025)), int(rng.integers(1024, 4097)),
                    int(rng.integers(1, 17))))
    return out


def shell_skull_3d(shape, dx, centre_px, r_in, thick_lo, thick_hi, rng, smooth_px=5.0):
    """3-D water / spherical skull shell / brain map; shell thickness varies
    smoothly in [thick_lo, thick_hi] with direction, speed field 2200-3000."""
    nz, ny, nx = shape
    r = node_radius_px(shape, centre_px)
    zz, yy, xx = np.meshgrid(np.arange(nz) - centre_px[2], np.arange(ny) - centre_px[1],
                             np.arange(nx) - centre_px[0], indexing="ij")
    th = np.arctan2(yy, xx)
    ph = np.arctan2(np.hypot(xx, yy), zz)
    g = fourier_curve(th, 3, rng) * 0.5 + 0.5 * np.cos(ph * rng.uniform(1, 3) + rng.uniform(0, 6))
    g = (g - g.min()) / (g.max() - g.min() + 1e-30)
    thick = thick_lo + (thick_hi - thick_lo) * g
    speed = np.full(shape, C_WATER, dtype=np.float64)
    speed[r < r_in] = C_BRAIN
    shell = (r >= r_in) & (r < r_in + thick)
    field = smooth_field(shape, smooth_px, rng)
    v = field[shell]
    v = (v - v.min()) / (v.max() - v.min() + 1e-30)
    speed[shell] = C_SKULL_LO + (C_SKULL_HI - C_SKULL_LO) * v
    return speed.astype(np.float32)


def config5_subject(subject, n_frames=1, n_sensors=1024, noise=0.01, shape=(96, 160, 160),
                    dx=0.25e-3, nt=2048, dt=20e-9, arrivals=None):
    """3-D serving subject: 160x160x96 at 0.25 mm, 1024 sensors on a Fibonacci
    hemisphere of radius 76 voxels centred at (79.5, 79.5, 8), spherical shell
    skull (inner radius 56, 5-8 voxels thick, 2200-3000 m/s), 2048 samples at
    20 ns, mask = all voxels.  A smaller `shape` scales every length."""
    s = shape[2] / 160.0
    origin = np.zeros(3)
    centre_px = (79.5 * s, 79.5 * s, 8.0 * s)
    speed = shell_skull_3d(shape, dx, centre_px, 56.0 * s, 5.0 * s, 8.0 * s,
                           rng_for(5, subject, 0, 1), smooth_px=5.0 * s)
    centre_m = np.array(centre_px) * dx
    sensors = fibonacci_hemisphere(n_sensors, 76.0 * s * dx, centre_m)
    mask = np.ones(shape, dtype=np.uint8)
    sig, p0 = [], []
    for f in range(n_frames):
        rng = rng_for(5, subject, f, 2)
        k = 8
        u = rng.standard_normal((k, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        u[:, 2] = np.abs(u[:, 2])
        c = centre_m[None, :] + u * (rng.uniform(0, 45.0 * s, k) * dx)[:, None]
        r = rng.uniform(1.0, 3.0, k) * dx
        a = rng.uniform(0.5, 1.0, k)
        sig.append(render_signals(speed, dx, origin, sensors, c, r, a, dt, nt, noise, rng,
                                  arrivals))
        p0.append(phantom_discs(shape, dx, origin, c, r, a))
    return Workload(f"c5_{subject}", speed, dx, origin, sensors, mask, dt, nt, np.stack(sig),
                    np.stack(p0))
