"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
of the eikonal equation (Sec. II-B), the discrete upwind equation the scheme
solves, brute-force fixed-point iteration, invariants of fast marching,
closed forms of the Eq. (BP) integrand and of linear interpolation, and the
qualitative claim of Sec. III.
"""
import math
import os

import numpy as np
import pytest

import oracle
from helpers import fmm_arrivals
from paper_1501_03869_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_numbers():
    out = {}
    with open(os.path.join(GOLDEN, "paper_numbers.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                out[k] = float(v)
    return out


# ----------------------------------------------------------- P1 homogeneous --
@pytest.mark.parametrize("ndim", [2, 3])
def test_p1_homogeneous_error_small_and_falls_with_dx(ndim):
    """Homogeneous medium: T = |r - r_s| / c up to first-order error, which is
    one-sided (upwind schemes overestimate) and shrinks when dx halves."""
    c, L = 1500.0, 1.0e-3
    src = np.array([0.31e-4, -0.17e-4, 0.23e-4])[:ndim]
    errs = []
    for n in ([33, 65, 129] if ndim == 2 else [17, 33]):
        h = 2 * L / (n - 1)
        origin = np.full(ndim, -L)
        sp = np.full((n,) * ndim, c)
        T = oracle.fmm_point(sp, h, origin, src)
        axes = [origin[d] + h * np.arange(n) for d in range(ndim)]
        mesh = np.meshgrid(*axes[::-1], indexing="ij")
        dist = np.sqrt(sum((mesh[ndim - 1 - d] - src[d]) ** 2 for d in range(ndim)))
        err = T - dist / c
        assert err.min() > -1e-12 * T.max()
        assert err.max() < 2.5 * h / c
        errs.append(err.max())
    for a, b in zip(errs, errs[1:]):
        assert b < 0.8 * a


# ------------------------------------------------- discrete upwind equation --
def _axis_minima(T, h):
    nd = T.ndim
    mins = []
    for ax in range(nd):
        lo = np.full(T.shape, np.inf)
        hi = np.full(T.shape, np.inf)
        sl_a = [slice(None)] * nd
        sl_b = [slice(None)] * nd
        sl_a[ax] = slice(1, None)
        sl_b[ax] = slice(None, -1)
        lo[tuple(sl_a)] = T[tuple(sl_b)]
        hi[tuple(sl_b)] = T[tuple(sl_a)]
        mins.append(np.minimum(lo, hi))
    return mins


def _heterogeneous(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(1000.0, 3000.0, shape)


def _corner_sources(shape, h, origin, src):
    """Enclosing-cell corners with distance times local slowness."""
    nd = len(shape)
    nx = shape[::-1]
    cell = [min(int(math.floor((src[d] - origin[d]) / h)), nx[d] - 2) for d in range(nd)]
    return cell


@pytest.mark.parametrize("shape,seed", [((23, 19), 1), ((9, 8, 7), 2)])
def test_upwind_equation_residual(shape, seed):
    """Every non-source node satisfies sum_d max(T - a_d, 0)^2 = (h/c)^2 with
    a_d the smaller neighbour along axis d: the first-order Godunov scheme,
    written as its defining equation rather than its closed-form roots."""
    h = 1e-4
    sp = _heterogeneous(shape, seed)
    nd = len(shape)
    origin = np.zeros(nd)
    src = np.array([(s - 1) * h * 0.37 for s in shape[::-1]])
    T = oracle.fmm_point(sp, h, origin, src)
    cell = _corner_sources(shape, h, origin, src)
    is_src = np.zeros(shape, dtype=bool)
    for m in range(1 << nd):
        idx = tuple(cell[d] + ((m >> d) & 1) for d in range(nd))[::-1]
        is_src[idx] = True
    mins = _axis_minima(T, h)
    res = sum(np.maximum(T - m, 0.0) ** 2 for m in mins)
    target = (h / sp) ** 2
    rel = np.abs(res - target) / target
    assert np.all(np.isfinite(T))
    assert rel[~is_src].max() < 1e-9


def _local_solve_bisect(avals, hf):
    """Root of sum max(T - a, 0)^2 = hf^2 by bisection (no closed form)."""
    a = [x for x in avals if np.isfinite(x)]
    if not a:
        return np.inf
    lo, hi = min(a), min(a) + hf
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        g = sum(max(mid - x, 0.0) ** 2 for x in a) - hf * hf
        if g > 0:
            hi = mid
        else:
            lo = mid
        if hi - lo <= 1e-17 * hi:
            break
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("shape,seed", [((14, 12), 3), ((6, 7, 5), 4)])
def test_p2_bruteforce_fixed_point_equals_fmm(shape, seed):
    """Gauss-Seidel sweeps of the local upwind solve (by bisection, using all
    neighbours) converge to the unique discrete solution; fast marching must
    reach the same values."""
    h = 1e-4
    nd = len(shape)
    sp = _heterogeneous(shape, seed)
    origin = np.zeros(nd)
    src = np.array([(s - 1) * h * 0.61 for s in shape[::-1]])
    T_fmm = oracle.fmm_point(sp, h, origin, src)

    cell = _corner_sources(shape, h, origin, src)
    T = np.full(shape, np.inf)
    fixed = np.zeros(shape, dtype=bool)
    for m in range(1 << nd):
        cx = [cell[d] + ((m >> d) & 1) for d in range(nd)]
        pos = np.array([origin[d] + cx[d] * h for d in range(nd)])
        idx = tuple(cx[::-1])
        T[idx] = np.linalg.norm(pos - src) / sp[idx]
        fixed[idx] = True
    nodes = [idx for idx in np.ndindex(*shape) if not fixed[idx]]
    for sweep in range(400):
        changed = 0.0
        order = nodes if sweep % 2 == 0 else nodes[::-1]
        for idx in order:
            avals = []
            for ax in range(nd):
                best = np.inf
                for side in (-1, 1):
                    j = list(idx)
                    j[ax] += side
                    if 0 <= j[ax] < shape[ax]:
                        best = min(best, T[tuple(j)])
                avals.append(best)
            t = _local_solve_bisect(avals, h / sp[idx])
            if t < T[idx]:
                changed = max(changed, (T[idx] - t) / t if np.isfinite(T[idx]) else 1.0)
                T[idx] = t
        if changed < 1e-15:
            break
    assert np.allclose(T_fmm, T, rtol=1e-12, atol=0.0)


# ---------------------------------------------------- P3 layered closed form --
def _layer_speed(depth_idx):
    if depth_idx <= 10:
        return 1500.0
    if depth_idx <= 30:
        return 2450.0
    return 1540.0


def test_p3_plane_wave_layers_matches_golden():
    """A plane source (the whole first row accepted at T = 0) through
    horizontal layers: T(depth) = sum of h / c over the rows crossed, exactly;
    checked against hand-written closed-form values (tests/golden)."""
    h = 1e-4
    ny, nx = 61, 9
    sp = np.array([[_layer_speed(r)] * nx for r in range(ny)], dtype=np.float64)
    src = np.arange(nx)
    T = oracle.fmm_sources(sp, h, src, np.zeros(nx))
    expect = np.zeros(ny)
    for r in range(1, ny):
        expect[r] = expect[r - 1] + h / _layer_speed(r)
    assert np.allclose(T, expect[:, None], rtol=1e-12, atol=0)
    with open(os.path.join(GOLDEN, "layered_plane.txt")) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    for depth_mm, t in rows:
        r = int(round(float(depth_mm) * 1e-3 / h))
        assert abs(T[r, 4] - float(t)) <= 1e-12 * float(t)


def test_p3_plane_wave_layers_3d():
    h = 1e-4
    nz, ny, nx = 41, 5, 4
    sp = np.empty((nz, ny, nx))
    for z in range(nz):
        sp[z] = _layer_speed(z)
    T = oracle.fmm_sources(sp, h, np.arange(nx * ny), np.zeros(nx * ny))
    expect = np.cumsum([0.0] + [h / _layer_speed(z) for z in range(1, nz)])
    assert np.allclose(T, expect[:, None, None], rtol=1e-12, atol=0)


def test_p3_point_source_normal_incidence():
    """Point source above horizontal layers: on the normal through the source
    the ray is straight, so T = sum d_i / c_i up to first-order error."""
    h = 1e-4
    n = 81
    sp = np.array([[_layer_speed(r)] * n for r in range(n)], dtype=np.float64)
    origin = np.array([0.0, 0.0])
    src = np.array([40 * h, 0.0])
    T = oracle.fmm_point(sp, h, origin, src)
    exact = np.zeros(n)
    for r in range(1, n):
        exact[r] = exact[r - 1] + h / _layer_speed(r)
    # along the normal only one axis contributes: the first-order scheme is
    # exact there up to the node-centred sampling of the interface (one cell)
    col = T[:, 40]
    assert np.all(np.abs(col - exact) <= h / 1500.0 + 1e-15)
    far = T[:, 0]
    assert np.all(far[1:] > col[1:])


# ------------------------------------------------------- P4 monotonicity --
@pytest.mark.parametrize("ndim", [2, 3])
def test_p4_monotone_accept_order_and_causality(ndim):
    h = 1e-4
    shape = (31, 27) if ndim == 2 else (11, 12, 13)
    sp = _heterogeneous(shape, 11 + ndim)
    origin = np.zeros(ndim)
    src = np.array([(s - 1) * h * 0.44 for s in shape[::-1]])
    T, order = oracle.fmm_point(sp, h, origin, src, return_order=True)
    t_order = T.ravel()[order]
    assert np.all(np.diff(t_order) >= 0)
    assert order.size + (1 << ndim) == T.size
    mins = _axis_minima(T, h)
    nb_min = np.minimum.reduce(mins)
    popped = np.zeros(T.size, dtype=bool)
    popped[order] = True
    popped = popped.reshape(shape)
    assert np.all(nb_min[popped] < T[popped])


def test_p4_homogeneous_increases_along_rays():
    h = 1e-4
    n = 41
    sp = np.full((n, n), 1540.0)
    T = oracle.fmm_point(sp, h, np.zeros(2), np.array([20 * h, 20 * h]))
    assert np.all(np.diff(T[20, 20:]) > 0) and np.all(np.diff(T[20, :21]) < 0)
    assert np.all(np.diff(np.diag(T)[20:]) > 0)


# --------------------------------------------------------- P5 reciprocity --
def test_p5_reciprocity():
    """Sec. II-B uses the sensor as the source since ray paths are
    reversible: T_A(B) ~ T_B(A) up to discretisation error."""
    h = 1e-4
    shape = (64, 64)
    rng = synth.rng_for(99, 0, 0, 0)
    sp = 1500.0 + 1000.0 * synth.smooth_field(shape, 6.0, rng)
    origin = np.zeros(2)
    pts = [(5, 7), (58, 50), (12, 55), (40, 3)]
    for (ax, ay) in pts:
        for (bx, by) in pts:
            if (ax, ay) >= (bx, by):
                continue
            TA = oracle.fmm_point(sp, h, origin, np.array([ax * h, ay * h]))
            TB = oracle.fmm_point(sp, h, origin, np.array([bx * h, by * h]))
            a2b, b2a = TA[by, bx], TB[ay, ax]
            assert abs(a2b - b2a) <= 0.02 * max(a2b, b2a) + 2 * h / 1500.0


# ----------------------------------------------------------- preprocessing --
def test_p6_linear_signal_gives_constant_integrand():
    """p = alpha + beta t  =>  2p - 2t dp/dt = 2 alpha at every sample (the
    one-sided ends are exact on a linear signal)."""
    dt, nt = 25e-9, 257
    t = np.arange(nt) * dt
    p = 0.7 - 3.1e5 * t
    b = oracle.preprocess(p, dt)
    assert np.allclose(b, 1.4, rtol=0, atol=1e-12)


def test_preprocess_quadratic_closed_form():
    """p = t^2: central difference is exact inside (b = -2t^2); the one-sided
    ends give b_0 = 0 and b_{N-1} = 2t^2 - 2t(t + t_{N-2})."""
    dt, nt = 1.0, 12
    t = np.arange(nt) * dt
    b = oracle.preprocess(t * t, dt)
    expect = -2 * t * t
    expect[0] = 0.0
    tn, tm = t[-1], t[-2]
    expect[-1] = 2 * tn * tn - 2 * tn * (tn + tm)
    assert np.allclose(b, expect, rtol=0, atol=1e-12)


def test_spherical_npulse_integrand_is_amplitude():
    """The spherical N-pulse p = A (T0 - t) / (2 T0) has 2p - 2t dp/dt = A
    inside its support (the synthetic signals rely on this)."""
    dt, nt = 10e-9, 400
    A, T0 = 0.8, 2.0e-6
    t = np.arange(nt) * dt
    p = np.where(np.abs(t - T0) <= 0.5e-6, A * (T0 - t) / (2 * T0), 0.0)
    b = oracle.preprocess(p, dt)
    inside = np.abs(t - T0) < 0.5e-6 - 1.5 * dt
    assert np.allclose(b[inside], A, rtol=0, atol=1e-12)


# ------------------------------------------------------------ interpolation --
def test_sample_linear_interpolation_and_window():
    nt = 50
    b = np.arange(nt, dtype=np.float64) * 2.0 + 1.0
    for u in [0.0, 0.25, 3.5, 17.999, 48.0, 48.75, 49.0]:
        assert abs(oracle.sample(b, u) - (2.0 * u + 1.0)) < 1e-12
    assert oracle.sample(b, 49.0 + 1e-9) == 0.0
    assert oracle.sample(b, 1e6) == 0.0


# ------------------------------------------------------- BP closed forms --
def _rand_table(ns, npix, nt, dt, seed, frac_out=0.1):
    rng = np.random.default_rng(seed)
    u = rng.uniform(0, nt - 1, (ns, npix))
    out = rng.uniform(0, 1, (ns, npix)) < frac_out
    u[out] = rng.uniform(nt - 1 + 1e-6, nt + 40, out.sum())
    u[0, 0] = nt - 1  # exactly the last sample
    return u * dt


def test_p6_polynomial_signals_image():
    """Linear signals p_s = alpha_s + beta_s t give an image equal to
    sum over in-window sensors of w_s 2 alpha_s, whatever the table."""
    ns, npix, nt, dt = 9, 40, 64, 1e-8
    T = _rand_table(ns, npix, nt, dt, 5)
    rng = np.random.default_rng(6)
    al, be = rng.normal(size=ns), rng.normal(size=ns) * 1e6
    t = np.arange(nt) * dt
    p = al[:, None] + be[:, None] * t[None, :]
    w = rng.uniform(0.5, 1.5, ns)
    img = oracle.bp(T, p, dt, w)
    inwin = (T / dt) <= nt - 1
    expect = (inwin * (w * 2 * al)[:, None]).sum(axis=0)
    assert np.allclose(img, expect, rtol=1e-12, atol=1e-12)
    img_default = oracle.bp(T, p, dt)
    assert np.allclose(img_default, (inwin * (2 * al / ns)[:, None]).sum(axis=0), atol=1e-12)


def test_p7_impulse_probe_reads_back_hat_function():
    """A unit sample at k0 on one sensor gives b = 2 at k0, -(k0-1) at k0-1 and
    k0+1 at k0+1; the image is w times the piecewise-linear interpolant of
    those three values at u = T/dt."""
    ns, npix, nt, dt, k0 = 3, 500, 40, 1e-8, 17
    rng = np.random.default_rng(7)
    u = rng.uniform(k0 - 3, k0 + 3, (ns, npix))
    T = u * dt
    p = np.zeros((ns, nt))
    p[1, k0] = 1.0
    w = np.array([0.3, 0.5, 0.2])
    img = oracle.bp(T, p, dt, w)
    bvals = {k0 - 1: -(k0 - 1.0), k0: 2.0, k0 + 1: k0 + 1.0}

    def bk(k):
        return bvals.get(k, 0.0)

    uu = u[1]
    i0 = np.floor(uu).astype(int)
    ph = uu - i0
    expect = 0.5 * np.array([(1 - f) * bk(i) + f * bk(i + 1) for i, f in zip(i0, ph)])
    assert np.allclose(img, expect, rtol=0, atol=1e-12)


def test_p8_bruteforce_bp_16x16():
    """Per-pixel oracle loop against a vectorised evaluation of the same sum
    on a 16x16 grid (a consistency check of the loop structure)."""
    n, dt, nt = 16, 20e-9, 300
    h = 0.2e-3
    sp = np.full((n, n), 1540.0)
    origin = synth.centred_origin((n, n), h)
    sensors = synth.ring_sensors(12, 7.0 * h)
    rng = np.random.default_rng(8)
    p = rng.normal(size=(12, nt))
    img = oracle.reconstruct(sp, h, origin, sensors, p, dt)
    T = oracle.travel_table(sp, h, origin, sensors, np.arange(n * n))
    b = np.empty_like(p)
    b[:, 1:-1] = 2 * p[:, 1:-1] - np.arange(1, nt - 1)[None, :] * (p[:, 2:] - p[:, :-2])
    b[:, 0] = 2 * p[:, 0]
    b[:, -1] = 2 * p[:, -1] - 2 * (nt - 1) * (p[:, -1] - p[:, -2])
    u = T / dt
    i0 = np.minimum(np.floor(u).astype(int), nt - 2)
    ph = u - i0
    rows = np.arange(12)[:, None]
    val = (1 - ph) * b[rows, i0] + ph * b[rows, i0 + 1]
    val[u > nt - 1] = 0
    assert np.allclose(img.ravel(), val.mean(axis=0), rtol=1e-12, atol=1e-12)


def test_p10_linearity():
    ns, npix, nt, dt = 7, 60, 80, 1e-8
    T = _rand_table(ns, npix, nt, dt, 9)
    rng = np.random.default_rng(10)
    p, q = rng.normal(size=(ns, nt)), rng.normal(size=(ns, nt))
    a, b = 1.7, -0.4
    lhs = oracle.bp(T, a * p + b * q, dt)
    rhs = a * oracle.bp(T, p, dt) + b * oracle.bp(T, q, dt)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


# ------------------------------------------------ P9 point absorber / skull --
def _peak_error(img, p0):
    """Distance (nodes) between the image argmax and the phantom argmax."""
    a = np.unravel_index(np.argmax(img), img.shape)
    b = np.unravel_index(np.argmax(p0), p0.shape)
    return math.hypot(a[0] - b[0], a[1] - b[1])


def test_p9_homogeneous_point_absorber_peak():
    """A single small absorber in a homogeneous medium reconstructs its peak
    at its own node, with a value near its amplitude."""
    n, h = 64, 0.2e-3
    shape = (n, n)
    sp = np.full(shape, 1540.0, dtype=np.float32)
    origin = synth.centred_origin(shape, h)
    sensors = synth.ring_sensors(64, 30 * h)
    centre = np.array([[origin[0] + 37 * h, origin[1] + 25 * h, 0.0]])
    dt, nt = 20e-9, 800
    p = synth.render_signals(sp, h, origin, sensors, centre, [2.0 * h], [1.0], dt, nt, 0.0,
                             np.random.default_rng(0))
    img = oracle.reconstruct(sp, h, origin, sensors, p, dt)
    iy, ix = np.unravel_index(np.argmax(img), shape)
    assert (ix, iy) == (37, 25)
    assert 0.5 < img.max() < 1.5


def test_p9_skull_fmm_beats_constant_speed():
    """Sec. III: with a skull, the fast-marching table localises absorbers
    better than a constant-speed (1560 m/s) table.  Signals are rendered at
    fast-marching arrival times from the absorber (the data a first-arrival
    forward model produces)."""
    g = golden_numbers()
    w = synth.config1(n_frames=1)
    # one absorber near the skull, where aberration is strongest
    centre = np.array([[w.origin[0] + 63.5 * w.dx + 38 * w.dx, w.origin[1] + 63.5 * w.dx, 0.0]])
    p = synth.render_signals(w.speed, w.dx, w.origin, w.sensors, centre, [1.5 * w.dx], [1.0],
                             w.dt, w.nt, 0.0, np.random.default_rng(0), arrivals=fmm_arrivals)
    pix = np.flatnonzero(w.mask.ravel())
    T = oracle.travel_table(w.speed, w.dx, w.origin, w.sensors, pix)
    img_fmm = oracle.reconstruct(w.speed, w.dx, w.origin, w.sensors, p, w.dt, w.mask, T=T)
    Tc = oracle.constant_table(w.speed.shape, w.dx, w.origin, w.sensors, pix, g["c_constant_bp"])
    img_c = oracle.reconstruct(w.speed, w.dx, w.origin, w.sensors, p, w.dt, w.mask, T=Tc)
    p0 = synth.phantom_discs(w.speed.shape, w.dx, w.origin, centre, [1.5 * w.dx], [1.0])
    e_fmm, e_c = _peak_error(img_fmm, p0), _peak_error(img_c, p0)
    assert e_fmm <= 1.0 and e_c > 3.0
    assert 0.9 < img_fmm.max() < 1.1 and img_c.max() < 0.5


# ------------------------------------------- constant-speed time of flight --
def test_constant_table_pythagorean_offsets_are_exact():
    """Conventional BP delays (Sec. II-C): node offsets (3, 4) and (2, 3, 6)
    node spacings from a sensor give 5 and 7 spacings over c0 exactly; in 2-D
    the sensor's z does not count."""
    h, c0 = 0.25e-3, 1560.0
    origin = (-1.0e-3, 2.0e-3, 0.5e-3)
    # 2-D: grid (ny, nx) = (9, 11); sensor on node (x=1, y=2) lifted off-plane
    sens = np.array([[origin[0] + 1 * h, origin[1] + 2 * h, 7.0e-3]])
    T = oracle.constant_table((9, 11), h, origin, sens, [6 * 11 + 4], c0)
    assert T[0, 0] * c0 / h == pytest.approx(5.0, rel=1e-15)
    T0 = oracle.constant_table((9, 11), h, origin, sens, [2 * 11 + 1], c0)
    assert T0[0, 0] == 0.0
    # 3-D: grid (nz, ny, nx) = (8, 6, 5); sensor on node (x=0, y=1, z=0)
    sens3 = np.array([[origin[0], origin[1] + h, origin[2]]])
    T3 = oracle.constant_table((8, 6, 5), h, origin, sens3, [(6 * 6 + 4) * 5 + 2], c0)
    assert T3[0, 0] * c0 / h == pytest.approx(7.0, rel=1e-15)


def test_constant_table_is_the_homogeneous_fast_marching_limit():
    """In a homogeneous medium the fast-marching table (Sec. II-B) converges
    to the constant-speed delays, from above, at first order in dx."""
    c0, L = 1560.0, 1.0e-3
    src = np.array([[0.21e-4, -0.37e-4, 0.0]])
    errs = []
    for n in (33, 65, 129):
        h = 2 * L / (n - 1)
        origin = (-L, -L, 0.0)
        pix = np.arange(n * n)
        Tf = oracle.travel_table(np.full((n, n), c0), h, origin, src, pix)
        Tc = oracle.constant_table((n, n), h, origin, src, pix, c0)
        err = Tf - Tc
        assert err.min() > -1e-12 * Tc.max()
        errs.append(err.max())
    assert errs[1] < 0.8 * errs[0] and errs[2] < 0.8 * errs[1]


def test_constant_speed_bp_of_homogeneous_absorber_recovers_it():
    """With the true constant speed the straight-ray delays are exact, and the
    Eq. (BP) integrand of a uniform absorber's N-shaped pulse is its amplitude
    inside it: the conventional back projection gives the amplitude at the
    absorber's node and its maximum lies inside the absorber."""
    n, h, c0 = 64, 0.2e-3, 1540.0
    shape = (n, n)
    sp = np.full(shape, c0, dtype=np.float32)
    origin = synth.centred_origin(shape, h)
    sensors = synth.ring_sensors(64, 30 * h)
    centre = np.array([[origin[0] + 26 * h, origin[1] + 36 * h, 0.0]])
    dt, nt = 20e-9, 800
    p = synth.render_signals(sp, h, origin, sensors, centre, [2.0 * h], [1.0], dt, nt, 0.0,
                             np.random.default_rng(3))
    pix = np.arange(n * n)
    T = oracle.constant_table(shape, h, origin, sensors, pix, c0)
    img = oracle.reconstruct(sp, h, origin, sensors, p, dt, T=T)
    assert img[36, 26] == pytest.approx(1.0, abs=1e-3)
    iy, ix = np.unravel_index(np.argmax(img), shape)
    assert math.hypot(ix - 26, iy - 36) <= 2.0
    assert img.max() < 1.0 + 1e-3


# ------------------------------------------------------ paper's numbers --
def test_paper_shaped_workload_matches_printed_numbers():
    g = golden_numbers()
    w = synth.config2(n_frames=1, n_lines=2)
    assert w.n_pix == int(g["n_pixels_coarse"])
    assert w.n_sensors == int(g["n_sensors"])
    # halving dx quadruples the pixel count of the same region (Sec. III)
    assert abs(g["n_pixels_fine"] / g["n_pixels_coarse"] - 4.0) < 0.01
    skull = (w.speed > 1600)
    assert w.speed[skull].min() >= g["c_skull_lo"] and w.speed[skull].max() <= g["c_skull_hi"]
    assert np.all(w.speed[w.mask.astype(bool)] == g["c_brain"])
    # record length covers the end time 1.5 d / c0 of Sec. III
    d = 2 * np.linalg.norm(w.sensors[0, :2])
    assert w.nt * w.dt >= g["end_time_factor"] * d / synth.C_WATER


# ------------------------------------------------------ speed-map errors --
@pytest.mark.parametrize("shape,seed", [((31, 27), 5), ((11, 13, 9), 6)])
def test_faster_medium_never_arrives_later(shape, seed):
    """The first-order upwind scheme is monotone: raising the speed at any set
    of nodes (here the Sec. III error model with its positive mean, clipped
    at zero) can only make arrivals earlier, at every node."""
    rng = np.random.default_rng(seed)
    sp = _heterogeneous(shape, seed)
    h = 1e-4
    origin = np.zeros(len(shape))
    src = np.array([(n - 1) * h * f for n, f in zip(shape[::-1], (0.3, 0.6, 0.4))])
    region = rng.uniform(0, 1, shape) < 0.5
    err = synth.speed_error(sp, rng, region=region).astype(np.float64)
    faster = np.maximum(err, sp)
    T = oracle.fmm_point(sp, h, origin, src)
    Tf = oracle.fmm_point(faster, h, origin, src)
    assert np.all(Tf <= T + 1e-15 * T.max())
    assert np.any(Tf < T)
    # and the error model itself: mean and spread 1.7 % of the maximum speed, on the region only
    d = (err - sp)[region]
    assert np.all(err[~region] == sp[~region].astype(np.float32))
    assert abs(d.mean() - 0.017 * sp.max()) < 0.2 * 0.017 * sp.max()
    assert abs(d.std() - 0.017 * sp.max()) < 0.2 * 0.017 * sp.max()


# ------------------------------------------------- second-order stencil --
@pytest.mark.parametrize("ndim", [2, 3])
def test_second_order_reproduces_an_oblique_plane_wave_exactly(ndim):
    """Both one-sided differences are exact for a linear arrival time, so with
    two exact layers accepted along every low face both orders reproduce an
    oblique plane wave to rounding (a wrong second-order weight or offset
    would not)."""
    n = 24 if ndim == 2 else 12
    shape = (n,) * ndim
    c, h = 1500.0, 1e-4
    k = np.array([0.8, 0.45, 0.39][:ndim])
    k = k / np.linalg.norm(k)
    idx = np.indices(shape)[::-1]  # x first
    T_exact = sum(k[d] * idx[d] * h for d in range(ndim)) / c
    src = np.flatnonzero(np.any(np.stack([idx[d] < 2 for d in range(ndim)]), axis=0).ravel())
    sp = np.full(shape, c)
    for order in (1, 2):
        T = oracle.fmm_sources(sp, h, src, T_exact.ravel()[src], order=order)
        assert np.abs(T - T_exact).max() <= 1e-10 * h / c


@pytest.mark.parametrize("ndim,sizes,min_ratio2", [(2, (41, 81, 161), 3.5), (3, (21, 41), 2.8)])
def test_second_order_converges_at_second_order(ndim, sizes, min_ratio2):
    """A circular (spherical) front accepted exactly inside 0.3 L of the
    source and marched outward: the order-1 error halves and the order-2 error
    falls about fourfold each time dx halves (observed orders 1 and 2)."""
    c, L = 1500.0, 1e-3
    src = np.array([0.13e-4, -0.07e-4, 0.05e-4])[:ndim]
    errs = {1: [], 2: []}
    for n in sizes:
        h = 2 * L / (n - 1)
        origin = np.full(ndim, -L)
        axes = [origin[d] + h * np.arange(n) for d in range(ndim)]
        mesh = np.meshgrid(*axes[::-1], indexing="ij")
        dist = np.sqrt(sum((mesh[ndim - 1 - d] - src[d]) ** 2 for d in range(ndim)))
        sp = np.full((n,) * ndim, c)
        init = np.flatnonzero((dist < 0.3 * L).ravel())
        for order in (1, 2):
            T = oracle.fmm_sources(sp, h, init, (dist / c).ravel()[init], order=order)
            errs[order].append(np.abs(T - dist / c)[dist >= 0.3 * L].max())
    for i in range(len(sizes) - 1):
        assert 1.8 < errs[1][i] / errs[1][i + 1] < 2.3
        assert errs[2][i] / errs[2][i + 1] > min_ratio2 or i < len(sizes) - 2
        assert errs[2][i] < 0.25 * errs[1][i]


def test_second_order_accept_order_and_causality():
    """P4 for the second-order march on a heterogeneous grid."""
    sp = _heterogeneous((29, 23), 3)
    h = 1e-4
    T, order = oracle.fmm_point(sp, h, np.zeros(2), np.array([7.3e-4, 9.1e-4]), return_order=True,
                                order=2)
    popped = T.ravel()[order]
    assert np.all(np.diff(popped) >= -1e-15 * popped.max())
    assert np.isfinite(T).all()


# ------------------------------------------------ exact back-projection weights --
# Sec. II-C: Eq. (BP) approximates the exact back projection, which weighs each
# sensor by the solid angle its element subtends at the pixel.  The weights are
# pinned by Gauss's theorem for angles: a closed curve (surface) is seen under
# the full angle 2 pi (4 pi) from every point inside it and under 0 from every
# point outside, so the weights of a closed array sum to 1 inside and 0 outside.
def _ring_geometry(n, radius, centre=(0.0, 0.0)):
    th = 2.0 * np.pi * (np.arange(n) + 0.25) / n
    sens = np.stack([centre[0] + radius * np.cos(th), centre[1] + radius * np.sin(th),
                     np.zeros(n)], axis=1)
    normals = -np.stack([np.cos(th), np.sin(th), np.zeros(n)], axis=1)
    return sens, normals, np.full(n, 2.0 * np.pi * radius / n)


def test_solid_angle_ring_sums_to_one_inside_and_zero_outside():
    shape, h = (41, 41), 1e-3
    origin = np.array([-20e-3, -20e-3, 0.0])
    R = 12.3e-3
    sens, nrm, elem = _ring_geometry(256, R)
    pix = np.arange(41 * 41)
    W = oracle.solid_angle_weights(shape, h, origin, sens, nrm, elem, 2.0 * np.pi, pix)
    r = np.linalg.norm(oracle.node_positions(shape, h, origin, pix)[:, :2], axis=1)
    tot = W.sum(axis=0)
    inside, outside = r < 0.7 * R, r > 1.3 * R
    assert inside.sum() > 100 and outside.sum() > 100
    assert np.abs(tot[inside] - 1.0).max() < 1e-12
    assert np.abs(tot[outside]).max() < 1e-12
    # the centre sees every element of the ring at the same angle: 1/N each
    c = np.argmin(r)
    assert r[c] == 0.0 and np.allclose(W[:, c], 1.0 / 256, rtol=1e-13, atol=0)


def test_solid_angle_ellipse_with_unequal_elements():
    """A non-circular array: an ellipse sampled at equal parameter steps, so the
    elements differ in length and the normals are not radial."""
    shape, h = (41, 41), 1e-3
    origin = np.array([-20e-3, -20e-3, 0.0])
    a, b, n = 15e-3, 9e-3, 512
    th = 2.0 * np.pi * np.arange(n) / n
    sens = np.stack([a * np.cos(th), b * np.sin(th), np.zeros(n)], axis=1)
    out_n = np.stack([b * np.cos(th), a * np.sin(th), np.zeros(n)], axis=1)
    speed = np.hypot(a * np.sin(th), b * np.cos(th))  # |dr/dtheta|
    elem = speed * 2.0 * np.pi / n
    pix = np.arange(41 * 41)
    W = oracle.solid_angle_weights(shape, h, origin, sens, -out_n, elem, 2.0 * np.pi, pix)
    pos = oracle.node_positions(shape, h, origin, pix)
    q = (pos[:, 0] / a) ** 2 + (pos[:, 1] / b) ** 2
    tot = W.sum(axis=0)
    assert np.abs(tot[q < 0.5] - 1.0).max() < 1e-10
    assert np.abs(tot[q > 2.0]).max() < 1e-10
    # outward normals see the full angle with the opposite sign
    Wout = oracle.solid_angle_weights(shape, h, origin, sens, out_n, elem, 2.0 * np.pi, pix)
    assert np.allclose(Wout, -W, rtol=0, atol=1e-15)


def _fibonacci_sphere(n, radius):
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    phi = np.pi * (1.0 + 5.0 ** 0.5) * k
    rho = np.sqrt(1.0 - z * z)
    return radius * np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def test_solid_angle_sphere_centre_exact_interior_converges():
    """3-D: equal-area elements of a sphere (Fibonacci lattice) with inward
    normals.  At the centre every weight is exactly 1/N; inside, the weights sum
    to 1 up to the lattice's quadrature error, which falls as N grows."""
    shape, h = (21, 21, 21), 1e-3
    origin = np.array([-10e-3] * 3)
    R = 30e-3
    pix = np.arange(21 ** 3)
    r = np.linalg.norm(oracle.node_positions(shape, h, origin, pix), axis=1)
    inner = r <= 0.5 * R
    errs = []
    for n in (500, 2000):
        S = _fibonacci_sphere(n, R)
        W = oracle.solid_angle_weights(shape, h, origin, S, -S / R, np.full(n, 4 * np.pi * R * R / n),
                                       4.0 * np.pi, pix)
        c = np.argmin(r)
        assert r[c] == 0.0 and np.allclose(W[:, c], 1.0 / n, rtol=1e-13, atol=0)
        errs.append(np.abs(W.sum(axis=0)[inner] - 1.0).max())
    assert errs[1] < 3e-5 and errs[1] < errs[0] / 3


def test_bp_with_pair_weights_reduces_to_sensor_weights():
    """Weights per (sensor, pixel) that do not depend on the pixel give the
    per-sensor sum bit for bit."""
    rng = np.random.default_rng(7)
    ns, npix, nt, dt = 9, 40, 64, 1e-8
    T = rng.uniform(-2, nt + 2, (ns, npix)) * dt
    p = rng.standard_normal((ns, nt))
    w = rng.uniform(0.1, 1.0, ns)
    a = oracle.bp(T, p, dt, w)
    b = oracle.bp(T, p, dt, np.repeat(w[:, None], npix, axis=1))
    assert np.array_equal(a, b)
