"""GPU parity of the conventional (constant-speed) back projection against the
FP64 oracle: Eq. (BP) with t_sj = |r_j - r_s| / c0 (Sec. II-C; Sec. III compares
at 1560 m/s), the delays computed in the gather kernel.

Tolerances are those of the stored-table path: FP32 signals rel-L2 <= 1e-5 and
max-abs <= 1e-4 * max|p0| per frame; 16-bit signals rel-L2 <= 5e-3 against the
oracle on the FP32 signals.  Facts that are integers (zeros outside the mask,
batch invariance, plan and eviction round trips) are checked bit for bit.
"""
import math

import numpy as np
import pytest

import oracle
from helpers import fmm_arrivals
from oracle_pool import travel_table
from paper_1501_03869_gb300 import BP, PatError, Plan, _lib, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_REL_L2 = 1e-5
FP32_MAX_ABS_FRAC = 1e-4
LOWP_REL_L2 = 5e-3
C_BP = 1560.0  # the constant speed of the paper's conventional back projection


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_03869_gb300.build import build
    build()
    torch.cuda.init()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_const(w, c0, signals=None, pix=None):
    """Oracle images [F, grid] (or [F, len(pix)] values at pix)."""
    sig = np.asarray(w.signals if signals is None else signals, dtype=np.float64)
    dense = pix is None
    if dense:
        pix = np.flatnonzero(w.mask.ravel()) if w.mask is not None else np.arange(w.speed.size)
    T = oracle.constant_table(w.speed.shape, w.dx, w.origin, w.sensors, pix, c0)
    vals = np.stack([oracle.bp(T, sig[f], w.dt) for f in range(sig.shape[0])])
    if not dense:
        return vals
    out = np.zeros((sig.shape[0], w.speed.size))
    out[:, pix] = vals
    return out.reshape((sig.shape[0],) + w.speed.shape)


def const_handle(w, c0, flags=0, sensors=None):
    return BP.constant(c0, w.speed.shape, w.dx, w.origin, w.sensors if sensors is None else sensors,
                       w.dt, w.nt, mask=w.mask, flags=flags)


def run(bp, sig, dtype="f32"):
    if dtype == "f32":
        s = torch.from_numpy(np.ascontiguousarray(sig, dtype=np.float32)).cuda()
        out = bp.reconstruct(s)
    else:
        codes, sc, _ = synth.quantise(sig, dtype)
        tdt = torch.bfloat16 if dtype == "bf16" else torch.float16
        s = torch.from_numpy(codes.astype(np.int16)).cuda().view(tdt)
        out = bp.reconstruct(s, scales=torch.from_numpy(sc).cuda())
    bp.sync()
    return out.cpu().numpy().astype(np.float64)


def gpu_const(w, c0, flags=0, signals=None, dtype="f32"):
    with const_handle(w, c0, flags) as bp:
        return run(bp, w.signals if signals is None else signals, dtype), dict(bp.info)


def assert_fp32_parity(got, ref, scale):
    for f in range(ref.shape[0]):
        e = rel_l2(got[f], ref[f])
        m = np.abs(got[f] - ref[f]).max()
        assert e <= FP32_REL_L2, f"frame {f}: rel-L2 {e:.3e}"
        assert m <= FP32_MAX_ABS_FRAC * scale, f"frame {f}: max-abs {m:.3e}"


def test_constant_c1_parity_and_no_table():
    w = synth.config1(n_frames=2)
    ref = oracle_const(w, C_BP)
    got, info = gpu_const(w, C_BP)
    assert info["delays"] == 1 and info["c0"] == C_BP
    # anchors (32 B per tile and sensor) and pixel terms (16 B per slot) only
    assert info["table_bytes"] == info["n_tiles"] * (((w.n_sensors + 3) // 4 * 4) * 32 + 128 * 16)
    assert_fp32_parity(got, ref, np.abs(w.p0).max())
    assert np.all(got[:, ~w.mask.astype(bool)] == 0.0)


def test_constant_c2_full_size_whole_image():
    """Paper-shaped frame (512 sensors, 21 323 pixels) at 1560 m/s."""
    w = synth.config2(n_frames=1)
    ref = oracle_const(w, C_BP)
    got, info = gpu_const(w, C_BP)
    assert info["n_pix"] == 21323
    assert_fp32_parity(got, ref, np.abs(w.p0).max())


def test_constant_3d_sensors_outside_the_grid():
    """A volume with every sensor outside the grid box (the fast-marching
    handle rejects those; straight-line delays need no grid around them)."""
    shape = (20, 28, 36)
    dx = 0.25e-3
    rng = np.random.default_rng(11)
    origin = synth.centred_origin(shape, dx)
    sens = synth.fibonacci_hemisphere(40, 30 * dx, np.zeros(3))
    half = np.array([(n - 1) / 2 * dx for n in shape[::-1]])
    outside = np.any(np.abs(sens) > half[None, :], axis=1)
    assert outside.all()
    nt, dt = 700, 20e-9
    t = np.arange(nt) * dt
    sig = (np.sin(t[None, None, :] * 4e6 + rng.uniform(0, 6, (2, 40, 1)))
           * np.exp(-t / 8e-6)[None, None, :]).astype(np.float32)
    mask = (rng.uniform(0, 1, shape) < 0.8).astype(np.uint8)
    w = synth.Workload("out", np.full(shape, 1500.0, np.float32), dx, origin, sens, mask, dt, nt,
                       sig, np.ones((2,) + shape, np.float32))
    with pytest.raises(PatError):
        BP(w.speed, dx, origin, sens, dt, nt, mask=mask)
    ref = oracle_const(w, 1500.0)
    got, _ = gpu_const(w, 1500.0)
    assert_fp32_parity(got, ref, np.abs(ref).max())


@pytest.mark.parametrize("ns,nt,F,shape,hole", [
    (1, 2, 1, (9, 7), False),
    (5, 3, 3, (20, 33), True),
    (37, 101, 9, (40, 45), True),
    (67, 640, 5, (64, 64), False),
    (13, 257, 2, (11, 13, 9), True),
])
def test_constant_ragged_and_degenerate_shapes(ns, nt, F, shape, hole):
    """Sensor counts off the stage size, records of 2-3 samples, partial frame
    groups, masks with holes, 2-D and 3-D; sensor 0 sits exactly on a mask
    node (a zero delay there)."""
    rng = np.random.default_rng(ns * 977 + nt)
    dx = 1e-4
    origin = synth.centred_origin(shape, dx)
    half = np.array([(n - 1) / 2 * dx for n in shape[::-1]])
    sens = np.zeros((ns, 3))
    sens[:, : len(shape)] = rng.uniform(-1.3, 1.3, (ns, len(shape))) * half
    mask = (rng.uniform(0, 1, shape) < (0.7 if hole else 1.0)).astype(np.uint8)
    node = np.unravel_index(int(np.flatnonzero(mask.ravel())[len(shape)]), shape)[::-1]
    sens[0, : len(shape)] = [origin[d] + node[d] * dx for d in range(len(shape))]
    c0 = 1500.0
    tmax = 2 * np.linalg.norm(half) / c0
    dt = tmax / max(nt - 1, 1) * 0.6
    t = np.arange(nt) * dt
    sig = (rng.standard_normal((F, ns, nt)) * 0.1 +
           np.sin(t[None, None, :] * 3e6 + rng.uniform(0, 6, (F, ns, 1)))).astype(np.float32)
    w = synth.Workload("rag", np.full(shape, c0, np.float32), dx, origin, sens, mask, dt, nt, sig,
                       np.ones((F,) + shape, np.float32))
    ref = oracle_const(w, c0)
    got, _ = gpu_const(w, c0)
    scale = np.abs(ref).max()
    for f in range(F):
        assert rel_l2(got[f], ref[f]) <= FP32_REL_L2
        assert np.abs(got[f] - ref[f]).max() <= FP32_MAX_ABS_FRAC * scale
    assert np.all(got[:, ~mask.astype(bool)] == 0.0)


@pytest.mark.parametrize("dtype,tol_kernel", [("bf16", 2e-3), ("f16", 5e-4)])
def test_constant_low_precision(dtype, tol_kernel):
    w = synth.config3(n_frames=64)
    ref = oracle_const(w, C_BP)
    got, _ = gpu_const(w, C_BP, dtype=dtype)
    _, _, deq = synth.quantise(w.signals, dtype)
    ref_q = oracle_const(w, C_BP, signals=deq)
    assert max(rel_l2(got[f], ref[f]) for f in range(64)) <= LOWP_REL_L2
    assert max(rel_l2(got[f], ref_q[f]) for f in range(64)) <= tol_kernel


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_constant_frame_result_independent_of_batch(dtype):
    w = synth.config1(n_frames=16)
    with const_handle(w, C_BP) as bp:
        alone = [run(bp, w.signals[f:f + 1], dtype)[0] for f in (0, 5, 15)]
        batch = run(bp, w.signals, dtype)
        three = run(bp, w.signals[3:6], dtype)
    for g, f in zip(alone, (0, 5, 15)):
        assert np.array_equal(g, batch[f])
    assert np.array_equal(three[2], batch[5])


def test_constant_tile256_and_compact():
    w = synth.config2(n_frames=1, n_lines=3)
    ref = oracle_const(w, C_BP)
    got, info = gpu_const(w, C_BP, flags=_lib.PAT_FLAG_TILE_256)
    assert info["tile_pix"] == 256
    assert_fp32_parity(got, ref, np.abs(w.p0).max())
    gc, _ = gpu_const(w, C_BP, flags=_lib.PAT_FLAG_COMPACT_OUT)
    pix = np.flatnonzero(w.mask.ravel())
    assert_fp32_parity(gc, ref.reshape(1, -1)[:, pix], np.abs(w.p0).max())


def test_constant_plan_equals_single_and_rejects_mixing():
    ws = [synth.config1(n_frames=3), synth.config1(n_frames=2, inst=1, cfg_id=7)]
    hs = [const_handle(w, C_BP) for w in ws]
    singles = [run(h, w.signals) for h, w in zip(hs, ws)]
    plan = Plan(hs, [3, 2], autotune=True, graph=True)
    sig = [torch.from_numpy(w.signals).cuda() for w in ws]
    outs = [torch.empty(shp, device="cuda") for shp in plan.out_shapes()]
    for _ in range(2):
        plan.execute(sig, outs)
        plan.sync()
        for o, s in zip(outs, singles):
            assert np.array_equal(o.cpu().numpy(), s)
    plan.close()
    fmm = BP(ws[0].speed, ws[0].dx, ws[0].origin, ws[0].sensors, ws[0].dt, ws[0].nt, mask=ws[0].mask)
    with pytest.raises(PatError) as e:
        Plan([hs[0], fmm], [1, 1])
    assert e.value.status == _lib.PAT_ERR_INVALID
    for h in hs + [fmm]:
        h.close()


def test_constant_evict_restore_and_no_table_readback():
    w = synth.config1(n_frames=2)
    with const_handle(w, C_BP, flags=_lib.PAT_FLAG_HOST_MIRROR) as bp:
        a = run(bp, w.signals)
        bp.evict()
        with pytest.raises(PatError):
            run(bp, w.signals)
        bp.restore()
        b = run(bp, w.signals)
        u, base, slot = bp.table()
        assert u is None and base.shape == (bp.info["n_tiles"], w.n_sensors)
        with pytest.raises(PatError):
            ctypes_u = np.empty(1, np.float32)
            _lib.check(bp._lib.pat_bp_table(bp.handle, ctypes_u.ctypes.data, None, None),
                       "pat_bp_table")
    assert np.array_equal(a, b)


def test_constant_noalloc_matches_reconstruct():
    w = synth.config1(n_frames=2)
    with const_handle(w, C_BP) as bp:
        s = torch.from_numpy(w.signals).cuda()
        ref = bp.reconstruct(s).cpu().numpy()
        out = torch.full(bp.out_shape(2), float("nan"), device="cuda")
        bp.reconstruct_noalloc(s, out)
        bp.sync()
        assert_fp32_parity(out.cpu().numpy(), ref, np.abs(w.p0).max())


def test_constant_linear_signals_and_after_record():
    """P6 through the computed delays: p_s = alpha_s + beta_s t gives the
    constant sum_s w_s 2 alpha_s wherever all arrivals fall in the record; a
    record that ends before every arrival gives zero."""
    w = synth.config2(n_frames=1, n_lines=1)
    rng = np.random.default_rng(5)
    al = rng.integers(-16, 17, w.n_sensors) / 16.0
    gam = rng.integers(-3, 4, w.n_sensors) * 2.0 ** -13
    k = np.arange(w.nt)
    sig = (al[:, None] + gam[:, None] * k[None, :])[None].astype(np.float32)
    got, _ = gpu_const(w, C_BP, signals=sig)
    vals = got[0][w.mask.astype(bool)]
    assert np.abs(vals - np.mean(2 * al)).max() <= 1e-5
    w1 = synth.config1(n_frames=1)
    w1.dt = 1e-12
    got, _ = gpu_const(w1, C_BP)
    assert np.all(got == 0.0)


def test_constant_full_3d_volume_sampled():
    """The serving volume at full size (160x160x96 voxels, all reconstructed)
    with all 1024 hemisphere sensors in water (1500 m/s), FP32 and BF16
    signals: 4096 sampled voxels against the oracle, one by one."""
    w = synth.config5_subject(4, n_frames=1, n_sensors=1024)
    rng = np.random.default_rng(7)
    pix = np.sort(rng.choice(w.speed.size, 4096, replace=False))
    ref = oracle_const(w, 1500.0, pix=pix)[0]
    with const_handle(w, 1500.0) as bp:
        assert bp.info["n_pix"] == 160 * 160 * 96
        got = run(bp, w.signals)[0].ravel()[pix]
        got16 = run(bp, w.signals, "bf16")[0].ravel()[pix]
    scale = np.abs(ref).max()
    assert rel_l2(got, ref) <= FP32_REL_L2
    assert np.abs(got - ref).max() <= FP32_MAX_ABS_FRAC * max(scale, np.abs(w.p0).max())
    assert rel_l2(got16, ref) <= LOWP_REL_L2


def _peak_error(img, p0):
    a = np.unravel_index(np.argmax(img), img.shape)
    b = np.unravel_index(np.argmax(p0), p0.shape)
    return math.hypot(a[0] - b[0], a[1] - b[1])


def test_fast_marching_beats_constant_speed_on_the_gpu():
    """Sec. III's comparison run through both GPU paths: with a skull, the
    fast-marching handle localises an absorber near the skull; the
    constant-speed (1560 m/s) handle misplaces and blurs it."""
    w = synth.config1(n_frames=1)
    centre = np.array([[w.origin[0] + 63.5 * w.dx + 38 * w.dx, w.origin[1] + 63.5 * w.dx, 0.0]])
    p = synth.render_signals(w.speed, w.dx, w.origin, w.sensors, centre, [1.5 * w.dx], [1.0],
                             w.dt, w.nt, 0.0, np.random.default_rng(0), arrivals=fmm_arrivals)
    with BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) as bp:
        img_fmm = run(bp, p[None])[0]
    with const_handle(w, C_BP) as bp:
        img_c = run(bp, p[None])[0]
    p0 = synth.phantom_discs(w.speed.shape, w.dx, w.origin, centre, [1.5 * w.dx], [1.0])
    assert _peak_error(img_fmm, p0) <= 1.0 and _peak_error(img_c, p0) > 3.0
    assert 0.9 < img_fmm.max() < 1.1 and img_c.max() < 0.5
    # the GPU images are the oracle's images of the same data
    pix = np.flatnonzero(w.mask.ravel())
    T = travel_table("c1", w.speed, w.dx, w.origin, w.sensors, pix)
    ref = np.zeros(w.speed.size)
    ref[pix] = oracle.bp(T, p, w.dt)
    assert rel_l2(img_fmm, ref.reshape(w.speed.shape)) <= FP32_REL_L2


def test_first_frame_after_device_memory_reuse():
    """Kernels that start before the previous kernel has finished must not
    read lines an earlier kernel left in L1: a handle whose buffers reuse the
    device memory of a closed handle gives, on its very first frame, the same
    bits through the unstaged and the staged gather."""
    w0 = synth.config5_subject(4, n_frames=1, n_sensors=512, shape=(24, 40, 40), nt=600)
    for fl in (0, _lib.PAT_FLAG_STAGED_SINGLE):
        with const_handle(w0, 1500.0, flags=fl) as bp:
            run(bp, w0.signals)
    w = synth.config5_subject(4, n_frames=1, n_sensors=1024)
    with const_handle(w, 1500.0) as a:
        first = run(a, w.signals)
    with const_handle(w, 1500.0, flags=_lib.PAT_FLAG_STAGED_SINGLE) as b:
        ref = run(b, w.signals)
    assert np.array_equal(first, ref)
