"""GPU parity of the CUDA path against the FP64 oracle (Eq. (BP), Sec. II-C).

Tolerances (from the precision budget of the method):
  FP32 signals:  rel-L2 <= 1e-5 and max-abs <= 1e-4 * max|p0| per frame;
  16-bit signals: rel-L2 <= 5e-3 per frame against the oracle on the original
  FP32 signals.
Integer facts (zeros outside the mask, batch invariance, determinism) are
checked bit for bit.
"""
import numpy as np
import pytest

import oracle
from oracle_pool import travel_table
from paper_1501_03869_gb300 import BP, _lib, synth, wait_timeout_probe

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_REL_L2 = 1e-5
FP32_MAX_ABS_FRAC = 1e-4
LOWP_REL_L2 = 5e-3


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


def oracle_images(w, key, sensors_idx=None, signals=None):
    """Oracle dense images [F, grid] of workload w (optionally a sensor subset)."""
    sens = w.sensors if sensors_idx is None else w.sensors[sensors_idx]
    pix = np.flatnonzero(w.mask.ravel())
    T = travel_table(key, w.speed, w.dx, w.origin, sens, pix)
    sig = w.signals if signals is None else signals
    if sensors_idx is not None:
        sig = sig[:, sensors_idx]
    return oracle.reconstruct(w.speed, w.dx, w.origin, sens, sig, w.dt, w.mask, T=T)


def gpu_images(w, sensors_idx=None, flags=0, signals=None, dtype="f32"):
    sens = w.sensors if sensors_idx is None else w.sensors[sensors_idx]
    sig = w.signals if signals is None else signals
    if sensors_idx is not None:
        sig = sig[:, sensors_idx]
    with BP(w.speed, w.dx, w.origin, sens, w.dt, w.nt, mask=w.mask, flags=flags) as bp:
        if dtype == "f32":
            s = torch.from_numpy(np.ascontiguousarray(sig, dtype=np.float32)).cuda()
            out = bp.reconstruct(s)
        else:
            codes, sc, _ = synth.quantise(sig, dtype)
            tdt = torch.bfloat16 if dtype == "bf16" else torch.float16
            s = torch.from_numpy(codes.astype(np.int16)).cuda().view(tdt)
            out = bp.reconstruct(s, scales=torch.from_numpy(sc).cuda())
        bp.sync()
        return out.cpu().numpy().astype(np.float64), dict(bp.info)


def assert_fp32_parity(got, ref, p0max):
    for f in range(ref.shape[0]):
        e = rel_l2(got[f], ref[f])
        m = np.abs(got[f] - ref[f]).max()
        assert e <= FP32_REL_L2, f"frame {f}: rel-L2 {e:.3e}"
        assert m <= FP32_MAX_ABS_FRAC * p0max, f"frame {f}: max-abs {m:.3e}"


def test_config1_fp32_parity():
    w = synth.config1(n_frames=2)
    ref = oracle_images(w, "c1")
    got, info = gpu_images(w)
    assert_fp32_parity(got, ref, np.abs(w.p0).max())
    outside = ~w.mask.astype(bool)
    assert np.all(got[:, outside] == 0.0)


def test_config2_fp32_parity_full_size():
    """Paper-shaped frame (512 sensors, 21 323 pixels) in the launch shape the
    benchmark times: the whole image against the oracle."""
    w = synth.config2(n_frames=1)
    ref = oracle_images(w, "c2")
    got, info = gpu_images(w)
    assert info["n_pix"] == 21323
    assert_fp32_parity(got, ref, np.abs(w.p0).max())


def test_config2_tile256_and_compact():
    w = synth.config2(n_frames=1, n_lines=3)
    sub = np.arange(0, 512, 5)
    ref = oracle_images(w, "c2_sub5", sensors_idx=sub)
    got, info = gpu_images(w, sensors_idx=sub, flags=_lib.PAT_FLAG_TILE_256)
    assert info["tile_pix"] == 256
    assert_fp32_parity(got, ref, np.abs(w.p0).max())
    gc, _ = gpu_images(w, sensors_idx=sub, flags=_lib.PAT_FLAG_COMPACT_OUT)
    pix = np.flatnonzero(w.mask.ravel())
    assert_fp32_parity(gc, ref.reshape(1, -1)[:, pix], np.abs(w.p0).max())


@pytest.mark.parametrize("ns,nt,F,shape,hole", [
    (1, 2, 1, (9, 7), False),
    (5, 3, 3, (20, 33), True),
    (37, 101, 9, (40, 45), True),
    (67, 640, 5, (64, 64), False),
    (13, 257, 2, (11, 13, 9), True),
])
def test_ragged_and_degenerate_shapes(ns, nt, F, shape, hole):
    """Sensor counts that are not multiples of the stage, records of 2-3
    samples, frame counts that leave partial frame groups, masks with holes,
    2-D and 3-D, single-tile and many-tile grids."""
    rng = np.random.default_rng(ns * 1000 + nt)
    dx = 1e-4
    origin = synth.centred_origin(shape, dx)
    speed = rng.uniform(1400, 3000, shape).astype(np.float32)
    half = np.array([(n - 1) / 2 * dx for n in shape[::-1]])
    sens = np.zeros((ns, 3))
    sens[:, : len(shape)] = rng.uniform(-0.9, 0.9, (ns, len(shape))) * half
    mask = (rng.uniform(0, 1, shape) < (0.7 if hole else 1.0)).astype(np.uint8)
    mask.ravel()[0] = 1
    # a record long enough that most, not all, arrivals fall inside it
    tmax = 2 * np.linalg.norm(half) / 1400
    dt = tmax / max(nt - 1, 1) * 0.6
    t = np.arange(nt) * dt
    sig = (rng.standard_normal((F, ns, nt)) * 0.1 +
           np.sin(t[None, None, :] * 3e6 + rng.uniform(0, 6, (F, ns, 1)))).astype(np.float32)
    w = synth.Workload("rag", speed, dx, origin, sens, mask, dt, nt, sig,
                       np.ones((F,) + shape, np.float32))
    ref = oracle_images(w, f"rag_{ns}_{nt}_{shape}")
    got, _ = gpu_images(w)
    scale = np.abs(ref).max()
    for f in range(F):
        assert rel_l2(got[f], ref[f]) <= FP32_REL_L2
        assert np.abs(got[f] - ref[f]).max() <= FP32_MAX_ABS_FRAC * scale
    assert np.all(got[:, ~mask.astype(bool)] == 0.0)
    if F <= 3:
        # frame by frame through the unstaged kernels: the windowed kernel
        # (default) and the one that gathers from L2 give the same bits
        alt, _ = gpu_images(w, flags=_lib.PAT_FLAG_NO_WINDOW)
        assert np.array_equal(got, alt)


def test_3d_volume_small():
    w = synth.config5_subject(1, n_frames=2, n_sensors=24, shape=(24, 40, 40), nt=600)
    ref = oracle_images(w, "c5_small")
    got, _ = gpu_images(w)
    assert_fp32_parity(got, ref, np.abs(w.p0).max())


@pytest.mark.parametrize("dtype,tol_kernel", [("bf16", 2e-3), ("f16", 5e-4)])
def test_config3_low_precision(dtype, tol_kernel):
    """64 frames sharing one table; per-frame error against the oracle on the
    original FP32 signals (the gate) and on the dequantised input (the kernel's
    own arithmetic)."""
    w = synth.config3(n_frames=64)
    ref = oracle_images(w, "c3")
    got, _ = gpu_images(w, dtype=dtype)
    _, _, deq = synth.quantise(w.signals, dtype)
    ref_q = oracle_images(w, "c3", signals=deq)
    errs = [rel_l2(got[f], ref[f]) for f in range(64)]
    errs_q = [rel_l2(got[f], ref_q[f]) for f in range(64)]
    assert max(errs) <= LOWP_REL_L2, max(errs)
    assert max(errs_q) <= tol_kernel, max(errs_q)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_frame_result_independent_of_batch(dtype):
    """A frame reconstructed alone and inside batches of 3 and 16 frames is
    bit-identical: the summation order is fixed per handle."""
    w = synth.config1(n_frames=16)
    alone = []
    for f in (0, 5, 15):
        g, _ = gpu_images(w, signals=w.signals[f:f + 1], dtype=dtype)
        alone.append(g[0])
    batch, _ = gpu_images(w, dtype=dtype)
    three, _ = gpu_images(w, signals=w.signals[3:6], dtype=dtype)
    for g, f in zip(alone, (0, 5, 15)):
        assert np.array_equal(g, batch[f])
    assert np.array_equal(three[2], batch[5])


def test_host_path_and_split_calls_match_device_path():
    w = synth.config1(n_frames=3)
    with BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) as bp:
        s = torch.from_numpy(w.signals).cuda()
        a = bp.reconstruct(s).cpu().numpy()
        b = bp.reconstruct_host(w.signals)
        bp.preprocess(s)
        out = torch.empty(bp.out_shape(3), device="cuda")
        c = bp.gather(3, out).cpu().numpy()
        d = bp.reconstruct(s).cpu().numpy()
        bp.sync()
    assert np.array_equal(a, b) and np.array_equal(a, c) and np.array_equal(a, d)


def test_linear_signals_give_constant_image_at_full_size():
    """P6 at the paper-shaped size: p_s = alpha_s + beta_s t gives 2p - 2t dp/dt
    = 2 alpha_s, so every pixel whose arrivals all fall in the record equals
    sum_s w_s 2 alpha_s, whatever the table."""
    w = synth.config2(n_frames=1, n_lines=1)
    rng = np.random.default_rng(3)
    # alpha_s = m/16 and slope j * 2^-13 per sample keep every sample, every
    # difference and 2 alpha_s exact in FP32
    al = rng.integers(-16, 17, w.n_sensors) / 16.0
    gam = rng.integers(-3, 4, w.n_sensors) * 2.0 ** -13
    k = np.arange(w.nt)
    sig = (al[:, None] + gam[:, None] * k[None, :])[None].astype(np.float32)
    assert np.array_equal(sig[0].astype(np.float64), al[:, None] + gam[:, None] * k[None, :])
    got, _ = gpu_images(w, signals=sig)
    expect = np.mean(2 * al)
    vals = got[0][w.mask.astype(bool)]
    assert np.abs(vals - expect).max() <= 1e-5


def test_everything_after_the_record_gives_zero():
    w = synth.config1(n_frames=1)
    w.dt = 1e-12  # every arrival lies after the last sample
    got, _ = gpu_images(w)
    assert np.all(got == 0.0)


def test_repeat_is_bitwise_deterministic():
    w = synth.config1(n_frames=4)
    a, _ = gpu_images(w)
    b, _ = gpu_images(w)
    assert np.array_equal(a, b)


def test_bounded_wait_reports_timeout_and_context_survives():
    assert wait_timeout_probe(1_000_000) == _lib.PAT_ERR_TIMEOUT
    w = synth.config1(n_frames=1)
    got, _ = gpu_images(w)
    assert np.isfinite(got).all()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_config5_full_grid_sensor_subset(dtype):
    """The serving volume at full size (160x160x96 voxels at 0.25 mm, all voxels
    reconstructed) with a 16-sensor sub-handle of the 1024-sensor hemisphere:
    every voxel against the oracle."""
    w = synth.config5_subject(3, n_frames=1, n_sensors=1024)
    sub = np.arange(0, 1024, 64)
    ref = oracle_images(w, "c5_full_sub16", sensors_idx=sub)
    got, info = gpu_images(w, sensors_idx=sub, dtype=dtype)
    assert info["n_pix"] == 160 * 160 * 96
    if dtype == "f32":
        assert_fp32_parity(got, ref, np.abs(w.p0).max())
    else:
        assert rel_l2(got[0], ref[0]) <= LOWP_REL_L2


@pytest.mark.parametrize("tile_flag", [0, _lib.PAT_FLAG_TILE_256])
def test_single_frame_unstaged_equals_staged_bitwise(tile_flag):
    """One frame goes through the unstaged gather by default; forcing the
    staged (TMA pipeline) kernel must give the same bits, for every signal
    dtype and both delay sources, with 8 sensor segments per tile."""
    w = synth.config2(n_frames=1, n_lines=3)
    sig = w.signals[:1]
    makers = {
        "table": lambda f: BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask,
                              flags=f | tile_flag),
        "constant": lambda f: BP.constant(1560.0, w.speed.shape, w.dx, w.origin, w.sensors, w.dt,
                                          w.nt, mask=w.mask, flags=f | tile_flag),
    }
    for kind, make in makers.items():
        with make(0) as a, make(_lib.PAT_FLAG_STAGED_SINGLE) as b, \
                make(_lib.PAT_FLAG_NO_WINDOW) as c:
            assert a.info["split"] == 8
            if kind == "table" and tile_flag != _lib.PAT_FLAG_TILE_256:
                # every window fits a slot: the default takes the windowed kernel
                assert a.info["window"] <= 288
            for dtype in ("f32", "bf16", "f16"):
                if dtype == "f32":
                    s = torch.from_numpy(np.ascontiguousarray(sig)).cuda()
                    sc = None
                else:
                    codes, scl, _ = synth.quantise(sig, dtype)
                    tdt = torch.bfloat16 if dtype == "bf16" else torch.float16
                    s = torch.from_numpy(codes.astype(np.int16)).cuda().view(tdt)
                    sc = torch.from_numpy(scl).cuda()
                ra = a.reconstruct(s, scales=sc).cpu().numpy()
                rb = b.reconstruct(s, scales=sc).cpu().numpy()
                rc = c.reconstruct(s, scales=sc).cpu().numpy()
                a.sync()
                b.sync()
                c.sync()
                assert np.array_equal(ra, rb), (kind, dtype)
                assert np.array_equal(ra, rc), (kind, dtype)
                assert np.isfinite(ra).all()


def test_single_fp32_frame_host_round_trip_and_split_calls():
    """One FP32 frame: pat_bp_reconstruct forms the integrand inside the
    gather; the host round trip (exactly sized staging buffers), the two-call
    API (preprocessing kernel, then gather) and the staged kernel give the same
    bits, with and without per-row scales."""
    w = synth.config2(n_frames=1, n_lines=2)
    sig = np.ascontiguousarray(w.signals[:1])
    sc = np.random.default_rng(4).uniform(0.5, 2.0, (1, w.n_sensors)).astype(np.float32)
    with BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) as bp, \
            BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask,
               flags=_lib.PAT_FLAG_STAGED_SINGLE) as st:
        s = torch.from_numpy(sig).cuda()
        for scales in (None, torch.from_numpy(sc).cuda()):
            a = bp.reconstruct(s, scales=scales).cpu().numpy()
            bp.preprocess(s, scales=scales)
            out = torch.empty(bp.out_shape(1), device="cuda")
            b = bp.gather(1, out).cpu().numpy()
            c = st.reconstruct(s, scales=scales).cpu().numpy()
            bp.sync()
            st.sync()
            assert np.array_equal(a, b) and np.array_equal(a, c)
        h = bp.reconstruct_host(sig)
        assert np.array_equal(h, bp.reconstruct(s).cpu().numpy())


def test_second_order_table_fp32_parity():
    """A handle built with the printed second-order stencil
    (PAT_FLAG_FMM_SECOND_ORDER) against the oracle's order-2 table."""
    w = synth.config1(n_frames=2)
    pix = np.flatnonzero(w.mask.ravel())
    T = travel_table("c1_order2", w.speed, w.dx, w.origin, w.sensors, pix, order=2)
    ref = oracle.reconstruct(w.speed, w.dx, w.origin, w.sensors, w.signals, w.dt, w.mask, T=T)
    got, _ = gpu_images(w, flags=_lib.PAT_FLAG_FMM_SECOND_ORDER)
    assert_fp32_parity(got, ref, np.abs(w.p0).max())
    first, _ = gpu_images(w)
    assert not np.array_equal(first, got)


def test_gather_only_hook():
    """pat_test_gather_only (the benchmark's hook for timing the gather kernel
    alone) refuses a handle without a one-frame preprocess, leaves the image
    alone, and a following gather gives the bits of the whole call."""
    import ctypes
    w = synth.config2(n_frames=1, n_lines=2)
    with BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) as bp:
        st = torch.cuda.current_stream()
        sp = ctypes.c_void_p(st.cuda_stream)
        assert bp._lib.pat_test_gather_only(bp._h, sp) == _lib.PAT_ERR_INVALID
        sig = torch.from_numpy(w.signals).cuda()
        ref = bp.reconstruct(sig).cpu().numpy()
        out = torch.full(bp.out_shape(1), 7.0, device="cuda")
        bp.preprocess(sig)
        assert bp._lib.pat_test_gather_only(bp._h, sp) == 0
        bp.sync()
        assert bool((out == 7.0).all())
        bp.gather(1, out)
        bp.sync()
        assert np.array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("dt_ns,wmin,wmax", [(40, 1, 128), (25, 129, 192), (18, 193, 288), (12, 289, 4096)])
def test_window_slot_sizes_against_l2_staged_and_oracle(dt_ns, wmin, wmax):
    """The 128^2 geometry sampled at 40, 25, 18 and 12 ns: the table's longest
    window (the largest one tile needs from one sensor) falls in each slot size
    of the windowed single-frame gather (128, 192, 288 rows) and beyond it (the
    L2 gather then runs).  The default path, the L2 gather (PAT_FLAG_NO_WINDOW)
    and the staged kernel give the same bits; the image matches the oracle."""
    w1 = synth.config1(n_frames=1)
    dt = dt_ns * 1e-9
    nt = int(round(w1.nt * w1.dt / dt))
    rng = np.random.default_rng(dt_ns)
    t = np.arange(nt) * dt
    sig = (np.sin(t[None, None, :] * rng.uniform(2e6, 6e6, (1, w1.n_sensors, 1)) +
                  rng.uniform(0, 6, (1, w1.n_sensors, 1))) +
           0.1 * rng.standard_normal((1, w1.n_sensors, nt))).astype(np.float32)
    w = synth.Workload("slots", w1.speed, w1.dx, w1.origin, w1.sensors, w1.mask, dt, nt, sig, w1.p0)
    imgs = {}
    for name, fl in (("default", 0), ("l2", _lib.PAT_FLAG_NO_WINDOW), ("staged", _lib.PAT_FLAG_STAGED_SINGLE)):
        imgs[name], info = gpu_images(w, flags=fl)
        assert wmin <= info["window"] <= wmax, info["window"]
    assert np.array_equal(imgs["default"], imgs["l2"])
    assert np.array_equal(imgs["default"], imgs["staged"])
    ref = oracle_images(w, "c1")
    assert_fp32_parity(imgs["default"], ref, np.abs(ref).max())
