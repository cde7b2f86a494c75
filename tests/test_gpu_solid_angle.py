"""GPU parity of the exact back projection (pat_bp_set_solid_angle) against the
FP64 oracle: Eq. (BP) with every term weighted by the share of the full angle
that the sensor's element subtends at the pixel (Sec. II-C: Eq. (BP)
approximates that exact form for a circular scan of large radius).  The
weights are evaluated in the gather kernel; the oracle forms them from their
definition (oracle.solid_angle_weights) and sums with oracle.bp.

Arrays: the paper-shaped ring of C1, a non-circular (elliptical) ring with
unequal elements on the skull map, and the 3-D hemisphere of the serving
subject through the constant-speed path.  Tolerances are those of the
stored-table path (FP32 rel-L2 <= 1e-5 and max-abs <= 1e-4 of the image's
peak, 16-bit rel-L2 <= 5e-3 on the FP32 signals); frame batching (the staged
kernel) against single frames (the unstaged one), plans, eviction and the
no-allocation entry are checked bit for bit.
"""
import math

import numpy as np
import pytest

import oracle
from oracle_pool import travel_table
from paper_1501_03869_gb300 import BP, PatError, Plan, _lib, synth

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


def ring_geometry(sensors):
    """Inward normals and equal arc elements of a ring centred at 0."""
    n = sensors.shape[0]
    R = float(np.linalg.norm(sensors[0, :2]))
    nrm = -sensors / np.linalg.norm(sensors, axis=1, keepdims=True)
    return nrm, np.full(n, 2.0 * math.pi * R / n)


def ellipse_array(n, a, b):
    """Sensors on an ellipse at equal parameter steps: unequal elements and
    normals that are not radial."""
    th = 2.0 * math.pi * (np.arange(n) + 0.5) / n
    sens = np.stack([a * np.cos(th), b * np.sin(th), np.zeros(n)], axis=1)
    out_n = np.stack([b * np.cos(th), a * np.sin(th), np.zeros(n)], axis=1)
    elem = np.hypot(a * np.sin(th), b * np.cos(th)) * 2.0 * math.pi / n
    return sens, -out_n, elem


def oracle_images(speed_shape, dx, origin, mask, sensors, nrm, elem, omega0, T, sig, dt):
    pix = np.flatnonzero(mask.ravel()) if mask is not None else np.arange(int(np.prod(speed_shape)))
    W = oracle.solid_angle_weights(speed_shape, dx, origin, sensors, nrm, elem, omega0, pix)
    out = np.zeros((sig.shape[0], int(np.prod(speed_shape))))
    for f in range(sig.shape[0]):
        out[f, pix] = oracle.bp(T, sig[f], dt, W)
    return out.reshape((sig.shape[0],) + tuple(speed_shape)), W


def check_fp32(img, ref):
    for f in range(ref.shape[0]):
        assert rel_l2(img[f], ref[f]) <= FP32_REL_L2
        assert np.abs(img[f] - ref[f]).max() <= FP32_MAX_ABS_FRAC * np.abs(ref[f]).max()


def test_ring_table_handle_matches_oracle():
    w = synth.config1(n_frames=2)
    nrm, elem = ring_geometry(w.sensors)
    pix = np.flatnonzero(w.mask.ravel())
    T = travel_table("c1", w.speed, w.dx, w.origin, w.sensors, pix)
    ref, W = oracle_images(w.speed.shape, w.dx, w.origin, w.mask, w.sensors, nrm, elem,
                           2.0 * math.pi, T, w.signals, w.dt)
    # inside the closed ring the weights of a pixel sum to 1 (the oracle's pin)
    assert np.abs(W.sum(axis=0) - 1.0).max() < 1e-6
    with BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, w.mask) as bp:
        assert bp.info["solid_angle"] == 0
        bp.set_solid_angle(nrm, elem, 2.0 * math.pi)
        assert bp.info["solid_angle"] == 1
        img = run(bp, w.signals)
    check_fp32(img, ref)
    assert np.all(img[:, w.mask == 0] == 0.0)


def test_elliptical_array_on_the_skull_map():
    """A non-circular array on C1's skull map: sensors on an ellipse (semi-axes
    60 and 54 pixels, outside the skull), signals rendered along straight rays."""
    base = synth.config1(n_frames=1)
    dx, origin = base.dx, base.origin
    sens, nrm, elem = ellipse_array(96, 60.0 * dx, 54.0 * dx)
    rng = synth.rng_for(41, 0, 0, 2)
    c = np.array([[4.0 * dx, -6.0 * dx, 0.0], [-10.0 * dx, 5.0 * dx, 0.0], [1.0 * dx, 20.0 * dx, 0.0]])
    sig = synth.render_signals(base.speed, dx, origin, sens, c, np.full(3, 2.0 * dx),
                               np.array([1.0, 0.7, 0.5]), base.dt, base.nt, 0.01, rng)[None]
    mask = (synth.node_radius_px(base.speed.shape) < 40.0).astype(np.uint8)
    pix = np.flatnonzero(mask.ravel())
    T = travel_table("c1_ellipse", base.speed, dx, origin, sens, pix)
    ref, W = oracle_images(base.speed.shape, dx, origin, mask, sens, nrm, elem, 2.0 * math.pi, T,
                           sig, base.dt)
    assert np.abs(W.sum(axis=0) - 1.0).max() < 1e-6
    with BP(base.speed, dx, origin, sens, base.dt, base.nt, mask) as bp:
        bp.set_solid_angle(nrm, elem, 2.0 * math.pi)
        img = run(bp, sig)
        img_bf16 = run(bp, sig, "bf16")
    check_fp32(img, ref)
    assert rel_l2(img_bf16[0], ref[0]) <= LOWP_REL_L2
    # the weights matter here: uniform weights give a different image
    with BP(base.speed, dx, origin, sens, base.dt, base.nt, mask) as bp:
        plain = run(bp, sig)
    assert rel_l2(plain[0], ref[0]) > 100 * FP32_REL_L2


def test_hemisphere_constant_speed_3d():
    """The serving subject's hemisphere (scaled to 34 x 54 x 54) through the
    constant-speed path, weights over the half space (omega0 = 2 pi)."""
    w = synth.config5_subject(0, n_frames=1, n_sensors=192, shape=(34, 54, 54), nt=1024)
    s = w.speed.shape[2] / 160.0
    centre = np.array([79.5 * s, 79.5 * s, 8.0 * s]) * w.dx
    R = 76.0 * s * w.dx
    nrm = (centre[None, :] - w.sensors) / R
    elem = np.full(w.sensors.shape[0], 2.0 * math.pi * R * R / w.sensors.shape[0])
    c0 = 1540.0
    pix = np.flatnonzero(w.mask.ravel())
    T = oracle.constant_table(w.speed.shape, w.dx, w.origin, w.sensors, pix, c0)
    ref, _ = oracle_images(w.speed.shape, w.dx, w.origin, w.mask, w.sensors, nrm, elem,
                           2.0 * math.pi, T, w.signals, w.dt)
    with BP.constant(c0, w.speed.shape, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) as bp:
        bp.set_solid_angle(nrm, elem, 2.0 * math.pi)
        img = run(bp, w.signals)
    check_fp32(img, ref)


def test_batched_frames_equal_single_frames_bitwise():
    """Frames in batches take the staged kernel (the weight anchors copied into
    each stage), single frames the unstaged one; both evaluate the weights with
    the same function and sum in the same order, so every frame has the same
    bits alone, in a batch of 3 or 8, through the no-allocation entry, and with
    PAT_FLAG_STAGED_SINGLE -- for table and constant-speed handles, FP32 and BF16."""
    w = synth.config1(n_frames=8)
    nrm, elem = ring_geometry(w.sensors)
    makers = [lambda fl: BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, w.mask, flags=fl),
              lambda fl: BP.constant(1560.0, w.speed.shape, w.dx, w.origin, w.sensors, w.dt, w.nt,
                                     mask=w.mask, flags=fl)]
    for make in makers:
        for dtype in ("f32", "bf16"):
            with make(0) as bp:
                bp.set_solid_angle(nrm, elem, 2.0 * math.pi)
                all8 = run(bp, w.signals, dtype)
                three = run(bp, w.signals[:3], dtype)
                singles = [run(bp, w.signals[f:f + 1], dtype)[0] for f in range(8)]
                if dtype == "f32":
                    s3 = torch.from_numpy(np.ascontiguousarray(w.signals[:3], dtype=np.float32)).cuda()
                    out = torch.empty((3,) + w.speed.shape, dtype=torch.float32, device="cuda")
                    bp.reconstruct_noalloc(s3, out=out)
                    bp.sync()
                    assert np.array_equal(out.cpu().numpy().astype(np.float64), three)
            for f in range(8):
                assert np.array_equal(all8[f], singles[f])
            for f in range(3):
                assert np.array_equal(three[f], singles[f])
            with make(_lib.PAT_FLAG_STAGED_SINGLE) as bp:
                bp.set_solid_angle(nrm, elem, 2.0 * math.pi)
                staged1 = run(bp, w.signals[:1], dtype)
            assert np.array_equal(staged1[0], singles[0])


def test_plan_of_weighted_handles_equals_the_handles():
    w = synth.config1(n_frames=4)
    sens2, nrm2, elem2 = ellipse_array(80, 60.0 * w.dx, 56.0 * w.dx)
    nrm, elem = ring_geometry(w.sensors)
    a = BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, w.mask).set_solid_angle(nrm, elem, 2 * math.pi)
    b = BP(w.speed, w.dx, w.origin, sens2, w.dt, w.nt, w.mask).set_solid_angle(nrm2, elem2, 2 * math.pi)
    rng = np.random.default_rng(5)
    sig_b = rng.standard_normal((2, 80, w.nt)).astype(np.float32)
    ref_a, ref_b = run(a, w.signals), run(b, sig_b)
    plan = Plan([a, b], [4, 2])
    outs = [torch.empty(s, dtype=torch.float32, device="cuda") for s in plan.out_shapes()]
    plan.execute([torch.from_numpy(np.ascontiguousarray(w.signals, dtype=np.float32)).cuda(),
                  torch.from_numpy(sig_b).cuda()], outs)
    plan.sync()
    assert np.array_equal(outs[0].cpu().numpy().astype(np.float64), ref_a)
    assert np.array_equal(outs[1].cpu().numpy().astype(np.float64), ref_b)
    plan.close()
    with BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, w.mask) as plain:
        with pytest.raises(PatError):
            Plan([a, plain], [1, 1])
    a.close()
    b.close()


def test_eviction_keeps_the_weights():
    w = synth.config1(n_frames=1)
    nrm, elem = ring_geometry(w.sensors)
    with BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, w.mask,
            flags=_lib.PAT_FLAG_HOST_MIRROR) as bp:
        bp.set_solid_angle(nrm, elem, 2.0 * math.pi)
        a = run(bp, w.signals)
        bp.evict()
        bp.restore()
        b = run(bp, w.signals)
    assert np.array_equal(a, b)


def test_bad_arguments_rejected():
    w = synth.config1(n_frames=1)
    nrm, elem = ring_geometry(w.sensors)
    with BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, w.mask) as bp:
        with pytest.raises(PatError):
            bp.set_solid_angle(np.zeros_like(nrm), elem, 2.0 * math.pi)
        with pytest.raises(PatError):
            bp.set_solid_angle(nrm, -elem, 2.0 * math.pi)
        with pytest.raises(PatError):
            bp.set_solid_angle(nrm, elem, 0.0)


def test_hemisphere_table_handle_3d():
    """Weights on a 3-D stored-table handle (pixel terms in node units): the
    scaled serving subject's speed map with 48 sensors on a hemisphere of
    radius 13 voxels inside the grid, the voxels within 10 of its centre,
    against the oracle's fast marching."""
    w = synth.config5_subject(1, n_frames=1, n_sensors=8, shape=(20, 32, 32), nt=512)
    centre = np.array([15.5, 15.5, 2.0]) * w.dx
    R = 13.0 * w.dx
    sens = synth.fibonacci_hemisphere(48, R, centre)
    nrm = (centre[None, :] - sens) / R
    elem = np.full(48, 2.0 * math.pi * R * R / 48)
    rng = synth.rng_for(43, 0, 0, 2)
    c = centre[None, :] + np.array([[2.0, -1.0, 3.0], [-3.0, 2.0, 5.0]]) * w.dx
    sig = synth.render_signals(w.speed, w.dx, w.origin, sens, c, np.full(2, 1.5 * w.dx),
                               np.array([1.0, 0.6]), w.dt, w.nt, 0.01, rng)[None]
    # voxels within 10 of the centre, 3 or more voxels from every element
    mask = (synth.node_radius_px(w.speed.shape, (15.5, 15.5, 2.0)) < 10.0).astype(np.uint8)
    pix = np.flatnonzero(mask.ravel())
    T = travel_table("c5_small_hemi48", w.speed, w.dx, w.origin, sens, pix)
    ref, _ = oracle_images(w.speed.shape, w.dx, w.origin, mask, sens, nrm, elem, 2.0 * math.pi, T,
                           sig, w.dt)
    with BP(w.speed, w.dx, w.origin, sens, w.dt, w.nt, mask) as bp:
        bp.set_solid_angle(nrm, elem, 2.0 * math.pi)
        img = run(bp, sig)
    check_fp32(img, ref)
