"""GPU checks of the multi-instance persistent form on the uneven workload
(32 instances: grids 96^2-384^2, 128-1024 sensors, 1024-4096 samples, 1-16
frames).  Every instance's image must be bit-identical to its own single-handle
reconstruction (the plan never changes a pixel's summation order), whatever
the tuned launch shape, the graph replay or the other instances; the cheapest
instances are also checked against the FP64 oracle at full size."""
import numpy as np
import pytest

import oracle
from oracle_pool import travel_table
from paper_1501_03869_gb300 import BP, Plan, reconstruct_multi, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_REL_L2 = 1e-5
FP32_MAX_ABS_FRAC = 1e-4


@pytest.fixture(scope="module")
def c4():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ws = [synth.config4_instance(i) for i in range(32)]
    bps = [BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) for w in ws]
    sig = [torch.from_numpy(w.signals).cuda() for w in ws]
    single = []
    for bp, s in zip(bps, sig):
        single.append(bp.reconstruct(s).cpu().numpy())
    for bp in bps:
        bp.sync()
    yield ws, bps, sig, single
    for bp in bps:
        bp.close()


def _outs(bps, ws):
    return [torch.full(bp.out_shape(w.n_frames), float("nan"), device="cuda") for bp, w in zip(bps, ws)]


def test_plan_tuned_graph_matches_single_handles(c4):
    ws, bps, sig, single = c4
    plan = Plan(bps, [w.n_frames for w in ws], autotune=True, graph=True)
    outs = _outs(bps, ws)
    plan.execute(sig, outs)
    plan.sync()
    info = plan.info
    assert info["tuned"] == 1 and info["graph"] == 1 and info["n_inst"] == 32
    # one class per frames-per-unit value the instances' frame counts give
    fbs = {min(8, 1 << (w.n_frames.bit_length() - 1)) for w in ws}
    assert info["n_classes"] == len(fbs) and info["fb_mask"] == sum(fbs)
    assert info["frames_per_unit"] == max(fbs)
    for i, o in enumerate(outs):
        assert np.array_equal(o.cpu().numpy(), single[i]), f"instance {i}"
    # replay with other inputs: every pointer is refreshed in the graph
    sig2 = [s.flip(0).contiguous() for s in sig]
    outs2 = _outs(bps, ws)
    plan.execute(sig2, outs2)
    plan.sync()
    for i, o in enumerate(outs2):
        assert np.array_equal(o.cpu().numpy(), single[i][::-1]), f"instance {i} (replay)"
    plan.close()


def test_one_shot_multi_and_untuned_plan(c4):
    ws, bps, sig, single = c4
    idx = [3, 7, 15, 21, 30]
    outs = _outs([bps[i] for i in idx], [ws[i] for i in idx])
    reconstruct_multi([bps[i] for i in idx], [sig[i] for i in idx], outs)
    torch.cuda.synchronize()
    for k, i in enumerate(idx):
        assert np.array_equal(outs[k].cpu().numpy(), single[i])
    plan = Plan([bps[i] for i in idx], [ws[i].n_frames for i in idx])
    outs = _outs([bps[i] for i in idx], [ws[i] for i in idx])
    plan.execute([sig[i] for i in idx], outs)
    plan.sync()
    for k, i in enumerate(idx):
        assert np.array_equal(outs[k].cpu().numpy(), single[i])
    plan.close()


def test_bf16_plan_matches_single_handles(c4):
    ws, bps, sig, single = c4
    idx = [0, 9, 12]
    sigq, scq, ref = [], [], []
    for i in idx:
        codes, sc, _ = synth.quantise(ws[i].signals, "bf16")
        s = torch.from_numpy(codes.astype(np.int16)).cuda().view(torch.bfloat16)
        scale = torch.from_numpy(sc).cuda()
        sigq.append(s)
        scq.append(scale)
        ref.append(bps[i].reconstruct(s, scales=scale).cpu().numpy())
    plan = Plan([bps[i] for i in idx], [ws[i].n_frames for i in idx], dtype="bf16", graph=True)
    outs = _outs([bps[i] for i in idx], [ws[i] for i in idx])
    plan.execute(sigq, outs, scales=scq)
    plan.sync()
    for k in range(len(idx)):
        assert np.array_equal(outs[k].cpu().numpy(), ref[k])
    plan.close()


def test_cheapest_instances_match_oracle(c4):
    ws, bps, sig, single = c4
    cost = sorted((w.n_sensors * w.speed.size, i) for i, w in enumerate(ws))
    for _, i in cost[:3]:
        w = ws[i]
        pix = np.flatnonzero(w.mask.ravel())
        T = travel_table(f"c4_{i}", w.speed, w.dx, w.origin, w.sensors, pix)
        ref = oracle.reconstruct(w.speed, w.dx, w.origin, w.sensors, w.signals, w.dt, w.mask, T=T)
        p0 = np.abs(w.p0).max()
        for f in range(w.n_frames):
            e = np.linalg.norm(single[i][f] - ref[f]) / np.linalg.norm(ref[f])
            assert e <= FP32_REL_L2, (i, f, e)
            assert np.abs(single[i][f] - ref[f]).max() <= FP32_MAX_ABS_FRAC * p0


def test_plan_follows_evict_restore_and_refuses_changed_weights():
    """A plan's descriptors follow its handles' buffers: after an eviction and
    a restore (which reallocate the table) the plan, graph-replayed, still
    gives the single-handle bits; a handle switched to solid-angle weights
    after the plan was made is refused instead of being read in the old mode."""
    import math
    from paper_1501_03869_gb300 import PatError, _lib
    a = synth.config1(n_frames=2)
    b = synth.config1(n_frames=3, inst=1, cfg_id=7)
    ha = BP(a.speed, a.dx, a.origin, a.sensors, a.dt, a.nt, a.mask, flags=_lib.PAT_FLAG_HOST_MIRROR)
    hb = BP(b.speed, b.dx, b.origin, b.sensors, b.dt, b.nt, b.mask)
    sa, sb = torch.from_numpy(a.signals).cuda(), torch.from_numpy(b.signals).cuda()
    ref_a, ref_b = ha.reconstruct(sa).cpu().numpy(), hb.reconstruct(sb).cpu().numpy()
    plan = Plan([ha, hb], [2, 3], graph=True)
    for rep in range(3):
        if rep == 1:
            ha.evict()
            junk = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")  # move the allocator on
            ha.restore()
            del junk
        outs = [torch.empty(s, dtype=torch.float32, device="cuda") for s in plan.out_shapes()]
        plan.execute([sa, sb], outs)
        plan.sync()
        assert np.array_equal(outs[0].cpu().numpy(), ref_a)
        assert np.array_equal(outs[1].cpu().numpy(), ref_b)
    nrm = -a.sensors / np.linalg.norm(a.sensors, axis=1, keepdims=True)
    elem = np.full(a.sensors.shape[0], 2 * math.pi * np.linalg.norm(a.sensors[0]) / a.sensors.shape[0])
    ha.set_solid_angle(nrm, elem, 2 * math.pi)
    outs = [torch.empty(s, dtype=torch.float32, device="cuda") for s in plan.out_shapes()]
    with pytest.raises(PatError):
        plan.execute([sa, sb], outs)
    plan.close()
    ha.close()
    hb.close()


def test_tile256_tuned_graph_plan_matches_single_handles_and_oracle():
    """The uneven workload with 256-pixel tiles (the benchmark's form): a tuned,
    graph-replayed plan over every instance gives each instance the bits of its
    own single-handle reconstruction; the cheapest instance matches the oracle."""
    from paper_1501_03869_gb300 import _lib
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ws = [synth.config4_instance(i) for i in range(32)]
    bps = [BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask,
              flags=_lib.PAT_FLAG_TILE_256) for w in ws]
    try:
        sig = [torch.from_numpy(w.signals).cuda() for w in ws]
        single = [bp.reconstruct(s).cpu().numpy() for bp, s in zip(bps, sig)]
        plan = Plan(bps, [w.n_frames for w in ws], autotune=True, graph=True)
        outs = _outs(bps, ws)
        plan.execute(sig, outs)
        plan.sync()
        assert bps[0].info["tile_pix"] == 256 and plan.info["graph"] == 1
        for i, o in enumerate(outs):
            assert np.array_equal(o.cpu().numpy(), single[i]), f"instance {i}"
        plan.close()
        i = min(range(32), key=lambda k: ws[k].n_frames * ws[k].n_sensors * ws[k].n_pix)
        w = ws[i]
        pix = np.flatnonzero(w.mask.ravel())
        T = travel_table(f"c4_{i}", w.speed, w.dx, w.origin, w.sensors, pix)
        ref = oracle.reconstruct(w.speed, w.dx, w.origin, w.sensors, w.signals, w.dt, w.mask, T=T)
        p0 = np.abs(w.p0).max()
        for f in range(w.n_frames):
            got = single[i][f].astype(np.float64).ravel()
            r = ref[f].ravel()
            assert np.linalg.norm(got - r) / np.linalg.norm(r) <= FP32_REL_L2
            assert np.abs(got - r).max() <= FP32_MAX_ABS_FRAC * p0
    finally:
        for bp in bps:
            bp.close()
