"""The entry point that allocates no device memory (pat_bp_reconstruct_noalloc).

It serves callers that may not allocate device memory: hosts that own all
device memory in their own pool, and per-frame loops that must not call the
CUDA allocator.  Its scratch lives in a fixed 16 MiB device array shared by
every call.  It runs the same kernels with the same launch shape and summation
order as pat_bp_reconstruct, so on two calls in a row with different frames
its images must equal pat_bp_reconstruct's bit for bit (FP32 and BF16
signals; stale scratch left by an earlier call on another handle would show
up as changed bits); one call is also compared with the FP64 oracle at the
FP32 tolerances of the other parity tests (rel-L2 <= 1e-5, max-abs <=
1e-4 max|p0|).  A reconstruction whose scratch would not fit is refused.
This file is collected last so that a stop-at-first-failure run has already
run every other test; it passes alone in a fresh process too.
"""
import numpy as np
import pytest

import oracle
from paper_1501_03869_gb300 import BP, PatError, _lib, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_REL_L2 = 1e-5
FP32_MAX_ABS_FRAC = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_03869_gb300.build import build
    build()


def _inputs(sig, dtype):
    if dtype == "f32":
        return torch.from_numpy(np.ascontiguousarray(sig, dtype=np.float32)).cuda(), None
    codes, sc, _ = synth.quantise(sig, "bf16")
    return (torch.from_numpy(codes.astype(np.int16)).cuda().view(torch.bfloat16),
            torch.from_numpy(sc).cuda())


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("cfg", ["c1", "c2"])
def test_noalloc_equals_reconstruct_on_two_calls(cfg, dtype):
    w = synth.config1(n_frames=4) if cfg == "c1" else synth.config2(n_frames=2, n_lines=4)
    # another handle's call first, so the shared array holds stale contents
    other = synth.config1(n_frames=3, inst=2, cfg_id=7)
    with BP(other.speed, other.dx, other.origin, other.sensors, other.dt, other.nt,
            mask=other.mask) as bo:
        s, sc = _inputs(other.signals, dtype)
        bo.reconstruct_noalloc(s, torch.empty(bo.out_shape(3), device="cuda"), scales=sc)
        bo.sync()
    with BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) as bp:
        calls = [w.signals[:2], w.signals[2:]] if cfg == "c1" else [w.signals[:1], w.signals[1:]]
        for sig in calls:
            s, sc = _inputs(sig, dtype)
            ref = bp.reconstruct(s, scales=sc).cpu().numpy()
            out = torch.full(bp.out_shape(s.shape[0]), float("nan"), device="cuda")
            bp.reconstruct_noalloc(s, out, scales=sc)
            bp.sync()
            assert np.array_equal(out.cpu().numpy(), ref)


def test_noalloc_matches_oracle():
    w = synth.config1(n_frames=2)
    ref = oracle.reconstruct(w.speed, w.dx, w.origin, w.sensors, w.signals, w.dt, w.mask)
    with BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) as bp:
        s = torch.from_numpy(w.signals).cuda()
        out = torch.full(bp.out_shape(2), float("nan"), device="cuda")
        bp.reconstruct_noalloc(s, out)
        bp.sync()
        got = out.cpu().numpy().astype(np.float64)
    p0 = np.abs(w.p0).max()
    for f in range(2):
        e = np.linalg.norm(got[f] - ref[f]) / np.linalg.norm(ref[f])
        assert e <= FP32_REL_L2, f"frame {f}: rel-L2 {e:.3e}"
        assert np.abs(got[f] - ref[f]).max() <= FP32_MAX_ABS_FRAC * p0


def test_noalloc_rejects_scratch_beyond_its_array():
    w = synth.config2(n_frames=1, n_lines=1)
    with BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) as bp:
        s = torch.zeros((8, w.n_sensors, w.nt), device="cuda")
        out = torch.empty(bp.out_shape(8), device="cuda")
        with pytest.raises(PatError) as e:
            bp.reconstruct_noalloc(s, out)
        assert e.value.status == _lib.PAT_ERR_INVALID
        assert "bytes of scratch" in str(e.value)
