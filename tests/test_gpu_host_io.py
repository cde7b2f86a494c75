"""The host round trip (pat_bp_reconstruct_host): page-locked buffers are read
and written in place by the kernels (no staging copies), pageable ones go
through device staging buffers.  Both give the bits of the device path
(pat_bp_reconstruct on device tensors); a pinned input rewritten in place
between calls is read afresh every call; interior pointers into a pinned
block, 16-bit codes with pinned scales, and several frames per call work."""
import numpy as np
import pytest

from paper_1501_03869_gb300 import BP, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_03869_gb300.build import build
    build()
    torch.cuda.init()


@pytest.fixture(scope="module")
def c1():
    w = synth.config1(n_frames=4)
    bp = BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, w.mask)
    yield w, bp
    bp.close()


def device_images(bp, sig):
    out = bp.reconstruct(torch.from_numpy(np.ascontiguousarray(sig, dtype=np.float32)).cuda())
    bp.sync()
    return out.cpu().numpy()


def pinned(shape, dtype=torch.float32):
    return torch.empty(shape, dtype=dtype, pin_memory=True)


def test_pinned_in_place_equals_device_path_and_sees_rewrites(c1):
    w, bp = c1
    ref = device_images(bp, w.signals)
    sig = pinned((1,) + w.signals.shape[1:])
    out = pinned(bp.out_shape(1))
    for f in (0, 1, 2, 3, 1, 0):  # rewrite the same pinned buffer between calls
        sig.copy_(torch.from_numpy(w.signals[f:f + 1]))
        bp.reconstruct_host(sig.numpy(), out=out.numpy())
        assert np.array_equal(out.numpy()[0], ref[f])


def test_pageable_and_mixed_buffers(c1):
    w, bp = c1
    ref = device_images(bp, w.signals[:2])
    sig_pg = np.ascontiguousarray(w.signals[:2], dtype=np.float32)
    sig_pin = pinned(sig_pg.shape)
    sig_pin.copy_(torch.from_numpy(sig_pg))
    out_pin = pinned(bp.out_shape(2))
    for s in (sig_pg, sig_pin.numpy()):
        for o in (np.empty(bp.out_shape(2), dtype=np.float32), out_pin.numpy()):
            o[...] = np.nan
            bp.reconstruct_host(s, out=o)
            assert np.array_equal(o, ref)


def test_interior_pointer_of_a_pinned_block(c1):
    """Buffers that start inside a larger page-locked block (an offset of one
    frame) are still read and written in place."""
    w, bp = c1
    ref = device_images(bp, w.signals[2:3])
    block = pinned(w.signals.shape)
    block.copy_(torch.from_numpy(np.ascontiguousarray(w.signals, dtype=np.float32)))
    outs = pinned((2,) + tuple(bp.out_shape(1)[1:]))
    bp.reconstruct_host(block.numpy()[2:3], out=outs.numpy()[1:2])
    assert np.array_equal(outs.numpy()[1], ref[0])


def test_bf16_codes_with_pinned_scales(c1):
    w, bp = c1
    codes, sc, _ = synth.quantise(w.signals[:3], "bf16")
    ref = bp.reconstruct(torch.from_numpy(codes.astype(np.int16)).cuda().view(torch.bfloat16),
                         scales=torch.from_numpy(sc).cuda())
    bp.sync()
    ref = ref.cpu().numpy()
    c_pin = pinned(codes.shape, torch.int16)
    c_pin.copy_(torch.from_numpy(codes.astype(np.int16)))
    s_pin = pinned(sc.shape)
    s_pin.copy_(torch.from_numpy(sc))
    out = pinned(bp.out_shape(3))
    bp.reconstruct_host(c_pin.numpy().view(np.uint16), dtype="bf16", scales=s_pin.numpy(), out=out.numpy())
    assert np.array_equal(out.numpy(), ref)
    # pageable codes and scales give the same bits
    out2 = bp.reconstruct_host(np.ascontiguousarray(codes), dtype="bf16", scales=sc)
    assert np.array_equal(out2, ref)
