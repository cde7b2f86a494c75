"""Sec. III's robustness study through the GPU path: the skull's speed map
carries an error (independent Gaussian noise per node, mean and spread 1.7 % of the
map's maximum), the table is rebuilt from the wrong map, and the same data are
reconstructed.  The wrong-map image still localises an absorber near the skull
as the true-map image does, and stays better than the constant-speed (1560 m/s)
conventional back projection; both GPU images match the oracle, and a serving
loop holding the true and the wrong subject returns each one's own image."""
import math

import numpy as np
import pytest

import oracle
from helpers import fmm_arrivals
from oracle_pool import travel_table
from paper_1501_03869_gb300 import BP, Server, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_REL_L2 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_03869_gb300.build import build
    build()


def _peak_error(img, p0):
    a = np.unravel_index(np.argmax(img), img.shape)
    b = np.unravel_index(np.argmax(p0), p0.shape)
    return math.hypot(a[0] - b[0], a[1] - b[1])


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("offset_px,seed", [(38, 0), (-36, 1)])
def test_speed_error_keeps_localisation(offset_px, seed):
    w = synth.config1(n_frames=1)
    centre = np.array([[w.origin[0] + (63.5 + offset_px) * w.dx, w.origin[1] + 63.5 * w.dx, 0.0]])
    p = synth.render_signals(w.speed, w.dx, w.origin, w.sensors, centre, [1.5 * w.dx], [1.0], w.dt,
                             w.nt, 0.01, np.random.default_rng(seed), arrivals=fmm_arrivals)
    p0 = synth.phantom_discs(w.speed.shape, w.dx, w.origin, centre, [1.5 * w.dx], [1.0])
    wrong = synth.speed_error(w.speed, np.random.default_rng(100 + seed))
    s = torch.from_numpy(p[None].astype(np.float32)).cuda()
    imgs = {}
    for name, sp in (("true", w.speed), ("wrong", wrong)):
        with BP(sp, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) as bp:
            imgs[name] = bp.reconstruct(s).cpu().numpy()[0].astype(np.float64)
    with BP.constant(1560.0, w.speed.shape, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) as bp:
        imgs["constant"] = bp.reconstruct(s).cpu().numpy()[0].astype(np.float64)
    e = {k: _peak_error(v, p0) for k, v in imgs.items()}
    assert e["true"] <= 1.5 and e["wrong"] <= 1.5 and e["constant"] > 3.0  # absorber radius 1.5 px
    assert imgs["wrong"].max() > 0.6 and imgs["constant"].max() < 0.5
    # the GPU image from the wrong map is the oracle's image from that map
    pix = np.flatnonzero(w.mask.ravel())
    T = travel_table(f"c1_wrong_{seed}", wrong, w.dx, w.origin, w.sensors, pix)
    ref = np.zeros(w.speed.size)
    ref[pix] = oracle.bp(T, p, w.dt)
    assert _rel(imgs["wrong"].ravel(), ref) <= FP32_REL_L2


def test_serving_holds_true_and_wrong_subjects():
    w = synth.config1(n_frames=3)
    wrong = synth.speed_error(w.speed, np.random.default_rng(7))
    singles = []
    for sp in (w.speed, wrong):
        with BP(sp, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) as bp:
            singles.append([bp.reconstruct(torch.from_numpy(w.signals[f:f + 1]).cuda()).cpu().numpy()[0]
                            for f in range(3)])
    srv = Server(hbm_budget=1 << 30, n_streams=2, max_batch_frames=2)
    ids = [srv.register(sp, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) for sp in (w.speed, wrong)]
    jobs = []
    for f in range(3):
        for k in (0, 1):
            out = np.empty(w.speed.shape, np.float32)
            jobs.append((srv.submit(ids[k], w.signals[f], out), out, k, f))
    for t, out, k, f in jobs:
        srv.wait(t)
        assert np.array_equal(out, singles[k][f])
    assert not np.array_equal(singles[0][0], singles[1][0])
    srv.close()
