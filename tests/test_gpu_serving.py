"""GPU checks of the serving loop: results equal single reconstructions bit
for bit (whatever the batching, the other subjects and the evictions), LRU
eviction under a small HBM budget, and host-side failure paths (unknown
subject or ticket, full queue, budget that can never fit, a stalled
scheduler) -- all made on the host, none faulting the GPU."""
import time

import numpy as np
import pytest

from paper_1501_03869_gb300 import BP, PatError, Server, _lib, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _subjects():
    a = synth.config1(n_frames=6)
    b = synth.config1(n_frames=6, inst=1, cfg_id=7)
    c = synth.config5_subject(2, n_frames=4, n_sensors=48, shape=(24, 40, 40), nt=512)
    return [a, b, c]


@pytest.fixture(scope="module")
def subjects():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ws = _subjects()
    refs = []
    for w in ws:
        with BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) as bp:
            alone = [bp.reconstruct(torch.from_numpy(w.signals[f:f + 1]).cuda()).cpu().numpy()[0]
                     for f in range(w.n_frames)]
            bp.sync()
        refs.append(alone)
    return ws, refs


def _register(srv, ws):
    return [srv.register(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) for w in ws]


def test_mixed_stream_is_bitwise_equal_to_alone(subjects):
    ws, refs = subjects
    # a 2 ms scheduler cycle lets requests pile up between admissions, so the
    # stream mixes single and batched frames of all subjects
    srv = Server(hbm_budget=8 << 30, n_streams=3, max_batch_frames=4, stall_us=2000)
    ids = _register(srv, ws)
    jobs = []
    rng = np.random.default_rng(0)
    order = [(k, f) for k in range(3) for f in range(ws[k].n_frames)] * 3
    rng.shuffle(order)
    for i, (k, f) in enumerate(order):
        out = np.full(ws[k].speed.shape, np.nan, dtype=np.float32)
        jobs.append((srv.submit(ids[k], ws[k].signals[f], out), out, k, f))
        if i % 5 == 4:
            time.sleep(0.0005)  # arrivals while earlier batches run
    for t, out, k, f in jobs:
        srv.wait(t)
        assert np.array_equal(out, refs[k][f]), (k, f)
    st = srv.stats()
    assert st["completed"] == len(order) and st["failed"] == 0
    assert st["batches"] < len(order)  # frames were batched
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    srv.close()


def test_lru_eviction_under_small_budget(subjects):
    ws, refs = subjects
    # room for about one config-1 subject at a time
    srv = Server(hbm_budget=3 << 20, n_streams=2, max_batch_frames=2)
    ids = _register(srv, ws[:2])
    jobs = []
    for rep in range(3):
        for k in (0, 1):
            out = np.empty(ws[k].speed.shape, dtype=np.float32)
            jobs.append((srv.submit(ids[k], ws[k].signals[rep], out), out, k, rep))
            srv.wait(jobs[-1][0])
    for t, out, k, f in jobs:
        assert np.array_equal(out, refs[k][f])
    st = srv.stats()
    assert st["evictions"] >= 2 and st["uploads"] >= 3
    assert st["resident_bytes"] <= st["budget_bytes"]
    srv.close()


def test_bf16_requests(subjects):
    ws, _ = subjects
    w = ws[0]
    codes, sc, _ = synth.quantise(w.signals, "bf16")
    with BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask) as bp:
        ref = [bp.reconstruct(torch.from_numpy(codes[f:f + 1].astype(np.int16)).cuda().view(torch.bfloat16),
                              scales=torch.from_numpy(sc[f:f + 1]).cuda()).cpu().numpy()[0]
               for f in range(3)]
    srv = Server(hbm_budget=1 << 30)
    sid = _register(srv, [w])[0]
    outs = [np.empty(w.speed.shape, np.float32) for _ in range(3)]
    ts = [srv.submit(sid, codes[f], outs[f], dtype="bf16", scales=sc[f]) for f in range(3)]
    for f, t in enumerate(ts):
        srv.wait(t)
        assert np.array_equal(outs[f], ref[f])
    srv.close()


def test_host_side_failures(subjects):
    ws, _ = subjects
    w = ws[0]
    srv = Server(hbm_budget=1 << 30, max_queue=2, stall_us=200000)
    sid = _register(srv, [w])[0]
    out = np.empty(w.speed.shape, np.float32)
    with pytest.raises(PatError) as e:
        srv.submit(sid + 5, w.signals[0], out)
    assert e.value.status == _lib.PAT_ERR_NOT_FOUND
    t1 = srv.submit(sid, w.signals[0], out)
    out2 = np.empty_like(out)
    srv.submit(sid, w.signals[1], out2)
    # the stalled scheduler has not admitted them yet: the queue is full
    with pytest.raises(PatError) as e:
        srv.submit(sid, w.signals[2], np.empty_like(out))
    assert e.value.status == _lib.PAT_ERR_BUSY
    assert srv.poll(t1, 0)[0] == _lib.PAT_PENDING
    srv.wait(t1)
    assert srv.poll(t1, 0)[0] == _lib.PAT_ERR_NOT_FOUND  # reported once
    srv.close()
    tiny = Server(hbm_budget=1 << 16)
    sid = _register(tiny, [w])[0]
    t = tiny.submit(sid, w.signals[0], out)
    st, _ = tiny.poll(t, 20_000_000)
    assert st == _lib.PAT_ERR_OOM
    tiny.close()


def test_subject_with_gpu_table(subjects):
    """A subject registered with its table solved on the GPU (PAT_FLAG_GPU_TABLE)
    serves the bits of a handle built the same way; the GPU-built table agrees
    with the host-built one to rounding, so the images agree to ~1e-6."""
    ws, refs = subjects
    w = ws[0]
    with BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask,
            flags=_lib.PAT_FLAG_GPU_TABLE) as bp:
        ref = [bp.reconstruct(torch.from_numpy(w.signals[f:f + 1]).cuda()).cpu().numpy()[0]
               for f in range(3)]
        bp.sync()
    srv = Server(hbm_budget=1 << 30, max_batch_frames=4)
    sid = srv.register(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, mask=w.mask,
                       flags=_lib.PAT_FLAG_GPU_TABLE)
    outs = [np.empty(w.speed.shape, np.float32) for _ in range(3)]
    ts = [srv.submit(sid, w.signals[f], outs[f]) for f in range(3)]
    for f, t in enumerate(ts):
        srv.wait(t)
        assert np.array_equal(outs[f], ref[f])
        host = refs[0][f]
        assert np.linalg.norm(outs[f] - host) <= 1e-6 * np.linalg.norm(host)
    srv.close()
