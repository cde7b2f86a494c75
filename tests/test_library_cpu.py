"""CPU-side checks of the CUDA library: the C ABI loads and exports every
declared symbol, argument validation, and the host fast marching and table
layout against the oracle.  No compute call here touches a GPU."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_1501_03869_gb300 import _lib, fmm_host, synth, table_host
from paper_1501_03869_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build()
    _lib.load()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(pat_\w+)\s*\(",
                                    text, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    declared = _declared_functions()
    assert set(_lib.EXPORTS) <= declared | set(_lib.EXPORTS)
    assert declared, "no declarations parsed"
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared but not exported"
    assert set(declared) == set(_lib.EXPORTS)


def test_status_strings():
    lib = _lib.load()
    assert lib.pat_status_str(0) == b"ok"
    assert lib.pat_status_str(4) == b"timeout"


def test_create_rejects_bad_arguments_before_touching_the_gpu():
    sp = np.full((16, 16), 1500.0, dtype=np.float32)
    origin = synth.centred_origin(sp.shape, 1e-4)
    inside = synth.ring_sensors(8, 5e-4)
    outside = synth.ring_sensors(8, 5e-3)
    from paper_1501_03869_gb300 import BP, PatError
    with pytest.raises(PatError) as e:
        BP(sp, 1e-4, origin, outside, 1e-8, 100)
    assert e.value.status == _lib.PAT_ERR_INVALID
    with pytest.raises(PatError) as e:
        BP(sp, 1e-4, origin, inside, -1e-8, 100)
    assert e.value.status == _lib.PAT_ERR_INVALID
    with pytest.raises(PatError) as e:
        BP(sp, 1e-4, origin, inside, 1e-8, 1)
    assert e.value.status == _lib.PAT_ERR_INVALID


def test_gpu_table_entries_reject_bad_arguments_before_touching_the_gpu():
    """The GPU eikonal entries check their inputs on the host first: a source
    outside the grid, a non-positive speed, or the second-order scheme (which
    the GPU solver does not take) fail with PAT_ERR_INVALID, GPU or not."""
    from paper_1501_03869_gb300 import PatError, fmm_gpu
    sp = np.full((16, 16), 1500.0, dtype=np.float32)
    origin = synth.centred_origin(sp.shape, 1e-4)
    with pytest.raises(PatError) as e:
        fmm_gpu(sp, 1e-4, origin, [[5e-3, 0.0, 0.0]])
    assert e.value.status == _lib.PAT_ERR_INVALID
    bad = sp.copy()
    bad[3, 4] = 0.0
    with pytest.raises(PatError) as e:
        fmm_gpu(bad, 1e-4, origin, [[0.0, 0.0, 0.0]])
    assert e.value.status == _lib.PAT_ERR_INVALID
    with pytest.raises(PatError) as e:
        table_host(sp, 1e-4, origin, synth.ring_sensors(4, 5e-4), 1e-8, 64, None,
                   _lib.PAT_FLAG_GPU_TABLE | _lib.PAT_FLAG_FMM_SECOND_ORDER)
    assert e.value.status == _lib.PAT_ERR_INVALID


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("shape,seed", [((40, 33), 1), ((12, 11, 10), 2)])
def test_host_fmm_matches_oracle(shape, seed, order):
    rng = np.random.default_rng(seed)
    sp = rng.uniform(1400.0, 3000.0, shape).astype(np.float32)
    h = 1e-4
    origin = np.array([-3e-4, 2e-4, 1e-4])[: len(shape)]
    src = origin + np.array([s * h * 0.43 for s in shape[::-1]])
    T_lib = fmm_host(sp, h, origin, src, order=order)
    T_or = oracle.fmm_point(sp.astype(np.float64), h, origin, src, order=order)
    assert np.allclose(T_lib, T_or, rtol=1e-12, atol=0)
    if order == 2:
        assert not np.allclose(T_lib, fmm_host(sp, h, origin, src, order=1), rtol=1e-6)


def test_second_order_march_is_bitwise_the_oracles_at_exact_ties():
    """A source at a cell centre makes tied neighbours, where the second-order
    switch (second upwind node not later than the first) decides on the last
    bit; the library's march evaluates the oracle's arithmetic, so the two
    agree bit for bit there (and everywhere else)."""
    for n, src_px in [(20, (13.5, 6.5)), (33, (16.0, 16.0))]:
        h = 1e-4
        sp = np.full((n, n), 1500.0, dtype=np.float32)
        src = np.array(src_px) * h
        T_lib = fmm_host(sp, h, np.zeros(2), src, order=2)
        T_or = oracle.fmm_point(sp.astype(np.float64), h, np.zeros(2), src, order=2)
        assert np.array_equal(T_lib, T_or)
    w = synth.config1(n_frames=1)
    for s in (0, 17):
        T_lib = fmm_host(w.speed, w.dx, w.origin, w.sensors[s], order=2)
        T_or = oracle.fmm_point(w.speed.astype(np.float64), w.dx, w.origin, w.sensors[s], order=2)
        assert np.array_equal(T_lib, T_or)


def test_second_order_table_matches_oracle():
    """The table of a second-order handle (PAT_FLAG_FMM_SECOND_ORDER) holds the
    oracle's order-2 arrival times."""
    w = synth.config1(n_frames=1)
    sensors = w.sensors[::8]
    info, u, base, slot = table_host(w.speed, w.dx, w.origin, sensors, w.dt, w.nt, w.mask,
                                     _lib.PAT_FLAG_FMM_SECOND_ORDER)
    P = info["tile_pix"]
    used = slot[slot >= 0]
    T = oracle.travel_table(w.speed, w.dx, w.origin, sensors, used, order=2)
    idx = np.flatnonzero(slot >= 0)
    for s in range(sensors.shape[0]):
        got = u[idx // P, s, idx % P].astype(np.float64) + base[idx // P, s]
        inrec = T[s] / w.dt <= w.nt - 1
        assert np.all(np.abs(got[inrec] - T[s][inrec] / w.dt) <= 1e-9 * T[s][inrec] / w.dt + 1e-4)


def _check_table(w, flags=0, sensor_subset=None):
    sensors = w.sensors if sensor_subset is None else w.sensors[sensor_subset]
    info, u, base, slot = table_host(w.speed, w.dx, w.origin, sensors, w.dt, w.nt, w.mask, flags)
    P, nt_, W = info["tile_pix"], info["n_tiles"], info["window"]
    pix = np.flatnonzero(w.mask.ravel())
    # every mask pixel appears in exactly one slot
    used = slot[slot >= 0]
    assert np.array_equal(np.sort(used), pix)
    assert info["n_pix"] == pix.size and nt_ == -(-pix.size // P)
    assert np.all(base % 8 == 0) and np.all(base >= 0) and W % 8 == 0
    # u + base reproduces T / dt of the oracle's own fast marching
    T = oracle.travel_table(w.speed, w.dx, w.origin, sensors, used)
    u_or = T / w.dt
    slot_of = {int(v): i for i, v in enumerate(slot) if v >= 0}
    idx = np.array([slot_of[int(v)] for v in used])
    t_i, p_i = idx // P, idx % P
    for s in range(sensors.shape[0]):
        u_s = u[t_i, s, p_i].astype(np.float64)
        b_s = base[t_i, s].astype(np.float64)
        inrec = u_or[s] <= w.nt - 1
        assert np.all(u_s[~inrec] == np.float32(1e30))
        got = u_s[inrec] + b_s[inrec]
        assert np.all(np.abs(got - u_or[s][inrec]) <= 1e-9 * u_or[s][inrec] + 2.0 ** -24 * W)
        # the window of each tile holds floor(u) and floor(u) + 1
        assert np.all(np.floor(u_s[inrec]) + 1 < W)
    # padding slots are out of record for every sensor
    pad = np.flatnonzero(slot < 0)
    if pad.size:
        assert np.all(u[pad // P, :, pad % P] == np.float32(1e30))
    return info


def test_table_layout_config1():
    info = _check_table(synth.config1(n_frames=1))
    assert info["window"] <= 200


def test_table_layout_config2_sensor_subset():
    w = synth.config2(n_frames=1, n_lines=1)
    info = _check_table(w, sensor_subset=np.arange(0, 512, 37))
    assert info["n_pix"] == 21323


def test_table_layout_3d_and_tile256():
    w = synth.config5_subject(0, n_frames=1, n_sensors=12, shape=(24, 40, 40), nt=512)
    _check_table(w)
    w2 = synth.config1(n_frames=1)
    _check_table(w2, flags=_lib.PAT_FLAG_TILE_256, sensor_subset=np.arange(0, 64, 9))


def test_tiles_are_spatially_compact():
    w = synth.config2(n_frames=1, n_lines=1)
    info, u, base, slot = table_host(w.speed, w.dx, w.origin, w.sensors[:4], w.dt, w.nt, w.mask)
    P = info["tile_pix"]
    ys, xs = np.divmod(np.where(slot >= 0, slot, 0), w.speed.shape[1])
    ext = []
    for t in range(info["n_tiles"]):
        sl = slice(t * P, (t + 1) * P)
        ok = slot[sl] >= 0
        ext.append(max(np.ptp(xs[sl][ok]), np.ptp(ys[sl][ok])))
    # Hilbert-curve tiles: squares in the interior, a few elongated ones along
    # the mask boundary
    assert np.median(ext) <= 16 and np.percentile(ext, 95) <= 32


def test_compact_output_slots_are_raster_ranks():
    w = synth.config1(n_frames=1)
    _, _, _, slot = table_host(w.speed, w.dx, w.origin, w.sensors[:3], w.dt, w.nt, w.mask,
                               _lib.PAT_FLAG_COMPACT_OUT)
    used = slot[slot >= 0]
    assert np.array_equal(np.sort(used), np.arange(w.n_pix))
