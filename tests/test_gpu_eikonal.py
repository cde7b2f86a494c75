"""The table's arrival times solved on the GPU (PAT_FLAG_GPU_TABLE,
pat_fmm_gpu): the first-order Godunov system of Sec. II-B iterated block by
block to its fixed point with the host march's local-solve arithmetic.  In
exact arithmetic that system has one solution, the fast marching one; in FP64
the iteration keeps the least value each node has seen, which may differ from
the march's by rounding (relative 1e-12 at most here).  The solve itself is
deterministic (blocks of one colour never share a node), so the table does not
change from run to run or with the batch a sensor is solved in.  The tables
agree with the host-built ones to the last place of the FP32 offsets with the
same windows, in 2-D and 3-D, with sensors on nodes, on the grid boundary and
at its far corner, a record that ends inside the grid, and a speed field with
strong contrast; one case checks the oracle directly."""
import numpy as np
import pytest

import oracle
from paper_1501_03869_gb300 import BP, PatError, _lib, fmm_gpu, fmm_host, synth, table_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GPU = _lib.PAT_FLAG_GPU_TABLE


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_03869_gb300.build import build
    build()


def _both(speed, dx, origin, sensors, dt, nt, mask, flags=0):
    host = table_host(speed, dx, origin, sensors, dt, nt, mask, flags)
    gpu = table_host(speed, dx, origin, sensors, dt, nt, mask, flags | GPU)
    assert host[0]["gpu_table"] == 0 and gpu[0]["gpu_table"] == 1
    return host, gpu


TIME_REL = 1e-11  # FP64 rounding accumulated along the front, with a wide margin


def _assert_same(host, gpu):
    (ih, uh, bh, sh), (ig, ug, bg, sg) = host, gpu
    assert np.array_equal(sh, sg)
    assert np.array_equal(bh, bg)
    assert ih["window"] == ig["window"]
    out = uh == np.float32(1e30)
    assert np.array_equal(out, ug == np.float32(1e30))
    # the times agree to TIME_REL, so an offset moves by that much of the time
    # it encodes plus the rounding to FP32 (one place)
    ns = uh.shape[1]
    t_abs = uh.astype(np.float64) + bh[:, :, None]
    du = np.abs(uh.astype(np.float64) - ug)
    tol = np.spacing(np.abs(uh)).astype(np.float64) + TIME_REL * t_abs
    bad = ~out & (du > tol)
    assert not bad.any(), f"{int(bad.sum())} offsets differ by more than rounding (of {ns} sensors)"


def _assert_same_times(Th, Tg):
    fin = np.isfinite(Th)
    assert np.array_equal(fin, np.isfinite(Tg))
    rel = np.abs(Th[fin] - Tg[fin]) / np.maximum(Th[fin], 1e-300)
    assert rel.max() <= TIME_REL, f"max rel {rel.max()}"


def test_arrival_times_match_host_2d():
    """Whole-grid times of single sources: pat_fmm_gpu against pat_fmm_host."""
    w = synth.config1(n_frames=1)
    Tg = fmm_gpu(w.speed, w.dx, w.origin, w.sensors[[0, 9, 33]])
    for k, s in enumerate((0, 9, 33)):
        _assert_same_times(fmm_host(w.speed, w.dx, w.origin, w.sensors[s]), Tg[k])


def test_arrival_times_deterministic():
    """Block order and batch make no difference to a single bit."""
    w = synth.config2(n_frames=1)
    a = fmm_gpu(w.speed, w.dx, w.origin, w.sensors[:40])
    b = fmm_gpu(w.speed, w.dx, w.origin, w.sensors[:40])
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    for k in (0, 17, 39):
        one = fmm_gpu(w.speed, w.dx, w.origin, w.sensors[k])
        assert np.array_equal(one.view(np.uint64), a[k].view(np.uint64))


def test_arrival_times_match_host_3d():
    w = synth.config5_subject(0, n_frames=1, n_sensors=16, shape=(34, 54, 54), nt=1024)
    Tg = fmm_gpu(w.speed, w.dx, w.origin, w.sensors[[0, 7]])
    for k, s in enumerate((0, 7)):
        _assert_same_times(fmm_host(w.speed, w.dx, w.origin, w.sensors[s]), Tg[k])


def test_c1_table():
    w = synth.config1(n_frames=1)
    _assert_same(*_both(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, w.mask))


def test_c1_table_matches_oracle():
    """The GPU times against the oracle's own fast marching, directly."""
    w = synth.config1(n_frames=1)
    sensors = w.sensors[::16]
    info, u, base, slot = table_host(w.speed, w.dx, w.origin, sensors, w.dt, w.nt, w.mask, GPU)
    P = info["tile_pix"]
    idx = np.flatnonzero(slot >= 0)
    T = oracle.travel_table(w.speed, w.dx, w.origin, sensors, slot[idx])
    for s in range(sensors.shape[0]):
        got = u[idx // P, s, idx % P].astype(np.float64) + base[idx // P, s]
        want = T[s] / w.dt
        inrec = want <= w.nt - 1
        assert np.all(np.abs(got[inrec] - want[inrec]) <= 1e-9 * want[inrec] + 1e-4)
        assert np.all(u[idx // P, s, idx % P][~inrec] == np.float32(1e30))


def test_c2_table():
    """The 256 x 256 skull frame, all 512 sensors, 2048 samples."""
    w = synth.config2(n_frames=1)
    host, gpu = _both(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, w.mask)
    print(f"\nC2 table, 512 sensors: GPU build {gpu[0]['build_seconds']:.3f} s, "
          f"host build {host[0]['build_seconds']:.3f} s")
    _assert_same(host, gpu)


def test_tile256_compact():
    w = synth.config1(n_frames=1)
    flags = _lib.PAT_FLAG_TILE_256 | _lib.PAT_FLAG_COMPACT_OUT
    _assert_same(*_both(w.speed, w.dx, w.origin, w.sensors[::4], w.dt, w.nt, w.mask, flags))


def test_contrast_field_awkward_sensors_short_record():
    """Speeds 800-4000 m/s on a 97 x 75 grid (ragged blocks on both axes),
    sensors on nodes, on the boundary and at the far corner, a record that ends
    half-way across the grid, no mask (every node a pixel)."""
    rng = np.random.default_rng(1234)
    shape, dx = (97, 75), 2.0 ** -13  # node coordinates exact in binary
    field = synth.smooth_field(shape, 3.0, rng)
    speed = (800.0 + 3200.0 * (field - field.min()) / np.ptp(field)).astype(np.float32)
    origin = np.array([0.0, 0.0, 0.0])
    ext = (np.array(shape[::-1]) - 1) * dx  # x runs along the last array axis
    sensors = np.array([
        [0.0, 0.0, 0.0],                     # grid corner
        [ext[0], ext[1], 0.0],               # far corner
        [ext[0], 0.37 * ext[1], 0.0],        # on the boundary
        [10 * dx, 20 * dx, 0.0],             # on a node
        [0.5 * ext[0] + 0.25 * dx, 0.5 * ext[1] + 0.75 * dx, 0.0],
        [0.123 * ext[0], 0.877 * ext[1], 0.0],
    ])
    dt = 20e-9
    _assert_same(*_both(speed, dx, origin, sensors, dt, 64, None))
    _assert_same(*_both(speed, dx, origin, sensors, dt, 2048, None))


def test_3d_shell():
    """The 3-D shell-skull subject at a third of the volume (ragged z blocks)."""
    w = synth.config5_subject(0, n_frames=1, n_sensors=96, shape=(34, 54, 54), nt=1024)
    _assert_same(*_both(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, w.mask))


def test_handle_from_gpu_table_reconstructs():
    w = synth.config1(n_frames=2)
    sig = torch.from_numpy(w.signals).cuda()
    a = BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, w.mask)
    b = BP(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, w.mask, flags=GPU)
    ia, ib = a.reconstruct(sig).cpu().numpy(), b.reconstruct(sig).cpu().numpy()
    assert np.linalg.norm(ia - ib) <= 1e-6 * np.linalg.norm(ia)
    ic = b.reconstruct(sig).cpu().numpy()
    assert np.array_equal(ib.view(np.uint32), ic.view(np.uint32))


def test_second_order_on_gpu_rejected():
    w = synth.config1(n_frames=1)
    with pytest.raises(PatError):
        table_host(w.speed, w.dx, w.origin, w.sensors[:2], w.dt, w.nt, w.mask,
                   GPU | _lib.PAT_FLAG_FMM_SECOND_ORDER)


def test_c5_full_table_build_time():
    """The 160 x 160 x 96 subject with 1024 sensors: the GPU build agrees with
    the host build on a sample of sensors and reports its build time."""
    w = synth.config5_subject(0, n_frames=1)
    gpu = table_host(w.speed, w.dx, w.origin, w.sensors, w.dt, w.nt, w.mask, GPU)
    pick = np.array([0, 1, 333, 777, 1023])
    host = table_host(w.speed, w.dx, w.origin, w.sensors[pick], w.dt, w.nt, w.mask)
    print(f"\nC5 table, 1024 sensors: GPU build {gpu[0]['build_seconds']:.2f} s, "
          f"host build of 5 sensors {host[0]['build_seconds']:.2f} s")
    ig, ug, bg, sg = gpu
    ig = dict(ig, window=host[0]["window"])  # the window bound is over all sensors
    _assert_same(host, (ig, np.ascontiguousarray(ug[:, pick]), bg[:, pick], sg))
    assert gpu[0]["window"] >= host[0]["window"]
