"""Oracle travel tables computed in a spawn-started process pool.

The pool uses the 'spawn' start method so that it never forks a process that
already holds a CUDA context.  Results are cached per test session.
"""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np

_cache = {}
_pool = None


def _chunk_table(args):
    speed, dx, origin, sensors, pix, order = args
    import oracle
    return oracle.travel_table(speed, dx, origin, sensors, pix, order=order)


def pool():
    global _pool
    if _pool is None:
        n = max(1, min(16, (os.cpu_count() or 2)))
        _pool = cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"))
    return _pool


def travel_table(key, speed, dx, origin, sensors, pix, order=1):
    """T[ns, npix] from the oracle (fast-marching order 1 or 2), split over
    sensors in the pool."""
    if key in _cache:
        return _cache[key]
    sensors = np.asarray(sensors, dtype=np.float64)
    n = sensors.shape[0]
    k = max(1, min(n, 4 * (os.cpu_count() or 2)))
    bounds = np.linspace(0, n, k + 1).astype(int)
    jobs = [(np.asarray(speed, dtype=np.float64), dx, np.asarray(origin), sensors[a:b],
             np.asarray(pix), int(order)) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
    parts = list(pool().map(_chunk_table, jobs))
    T = np.concatenate(parts, axis=0)
    _cache[key] = T
    return T
