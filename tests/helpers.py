"""Test-side helpers that combine the synthetic generator with the oracle."""
import numpy as np

import oracle


def fmm_arrivals(speed, dx, origin, centres, sensors):
    """Arrival times [na, ns]: one oracle fast-marching run from each absorber
    centre (ray paths are reversible, Sec. II-B), read at the sensor positions
    by multilinear interpolation of the node values."""
    speed = np.asarray(speed)
    nd = speed.ndim
    centres = np.asarray(centres, dtype=np.float64)
    sensors = np.asarray(sensors, dtype=np.float64)
    shape_x = speed.shape[::-1]
    g = (sensors[:, :nd] - np.asarray(origin)[:nd]) / dx
    i0 = [np.clip(np.floor(g[:, d]).astype(np.int64), 0, shape_x[d] - 2) for d in range(nd)]
    fr = [g[:, d] - i0[d] for d in range(nd)]
    out = np.empty((centres.shape[0], sensors.shape[0]))
    for a in range(centres.shape[0]):
        T = oracle.fmm_point(speed, dx, origin, centres[a, :nd]).ravel()
        acc = np.zeros(sensors.shape[0])
        for corner in range(1 << nd):
            w = np.ones(sensors.shape[0])
            idx = np.zeros(sensors.shape[0], dtype=np.int64)
            stride = 1
            for d in range(nd):
                bit = (corner >> d) & 1
                w = w * (fr[d] if bit else 1.0 - fr[d])
                idx += (i0[d] + bit) * stride
                stride *= shape_x[d]
            acc += w * T[idx]
        out[a] = acc
    return out
