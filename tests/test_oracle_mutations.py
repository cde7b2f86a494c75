"""The oracle's pins catch plausible mistakes.  Each case plants one mistake
(a dropped factor, a wrong sign, an off-by-one index, a transposed operand, a
missing normalisation ...) in a temporary copy of the oracle and runs the pins
(tests/test_oracle_pins.py) against it: every copy must fail at least one pin,
while the untouched copy passes them all.  Everything runs on the CPU."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (file under oracle/, text to replace, replacement)
MUTATIONS = [
    # first-order Godunov update: one-axis step, two-axis discriminant, three-axis constant
    ("oracle.c", "double t = a[0] + hf;", "double t = a[0] + 0.5 * hf;"),
    ("oracle.c", "sqrt(2.0 * hf * hf - diff * diff)", "sqrt(2.0 * hf * hf + diff * diff)"),
    ("oracle.c", "3.0 * (q - hf * hf)", "3.0 * (q + hf * hf)"),
    # upwind neighbour: the larger instead of the smaller value on the upper side
    ("oracle.c", "if (state[w] == KNOWN && T[w] < best) best = T[w];\n    }\n    if (best",
     "if (state[w] == KNOWN && T[w] > best) best = T[w];\n    }\n    if (best"),
    # point source: distance times speed instead of over it
    ("oracle.c", "t0[m] = sqrt(dist2) / speed[v];", "t0[m] = sqrt(dist2) * speed[v];"),
    # second-order stencil: weight, extrapolated offset, applicability test
    ("oracle.c", "alpha = 9.0 / 4.0;", "alpha = 9.0 / 2.0;"),
    ("oracle.c", "ad = (4.0 * t1 - T[v2]) / 3.0;", "ad = (4.0 * t1 + T[v2]) / 3.0;"),
    ("oracle.c", "T[v2] <= t1)", "T[v2] >= t1)"),
    # integrand: central difference without its 2, the t-term without its 2, end index
    ("oracle.c", "dp = (p[k + 1] - p[k - 1]) / (2.0 * dt);", "dp = (p[k + 1] - p[k - 1]) / dt;"),
    ("oracle.c", "b[k] = 2.0 * p[k] - 2.0 * t * dp;", "b[k] = 2.0 * p[k] - t * dp;"),
    ("oracle.c", "dp = (p[nt - 1] - p[nt - 2]) / dt;", "dp = (p[nt - 1] - p[nt - 3]) / dt;"),
    # sampling: interpolation weight on the wrong sample, record end off by one
    ("oracle.c", "return (1.0 - phi) * b[i0] + phi * b[i0 + 1];",
     "return (1.0 - phi) * b[i0] + phi * b[i0];"),
    ("oracle.c", "if (!(u >= 0.0) || u > (double)(nt - 1)) return 0.0;",
     "if (!(u >= 0.0) || u > (double)nt) return 0.0;"),
    # back projection: default weight
    ("oracle.c", "double ws = w ? w[s] : 1.0 / (double)ns;", "double ws = w ? w[s] : 1.0 / (double)(ns - 1);"),
    # per-pair sum: transposed weights, time not divided by dt
    ("oracle.c", "acc += W[s * npix + j] * oracle_sample(b + s * nt, nt, T[s * npix + j] / dt);",
     "acc += W[j * ns + s] * oracle_sample(b + s * nt, nt, T[s * npix + j] / dt);"),
    ("oracle.c", "acc += W[s * npix + j] * oracle_sample(b + s * nt, nt, T[s * npix + j] / dt);",
     "acc += W[s * npix + j] * oracle_sample(b + s * nt, nt, T[s * npix + j]);"),
    # node positions without the origin; constant-speed delay times c0
    ("__init__.py", "pos[:, d] = float(origin[d]) + i.astype(np.float64) * float(h)",
     "pos[:, d] = i.astype(np.float64) * float(h)"),
    ("__init__.py", "out[s] = np.sqrt(np.sum(diff * diff, axis=1)) / float(c0)",
     "out[s] = np.sqrt(np.sum(diff * diff, axis=1)) * float(c0)"),
    # solid-angle weights: power, normal, normalisation, direction, element, full angle
    ("__init__.py", "out[s] = elem[s] * (v @ n) / r ** nd / float(omega0)",
     "out[s] = elem[s] * (v @ n) / r ** (nd + 1) / float(omega0)"),
    ("__init__.py", "out[s] = elem[s] * (v @ n) / r ** nd / float(omega0)",
     "out[s] = elem[s] * r / r ** nd / float(omega0)"),
    ("__init__.py", "n = normals[s, :nd] / np.sqrt(np.sum(normals[s, :nd] ** 2))", "n = normals[s, :nd]"),
    ("__init__.py", "v = pos - sensors[s, :nd]", "v = sensors[s, :nd] - pos"),
    ("__init__.py", "out[s] = elem[s] * (v @ n) / r ** nd / float(omega0)",
     "out[s] = (v @ n) / r ** nd / float(omega0)"),
    ("__init__.py", "out[s] = elem[s] * (v @ n) / r ** nd / float(omega0)",
     "out[s] = elem[s] * (v @ n) / r ** nd"),
]


def _run_pins(mutation):
    """Exit code of the pins on a copy of the oracle with `mutation` planted
    (None: an untouched copy)."""
    d = tempfile.mkdtemp(prefix="oracle_mut_")
    try:
        shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(d, "oracle"),
                        ignore=shutil.ignore_patterns("_build", "__pycache__"))
        shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(d, "tests"),
                        ignore=shutil.ignore_patterns("__pycache__"))
        if mutation is not None:
            fname, old, new = mutation
            f = os.path.join(d, "oracle", fname)
            with open(f) as fh:
                src = fh.read()
            assert src.count(old) >= 1, f"mutation target not found: {old!r}"
            with open(f, "w") as fh:
                fh.write(src.replace(old, new, 1))
        env = dict(os.environ, PYTHONPATH=d + os.pathsep + ROOT)
        r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(d, "tests", "test_oracle_pins.py"),
                            "-x", "-q", "-p", "no:cacheprovider"], cwd=d, env=env,
                           capture_output=True, text=True, timeout=600)
        return r.returncode, r.stdout[-400:]
    finally:
        shutil.rmtree(d, ignore_errors=True)


def test_pins_catch_every_planted_mistake():
    jobs = [None] + MUTATIONS
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(_run_pins, jobs))
    rc0, out0 = results[0]
    assert rc0 == 0, f"the untouched oracle copy must pass its pins: {out0}"
    # caught = a pin failed (exit code 1 with a failure), not an error of the copy
    survivors = [m for m, (rc, out) in zip(MUTATIONS, results[1:])
                 if not (rc == 1 and " failed" in out and " error" not in out)]
    assert not survivors, f"mutations no pin caught: {survivors}"
