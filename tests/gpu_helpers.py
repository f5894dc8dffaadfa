"""Shared helpers of the GPU parity tests."""
import math

import numpy as np

# Tolerances of the FP32 path against the FP64 oracle: RMS wrapped phase error
# per iteration and on the final map (radians), and absolute e / u error.
TOL_PHASE_RMS = 1e-3
TOL_EU = 1e-3
# The FP64 GPU baseline computes the same sums as the oracle in another order.
TOL_FP64_PHASE = 1e-9
# ... and writes its map as float32: half an ulp of 2 pi is 2.4e-7 rad.
TOL_FP64_MAP = 2e-7
TOL_FP64_EU = 1e-11


def wrap(d):
    return (np.asarray(d, dtype=np.float64) + np.pi) % (2 * np.pi) - np.pi


def rms_wrapped(a, b):
    d = wrap(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64))
    return float(math.sqrt(np.mean(d * d)))


def oracle_states(oracle, pb, iterations, full_iterations=2):
    """(w, theta) at the start of every iteration j = 1..iterations+1, from the oracle."""
    w = np.ones(pb.N)
    th = oracle.theta0(pb.N, pb.seed)
    states = [(w, th)]
    for j in range(1, iterations + 1):
        full = 1 if j > iterations - full_iterations else 0
        r = oracle.solve(pb.P, pb.xyz, pb.amp, c=pb.c, iterations=1, seed=pb.seed, theta_in=th, w_in=w,
                         first_j=j, final_pass=False, full_iterations=full)
        w, th = r["w"], r["theta"]
        states.append((w, th))
    return states


def write_pinned_tune_cache(path, threads, ppt, full, half=False, batch_pow2=range(0, 7), strip=None):
    """A tune cache that pins every key these tests can reach to one launch
    shape: P rounded up to 128 (128 .. 2048), N and the batch size to powers of
    two, and the subset fraction to the nearest power of two (c = 1 .. 2^-16).
    strip: the tensor-core launches' tiles per work item (None: chosen per
    launch)."""
    import json
    shape = [threads, ppt, full] + ([] if strip is None else [strip])
    entries = {"P%d_N%d_B%d_c%d%s" % (128 * p, 2 ** n, 2 ** b, c, "_H" if half else ""): shape
               for p in range(1, 17) for n in range(4, 11) for b in batch_pow2 for c in range(0, 17)}
    path.write_text(json.dumps({"format": "cswgs-tune-3", "entries": entries}))
    return str(path)
