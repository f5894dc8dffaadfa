"""FP64 CPU oracle for CS-WGS (test infrastructure only).

This package is the slow, plain reference that the CUDA library is checked
against.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the product path never does.  It shares no code
with the CUDA library.  The arithmetic lives in ``cswgs_oracle.c`` (plain C,
double precision, optional OpenMP); this module compiles it with gcc on first
use and wraps it with ctypes and numpy.

Each wrapper names the passage of the paper the C function follows:
Eq. 1 (back-propagation), Eq. 2 (lens-and-prism phase), Eq. 3 (forward
projection), Eqs. 4-6 (weighted update), Eq. 7 (uniformity), Section 2
(CS-WGS schedule) and Section 3 "Compressed sensing" (random pixel order).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cswgs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no -ffast-math); returns the .so path."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # CSWGS_ORACLE_LIB: a deliberately broken build of this file, loaded by
        # the mutation tests to show that the pins catch each planted mistake
        path = os.environ.get("CSWGS_ORACLE_LIB")
        if not path:
            path = build()
        lib = ctypes.CDLL(path)
        d = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.POINTER(ctypes.c_int64)
        u64 = ctypes.c_uint64
        lib.oracle_splitmix64.argtypes = [u64, u64]
        lib.oracle_splitmix64.restype = u64
        lib.oracle_fmix32.argtypes = [ctypes.c_uint32]
        lib.oracle_fmix32.restype = ctypes.c_uint32
        lib.oracle_theta0.argtypes = [ctypes.c_int, u64, d]
        lib.oracle_permute.argtypes = [ctypes.c_int, u64, ctypes.c_int, ctypes.c_int64]
        lib.oracle_permute.restype = ctypes.c_int64
        lib.oracle_permute_domain.argtypes = [ctypes.c_int64, u64, ctypes.c_int, ctypes.c_int64]
        lib.oracle_permute_domain.restype = ctypes.c_int64
        lib.oracle_in_pupil.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64]
        lib.oracle_in_pupil.restype = ctypes.c_int
        lib.oracle_pupil_amplitude.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int64]
        lib.oracle_pupil_amplitude.restype = ctypes.c_double
        lib.oracle_pupil_pixels.argtypes = [ctypes.c_int, ctypes.c_int, i64]
        lib.oracle_pupil_pixels.restype = ctypes.c_int64
        lib.oracle_subset_pupil.argtypes = [ctypes.c_int64, i64, ctypes.c_int64, u64, ctypes.c_int, ctypes.c_int, i64]
        lib.oracle_forward_pupil.argtypes = [ctypes.c_int, ctypes.c_int, d, ctypes.c_int64, i64, d, d,
                                             ctypes.c_double, d]
        lib.oracle_metrics_pupil.argtypes = [ctypes.c_int, ctypes.c_int, d, d, ctypes.c_int, ctypes.c_double,
                                             d, d, d, d]
        lib.oracle_solve_pupil.argtypes = [ctypes.c_int, ctypes.c_int, d, d, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_int, u64, d, d, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_int, d, d, d, d, d, d]
        lib.oracle_solve_pupil.restype = ctypes.c_int
        lib.oracle_subset.argtypes = [ctypes.c_int, ctypes.c_int64, u64, ctypes.c_int, i64]
        lib.oracle_spot_phase.argtypes = [ctypes.c_int, d, ctypes.c_int, ctypes.c_int64]
        lib.oracle_spot_phase.restype = ctypes.c_double
        lib.oracle_back.argtypes = [ctypes.c_int, ctypes.c_int, d, d, d, ctypes.c_int64, i64, d]
        lib.oracle_forward.argtypes = [ctypes.c_int, ctypes.c_int, d, ctypes.c_int64, i64, d, d]
        lib.oracle_update.argtypes = [ctypes.c_int, d, d, d]
        lib.oracle_metrics.argtypes = [ctypes.c_int, ctypes.c_int, d, d, d, d, d, d]
        lib.oracle_solve.argtypes = [ctypes.c_int, ctypes.c_int, d, d, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int, u64, d, d, ctypes.c_int, ctypes.c_int, d, d, d, d, d, d]
        lib.oracle_solve.restype = ctypes.c_int
        lib.oracle_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
        return lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def threads() -> int:
    return _load().oracle_threads()


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def splitmix64(seed: int, k: int) -> int:
    """Output k of SplitMix64 started from `seed` (counter-based form)."""
    return int(_load().oracle_splitmix64(seed & (2**64 - 1), k & (2**64 - 1)))


def fmix32(h: int) -> int:
    """MurmurHash3 32-bit finaliser."""
    return int(_load().oracle_fmix32(h & 0xFFFFFFFF))


def theta0(N: int, seed: int) -> np.ndarray:
    """theta_n^0 ~ U[0, 2 pi) drawn from the seed (Eq. 1, random superposition)."""
    out = np.empty(N)
    _load().oracle_theta0(N, seed & (2**64 - 1), _dp(out))
    return out


def permute(P: int, seed: int, j: int, k: int) -> int:
    """pi_{seed,j}(k): keyed bijection on [0, P^2) (Section 3, compressed sensing)."""
    return int(_load().oracle_permute(P, seed & (2**64 - 1), j, k))


def permute_domain(D: int, seed: int, j: int, k: int) -> int:
    """pi_{seed,j}(k): keyed bijection on [0, D) (Feistel network plus cycle walking)."""
    return int(_load().oracle_permute_domain(D, seed & (2**64 - 1), j, k))


APERTURES = {"square": 0, "round": 1}
SUBSET_MODES = {"fresh": 0, "windows": 1}


def pupil_pixels(P: int, aperture: str = "square") -> np.ndarray:
    """The pupil's pixels Omega in row-major order (Section 4: a round aperture of P pixels)."""
    lib = _load()
    ap = APERTURES[aperture]
    D = int(lib.oracle_pupil_pixels(P, ap, None))
    out = np.empty(D, dtype=np.int64)
    lib.oracle_pupil_pixels(P, ap, _ip(out))
    return out


def pupil_amplitude(P: int, waist: float = 0.0) -> np.ndarray:
    """A at every pixel (P*P): exp(-rho^2 / waist^2), or 1 for waist <= 0."""
    lib = _load()
    return np.array([lib.oracle_pupil_amplitude(P, float(waist), m) for m in range(P * P)])


def subset(P: int, Mp: int, seed: int, j: int, aperture: str = "square", mode: str = "fresh") -> np.ndarray:
    """S_j: the Mp pixel indices of iteration j (Section 2, CS-WGS), drawn from
    the pupil's pixels; mode "windows" takes window j of one fixed permutation."""
    out = np.empty(Mp, dtype=np.int64)
    if aperture == "square" and mode == "fresh":
        _load().oracle_subset(P, Mp, seed & (2**64 - 1), j, _ip(out))
        return out
    omega = pupil_pixels(P, aperture)
    _load().oracle_subset_pupil(omega.shape[0], _ip(omega), Mp, seed & (2**64 - 1), j, SUBSET_MODES[mode],
                                _ip(out))
    return out


def spot_phase(P: int, xyz, n: int, m: int) -> float:
    """phi_n at pixel m (Eq. 2, normalised units), radians."""
    xyz = _f64(xyz, (-1, 3))
    return float(_load().oracle_spot_phase(P, _dp(xyz), n, m))


def back(P: int, xyz, amp, theta, pix=None) -> np.ndarray:
    """Eq. 1: Phi at the listed pixels (all pixels when pix is None), in (-pi, pi]."""
    xyz = _f64(xyz, (-1, 3))
    N = xyz.shape[0]
    amp = _f64(amp)
    theta = _f64(theta)
    if pix is None:
        cnt = P * P
    else:
        pix = np.ascontiguousarray(pix, dtype=np.int64)
        cnt = pix.shape[0]
    out = np.empty(cnt)
    _load().oracle_back(P, N, _dp(xyz), _dp(amp), _dp(theta), cnt, _ip(pix), _dp(out))
    return out


def forward(P: int, xyz, phi, pix=None) -> np.ndarray:
    """Eq. 3 (sign reading +i): complex V_n over the listed pixels, normalised 1/count."""
    xyz = _f64(xyz, (-1, 3))
    N = xyz.shape[0]
    phi = _f64(phi)
    if pix is None:
        cnt = P * P
    else:
        pix = np.ascontiguousarray(pix, dtype=np.int64)
        cnt = pix.shape[0]
    assert phi.shape[0] == cnt
    V = np.empty(2 * N)
    _load().oracle_forward(P, N, _dp(xyz), cnt, _ip(pix), _dp(phi), _dp(V))
    return V[0::2] + 1j * V[1::2]


def forward_pupil(P: int, xyz, phi, pix, A, norm: float) -> np.ndarray:
    """Eq. 3 with pupil amplitudes: (1/norm) sum_k A_k e^{i (Phi_k - phi_n(m_k))}."""
    xyz = _f64(xyz, (-1, 3))
    N = xyz.shape[0]
    phi = _f64(phi)
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    A = _f64(A)
    assert phi.shape[0] == pix.shape[0] == A.shape[0]
    V = np.empty(2 * N)
    _load().oracle_forward_pupil(P, N, _dp(xyz), pix.shape[0], _ip(pix), _dp(phi), _dp(A), float(norm), _dp(V))
    return V[0::2] + 1j * V[1::2]


def update(V, w, theta):
    """Eqs. 4-6: returns the updated (w, theta)."""
    V = np.asarray(V, dtype=np.complex128)
    Vi = np.empty(2 * V.shape[0])
    Vi[0::2] = V.real
    Vi[1::2] = V.imag
    w = _f64(w).copy()
    theta = _f64(theta).copy()
    _load().oracle_update(V.shape[0], _dp(Vi), _dp(w), _dp(theta))
    return w, theta


def metrics(P: int, xyz, phi_full, aperture: str = "square", waist: float = 0.0):
    """Efficiency e, uniformity u (Eq. 7), spot intensities I_n and fields V_n
    over the pupil (normalised by the pupil's sum of A)."""
    xyz = _f64(xyz, (-1, 3))
    N = xyz.shape[0]
    phi_full = _f64(phi_full)
    assert phi_full.shape[0] == P * P
    V = np.empty(2 * N)
    In = np.empty(N)
    e = ctypes.c_double()
    u = ctypes.c_double()
    lib = _load()
    if aperture == "square" and not waist > 0:
        lib.oracle_metrics(P, N, _dp(xyz), _dp(phi_full), _dp(V), _dp(In), ctypes.byref(e), ctypes.byref(u))
    else:
        lib.oracle_metrics_pupil(P, N, _dp(xyz), _dp(phi_full), APERTURES[aperture], float(waist), _dp(V),
                                 _dp(In), ctypes.byref(e), ctypes.byref(u))
    return e.value, u.value, In, V[0::2] + 1j * V[1::2]


def solve(P: int, xyz, amp=None, c: float = 1.0, iterations: int = 0, seed: int = 0,
          theta_in=None, w_in=None, first_j: int = 1, final_pass: bool = True,
          full_iterations: int = 2, aperture: str = "square", waist: float = 0.0,
          subset_mode: str = "fresh"):
    """The whole CS-WGS method (Section 2).

    The last `full_iterations` of the `iterations` run over all pupil pixels
    (the paper ends with two such iterations); the others over the subsets S_j.
    aperture "round", waist > 0 and subset_mode "windows" are the paper's own
    setup (Section 4: round aperture, Gaussian beam; Section 3: one random
    reordering of the pupil's pixels).

    Returns a dict with phase (P*P, [0, 2 pi), or None without the final pass),
    e, u, w, theta (final state) and I (spot intensities)."""
    xyz = _f64(xyz, (-1, 3))
    N = xyz.shape[0]
    amp = _f64(amp)
    theta_in = _f64(theta_in)
    w_in = _f64(w_in)
    M = P * P
    phase = np.empty(M) if final_pass else None
    w = np.empty(N)
    th = np.empty(N)
    In = np.empty(N) if final_pass else None
    e = ctypes.c_double(float("nan"))
    u = ctypes.c_double(float("nan"))
    if aperture == "square" and not waist > 0 and subset_mode == "fresh":
        rc = _load().oracle_solve(P, N, _dp(xyz), _dp(amp), float(c), int(iterations),
                                  int(full_iterations), seed & (2**64 - 1), _dp(theta_in), _dp(w_in), int(first_j),
                                  1 if final_pass else 0, _dp(phase), ctypes.byref(e),
                                  ctypes.byref(u), _dp(w), _dp(th), _dp(In))
    else:
        rc = _load().oracle_solve_pupil(P, N, _dp(xyz), _dp(amp), float(c), int(iterations),
                                        int(full_iterations), seed & (2**64 - 1), _dp(theta_in), _dp(w_in),
                                        int(first_j), 1 if final_pass else 0, APERTURES[aperture], float(waist),
                                        SUBSET_MODES[subset_mode], _dp(phase), ctypes.byref(e),
                                        ctypes.byref(u), _dp(w), _dp(th), _dp(In))
    if rc != 0:
        raise ValueError("oracle_solve rejected its arguments")
    return {"phase": phase, "e": e.value, "u": u.value, "w": w, "theta": th, "I": In}


def subset_size(P: int, c: float, aperture: str = "square") -> int:
    """Mp = floor(c D), the size of every subset (Section 2, CS-WGS), D the
    pupil's pixel count (M for the square grid)."""
    import math
    D = P * P if aperture == "square" else int(_load().oracle_pupil_pixels(P, APERTURES[aperture], None))
    return int(math.floor(c * D))


def slm_gray(phase_f32, lut, levels: int):
    """Gray frame of a float32 phase map (Section 3: phase to gray-scale lookup
    table of the SLM).  The level decision is made in float32, as the library
    defines it: l = rint(Phi * s) mod levels, s = float32(levels / (2 pi)),
    gray = lut[l].  Takes the phase the decision is made from, so that both
    sides decide from the same float."""
    ph = np.asarray(phase_f32, dtype=np.float32)
    s = np.float32(levels / (2.0 * np.pi))
    lvl = np.rint(ph * s).astype(np.int64)
    lvl = np.where(lvl >= levels, lvl - levels, lvl)
    return np.asarray(lut, dtype=np.uint8)[lvl]
