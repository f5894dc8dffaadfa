"""Seeded synthetic inputs for CS-WGS: spot clouds, batches and arrival streams.

This module holds no arithmetic of the method itself.  It only draws the
workload data (spot coordinates, amplitudes, hologram sizes, arrival times)
that both the CUDA library and the oracle take as inputs, with numpy's PCG64
seeded generator.  The method's own random draws (theta^0 and the pixel
subsets) are made from the `seed` argument inside each side.

Spot units are normalised: (alpha, beta) in cycles across the aperture,
gamma in waves of defocus at the aperture edge, so that the lens-and-prism
phase of Eq. 2 becomes 2 pi [(alpha x' + beta y')/P + gamma rho^2/(P/2)^2].

The five workloads follow the paper's regime (Section 5: 100- and 36-spot
patterns, compression rates 2^-1 .. 2^-8, a 1152-pixel aperture):

  tiny     P=64,   N=10,  gamma ~ U[-5, 5],   c=1/4, I=10
  medium   P=512,  N=100, gamma ~ U[-10, 10], c=1/8, I=30
  large    P=1152, N in {100, 300}, gamma ~ U[-10, 10], c in {1/4, 1/8, 1/16}, I=30
  batch    64 holograms, P in {512, 768, 1024, 1152}, N ~ U{10..300}, c=1/8, I=30
  serve    Poisson arrivals; P in {768, 1024, 1152}, N in {10, 100, 1000},
           gamma ~ U[-20, 20], c=1/8, I=20
with alpha, beta ~ U[-P/4, P/4] and a_n = 1 throughout.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = ["Problem", "spots", "problem", "TINY", "MEDIUM", "LARGE", "batch", "arrivals", "scenario",
           "SCENARIOS"]


@dataclass
class Problem:
    """One hologram request: spot cloud plus the solver's scalar arguments."""
    P: int
    xyz: np.ndarray            # (N, 3) float64: alpha, beta (cycles), gamma (waves)
    amp: np.ndarray | None     # (N,) float64 or None (all ones)
    c: float
    iterations: int
    seed: int
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def M(self) -> int:
        return self.P * self.P


def spots(P: int, N: int, gamma_max: float, seed: int) -> np.ndarray:
    """(N, 3) float64 spots: alpha, beta ~ U[-P/4, P/4], gamma ~ U[-g, g]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xyz = np.empty((N, 3), dtype=np.float64)
    xyz[:, 0] = rng.uniform(-P / 4.0, P / 4.0, N)
    xyz[:, 1] = rng.uniform(-P / 4.0, P / 4.0, N)
    xyz[:, 2] = rng.uniform(-gamma_max, gamma_max, N)
    return xyz


def problem(P: int, N: int, gamma_max: float, c: float, iterations: int, seed: int) -> Problem:
    return Problem(P=P, xyz=spots(P, N, gamma_max, seed), amp=None, c=c,
                   iterations=iterations, seed=seed)


# name -> (P, N, gamma_max, c, iterations)
TINY = dict(P=64, N=10, gamma_max=5.0, c=0.25, iterations=10)
MEDIUM = dict(P=512, N=100, gamma_max=10.0, c=0.125, iterations=30)
LARGE = dict(P=1152, N=100, gamma_max=10.0, c=0.125, iterations=30)
LARGE_N = (100, 300)
LARGE_C = (0.25, 0.125, 0.0625)


def batch(count: int = 64, seed: int = 0, P_choices=(512, 768, 1024, 1152), N_lo: int = 10,
          N_hi: int = 300, gamma_max: float = 10.0, c: float = 0.125, iterations: int = 30):
    """`count` independent holograms of uneven size, each with its own seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for h in range(count):
        P = int(rng.choice(P_choices))
        N = int(rng.integers(N_lo, N_hi + 1))
        hs = int(rng.integers(0, 2**63 - 1))
        out.append(problem(P, N, gamma_max, c, iterations, hs))
    return out


def arrivals(rate_hz: float, duration_s: float, seed: int = 0, P_choices=(768, 1024, 1152),
             N_choices=(10, 100, 1000), gamma_max: float = 20.0, c: float = 0.125,
             iterations: int = 20):
    """Poisson arrival stream: list of (arrival time in s, Problem).

    N is drawn uniformly from N_choices, i.e. log-uniformly on that grid."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    while True:
        t += float(rng.exponential(1.0 / rate_hz))
        if t >= duration_s:
            break
        P = int(rng.choice(P_choices))
        N = int(rng.choice(N_choices))
        hs = int(rng.integers(0, 2**63 - 1))
        out.append((t, problem(P, N, gamma_max, c, iterations, hs)))
    return out


# The paper's test scenarios (Section 5), as seeded synthetic stand-ins: a
# regular 10 x 10 and a 6 x 6 grid of spots rotated in 3D, and a less regular
# 3D cloud of spots in two cubes.  Each seed draws a new orientation (the
# paper repeats every scenario with 10 orientations and initial phases).
# Lateral coordinates are in cycles across the aperture; the axial one is
# turned into waves of defocus at the aperture edge with KAPPA waves per cycle
# (the ratio of the two scales for an objective of NA ~ 0.8).
KAPPA = 0.2
SCENARIOS = ("grid100", "grid36", "cubes100")


def _rotation(rng):
    a, b, c = rng.uniform(0.0, 2.0 * np.pi, 3)

    def rz(t):
        return np.array([[np.cos(t), -np.sin(t), 0.0], [np.sin(t), np.cos(t), 0.0], [0.0, 0.0, 1.0]])

    def rx(t):
        return np.array([[1.0, 0.0, 0.0], [0.0, np.cos(t), -np.sin(t)], [0.0, np.sin(t), np.cos(t)]])

    return rz(a) @ rx(b) @ rz(c)


def scenario(name: str, P: int, seed: int, c: float = 0.125, iterations: int = 30) -> Problem:
    """One of SCENARIOS at grid side P, orientation drawn from `seed`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if name in ("grid100", "grid36"):
        n = 10 if name == "grid100" else 6
        spacing = P / (4.0 * n)                  # the grid spans ~P/4 cycles
        g = (np.arange(n) - (n - 1) / 2.0) * spacing
        pts = np.array([[x, y, 0.0] for x in g for y in g])
    elif name == "cubes100":
        side = P / 10.0
        pts = np.concatenate([rng.uniform(-side / 2, side / 2, (50, 3)) + np.array([dx * 0.8 * side, 0.0, 0.0])
                              for dx in (-1.0, 1.0)])
    else:
        raise ValueError("unknown scenario %r" % name)
    pts = pts @ _rotation(rng).T
    xyz = np.stack([pts[:, 0], pts[:, 1], KAPPA * pts[:, 2]], axis=1)
    return Problem(P=P, xyz=xyz, amp=None, c=c, iterations=iterations, seed=seed, extra={"scenario": name})
