"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, x and y swapped, a wrong normalisation, an off-by-one in the pixel
grid) fails at least one of them:

* published generator test vectors (SplitMix64, MurmurHash3 finaliser);
* the unit definitions of Eq. 2 in the normalised workload units;
* the 2D DFT identities for on-grid spots (numpy.fft), for Eq. 1 and Eq. 3;
* Parseval's theorem for the efficiency;
* closed forms: a single spot (N = 1), the projection of a one-spot hologram,
  a worked example of Eqs. 4-6;
* convergence of WGS on well-separated spots (the paper's u > 0.9 claim);
* a brute-force re-run of the whole method in 40-digit arithmetic on a tiny grid.
"""
import math
import os

import numpy as np
import pytest

import oracle


def wrap(d):
    return (np.asarray(d) + np.pi) % (2 * np.pi) - np.pi


# --------------------------------------------------------------------------
# generators

def _golden(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "prng_vectors.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_prng_published_vectors(golden_dir):
    rows = _golden(golden_dir)
    assert len(rows) == 8
    for name, a, b, out in rows:
        if name == "splitmix64":
            assert oracle.splitmix64(int(a), int(b)) == int(out)
        else:
            assert oracle.fmix32(int(a, 16)) == int(out, 16)


def test_theta0_draw():
    th = oracle.theta0(5, 1234567)
    # draw n is 2 pi * (splitmix64(seed, n) >> 11) * 2^-53
    assert th[0] == pytest.approx(2 * math.pi * ((6457827717110365317 >> 11) * 2.0**-53), abs=1e-15)
    th = oracle.theta0(1000, 7)
    assert np.all(th >= 0) and np.all(th < 2 * np.pi)
    assert np.array_equal(th, oracle.theta0(1000, 7))
    assert not np.array_equal(th, oracle.theta0(1000, 8))
    # U[0, 2 pi): mean pi, variance (2 pi)^2 / 12 within 5 sigma
    assert abs(th.mean() - np.pi) < 5 * (2 * np.pi / math.sqrt(12)) / math.sqrt(1000)


# --------------------------------------------------------------------------
# subsets (Section 2, CS-WGS; Section 3 "Compressed sensing")

@pytest.mark.parametrize("P", [2, 4, 6, 8, 64, 130])
def test_permutation_is_bijection(P):
    for j in (1, 2, 17):
        s = oracle.subset(P, P * P, 99, j)
        assert np.array_equal(np.sort(s), np.arange(P * P))


def test_subset_properties():
    P, c = 64, 0.25
    Mp = oracle.subset_size(P, c)
    assert Mp == 1024
    s1 = oracle.subset(P, Mp, 5, 1)
    assert len(np.unique(s1)) == Mp and s1.min() >= 0 and s1.max() < P * P
    assert np.array_equal(s1, oracle.subset(P, Mp, 5, 1))          # reproducible
    s2 = oracle.subset(P, Mp, 5, 2)
    s1b = oracle.subset(P, Mp, 6, 1)
    assert not np.array_equal(np.sort(s1), np.sort(s2))             # new draw per iteration
    assert not np.array_equal(np.sort(s1), np.sort(s1b))            # and per seed
    # overlap of two independent c-subsets ~ hypergeometric with mean c * Mp
    ov = len(np.intersect1d(s1, s2))
    sd = math.sqrt(Mp * c * (1 - c))
    assert abs(ov - c * Mp) < 6 * sd
    # prefix property: the first k entries of S_j are the subset of size k
    assert np.array_equal(oracle.subset(P, 100, 5, 1), s1[:100])


def test_subset_spatially_uniform():
    # counts per 8x8 block of the pupil ~ Binomial(64, c) (hypergeometric, smaller var)
    P, c = 128, 0.125
    Mp = oracle.subset_size(P, c)
    for j in (1, 2, 3):
        s = oracle.subset(P, Mp, 11, j)
        r, i = s // P, s % P
        counts = np.zeros((P // 8, P // 8))
        np.add.at(counts, (r // 8, i // 8), 1)
        exp = 64 * c
        chi2 = ((counts - exp) ** 2 / (exp * (1 - c))).sum()
        dof = counts.size - 1
        assert abs(chi2 - dof) < 6 * math.sqrt(2 * dof)
        # rows and columns each get their share too
        rows = np.bincount(r, minlength=P)
        assert abs(rows.mean() - c * P) < 1e-9
        assert rows.std() < 3 * math.sqrt(P * c * (1 - c))


# --------------------------------------------------------------------------
# Eq. 2 in normalised units

def test_spot_phase_units():
    P = 64
    a, b, g = 3.7, -5.2, 2.3
    xyz = np.array([[a, b, g]])
    centre = (P // 2) * P + P // 2                    # x' = y' = 0
    assert oracle.spot_phase(P, xyz, 0, centre) == 0.0
    # tilt: alpha cycles across the P-pixel aperture -> 2 pi alpha / P per pixel in x
    lin = np.array([[a, b, 0.0]])
    d = oracle.spot_phase(P, lin, 0, centre + 1) - oracle.spot_phase(P, lin, 0, centre)
    assert d == pytest.approx(2 * math.pi * a / P, rel=1e-12)
    d = oracle.spot_phase(P, lin, 0, centre + P) - oracle.spot_phase(P, lin, 0, centre)
    assert d == pytest.approx(2 * math.pi * b / P, rel=1e-12)
    # defocus: gamma waves at the aperture edge (rho = P/2), rotationally symmetric
    foc = np.array([[0.0, 0.0, g]])
    edge_x = (P // 2) * P + 0                         # x' = -P/2, y' = 0
    edge_y = 0 * P + P // 2                           # x' = 0, y' = -P/2
    assert oracle.spot_phase(P, foc, 0, edge_x) == pytest.approx(2 * math.pi * g, rel=1e-12)
    assert oracle.spot_phase(P, foc, 0, edge_y) == pytest.approx(2 * math.pi * g, rel=1e-12)
    # second difference of a quadratic along x: 2 * 2 pi g / (P/2)^2
    p = [oracle.spot_phase(P, foc, 0, centre + k) for k in (-1, 0, 1)]
    assert p[0] - 2 * p[1] + p[2] == pytest.approx(4 * math.pi * g / (P / 2) ** 2, rel=1e-9)


# --------------------------------------------------------------------------
# Eq. 1 and Eq. 3 against the 2D DFT (numpy.fft)

def _on_grid_spots(P, N, rng):
    modes = rng.choice(P * P, size=N, replace=False)
    a = (modes % P) - P // 2
    b = (modes // P) - P // 2
    return np.stack([a, b, np.zeros(N)], axis=1).astype(np.float64)


@pytest.mark.parametrize("P", [8, 16, 32])
def test_back_is_inverse_dft(P):
    rng = np.random.default_rng(P)
    N = 7
    xyz = _on_grid_spots(P, N, rng)
    amp = rng.uniform(0.5, 2.0, N)
    theta = rng.uniform(0, 2 * np.pi, N)
    phi = oracle.back(P, xyz, amp, theta)
    # S[r, i] = sum_n a_n e^{i theta_n} e^{2 pi i (alpha (i - P/2) + beta (r - P/2)) / P}
    X = np.zeros((P, P), dtype=complex)
    for (al, be, _), an, tn in zip(xyz, amp, theta):
        X[int(be) % P, int(al) % P] += an * np.exp(1j * tn) * np.exp(-1j * np.pi * (al + be))
    S = np.fft.ifft2(X) * P * P
    ref = np.angle(S).reshape(-1)
    assert np.max(np.abs(wrap(phi - ref))) < 1e-10


@pytest.mark.parametrize("P,gamma", [(8, 0.0), (16, 0.0), (16, 1.7), (32, -3.1)])
def test_forward_is_dft(P, gamma):
    rng = np.random.default_rng(100 + P)
    N = 9
    xyz = _on_grid_spots(P, N, rng)
    xyz[:, 2] = gamma
    phi = rng.uniform(-np.pi, np.pi, P * P)
    V = oracle.forward(P, xyz, phi)
    r, i = np.divmod(np.arange(P * P), P)
    rho2 = (i - P / 2) ** 2 + (r - P / 2) ** 2
    field = (np.exp(1j * phi) * np.exp(-2j * np.pi * gamma * rho2 / (P / 2) ** 2)).reshape(P, P)
    F = np.fft.fft2(field) / (P * P)
    for n, (al, be, _) in enumerate(xyz):
        ref = np.exp(1j * np.pi * (al + be)) * F[int(be) % P, int(al) % P]
        assert abs(V[n] - ref) < 1e-12


def test_forward_subset_normalisation():
    # over a subset the field is the mean over the listed pixels
    P = 16
    rng = np.random.default_rng(3)
    xyz = _on_grid_spots(P, 3, rng)
    phi_full = rng.uniform(-np.pi, np.pi, P * P)
    pix = oracle.subset(P, 40, 1, 1)
    V = oracle.forward(P, xyz, phi_full[pix], pix)
    r, i = np.divmod(pix, P)
    for n, (al, be, _) in enumerate(xyz):
        ref = np.mean(np.exp(1j * (phi_full[pix] - 2 * np.pi * (al * (i - P / 2) + be * (r - P / 2)) / P)))
        assert abs(V[n] - ref) < 1e-13


def test_projection_of_single_spot_hologram():
    # Phi = phi_k projects to |V_k| = 1 (off-grid, defocused spot)
    P = 48
    xyz = np.array([[3.3, -7.9, 2.6], [-8.1, 4.4, -1.2], [10.5, 10.2, 0.4]])
    m = np.arange(P * P)
    for k in range(3):
        phi_k = np.array([oracle.spot_phase(P, xyz, k, int(q)) for q in m])
        V = oracle.forward(P, xyz, phi_k)
        assert abs(abs(V[k]) - 1.0) < 1e-12
        assert abs(V[k] - 1.0) < 1e-12
        others = [abs(V[n]) for n in range(3) if n != k]
        assert max(others) < 0.5


def test_parseval_efficiency():
    # all P^2 on-grid modes as spots: e = sum |V|^2 = 1 for any phase map
    P = 4
    a = np.arange(P * P) % P - P // 2
    b = np.arange(P * P) // P - P // 2
    xyz = np.stack([a, b, np.zeros(P * P)], axis=1).astype(float)
    rng = np.random.default_rng(0)
    for _ in range(3):
        phi = rng.uniform(0, 2 * np.pi, P * P)
        e, u, In, V = oracle.metrics(P, xyz, phi)
        assert e == pytest.approx(1.0, abs=1e-13)
        assert 0.0 <= u <= 1.0
        assert np.all(In >= 0)


# --------------------------------------------------------------------------
# Eqs. 4-6 and Eq. 7

def test_update_worked_example():
    # |V| = (2, 1): mean 1.5, so w <- w * (0.75, 1.5); theta <- arg V = (0, pi/2)
    w, th = oracle.update(np.array([2.0 + 0j, 1j]), np.array([1.0, 2.0]), np.array([0.3, 0.3]))
    assert np.allclose(w, [0.75, 3.0], atol=1e-15)
    assert np.allclose(th, [0.0, np.pi / 2], atol=1e-15)
    # a zero field keeps its phase and is clamped
    w, th = oracle.update(np.array([0j, 1.0 + 0j]), np.array([1.0, 1.0]), np.array([0.7, 0.1]))
    assert th[0] == 0.7 and np.isfinite(w[0]) and w[0] > 1e20


def test_uniformity_eq7():
    # two on-grid spots with amplitudes set so I = (4/9, ...) -> u from Eq. 7 by hand
    P = 8
    xyz = np.array([[1.0, 0.0, 0.0], [-2.0, 1.0, 0.0]])
    amp = np.array([2.0, 1.0])
    phi = oracle.back(P, xyz, amp, np.zeros(2))
    e, u, In, _ = oracle.metrics(P, xyz, phi)
    assert u == pytest.approx(1 - (In.max() - In.min()) / (In.max() + In.min()), abs=1e-15)
    assert In[0] > In[1] and 0 < u < 1
    assert e == pytest.approx(In.sum(), abs=1e-15) and e <= 1 + 1e-12


# --------------------------------------------------------------------------
# whole method

@pytest.mark.parametrize("iters,c", [(0, 1.0), (5, 0.25), (3, 1.0)])
def test_single_spot_closed_form(iters, c):
    # N = 1, theta^0 = 0: Phi = phi_1 mod 2 pi, theta stays a fixed point, e = u = 1
    P = 32
    xyz = np.array([[4.3, -2.8, 1.9]])
    res = oracle.solve(P, xyz, c=c, iterations=iters, seed=3, theta_in=np.zeros(1))
    ref = np.array([oracle.spot_phase(P, xyz, 0, m) for m in range(P * P)]) % (2 * np.pi)
    assert np.max(np.abs(wrap(res["phase"] - ref))) < 1e-12
    assert np.all(res["phase"] >= 0) and np.all(res["phase"] < 2 * np.pi)
    assert res["e"] == pytest.approx(1.0, abs=1e-12)
    assert res["u"] == pytest.approx(1.0, abs=1e-12)
    assert abs(res["theta"][0]) < 1e-12 and res["w"][0] == pytest.approx(1.0, abs=1e-12)


def test_rs_is_zero_iterations():
    P = 16
    xyz = np.array([[1.5, 2.5, 0.3], [-3.0, 1.0, -0.7]])
    res = oracle.solve(P, xyz, c=0.5, iterations=0, seed=9)
    th0 = oracle.theta0(2, 9)
    ref = oracle.back(P, xyz, np.ones(2), th0) % (2 * np.pi)
    assert np.max(np.abs(wrap(res["phase"] - ref))) < 1e-13
    assert np.array_equal(res["theta"], th0)


def test_wgs_converges_on_separated_spots():
    # plain WGS (c = 1) on well-separated on-grid spots drives u to 1 (Section 1: WGS
    # gives high uniformity); RS from the same start is far less uniform.  With
    # only six spots a phase-only hologram cannot put much more than ~85% of the
    # power into them, so e is only bounded loosely here.
    P = 32
    xyz = np.array([[-8, -8, 0], [8, -8, 0], [-8, 8, 0], [8, 8, 0], [0, 0, 0], [4, -11, 0]], float)
    rs = oracle.solve(P, xyz, c=1.0, iterations=0, seed=1)
    wgs = oracle.solve(P, xyz, c=1.0, iterations=30, seed=1)
    assert wgs["u"] > 0.99 and wgs["u"] > rs["u"]
    assert wgs["e"] > 0.75 and wgs["e"] >= rs["e"] - 1e-9 and wgs["e"] <= 1 + 1e-12
    assert np.all(wgs["w"] > 0)


def test_cs_wgs_quality_small():
    # CS-WGS on a random 3D cloud reaches the WGS-like quality claimed in Section 1
    import workloads
    # (two full iterations at the end, as in Section 2); with only the compressed
    # iterations the subset sampling noise stays in the weights and u drops
    pb = workloads.problem(128, 20, 5.0, 0.25, 30, seed=4)
    res = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed)
    cs_only = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed,
                           full_iterations=0)
    assert res["e"] > 0.8 and res["u"] > 0.97
    assert cs_only["u"] < res["u"]


def test_resume_is_exact():
    # state (w, theta, j) fully determines the rest: 4 + 3 iterations == 7 iterations
    P = 16
    xyz = np.array([[1.2, -3.4, 0.5], [2.5, 4.1, -1.0], [-5.0, 0.3, 0.2]])
    full = oracle.solve(P, xyz, c=0.25, iterations=7, seed=21)
    a = oracle.solve(P, xyz, c=0.25, iterations=4, seed=21, final_pass=False, full_iterations=0)
    b = oracle.solve(P, xyz, c=0.25, iterations=3, seed=21, theta_in=a["theta"], w_in=a["w"], first_j=5)
    assert np.array_equal(full["phase"], b["phase"])
    assert full["e"] == b["e"] and full["u"] == b["u"]


def test_bruteforce_high_precision_tiny():
    # the whole method re-run in 40-digit arithmetic on a 6x6 grid (RS start,
    # 3 CS iterations with c = 1/2, final pass, metrics)
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    P, c, I, seed = 6, 0.5, 3, 77
    xyz = np.array([[0.7, -1.1, 0.4], [-1.3, 0.9, -0.6]])
    N, M = 2, P * P
    res = oracle.solve(P, xyz, c=c, iterations=I, seed=seed, full_iterations=1)
    pi = mp.pi

    def phase(n, m):
        xp = mp.mpf(int(m % P)) - P // 2
        yp = mp.mpf(int(m // P)) - P // 2
        a, b, g = (mp.mpf(float(v)) for v in xyz[n])
        return 2 * pi * ((a * xp + b * yp) / P + g * (xp * xp + yp * yp) / mp.mpf(P // 2) ** 2)

    w = [mp.mpf(1)] * N
    th = [mp.mpf(float(t)) for t in oracle.theta0(N, seed)]
    Mp = int(math.floor(c * M))
    for j in range(1, I + 1):
        # the last iteration runs over all pixels (Section 2 schedule)
        pix = list(range(M)) if j == I else [int(q) for q in oracle.subset(P, Mp, seed, j)]
        Phi = {}
        for m in pix:
            s = sum(w[n] * mp.expj(phase(n, m) + th[n]) for n in range(N))
            Phi[m] = mp.atan2(s.imag, s.real)
        V = [sum(mp.expj(Phi[m] - phase(n, m)) for m in pix) / len(pix) for n in range(N)]
        mean = sum(abs(v) for v in V) / N
        w = [w[n] * mean / abs(V[n]) for n in range(N)]
        th = [mp.atan2(V[n].imag, V[n].real) for n in range(N)]
    Phi = []
    for m in range(M):
        s = sum(w[n] * mp.expj(phase(n, m) + th[n]) for n in range(N))
        Phi.append(mp.atan2(s.imag, s.real))
    In = [abs(sum(mp.expj(Phi[m] - phase(n, m)) for m in range(M)) / M) ** 2 for n in range(N)]
    e_ref = float(sum(In))
    u_ref = float(1 - (max(In) - min(In)) / (max(In) + min(In)))
    phi_ref = np.array([float(p) for p in Phi])
    assert np.max(np.abs(wrap(res["phase"] - phi_ref))) < 1e-12
    assert res["e"] == pytest.approx(e_ref, abs=1e-13)
    assert res["u"] == pytest.approx(u_ref, abs=1e-13)
    assert np.allclose(res["w"], [float(x) for x in w], rtol=1e-12)
    assert np.max(np.abs(wrap(res["theta"] - np.array([float(t) for t in th])))) < 1e-12


def test_rejects_bad_arguments():
    xyz = np.array([[1.0, 1.0, 0.0]])
    for kw in (dict(P=7), dict(P=0), dict(c=0.0), dict(c=1.5), dict(iterations=-1)):
        args = dict(P=8, c=0.5, iterations=1)
        args.update(kw)
        with pytest.raises(ValueError):
            oracle.solve(args["P"], xyz, c=args["c"], iterations=args["iterations"])


# --------------------------------------------------------------------------
# pupil (Section 4: round aperture of P pixels, Gaussian beam; Eq. 3's A) and
# the subset readings over it (Section 3, "Compressed sensing")

# Lattice points with x^2 + y^2 <= r^2, r = 1 .. 12 (the Gauss circle problem,
# OEIS A000328).  The round pupil of a P-pixel grid is that disc of radius P/2
# less its two points at x' = P/2 or y' = P/2, which fall off the grid.
GAUSS_CIRCLE = [5, 13, 29, 49, 81, 113, 149, 197, 253, 317, 377, 441]


def test_round_pupil_counts_gauss_circle():
    for r, n in enumerate(GAUSS_CIRCLE, start=1):
        P = 2 * r
        om = oracle.pupil_pixels(P, "round")
        assert om.shape[0] == n - 2
        assert np.all(np.diff(om) > 0) and om.min() >= 0 and om.max() < P * P
    assert np.array_equal(oracle.pupil_pixels(10, "square"), np.arange(100))
    # the disc's area, to within its perimeter
    P = 1152
    D = oracle.subset_size(P, 1.0, "round")
    assert abs(D - math.pi * (P / 2) ** 2) < 2 * math.pi * (P / 2)


def test_gaussian_amplitude_is_beam_radius():
    # A = 1 on the axis and 1/e at rho = waist (intensity 1/e^2 there), separable
    P, w = 32, 10.0
    A = oracle.pupil_amplitude(P, w).reshape(P, P)
    assert A[P // 2, P // 2] == 1.0
    assert A[P // 2, P // 2 + 10] == pytest.approx(math.exp(-1.0), rel=1e-15)
    assert A[P // 2 + 6, P // 2 + 8] == pytest.approx(math.exp(-1.0), rel=1e-15)   # 6-8-10 triangle
    assert np.allclose(A, np.outer(A[:, P // 2], A[P // 2, :]), rtol=1e-14)
    assert np.all(oracle.pupil_amplitude(P, 0.0) == 1.0)


@pytest.mark.parametrize("D", [1, 2, 3, 5, 47, 79, 195, 1000, 4093, 12345])
def test_permutation_on_any_domain_is_bijection(D):
    for j in (0, 1, 9):
        img = np.array([oracle.permute_domain(D, 31, j, k) for k in range(D)])
        assert np.array_equal(np.sort(img), np.arange(D))
    if D > 100:
        a = [oracle.permute_domain(D, 31, 1, k) for k in range(100)]
        b = [oracle.permute_domain(D, 31, 2, k) for k in range(100)]
        assert a != b


def test_permutation_of_square_domain_is_the_grid_permutation():
    P = 24
    for k in range(0, P * P, 7):
        assert oracle.permute_domain(P * P, 5, 3, k) == oracle.permute(P, 5, 3, k)


def test_subsets_stay_in_round_pupil():
    P, c = 64, 0.125
    Mp = oracle.subset_size(P, c, "round")
    om = set(oracle.pupil_pixels(P, "round").tolist())
    for mode in ("fresh", "windows"):
        for j in (1, 2, 7):
            s = oracle.subset(P, Mp, 4, j, "round", mode)
            assert len(set(s.tolist())) == Mp and set(s.tolist()) <= om
            r, i = np.divmod(s, P)
            assert np.all((i - P // 2) ** 2 + (r - P // 2) ** 2 <= (P // 2) ** 2)


def test_windows_partition_one_permutation():
    # window j is entries (j-1) Mp .. j Mp - 1 of one fixed order of the pupil's
    # pixels: windows 1 .. 1/c are disjoint, the first is the prefix of that
    # order (the fresh draw with key 0), and they wrap around after the last
    P, c = 16, 0.25
    om = oracle.pupil_pixels(P, "round")
    D = om.shape[0]
    Mp = oracle.subset_size(P, c, "round")
    wins = [oracle.subset(P, Mp, 8, j, "round", "windows") for j in range(1, 5)]
    allw = np.concatenate(wins)
    assert len(np.unique(allw)) == 4 * Mp
    order = om[[oracle.permute_domain(D, 8, 0, k) for k in range(D)]]
    assert np.array_equal(wins[0], order[:Mp])
    assert np.array_equal(wins[2], order[2 * Mp:3 * Mp])
    w5 = oracle.subset(P, Mp, 8, 5, "round", "windows")
    assert np.array_equal(w5, order[(4 * Mp + np.arange(Mp)) % D])


def test_forward_with_pupil_is_weighted_dft():
    # Eq. 3 with A: V_n (times the norm) is the DFT of 1_Omega A e^{i Phi} at the spot's bin
    P, w = 16, 5.0
    rng = np.random.default_rng(77)
    xyz = _on_grid_spots(P, 6, rng)
    phi = rng.uniform(-np.pi, np.pi, P * P)
    om = oracle.pupil_pixels(P, "round")
    A = oracle.pupil_amplitude(P, w)
    V = oracle.forward_pupil(P, xyz, phi[om], om, A[om], 2.5)
    field = np.zeros(P * P, dtype=complex)
    field[om] = A[om] * np.exp(1j * phi[om])
    F = np.fft.fft2(field.reshape(P, P)) / 2.5
    for n, (al, be, _) in enumerate(xyz):
        ref = np.exp(1j * np.pi * (al + be)) * F[int(be) % P, int(al) % P]
        assert abs(V[n] - ref) < 1e-12


@pytest.mark.parametrize("aperture,waist", [("round", 0.0), ("round", 9.0), ("square", 7.0)])
def test_metrics_with_pupil_parseval(aperture, waist):
    # all P^2 on-grid modes as spots: sum_n I_n = P^2 sum A^2 / (sum A)^2 over the
    # pupil (Parseval with the single-spot normalisation), for any phase map
    P = 8
    a = np.arange(P * P) % P - P // 2
    b = np.arange(P * P) // P - P // 2
    xyz = np.stack([a, b, np.zeros(P * P)], axis=1).astype(float)
    om = oracle.pupil_pixels(P, aperture)
    A = oracle.pupil_amplitude(P, waist)[om]
    rng = np.random.default_rng(5)
    phi = rng.uniform(0, 2 * np.pi, P * P)
    e, u, In, V = oracle.metrics(P, xyz, phi, aperture, waist)
    assert e == pytest.approx(P * P * np.sum(A ** 2) / np.sum(A) ** 2, rel=1e-12)


@pytest.mark.parametrize("mode", ["fresh", "windows"])
def test_single_spot_closed_form_round_gaussian_pupil(mode):
    # N = 1, theta^0 = 0: Phi = phi_1 mod 2 pi on the pupil, 0 outside it; the
    # spot takes all the light, e = u = 1, whatever A is
    P = 32
    xyz = np.array([[4.3, -2.8, 1.9]])
    res = oracle.solve(P, xyz, c=0.25, iterations=4, seed=3, theta_in=np.zeros(1), aperture="round",
                       waist=11.0, subset_mode=mode)
    om = oracle.pupil_pixels(P, "round")
    out = np.setdiff1d(np.arange(P * P), om)
    ref = np.array([oracle.spot_phase(P, xyz, 0, int(m)) for m in om]) % (2 * np.pi)
    assert np.max(np.abs(wrap(res["phase"][om] - ref))) < 1e-12
    assert np.all(res["phase"][out] == 0.0)
    assert res["e"] == pytest.approx(1.0, abs=1e-12)
    assert res["u"] == pytest.approx(1.0, abs=1e-12)


def test_wide_beam_is_uniform_pupil():
    # a beam far wider than the aperture: A -> 1, the uniform result
    P = 16
    xyz = np.array([[1.2, -3.4, 0.5], [2.5, 4.1, -1.0], [-5.0, 0.3, 0.2]])
    a = oracle.solve(P, xyz, c=0.5, iterations=4, seed=2, aperture="round", waist=1e9)
    b = oracle.solve(P, xyz, c=0.5, iterations=4, seed=2, aperture="round")
    assert np.max(np.abs(wrap(a["phase"] - b["phase"]))) < 1e-9
    assert a["e"] == pytest.approx(b["e"], abs=1e-12) and a["u"] == pytest.approx(b["u"], abs=1e-12)


def test_wgs_converges_in_round_gaussian_pupil():
    P = 32
    xyz = np.array([[-7, -7, 0], [7, -7, 0], [-7, 7, 0], [7, 7, 0], [0, 0, 0]], float)
    rs = oracle.solve(P, xyz, c=1.0, iterations=0, seed=1, aperture="round", waist=14.0)
    wgs = oracle.solve(P, xyz, c=1.0, iterations=30, seed=1, aperture="round", waist=14.0)
    assert wgs["u"] > 0.99 and wgs["u"] > rs["u"]
    assert 0.5 < wgs["e"] <= 1 + 1e-9 and np.all(wgs["w"] > 0)


def test_bruteforce_high_precision_round_gaussian_windows():
    # the whole method with the paper's own pupil and subset reading, re-run in
    # 40-digit arithmetic on an 8x8 grid: round aperture (47 pixels), Gaussian
    # A, windows of one permutation, 2 compressed + 1 full iteration
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    P, c, I, seed, waist = 8, 0.5, 3, 12, 3.0
    xyz = np.array([[0.7, -1.1, 0.4], [-1.3, 0.9, -0.6]])
    N = 2
    res = oracle.solve(P, xyz, c=c, iterations=I, seed=seed, full_iterations=1, aperture="round",
                       waist=waist, subset_mode="windows")
    pi = mp.pi
    half = P // 2

    def coords(m):
        return mp.mpf(int(m % P) - half), mp.mpf(int(m // P) - half)

    def phase(n, m):
        xp, yp = coords(m)
        a, b, g = (mp.mpf(float(v)) for v in xyz[n])
        return 2 * pi * ((a * xp + b * yp) / P + g * (xp * xp + yp * yp) / mp.mpf(half) ** 2)

    def amp(m):
        xp, yp = coords(m)
        return mp.exp(-(xp * xp + yp * yp) / mp.mpf(waist) ** 2)

    omega = [m for m in range(P * P) if (m % P - half) ** 2 + (m // P - half) ** 2 <= half * half]
    assert len(omega) == 47
    D = len(omega)
    Mp = int(math.floor(c * D))
    w = [mp.mpf(1)] * N
    th = [mp.mpf(float(t)) for t in oracle.theta0(N, seed)]
    for j in range(1, I + 1):
        if j == I:
            pix = omega
        else:
            pix = [omega[oracle.permute_domain(D, seed, 0, ((j - 1) * Mp + k) % D)] for k in range(Mp)]
        Phi = {}
        for m in pix:
            s = sum(w[n] * mp.expj(phase(n, m) + th[n]) for n in range(N))
            Phi[m] = mp.atan2(s.imag, s.real)
        V = [sum(amp(m) * mp.expj(Phi[m] - phase(n, m)) for m in pix) for n in range(N)]
        mean = sum(abs(v) for v in V) / N
        w = [w[n] * mean / abs(V[n]) for n in range(N)]
        th = [mp.atan2(V[n].imag, V[n].real) for n in range(N)]
    Phi = {}
    for m in omega:
        s = sum(w[n] * mp.expj(phase(n, m) + th[n]) for n in range(N))
        Phi[m] = mp.atan2(s.imag, s.real)
    norm = sum(amp(m) for m in omega)
    In = [abs(sum(amp(m) * mp.expj(Phi[m] - phase(n, m)) for m in omega) / norm) ** 2 for n in range(N)]
    phi_ref = np.zeros(P * P)
    for m in omega:
        phi_ref[m] = float(Phi[m])
    assert np.max(np.abs(wrap(res["phase"] - phi_ref))) < 1e-12
    assert np.all(res["phase"][np.setdiff1d(np.arange(P * P), omega)] == 0.0)
    assert res["e"] == pytest.approx(float(sum(In)), abs=1e-13)
    assert res["u"] == pytest.approx(float(1 - (max(In) - min(In)) / (max(In) + min(In))), abs=1e-13)
    assert np.allclose(res["w"], [float(x) for x in w], rtol=1e-12)


def test_slm_gray_levels():
    # identity table of 256 levels: phase 2 pi k / 256 -> k, half a level rounds
    # to even, the top of the range wraps to level 0
    lut = np.arange(256, dtype=np.uint8)
    k = np.arange(256)
    ph = (2 * np.pi * k / 256).astype(np.float32)
    assert np.array_equal(oracle.slm_gray(ph, lut, 256), k.astype(np.uint8))
    assert oracle.slm_gray(np.float32(np.pi), lut, 256) == 128
    assert oracle.slm_gray(np.float32(2 * np.pi * 255.7 / 256), lut, 256) == 0
    assert oracle.slm_gray(np.float32(2 * np.pi * 0.3 / 256), lut, 256) == 0
    # a non-trivial table: gray = lut[level]
    lut2 = (255 - np.arange(16) * 17).astype(np.uint8)
    ph = (2 * np.pi * np.arange(16) / 16).astype(np.float32)
    assert np.array_equal(oracle.slm_gray(ph, lut2, 16), lut2)
