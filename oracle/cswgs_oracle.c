/*
 * CS-WGS oracle: a plain, slow, double-precision CPU restatement of the
 * compressed-sensing weighted Gerchberg-Saxton method (Pozzi & Mapelli,
 * "Real time computer generation of three-dimensional point cloud holograms
 * through GPU implementation of compressed sensing Gerchberg-Saxton algorithm").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or constant generator
 * with the CUDA library.
 *
 * Every function below states the passage of the paper it follows.  Where the
 * paper is silent or garbled, the reading taken is stated at the function.
 *
 * Grid and units (Section 2, Eq. 2, in the normalised units of the synthetic
 * workloads): a P x P grid, pixel m = r*P + i, x' = i - P/2, y' = r - P/2.
 * The pupil is the whole grid with amplitude A = 1 unless a round aperture
 * or a Gaussian amplitude is asked for (Section 4's optical setup).  Spot n is (alpha, beta, gamma):
 * alpha, beta in cycles across the aperture, gamma in waves of defocus at the
 * aperture edge, so
 *     phi_n(x', y') = 2 pi [ (alpha x' + beta y') / P
 *                          + gamma (x'^2 + y'^2) / (P/2)^2 ].
 *
 * Parallelism (optional OpenMP) never changes a result: pixel loops write
 * disjoint outputs, and every per-spot sum over pixels is taken by one thread
 * in increasing pixel order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------------ */
/* Seeded draws.  The paper draws theta^0 at random (Section 2, RS) and the   */
/* pixel subsets at random (Section 2, CS-WGS; Section 3 "Compressed          */
/* sensing") but fixes no generator.  Reading: counter-based SplitMix64.      */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014; the 64-bit C form published
 * with the xoshiro generators).  Output k (k = 0, 1, ...) of the sequence
 * started from state `seed`: the state is advanced k+1 times by the golden
 * gamma and the result passed through the output mix. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* MurmurHash3 32-bit finaliser (fmix32, A. Appleby, public domain). */
uint32_t oracle_fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

/* Initial spot phases theta_n^0 ~ U[0, 2 pi) (Section 2, Eq. 1 with random
 * theta^0; the RS hologram is CS-WGS's starting point).  Draw n is
 * 2 pi * (splitmix64(seed, n) >> 11) * 2^-53. */
void oracle_theta0(int N, uint64_t seed, double *theta)
{
    for (int n = 0; n < N; ++n) {
        uint64_t x = oracle_splitmix64(seed, (uint64_t)n);
        theta[n] = ORACLE_TWO_PI * ((double)(x >> 11) * 0x1.0p-53);
    }
}

/* Round key r (0..3) of the subset permutation of iteration j. */
static uint32_t subset_key(uint64_t seed, int j, int r)
{
    uint64_t k = 0x100000000ull + 4ull * (uint64_t)(uint32_t)j + (uint64_t)r;
    return (uint32_t)(oracle_splitmix64(seed, k) >> 32);
}

/* Keyed bijection pi_{seed,j} on [0, D) (Section 2, CS-WGS: a random pixel
 * subset per iteration; Section 3, "Compressed sensing": the pupil's pixels
 * taken in a random order).  Reading: a Feistel network over a near-square
 * rectangle, walked back into range.
 *   a = the smallest integer with a^2 >= D, b = ceil(D / a), so a b >= D;
 *   k = L b + R with L in [0, a), R in [0, b);
 *   four rounds (L, R) -> (R, (L + F_r(R)) mod p), where p is the modulus of
 *   the incoming L (a in rounds 0 and 2, b in rounds 1 and 3) and
 *   F_r(R) = floor(fmix32(R ^ K_r) p / 2^32);  result L b + R.
 * Each round is a bijection, so the network permutes [0, a b); values >= D
 * are sent through it again (cycle walking, Black & Rogaway 2002), which
 * leaves a permutation of [0, D).  For a square grid (D = P^2) a = b = P and
 * no value leaves the range. */
int64_t oracle_permute_domain(int64_t D, uint64_t seed, int j, int64_t k)
{
    int64_t a = (int64_t)sqrt((double)D);
    while (a * a < D) ++a;
    while (a > 1 && (a - 1) * (a - 1) >= D) --a;
    int64_t b = (D + a - 1) / a;
    int64_t y = k;
    do {
        uint64_t L = (uint64_t)(y / b), R = (uint64_t)(y % b);
        uint64_t p = (uint64_t)a, q = (uint64_t)b;
        for (int r = 0; r < 4; ++r) {
            uint64_t F = ((uint64_t)oracle_fmix32((uint32_t)R ^ subset_key(seed, j, r)) * p) >> 32;
            uint64_t nl = R;
            uint64_t nr = (L + F) % p;
            L = nl;
            R = nr;
            uint64_t t = p;
            p = q;
            q = t;
        }
        y = (int64_t)(L * (uint64_t)b + R);
    } while (y >= D);
    return y;
}

/* The square grid's permutation: pi_{seed,j} on [0, P^2). */
int64_t oracle_permute(int P, uint64_t seed, int j, int64_t k)
{
    return oracle_permute_domain((int64_t)P * P, seed, j, k);
}

/* S_j = { pi_{seed,j}(k) : 0 <= k < Mp }, Mp = floor(c M) distinct pixels. */
void oracle_subset(int P, int64_t Mp, uint64_t seed, int j, int64_t *out)
{
    for (int64_t k = 0; k < Mp; ++k) out[k] = oracle_permute(P, seed, j, k);
}

/* ------------------------------------------------------------------------ */
/* Pupil (Section 4: the hologram is computed on a round region of the panel */
/* P pixels in diameter, lit by a Gaussian beam; Eq. 3: the field is summed  */
/* over the pupil's pixels Omega with the pupil amplitude A).                */
/* ------------------------------------------------------------------------ */

/* Pixel m lies in the pupil: every pixel of the square grid, or, for the
 * round aperture, x'^2 + y'^2 <= (P/2)^2. */
int oracle_in_pupil(int P, int round_ap, int64_t m)
{
    if (!round_ap) return 1;
    int64_t xp = m % P - P / 2, yp = m / P - P / 2;
    return xp * xp + yp * yp <= (int64_t)(P / 2) * (P / 2);
}

/* Pupil amplitude A at pixel m: a Gaussian beam of radius `waist` pixels
 * (intensity |A|^2 falls to 1/e^2 at rho = waist), A = exp(-rho^2 / waist^2);
 * waist <= 0 means a uniform pupil, A = 1. */
double oracle_pupil_amplitude(int P, double waist, int64_t m)
{
    if (!(waist > 0.0)) return 1.0;
    double xp = (double)(m % P - P / 2), yp = (double)(m / P - P / 2);
    return exp(-(xp * xp + yp * yp) / (waist * waist));
}

/* The pupil's pixels in row-major order (the paper's per-pixel position
 * array); returns their number D.  `out` may be NULL. */
int64_t oracle_pupil_pixels(int P, int round_ap, int64_t *out)
{
    int64_t D = 0;
    for (int64_t m = 0; m < (int64_t)P * P; ++m)
        if (oracle_in_pupil(P, round_ap, m)) {
            if (out) out[D] = m;
            ++D;
        }
    return D;
}

/* S_j over a pupil of D pixels listed in `omega` (NULL: the square grid's
 * pixels in order, D = P^2).  Two readings of Section 3's random order:
 *   windows = 0: a new permutation per iteration,
 *                S_j = { omega[pi_{seed,j}(k)] : 0 <= k < Mp };
 *   windows = 1: the paper's single reordering made once at start-up, with
 *                iteration j taking the next Mp entries (wrapping around),
 *                S_j = { omega[pi_{seed,0}(((j-1) Mp + k) mod D)] }. */
void oracle_subset_pupil(int64_t D, const int64_t *omega, int64_t Mp, uint64_t seed, int j, int windows,
                         int64_t *out)
{
    int64_t off = 0;
    if (windows) {
        off = (((int64_t)(j - 1) % D) * (Mp % D)) % D;
        if (off < 0) off += D;
    }
    for (int64_t k = 0; k < Mp; ++k) {
        int64_t q = windows ? oracle_permute_domain(D, seed, 0, (off + k) % D)
                            : oracle_permute_domain(D, seed, j, k);
        out[k] = omega ? omega[q] : q;
    }
}

/* ------------------------------------------------------------------------ */
/* Optics                                                                    */
/* ------------------------------------------------------------------------ */

/* Lens-and-prism phase of spot n at pixel m (Eq. 2, normalised units). */
double oracle_spot_phase(int P, const double *xyz, int n, int64_t m)
{
    double xp = (double)(m % P) - 0.5 * P;
    double yp = (double)(m / P) - 0.5 * P;
    double half = 0.5 * P;
    return ORACLE_TWO_PI * ((xyz[3 * n] * xp + xyz[3 * n + 1] * yp) / P
                            + xyz[3 * n + 2] * (xp * xp + yp * yp) / (half * half));
}

/* Back-propagation (Eq. 1): Phi_m = arg sum_n a_n e^{i (phi_n(m) + theta_n)}
 * for the `cnt` pixels listed in `pix` (all pixels in order when pix is NULL).
 * `amp` holds the amplitudes a_n of the current iteration, a_n = w_n a_n^0
 * (Eq. 5).  arg is atan2, in (-pi, pi]; atan2(0, 0) = 0. */
void oracle_back(int P, int N, const double *xyz, const double *amp, const double *theta,
                 int64_t cnt, const int64_t *pix, double *phi_out)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < cnt; ++k) {
        int64_t m = pix ? pix[k] : k;
        double sr = 0.0, si = 0.0;
        for (int n = 0; n < N; ++n) {
            double ph = oracle_spot_phase(P, xyz, n, m) + theta[n];
            sr += amp[n] * cos(ph);
            si += amp[n] * sin(ph);
        }
        phi_out[k] = atan2(si, sr);
    }
}

/* Forward projection (Eq. 3) over the listed pixels with pupil amplitudes
 * A_k (NULL: A = 1), divided by `norm`:
 *     V_n = (1/norm) sum_k A_k e^{i (Phi_k - phi_n(m_k))}.
 * Reading of the sign: Eq. 3 prints e^{-i(Phi - phi_n)}; with theta_n = arg E_n
 * (Eq. 6) that would negate theta every iteration (for N = 1 theta -> -theta),
 * so the self-consistent e^{+i(Phi - phi_n)} is taken.  The normalisation does
 * not change w or theta; for the metrics it makes |V_n|^2 a power fraction.
 * V is returned interleaved (re, im) per spot. */
void oracle_forward_pupil(int P, int N, const double *xyz, int64_t cnt, const int64_t *pix,
                          const double *phi, const double *A, double norm, double *V)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int n = 0; n < N; ++n) {
        double vr = 0.0, vi = 0.0;
        for (int64_t k = 0; k < cnt; ++k) {
            int64_t m = pix ? pix[k] : k;
            double d = phi[k] - oracle_spot_phase(P, xyz, n, m);
            double a = A ? A[k] : 1.0;
            vr += a * cos(d);
            vi += a * sin(d);
        }
        V[2 * n] = vr / norm;
        V[2 * n + 1] = vi / norm;
    }
}

/* The uniform-pupil form, V_n = (1/cnt) sum_k e^{i (Phi_k - phi_n(m_k))}. */
void oracle_forward(int P, int N, const double *xyz, int64_t cnt, const int64_t *pix,
                    const double *phi, double *V)
{
    oracle_forward_pupil(P, N, xyz, cnt, pix, phi, NULL, (double)cnt, V);
}

/* Weighted GS update (Eqs. 4-6): w_n <- w_n <|V|>_n / |V_n|, theta_n <- arg V_n.
 * Readings: the update uses the field just projected (the E^{j-1} index of
 * Eq. 4 counts the hologram it came from); the mean is over amplitudes |V|.
 * Degenerate spot: |V_n| is clamped to 1e-30 and theta_n kept when V_n = 0. */
void oracle_update(int N, const double *V, double *w, double *theta)
{
    double mean = 0.0;
    for (int n = 0; n < N; ++n) mean += hypot(V[2 * n], V[2 * n + 1]);
    mean /= (double)N;
    for (int n = 0; n < N; ++n) {
        double mag = hypot(V[2 * n], V[2 * n + 1]);
        w[n] = w[n] * mean / (mag > 1e-30 ? mag : 1e-30);
        if (mag > 0.0) theta[n] = atan2(V[2 * n + 1], V[2 * n]);
    }
}

/* Efficiency and uniformity of a full hologram (Section 2; Eq. 7).  The
 * field of spot n is the forward projection over the pupil, normalised so
 * that a hologram focusing all light into one spot gives 1:
 *     V_n = sum_{m in Omega} A_m e^{i(Phi_m - phi_n(m))} / sum_{m in Omega} A_m,
 * I_n = |V_n|^2, e = sum_n I_n, u = 1 - (max I - min I) / (max I + min I).
 * Reading: the paper defines e only in words (the fraction of the power sent
 * to the spots).  For the square uniform pupil V_n = (1/M) sum_m ..., and the
 * squared DFT coefficients of e^{i Phi} sum to 1 (Parseval), so e is the
 * fraction of the power in the N spot modes.  For a round or Gaussian pupil
 * the normalisation by the pupil's own peak keeps e = 1 for a single
 * perfect spot (the power fraction per DFT bin would cap it below 1).
 * phi_full holds all P^2 pixels.  V (2N) and I (N) may be NULL. */
void oracle_metrics_pupil(int P, int N, const double *xyz, const double *phi_full, int round_ap,
                          double waist, double *V, double *I, double *e, double *u)
{
    int64_t D = oracle_pupil_pixels(P, round_ap, NULL);
    int64_t *omega = (int64_t *)malloc(sizeof(int64_t) * (size_t)D);
    double *A = (double *)malloc(sizeof(double) * (size_t)D);
    double *ph = (double *)malloc(sizeof(double) * (size_t)D);
    oracle_pupil_pixels(P, round_ap, omega);
    double norm = 0.0;
    for (int64_t k = 0; k < D; ++k) {
        A[k] = oracle_pupil_amplitude(P, waist, omega[k]);
        ph[k] = phi_full[omega[k]];
        norm += A[k];
    }
    double *Vl = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    oracle_forward_pupil(P, N, xyz, D, omega, ph, A, norm, Vl);
    double sum = 0.0, imax = -1.0, imin = 1e300;
    for (int n = 0; n < N; ++n) {
        double in = Vl[2 * n] * Vl[2 * n] + Vl[2 * n + 1] * Vl[2 * n + 1];
        if (I) I[n] = in;
        sum += in;
        if (in > imax) imax = in;
        if (in < imin) imin = in;
    }
    if (V) memcpy(V, Vl, sizeof(double) * 2 * (size_t)N);
    *e = sum;
    *u = (imax + imin) > 0.0 ? 1.0 - (imax - imin) / (imax + imin) : 0.0;
    free(Vl); free(ph); free(A); free(omega);
}

/* The square uniform pupil's metrics. */
void oracle_metrics(int P, int N, const double *xyz, const double *phi_full,
                    double *V, double *I, double *e, double *u)
{
    oracle_metrics_pupil(P, N, xyz, phi_full, 0, 0.0, V, I, e, u);
}

/* ------------------------------------------------------------------------ */
/* The whole method                                                          */
/* ------------------------------------------------------------------------ */

/* CS-WGS (Section 2): start from w = 1 (Eq. 4) and random theta^0 (the RS
 * hologram of Eq. 1); then for each of the I iterations j = first_j, ...:
 *   the pixel set of the iteration: the subset S_j (oracle_subset_pupil) for
 *   the first I - n_full iterations, all pupil pixels for the last n_full;
 *   Phi on that set by Eq. 1 with a_n = w_n a_n^0, V on it by Eq. 3 (with the
 *   pupil amplitude A), and the update of Eqs. 4-6;
 * then one full back-propagation (Eq. 1 over the pupil) giving the phase map
 * in [0, 2 pi) (0 outside the pupil, where no light falls), and the metrics.
 * Schedule: Section 2 ends CS-WGS with two iterations over all pixels
 * ("N-2" compressed iterations there counts iterations, the spot symbol being
 * a misprint for I), so the paper's schedule is n_full = 2; n_full = 0 gives
 * I compressed iterations followed by the full back-propagation alone.
 * I = 0 gives the random-superposition hologram; c = 1 gives plain WGS.
 *
 * Pupil (Section 4): round_ap = 0 is the square P x P grid, 1 the round
 * aperture of diameter P; waist > 0 a Gaussian amplitude (oracle_pupil_amplitude);
 * windows selects the subset reading (oracle_subset_pupil).  Mp = floor(c D)
 * with D the pupil's pixel count (D = M = P^2 for the square grid).
 *
 * amp0: a_n^0 (NULL -> 1).  theta_in / w_in: optional start state (NULL ->
 * drawn theta^0 / w = 1), used to resume or teacher-force.  first_j: index of
 * the first iteration (its subset key).  final_pass = 0 skips the full pass
 * and the metrics.  Outputs may be NULL.  Returns 0, or -1 on bad arguments. */
int oracle_solve_pupil(int P, int N, const double *xyz, const double *amp0, double c, int I,
                       int n_full, uint64_t seed, const double *theta_in, const double *w_in, int first_j,
                       int final_pass, int round_ap, double waist, int windows, double *phase_out,
                       double *e, double *u, double *w_out, double *theta_out, double *I_out)
{
    if (P < 2 || (P & 1) || N < 1 || !(c > 0.0 && c <= 1.0) || I < 0 || n_full < 0) return -1;
    int64_t M = (int64_t)P * P;
    int64_t D = oracle_pupil_pixels(P, round_ap, NULL);
    int64_t Mp = (int64_t)floor(c * (double)D);
    if (Mp < 1) return -1;
    int plain = !round_ap && !(waist > 0.0);   /* square uniform pupil: no lists needed */

    double *w = (double *)malloc(sizeof(double) * N);
    double *th = (double *)malloc(sizeof(double) * N);
    double *amp = (double *)malloc(sizeof(double) * N);
    double *V = (double *)malloc(sizeof(double) * 2 * N);
    int64_t *pix = (int64_t *)malloc(sizeof(int64_t) * (size_t)Mp);
    int64_t *omega = plain ? NULL : (int64_t *)malloc(sizeof(int64_t) * (size_t)D);
    double *A = plain ? NULL : (double *)malloc(sizeof(double) * (size_t)D);
    double *phi = (double *)malloc(sizeof(double) * (size_t)M);
    if (omega) oracle_pupil_pixels(P, round_ap, omega);

    for (int n = 0; n < N; ++n) w[n] = w_in ? w_in[n] : 1.0;
    if (theta_in) memcpy(th, theta_in, sizeof(double) * N);
    else oracle_theta0(N, seed, th);

    for (int it = 0; it < I; ++it) {
        int j = first_j + it;
        int full = it >= I - n_full;
        for (int n = 0; n < N; ++n) amp[n] = w[n] * (amp0 ? amp0[n] : 1.0);
        const int64_t *set = full ? omega : pix;
        int64_t cnt = full ? D : Mp;
        if (!full) oracle_subset_pupil(D, omega, Mp, seed, j, windows, pix);
        if (A)
            for (int64_t k = 0; k < cnt; ++k) A[k] = oracle_pupil_amplitude(P, waist, set ? set[k] : k);
        oracle_back(P, N, xyz, amp, th, cnt, set, phi);
        oracle_forward_pupil(P, N, xyz, cnt, set, phi, A, (double)cnt, V);
        oracle_update(N, V, w, th);
    }

    if (final_pass) {
        for (int n = 0; n < N; ++n) amp[n] = w[n] * (amp0 ? amp0[n] : 1.0);
        if (plain) {
            oracle_back(P, N, xyz, amp, th, M, NULL, phi);
        } else {
            double *pp = (double *)malloc(sizeof(double) * (size_t)D);
            oracle_back(P, N, xyz, amp, th, D, omega, pp);
            for (int64_t m = 0; m < M; ++m) phi[m] = 0.0;
            for (int64_t k = 0; k < D; ++k) phi[omega[k]] = pp[k];
            free(pp);
        }
        for (int64_t m = 0; m < M; ++m) {
            double p = phi[m];
            if (p < 0.0) p += ORACLE_TWO_PI;
            if (p >= ORACLE_TWO_PI) p -= ORACLE_TWO_PI;
            phi[m] = p;
        }
        double ee, uu;
        oracle_metrics_pupil(P, N, xyz, phi, round_ap, waist, NULL, I_out, &ee, &uu);
        if (e) *e = ee;
        if (u) *u = uu;
        if (phase_out) memcpy(phase_out, phi, sizeof(double) * (size_t)M);
    }
    if (w_out) memcpy(w_out, w, sizeof(double) * N);
    if (theta_out) memcpy(theta_out, th, sizeof(double) * N);

    free(w); free(th); free(amp); free(V); free(pix); free(phi); free(omega); free(A);
    return 0;
}

/* CS-WGS on the square uniform pupil (all M pixels, A = 1), Mp = floor(c M). */
int oracle_solve(int P, int N, const double *xyz, const double *amp0, double c, int I,
                 int n_full, uint64_t seed, const double *theta_in, const double *w_in, int first_j,
                 int final_pass, double *phase_out, double *e, double *u,
                 double *w_out, double *theta_out, double *I_out)
{
    return oracle_solve_pupil(P, N, xyz, amp0, c, I, n_full, seed, theta_in, w_in, first_j, final_pass,
                              0, 0.0, 0, phase_out, e, u, w_out, theta_out, I_out);
}

/* Number of OpenMP threads the oracle runs on (1 without OpenMP). */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
