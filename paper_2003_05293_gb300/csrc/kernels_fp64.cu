// Plain double-precision CS-WGS on the GPU: the baseline solver.
//
// Straightforward kernels, one per step, one hologram at a time:
//   prep     per spot: coefficients of Eq. 2 in turns per pixel, w = 1,
//            theta^0 drawn from the seed (Eq. 1, random superposition);
//   back     per pixel of the pass: Phi = arg sum_n w_n a_n e^{i(phi_n + theta_n)} (Eq. 1);
//   forward  per (pixel chunk, spot): sum of e^{i(Phi - phi_n)} (Eq. 3);
//   update   one block: w_n <- w_n <|V|>/|V_n|, theta_n <- arg V_n (Eqs. 4-6);
//   metrics  one block: I_n = |V_n|^2, e = sum I_n, u (Eq. 7).
// Phases are evaluated in FP64 with the range reduction done in turns
// (t - rint(t)) before the double-precision sincos.
#include "cswgs_device.cuh"
#include "cswgs_internal.h"

namespace cswgs {

constexpr int kF64Threads = 256;
constexpr int kF64PixPerBlock = 4096;

__global__ void fp64_prep(const double *xyz, const double *init_w, const double *init_th, int N, int P,
                          uint64_t seed, double *coef, double *w, double *theta)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double half = 0.5 * (double)P;
    coef[3 * n] = xyz[3 * n] / (double)P;
    coef[3 * n + 1] = xyz[3 * n + 1] / (double)P;
    coef[3 * n + 2] = xyz[3 * n + 2] / (half * half);
    w[n] = init_w ? init_w[n] : 1.0;
    theta[n] = init_th ? init_th[n] : kTwoPi * theta0_turns(seed, n);
}

__device__ __forceinline__ double spot_phase64(const double *coef, int n, double xp, double yp)
{
    double t = coef[3 * n] * xp + coef[3 * n + 1] * yp + coef[3 * n + 2] * (xp * xp + yp * yp);
    return kTwoPi * (t - rint(t));
}

__global__ void fp64_back(int P, int N, const double *coef, const double *w, const double *amp,
                          const double *theta, int64_t count, int subset, uint64_t seed, int j,
                          double *phi, int32_t *pix)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= count) return;
    int64_t m = k;
    if (subset) {
        SubsetKeys K = subset_keys(seed, j);
        m = permute((uint32_t)k, (uint32_t)P, K);
        pix[k] = (int32_t)m;
    }
    double xp = (double)(m % P) - 0.5 * P;
    double yp = (double)(m / P) - 0.5 * P;
    double sr = 0.0, si = 0.0;
    for (int n = 0; n < N; ++n) {
        double s, c;
        sincos(spot_phase64(coef, n, xp, yp) + theta[n], &s, &c);
        double a = w[n] * (amp ? amp[n] : 1.0);
        sr += a * c;
        si += a * s;
    }
    phi[k] = atan2(si, sr);
}

__global__ void fp64_forward(int P, int N, const double *coef, int64_t count, const int32_t *pix,
                             const double *phi, double2 *part)
{
    __shared__ double s_r[kF64Threads], s_i[kF64Threads];
    const int n = blockIdx.y;
    const int64_t k0 = (int64_t)blockIdx.x * kF64PixPerBlock;
    int64_t k1 = k0 + kF64PixPerBlock;
    if (k1 > count) k1 = count;
    double vr = 0.0, vi = 0.0;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        int64_t m = pix ? (int64_t)pix[k] : k;
        double xp = (double)(m % P) - 0.5 * P;
        double yp = (double)(m / P) - 0.5 * P;
        double s, c;
        sincos(phi[k] - spot_phase64(coef, n, xp, yp), &s, &c);
        vr += c;
        vi += s;
    }
    s_r[threadIdx.x] = vr;
    s_i[threadIdx.x] = vi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s_r[threadIdx.x] += s_r[threadIdx.x + o];
            s_i[threadIdx.x] += s_i[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * N + n] = make_double2(s_r[0], s_i[0]);
}

__global__ void fp64_update(int N, int chunks, int64_t count, const double2 *part, double *w,
                            double *theta)
{
    extern __shared__ double s_mag[];
    __shared__ double s_mean;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        double vr = 0.0, vi = 0.0;
        for (int c = 0; c < chunks; ++c) {
            vr += part[(size_t)c * N + n].x;
            vi += part[(size_t)c * N + n].y;
        }
        vr /= (double)count;
        vi /= (double)count;
        s_mag[n] = hypot(vr, vi);
        s_mag[N + n] = atan2(vi, vr);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mean = 0.0;
        for (int n = 0; n < N; ++n) mean += s_mag[n];
        s_mean = mean / (double)N;
    }
    __syncthreads();
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        double mag = s_mag[n];
        w[n] = w[n] * s_mean / (mag > 1e-30 ? mag : 1e-30);
        if (mag > 0.0) theta[n] = s_mag[N + n];
    }
}

__global__ void fp64_phase_out(int64_t M, const double *phi, float *out)
{
    int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= M) return;
    double p = phi[m];
    if (p < 0.0) p += kTwoPi;
    float o = (float)p;
    if (o >= kTwoPiF) o = 0.f;
    out[m] = o;
}

__global__ void fp64_metrics(int N, int chunks, int64_t M, const double2 *part, double *metrics)
{
    if (threadIdx.x != 0) return;
    double e = 0.0, imax = -1.0, imin = 1e300;
    for (int n = 0; n < N; ++n) {
        double vr = 0.0, vi = 0.0;
        for (int c = 0; c < chunks; ++c) {
            vr += part[(size_t)c * N + n].x;
            vi += part[(size_t)c * N + n].y;
        }
        vr /= (double)M;
        vi /= (double)M;
        double in = vr * vr + vi * vi;
        metrics[2 + n] = in;
        e += in;
        imax = fmax(imax, in);
        imin = fmin(imin, in);
    }
    metrics[0] = e;
    metrics[1] = (imax + imin) > 0.0 ? 1.0 - (imax - imin) / (imax + imin) : 0.0;
}

static unsigned blocks_for(int64_t n, int threads)
{
    return (unsigned)((n + threads - 1) / threads);
}

cudaError_t fp64_solve(const Fp64Work &wk, int P, int N, int Mp, int iterations, int n_full,
                       int first_j, uint64_t seed, int final_pass, float *phase_out, cudaStream_t s)
{
    const int64_t M = (int64_t)P * P;
    (void)cudaGetLastError();   // report these launches, not an earlier call's error
    fp64_prep<<<blocks_for(N, 128), 128, 0, s>>>(wk.xyz, wk.init_w, wk.init_th, N, P, seed, wk.coef,
                                                 wk.w, wk.theta);
    for (int it = 0; it < iterations; ++it) {
        const int full = it >= iterations - n_full;
        const int64_t count = full ? M : (int64_t)Mp;
        const int chunks = (int)((count + kF64PixPerBlock - 1) / kF64PixPerBlock);
        fp64_back<<<blocks_for(count, kF64Threads), kF64Threads, 0, s>>>(
            P, N, wk.coef, wk.w, wk.amp, wk.theta, count, full ? 0 : 1, seed, first_j + it, wk.phi, wk.pix);
        fp64_forward<<<dim3((unsigned)chunks, (unsigned)N), kF64Threads, 0, s>>>(
            P, N, wk.coef, count, full ? nullptr : wk.pix, wk.phi, wk.part);
        fp64_update<<<1, 256, sizeof(double) * 2 * N, s>>>(N, chunks, count, wk.part, wk.w, wk.theta);
    }
    if (final_pass) {
        const int chunks = (int)((M + kF64PixPerBlock - 1) / kF64PixPerBlock);
        fp64_back<<<blocks_for(M, kF64Threads), kF64Threads, 0, s>>>(
            P, N, wk.coef, wk.w, wk.amp, wk.theta, M, 0, seed, 0, wk.phi, wk.pix);
        if (phase_out) fp64_phase_out<<<blocks_for(M, 256), 256, 0, s>>>(M, wk.phi, phase_out);
        fp64_forward<<<dim3((unsigned)chunks, (unsigned)N), kF64Threads, 0, s>>>(
            P, N, wk.coef, M, nullptr, wk.phi, wk.part);
        fp64_metrics<<<1, 32, 0, s>>>(N, chunks, M, wk.part, wk.metrics);
    }
    return cudaGetLastError();
}

}  // namespace cswgs
