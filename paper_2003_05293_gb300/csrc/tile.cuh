// Device side of the fused CS-WGS iteration: the per-tile work (back-
// propagation, forward projection, tile partials), the per-hologram tails
// (weighted update, metrics) and the per-spot preparation.  Included by the
// kernel files; every function here is __device__.
#pragma once

#include "cswgs_device.cuh"
#include "cswgs_internal.h"

namespace cswgs {

constexpr int kSpotChunk = 128;   // spots per forward-reduction round

template <int THREADS>
__device__ __forceinline__ double block_sum_f64(double v, double *s_red)
{
    constexpr int W = THREADS / 32;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    double r = 0.0;
    for (int w = 0; w < W; ++w) r += s_red[w];
    return r;
}

template <int THREADS>
__device__ __forceinline__ double block_max_f64(double v, double *s_red)
{
    constexpr int W = THREADS / 32;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    double r = s_red[0];
    for (int w = 1; w < W; ++w) r = fmax(r, s_red[w]);
    return r;
}

// Weighted update (Eqs. 4-6) from the per-tile partial fields of one pass:
// V_n = (1/count) sum_tiles part; w_n <- w_n <|V|> / |V_n|; theta_n <- arg V_n.
// The tile partials are summed with Kahan compensation.
template <int THREADS>
__device__ void tail_update(const HoloDev &H, const LaunchSlot &sl, float2 *s_v, double *s_red)
{
    const int N = H.N;
    const float inv = 1.0f / (float)sl.count;
    double local = 0.0;
    for (int n = threadIdx.x; n < N; n += THREADS) {
        float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
        for (int t = 0; t < sl.tiles; ++t) {
            float2 p = __ldcg(&H.part[(size_t)t * N + n]);
            float yr = p.x - cr, tr = sr + yr;
            cr = (tr - sr) - yr;
            sr = tr;
            float yi = p.y - ci, ti = si + yi;
            ci = (ti - si) - yi;
            si = ti;
        }
        float2 v = make_float2(sr * inv, si * inv);
        s_v[n] = v;
        local += (double)hypotf(v.x, v.y);
    }
    const double mean = block_sum_f64<THREADS>(local, s_red) / (double)N;
    for (int n = threadIdx.x; n < N; n += THREADS) {
        float2 v = s_v[n];
        float mag = hypotf(v.x, v.y);
        SpotState st = H.state[n];
        st.w = (float)((double)st.w * mean / (double)fmaxf(mag, 1e-30f));
        if (mag > 0.f) st.theta = rad_to_fix(atan2f(v.y, v.x));
        H.state[n] = st;
    }
}

// Metrics of the final pass: V_n = (1/M) sum over all pixels (FP64 partials),
// I_n = |V_n|^2, e = sum_n I_n, u by Eq. 7.
template <int THREADS>
__device__ void tail_metrics(const HoloDev &H, const LaunchSlot &sl, double *s_red)
{
    const int N = H.N;
    const double inv = 1.0 / (double)sl.count;
    double e = 0.0, imax = -1.0, imin = 1e300;
    for (int n = threadIdx.x; n < N; n += THREADS) {
        double vr = 0.0, vi = 0.0;
        for (int t = 0; t < sl.tiles; ++t) {
            double2 p = __ldcg(&H.part64[(size_t)t * N + n]);
            vr += p.x;
            vi += p.y;
        }
        vr *= inv;
        vi *= inv;
        double in = vr * vr + vi * vi;
        H.metrics[2 + n] = in;
        e += in;
        imax = fmax(imax, in);
        imin = fmin(imin, in);
    }
    e = block_sum_f64<THREADS>(e, s_red);
    imax = block_max_f64<THREADS>(imax, s_red);
    imin = -block_max_f64<THREADS>(-imin, s_red);
    if (threadIdx.x == 0) {
        H.metrics[0] = e;
        H.metrics[1] = (imax + imin) > 0.0 ? 1.0 - (imax - imin) / (imax + imin) : 0.0;
    }
}

// Spots per warp-transposed reduction round, and the padded row length of the
// per-warp transpose buffer (17 float2: conflict-free column reads).
constexpr int kWarpChunk = 16;
constexpr int kWarpRow = kWarpChunk + 1;

template <int THREADS, int PPT>
__device__ void process_tile(const HoloDev &H, const LaunchSlot &sl, int t, int maxN,
                             unsigned char *smem, double *s_red, int *s_last)
{
    constexpr int W = THREADS / 32;
    int4 *s_coef = reinterpret_cast<int4 *>(smem);
    uint2 *s_bw = reinterpret_cast<uint2 *>(s_coef + maxN);
    float2 *s_v = reinterpret_cast<float2 *>(s_bw + maxN);
    float2 *s_part = s_v + maxN;                       // W x kSpotChunk
    float2 *s_wbuf = s_part + W * kSpotChunk;          // W x 32 x kWarpRow

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int P = H.P, N = H.N;
    const int pass = sl.pass;
    const int count = sl.count;

    // spot tables: fixed-point coefficients and (theta addend, w a0)
    for (int n = tid; n < N; n += THREADS) {
        s_coef[n] = H.coef[n];
        SpotState st = H.state[n];
        s_bw[n] = make_uint2(st.theta + kFixRound, __float_as_uint(st.w * st.a0));
    }

    // this thread's pixels
    SubsetKeys K = {0u, 0u, 0u, 0u};
    if (pass == kPassSubset) K = subset_keys(H.seed, sl.j);
    const int half = P >> 1;
    int32_t xp[PPT], yp[PPT];
    uint32_t r2[PPT];
    float qf[PPT], msk[PPT];
    int mix[PPT];
    const int base = t * (THREADS * PPT);
#pragma unroll
    for (int s = 0; s < PPT; ++s) {
        int idx = base + s * THREADS + tid;
        bool valid = idx < count;
        uint32_t k = valid ? (uint32_t)idx : 0u;
        uint32_t m = pass == kPassSubset ? permute(k, (uint32_t)P, K) : k;
        int r = (int)(m / (uint32_t)P);
        int i = (int)m - r * P;
        xp[s] = i - half;
        yp[s] = r - half;
        r2[s] = (uint32_t)(xp[s] * xp[s] + yp[s] * yp[s]);
        qf[s] = (float)r2[s];
        msk[s] = valid ? 1.f : 0.f;
        mix[s] = valid ? (int)m : -1;
    }
    __syncthreads();

    // back-propagation, Eq. 1
    float sr[PPT], si[PPT];
#pragma unroll
    for (int s = 0; s < PPT; ++s) { sr[s] = 0.f; si[s] = 0.f; }
    for (int n = 0; n < N; ++n) {
        const int4 c = s_coef[n];
        const uint2 bw = s_bw[n];
        const float wn = __uint_as_float(bw.y);
        const float gl = __int_as_float(c.w);
        const SpotFix f = {c.x, c.y, c.z, gl};
#pragma unroll
        for (int s = 0; s < PPT; ++s) {
            float sn, cs;
            sincos_fix(fix_phase(f, xp[s], yp[s], r2[s], bw.x), fmaf(gl, qf[s], -kTwoPiF), sn, cs);
            sr[s] = fmaf(wn, cs, sr[s]);
            si[s] = fmaf(wn, sn, si[s]);
        }
    }

    // Phi_m = arg S_m; the forward pass needs -Phi_m as a fixed-point addend
    uint32_t padd[PPT];
#pragma unroll
    for (int s = 0; s < PPT; ++s) {
        float ph = atan2f(si[s], sr[s]);
        padd[s] = kFixRound - rad_to_fix(ph);
        if (pass == kPassFinal && mix[s] >= 0 && H.phase_out) {
            float o = ph < 0.f ? ph + kTwoPiF : ph;
            if (o >= kTwoPiF) o = 0.f;
            H.phase_out[mix[s]] = o;
        }
    }

    // forward projection, Eq. 3: conj of sum_m e^{i (phi_n(m) - Phi_m)}.
    // Per spot each thread sums its PPT pixels; the warp's 32 partials of 16
    // spots go through a transposed shared buffer (lane q sums spot q), the
    // warps' totals through s_part, and one partial per (tile, spot) leaves.
    float2 *wbuf = s_wbuf + warp * 32 * kWarpRow;
    for (int n0 = 0; n0 < N; n0 += kSpotChunk) {
        const int nc = min(kSpotChunk, N - n0);
        for (int q0 = 0; q0 < nc; q0 += kWarpChunk) {
            const int qc = min(kWarpChunk, nc - q0);
            for (int q = 0; q < qc; ++q) {
                const int4 c = s_coef[n0 + q0 + q];
                const float gl = __int_as_float(c.w);
                const SpotFix f = {c.x, c.y, c.z, gl};
                float vr = 0.f, vi = 0.f;
#pragma unroll
                for (int s = 0; s < PPT; ++s) {
                    float sn, cs;
                    sincos_fix(fix_phase(f, xp[s], yp[s], r2[s], padd[s]), fmaf(gl, qf[s], -kTwoPiF), sn, cs);
                    vr = fmaf(msk[s], cs, vr);
                    vi = fmaf(msk[s], sn, vi);
                }
                wbuf[lane * kWarpRow + q] = make_float2(vr, vi);
            }
            __syncwarp();
            // lane = 16 h + q sums rows 16 h .. 16 h + 15 of column q
            const int q = lane & (kWarpChunk - 1), h = lane >> 4;
            float ar = 0.f, ai = 0.f;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                float2 p = wbuf[(h * 16 + i) * kWarpRow + q];
                ar += p.x;
                ai += p.y;
            }
            ar += __shfl_xor_sync(0xffffffffu, ar, 16);
            ai += __shfl_xor_sync(0xffffffffu, ai, 16);
            if (h == 0 && q < qc) s_part[warp * kSpotChunk + q0 + q] = make_float2(ar, -ai);
            __syncwarp();
        }
        __syncthreads();
        for (int q = tid; q < nc; q += THREADS) {
            const size_t o = (size_t)t * N + n0 + q;
            if (pass == kPassFinal) {
                double ar = 0.0, ai = 0.0;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    float2 p = s_part[w * kSpotChunk + q];
                    ar += (double)p.x;
                    ai += (double)p.y;
                }
                H.part64[o] = make_double2(ar, ai);
            } else {
                float ar = 0.f, ai = 0.f;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    float2 p = s_part[w * kSpotChunk + q];
                    ar += p.x;
                    ai += p.y;
                }
                H.part[o] = make_float2(ar, ai);
            }
        }
        __syncthreads();
    }

    // the last tile of this hologram's pass runs the update / metrics
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        unsigned prev = atomicAdd(H.counter, 1u);
        *s_last = (prev == (unsigned)(sl.tiles - 1)) ? 1 : 0;
    }
    __syncthreads();
    if (*s_last) {
        __threadfence();
        if (pass == kPassFinal) tail_metrics<THREADS>(H, sl, s_red);
        else tail_update<THREADS>(H, sl, s_v, s_red);
        __syncthreads();
        if (tid == 0) *H.counter = 0u;
    }
    __syncthreads();
}

// Spot preparation (step 1 of the path) for spot n of hologram H: fixed-point
// coefficients of Eq. 2, theta^0 drawn from the seed (or the caller's start
// state), w = 1 (or the caller's start weights).
__device__ __forceinline__ void prep_spot(const HoloDev &H, int n)
{
    SpotFix f = spot_fix(H.xyz[3 * n], H.xyz[3 * n + 1], H.xyz[3 * n + 2], H.P);
    H.coef[n] = make_int4(f.A, f.B, f.Gh, __float_as_int(f.gl));
    double th = H.init_th ? H.init_th[n] / kTwoPi : theta0_turns(H.seed, n);
    SpotState st;
    st.theta = turns_to_fix(th);
    st.w = H.init_w ? (float)H.init_w[n] : 1.0f;
    st.a0 = H.amp ? (float)H.amp[n] : 1.0f;
    st.pad = 0.f;
    H.state[n] = st;
}

// Dynamic shared memory of process_tile for THREADS threads and up to maxN spots.
__host__ __device__ constexpr size_t tile_smem_bytes(int threads, int maxN)
{
    return (size_t)maxN * (sizeof(int4) + sizeof(uint2) + sizeof(float2)) +
           (size_t)(threads / 32) * kSpotChunk * sizeof(float2) +
           (size_t)(threads / 32) * 32 * kWarpRow * sizeof(float2);
}

}  // namespace cswgs
