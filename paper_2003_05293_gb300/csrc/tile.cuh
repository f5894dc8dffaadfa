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
// Compensated sum of spot n's tile partials t = t0, t0 + dt, ... (8 loads in flight).
__device__ __forceinline__ float4 tile_sum(const HoloDev &H, int n, int t0, int dt, int tiles)
{
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
#pragma unroll 8   // loads issued ahead of the compensated sum's chain
    for (int t = t0; t < tiles; t += dt) {
        float2 p = __ldcg(&H.part[(size_t)t * H.N + n]);
        float yr = p.x - cr, tr = sr + yr;
        cr = (tr - sr) - yr;
        sr = tr;
        float yi = p.y - ci, ti = si + yi;
        ci = (ti - si) - yi;
        si = ti;
    }
    return make_float4(sr, cr, si, ci);
}

// With SPLIT (a block of its own per hologram), G groups of threads share a
// spot's tiles (t = g, g + G, ...) when the block has threads to spare, for
// G times the loads in flight; each group's compensated sum (s, c) stands for
// s - c, and the G of them are summed with compensation again.
template <int THREADS, bool SPLIT = false>
__device__ void tail_update(const HoloDev &H, const LaunchSlot &sl, float2 *s_v, double *s_red)
{
    const int N = H.N;
    const float inv = 1.0f / (float)sl.count;
    const int G = SPLIT ? max(1, min(16, THREADS / max(1, N))) : 1;
    float4 *s_grp = nullptr;
    if constexpr (SPLIT) {
        __shared__ double2 s_grp_buf[THREADS];
        s_grp = reinterpret_cast<float4 *>(s_grp_buf);
        if (G > 1) {
            const int n = threadIdx.x % N, g = threadIdx.x / N;
            if (g < G) s_grp[g * N + n] = tile_sum(H, n, g, G, sl.tiles);
            __syncthreads();
        }
    }
    double local = 0.0;
    for (int n = threadIdx.x; n < N; n += THREADS) {
        float4 q;
        if (G > 1) {
            float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
            for (int g = 0; g < G; ++g) {
                const float4 p = s_grp[g * N + n];
                float yr = (p.x - p.y) - cr, tr = sr + yr;
                cr = (tr - sr) - yr;
                sr = tr;
                float yi = (p.z - p.w) - ci, ti = si + yi;
                ci = (ti - si) - yi;
                si = ti;
            }
            q = make_float4(sr, cr, si, ci);
        } else {
            q = tile_sum(H, n, 0, 1, sl.tiles);
        }
        float2 v = make_float2(q.x * inv, q.z * inv);
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

// Metrics of the final pass: V_n = sum over the pupil of A e^{i(Phi - phi_n)}
// (FP64 partials) divided by the pupil's sum of A, I_n = |V_n|^2,
// e = sum_n I_n, u by Eq. 7.
// With SPLIT, G groups of threads share a spot's tiles as in tail_update.
template <int THREADS, bool SPLIT = false>
__device__ void tail_metrics(const HoloDev &H, const LaunchSlot &sl, double *s_red)
{
    const int N = H.N;
    const double inv = 1.0 / H.norm;   // sum of A over the pupil (P^2 for the square uniform grid)
    const int G = SPLIT ? max(1, min(16, THREADS / max(1, N))) : 1;
    auto sum = [&](int n, int t0, int dt) {
        double vr = 0.0, vi = 0.0;
#pragma unroll 8
        for (int t = t0; t < sl.tiles; t += dt) {
            double2 p = __ldcg(&H.part64[(size_t)t * N + n]);
            vr += p.x;
            vi += p.y;
        }
        return make_double2(vr, vi);
    };
    double2 *s_grp = nullptr;
    if constexpr (SPLIT) {
        __shared__ double2 s_grp_buf[THREADS];
        s_grp = s_grp_buf;
        if (G > 1) {
            const int n = threadIdx.x % N, g = threadIdx.x / N;
            if (g < G) s_grp[g * N + n] = sum(n, g, G);
            __syncthreads();
        }
    }
    double e = 0.0, imax = -1.0, imin = 1e300;
    for (int n = threadIdx.x; n < N; n += THREADS) {
        double vr = 0.0, vi = 0.0;
        if (G > 1) {
            for (int g = 0; g < G; ++g) {
                vr += s_grp[g * N + n].x;
                vi += s_grp[g * N + n].y;
            }
        } else {
            const double2 v = sum(n, 0, 1);
            vr = v.x;
            vi = v.y;
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

// Separable full-pass tiles: THREADS / 4 rows x kFullCols columns, each thread
// a 4 x 4 block of pixels (16 threads across a row of the tile).  Row factors
// are stored in row order (a thread's 4 rows: two 16-byte loads, broadcast to
// the 16 threads of its row); column factors are interleaved so that the
// 16-byte halves of each thread's 4 columns sit side by side (every load is a
// contiguous 256-byte row).  Spot factors are made kFactorChunk spots at a time.
constexpr int kFullCols = 64;
constexpr int kFactorChunk = 16;

__host__ __device__ inline int full_pass_tiles(int P, int threads)
{
    const int rows = threads / 4;
    return ((P + rows - 1) / rows) * ((P + kFullCols - 1) / kFullCols);
}

// Position of column x (0..63) of a spot's column factors: 16-byte half h of
// thread x / 4 at float2 index 32 h + 2 (x / 4) + (x % 2).
__host__ __device__ constexpr int col_slot(int x) { return 32 * ((x >> 1) & 1) + 2 * (x >> 2) + (x & 1); }

// Shared-memory layout of a tile (both tile processors).
struct TileSmem {
    int4 *coef;      // maxN: fixed-point spot coefficients
    uint2 *bw;       // maxN: (theta addend, w a0)
    float2 *v;       // maxN: tail scratch
    float2 *part;    // W x kSpotChunk: per-warp spot totals
    float2 *wbuf;    // W x 32 x kWarpRow: per-warp transpose buffers
    float2 *fac;     // kFactorChunk x (THREADS / 4 + kFullCols): separable spot factors
};

template <int THREADS>
__device__ __forceinline__ TileSmem tile_smem(unsigned char *smem, int maxN)
{
    constexpr int W = THREADS / 32;
    TileSmem m;
    m.coef = reinterpret_cast<int4 *>(smem);
    m.bw = reinterpret_cast<uint2 *>(m.coef + maxN);
    m.v = reinterpret_cast<float2 *>(m.bw + maxN);
    m.part = m.v + maxN;
    m.wbuf = m.part + W * kSpotChunk;
    m.fac = m.wbuf + W * 32 * kWarpRow;
    return m;
}

// Spot tables of hologram H into shared memory.
template <int THREADS>
__device__ __forceinline__ void load_spot_tables(const HoloDev &H, const TileSmem &m)
{
    for (int n = threadIdx.x; n < H.N; n += THREADS) {
        m.coef[n] = H.coef[n];
        SpotState st = H.state[n];
        m.bw[n] = make_uint2(st.theta + kFixRound, __float_as_uint(st.w * st.a0));
    }
}

// The warp's 32 lane partials of qc <= 16 spots sit in wbuf (row = lane,
// column = spot).  Lane 16 h + q sums rows 16 h .. 16 h + 15 of column q, the
// two halves meet by one shuffle, and lane q < qc stores the warp total.
__device__ __forceinline__ void warp_transpose_reduce(const float2 *wbuf, int lane, int qc, float2 *dst)
{
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
    if (h == 0 && q < qc) dst[q] = make_float2(ar, ai);
}

// Sums the warps' totals of spots n0 .. n0 + nc - 1 and writes the tile's
// partial fields (FP64 for the metrics pass).
template <int THREADS>
__device__ __forceinline__ void store_tile_partials(const HoloDev &H, int pass, int t, int n0, int nc,
                                                    const float2 *s_part)
{
    constexpr int W = THREADS / 32;
    for (int q = threadIdx.x; q < nc; q += THREADS) {
        const size_t o = (size_t)t * H.N + n0 + q;
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
}

// After a tile's partials are written: the last tile of this hologram's pass
// (arrival counter) runs the update or the metrics, then resets the counter.
template <int THREADS>
__device__ __forceinline__ void finish_tile(const HoloDev &H, const LaunchSlot &sl, float2 *s_v, double *s_red,
                                            int *s_last)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(H.counter, 1u);
        *s_last = (prev == (unsigned)(sl.tiles - 1)) ? 1 : 0;
    }
    __syncthreads();
    if (*s_last) {
        __threadfence();
        if (sl.pass == kPassFinal) tail_metrics<THREADS>(H, sl, s_red);
        else tail_update<THREADS>(H, sl, s_v, s_red);
        __syncthreads();
        if (threadIdx.x == 0) *H.counter = 0u;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- pupil --
// The subset draw of iteration j (Section 3, "Compressed sensing"): the
// permutation's keys, and for the windows reading (one order made at the
// start, keyed by j = 0) the window's offset ((j - 1) Mp) mod D.
struct SubsetDraw {
    SubsetKeys K;
    uint32_t off;
    UDiv fb;   // the permutation rectangle's b, as a divisor
};

__device__ __forceinline__ SubsetDraw subset_draw(const HoloDev &H, int j)
{
    SubsetDraw d;
    d.K = subset_keys(H.seed, H.windows ? 0 : j);
    d.off = 0u;
    d.fb = udiv_of(H.fb);
    if (H.windows) {
        const int64_t D = H.D;
        int64_t t = (((int64_t)(j - 1) % D) * ((int64_t)H.Mp % D)) % D;
        d.off = (uint32_t)(t < 0 ? t + D : t);
    }
    return d;
}

// Grid pixel m = r P + i of pupil pixel q (the pupil's pixels in row-major
// order).  Round aperture: the row is found by binary search in the row
// table (first pupil index of each row, monotone), then the column offset.
__device__ __forceinline__ uint32_t pupil_pixel(const HoloDev &H, uint32_t q)
{
    if (H.aperture == 0) return q;
    int lo = 0, hi = H.P - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((uint32_t)__ldg(&H.rows[mid].x) <= q) lo = mid;
        else hi = mid - 1;
    }
    const int2 rw = __ldg(&H.rows[lo]);
    return (uint32_t)lo * (uint32_t)H.P + (uint32_t)rw.y + (q - (uint32_t)rw.x);
}

// Pixel k (< Mp) of the subset S_j.
__device__ __forceinline__ uint32_t subset_pixel(const HoloDev &H, const SubsetDraw &d, uint32_t k)
{
    uint32_t kk = k + d.off;
    kk = kk >= (uint32_t)H.D ? kk - (uint32_t)H.D : kk;
    return pupil_pixel(H, permute_domain(kk, (uint32_t)H.D, H.fa, d.fb, d.K));
}

// The subset mask of iteration j of a compressed pass on the tensor cores or
// the subset-only gather kernel: bit c of word r * mask_words + c / 32 is set
// when pixel r P + c belongs to S_j (two masks per hologram, by the parity of j).
__device__ __forceinline__ uint32_t *subset_mask(const HoloDev &H, int j)
{
    return H.mask + (size_t)(j & 1) * (size_t)H.mask_stride;
}

// Pupil amplitude A = exp(-rho^2 / waist^2) = exp2(-kA rho^2) (Eq. 3's A;
// Section 4's Gaussian beam), 1 for a uniform pupil.
__device__ __forceinline__ float pupil_amp(const HoloDev &H, float rho2)
{
    return H.kA != 0.f ? exp2f(-H.kA * rho2) : 1.f;
}

// A tile of a compressed iteration: THREADS * PPT pixels of the subset S_j,
// each phasor evaluated directly (fixed-point phase, hardware sine/cosine).
template <int THREADS, int PPT>
__device__ void process_tile(const HoloDev &H, const LaunchSlot &sl, int t, int maxN,
                             unsigned char *smem, double *s_red, int *s_last)
{
    const TileSmem m = tile_smem<THREADS>(smem, maxN);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int P = H.P, N = H.N;
    const int pass = sl.pass;   // kPassSubset
    const int count = sl.count;

    load_spot_tables<THREADS>(H, m);

    // this thread's pixels of S_j, with their pupil amplitudes (0 past the end)
    const SubsetDraw dr = subset_draw(H, sl.j);
    const int half = P >> 1;
    int32_t xp[PPT], yp[PPT];
    uint32_t r2[PPT];
    float qf[PPT], msk[PPT];
    const int base = t * (THREADS * PPT);
#pragma unroll
    for (int s = 0; s < PPT; ++s) {
        int idx = base + s * THREADS + tid;
        bool valid = idx < count;
        uint32_t mm = subset_pixel(H, dr, valid ? (uint32_t)idx : 0u);
        int r = (int)(mm / (uint32_t)P);
        int i = (int)mm - r * P;
        xp[s] = i - half;
        yp[s] = r - half;
        r2[s] = (uint32_t)(xp[s] * xp[s] + yp[s] * yp[s]);
        qf[s] = (float)r2[s];
        msk[s] = valid ? pupil_amp(H, qf[s]) : 0.f;
    }
    __syncthreads();

    // back-propagation, Eq. 1
    float sr[PPT], si[PPT];
#pragma unroll
    for (int s = 0; s < PPT; ++s) { sr[s] = 0.f; si[s] = 0.f; }
    for (int n = 0; n < N; ++n) {
        const int4 c = m.coef[n];
        const uint2 bw = m.bw[n];
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
    for (int s = 0; s < PPT; ++s) padd[s] = kFixRound - rad_to_fix(atan2f(si[s], sr[s]));

    // forward projection, Eq. 3: each thread's phasor is e^{i (phi_n - Phi_m)},
    // the conjugate of the term; per spot the thread sums its PPT pixels, the
    // warp's partials go through the transpose buffer, the warps' totals
    // through m.part, and one partial per (tile, spot) leaves.
    float2 *wbuf = m.wbuf + warp * 32 * kWarpRow;
    for (int n0 = 0; n0 < N; n0 += kSpotChunk) {
        const int nc = min(kSpotChunk, N - n0);
        for (int q0 = 0; q0 < nc; q0 += kWarpChunk) {
            const int qc = min(kWarpChunk, nc - q0);
            for (int q = 0; q < qc; ++q) {
                const int4 c = m.coef[n0 + q0 + q];
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
                wbuf[lane * kWarpRow + q] = make_float2(vr, -vi);
            }
            __syncwarp();
            warp_transpose_reduce(wbuf, lane, qc, m.part + warp * kSpotChunk + q0);
            __syncwarp();
        }
        __syncthreads();
        store_tile_partials<THREADS>(H, pass, t, n0, nc, m.part);
        __syncthreads();
    }
    finish_tile<THREADS>(H, sl, m.v, s_red, s_last);
}

// A tile of a compressed iteration with the half-precision sincos option
// (sincos_fix_h2): as process_tile, with each pair of pixels' phasors made by
// one packed FP16 evaluation.  The back-propagation sums run in FP16 over 8
// spots at a time and are flushed into FP32; the forward sums over the
// thread's PPT pixels run in FP16 and are converted before the reductions.
template <int THREADS, int PPT>
__device__ void process_tile_h2(const HoloDev &H, const LaunchSlot &sl, int t, int maxN,
                                unsigned char *smem, double *s_red, int *s_last)
{
    static_assert(PPT % 2 == 0, "pixels go in pairs");
    constexpr int NP = PPT / 2;
    constexpr int kFlush = 8;
    const TileSmem m = tile_smem<THREADS>(smem, maxN);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int P = H.P, N = H.N;
    const int count = sl.count;

    load_spot_tables<THREADS>(H, m);

    const SubsetDraw dr = subset_draw(H, sl.j);
    const int half = P >> 1;
    int32_t xp[PPT], yp[PPT];
    uint32_t r2[PPT];
    __half2 msk[NP];
    float amp_prev = 0.f;
    const int base = t * (THREADS * PPT);
#pragma unroll
    for (int s = 0; s < PPT; ++s) {
        int idx = base + s * THREADS + tid;
        bool valid = idx < count;
        uint32_t mm = subset_pixel(H, dr, valid ? (uint32_t)idx : 0u);
        int r = (int)(mm / (uint32_t)P);
        int i = (int)mm - r * P;
        xp[s] = i - half;
        yp[s] = r - half;
        r2[s] = (uint32_t)(xp[s] * xp[s] + yp[s] * yp[s]);
        const float a = valid ? pupil_amp(H, (float)r2[s]) : 0.f;
        if (s & 1) msk[s / 2] = __floats2half2_rn(amp_prev, a);
        amp_prev = a;
    }
    __syncthreads();

    // back-propagation, Eq. 1
    float sr[PPT], si[PPT];
    __half2 hr[NP], hi[NP];
#pragma unroll
    for (int s = 0; s < PPT; ++s) { sr[s] = 0.f; si[s] = 0.f; }
#pragma unroll
    for (int k = 0; k < NP; ++k) { hr[k] = __float2half2_rn(0.f); hi[k] = __float2half2_rn(0.f); }
    for (int n0 = 0; n0 < N; n0 += kFlush) {
        const int n1 = min(n0 + kFlush, N);
        for (int n = n0; n < n1; ++n) {
            const int4 c = m.coef[n];
            const uint2 bw = m.bw[n];
            const uint32_t add = bw.x - kFixRound + kHalfAddend;
            const __half2 w2 = __float2half2_rn(__uint_as_float(bw.y));
            const SpotFix f = {c.x, c.y, c.z, 0.f};
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                __half2 sn, cs;
                sincos_fix_h2(fix_phase(f, xp[2 * k], yp[2 * k], r2[2 * k], add),
                              fix_phase(f, xp[2 * k + 1], yp[2 * k + 1], r2[2 * k + 1], add), sn, cs);
                hr[k] = __hfma2(w2, cs, hr[k]);
                hi[k] = __hfma2(w2, sn, hi[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float2 a = __half22float2(hr[k]), b = __half22float2(hi[k]);
            sr[2 * k] += a.x;
            sr[2 * k + 1] += a.y;
            si[2 * k] += b.x;
            si[2 * k + 1] += b.y;
            hr[k] = __float2half2_rn(0.f);
            hi[k] = __float2half2_rn(0.f);
        }
    }

    // Phi_m = arg S_m; the forward pass needs -Phi_m as a fixed-point addend
    uint32_t padd[PPT];
#pragma unroll
    for (int s = 0; s < PPT; ++s) padd[s] = kHalfAddend - rad_to_fix(atan2f(si[s], sr[s]));

    // forward projection, Eq. 3 (conjugate phasors, as in process_tile)
    float2 *wbuf = m.wbuf + warp * 32 * kWarpRow;
    for (int n0 = 0; n0 < N; n0 += kSpotChunk) {
        const int nc = min(kSpotChunk, N - n0);
        for (int q0 = 0; q0 < nc; q0 += kWarpChunk) {
            const int qc = min(kWarpChunk, nc - q0);
            for (int q = 0; q < qc; ++q) {
                const int4 c = m.coef[n0 + q0 + q];
                const SpotFix f = {c.x, c.y, c.z, 0.f};
                __half2 vr2 = __float2half2_rn(0.f), vi2 = __float2half2_rn(0.f);
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    __half2 sn, cs;
                    sincos_fix_h2(fix_phase(f, xp[2 * k], yp[2 * k], r2[2 * k], padd[2 * k]),
                                  fix_phase(f, xp[2 * k + 1], yp[2 * k + 1], r2[2 * k + 1], padd[2 * k + 1]), sn, cs);
                    vr2 = __hfma2(msk[k], cs, vr2);
                    vi2 = __hfma2(msk[k], sn, vi2);
                }
                const float2 a = __half22float2(vr2), b = __half22float2(vi2);
                wbuf[lane * kWarpRow + q] = make_float2(a.x + a.y, -(b.x + b.y));
            }
            __syncwarp();
            warp_transpose_reduce(wbuf, lane, qc, m.part + warp * kSpotChunk + q0);
            __syncwarp();
        }
        __syncthreads();
        store_tile_partials<THREADS>(H, sl.pass, t, n0, nc, m.part);
        __syncthreads();
    }
    finish_tile<THREADS>(H, sl, m.v, s_red, s_last);
}

// One spot factor of a separable tile: e^{i 2 pi (c u + G u^2)} for pixel
// coordinate u (x' with the tilt A, or y' with the tilt B) plus an addend,
// scaled by w.  The fixed-point split is that of fix_phase.
__device__ __forceinline__ float2 spot_factor(int32_t tilt, int32_t Gh, float gl, int32_t u, uint32_t addend, float w)
{
    const uint32_t u2 = (uint32_t)(u * u);
    uint32_t T = addend + (uint32_t)tilt * (uint32_t)u;
    T += (uint32_t)Gh * u2;
    float s, c;
    sincos_fix(T, fmaf(gl, (float)u2, -kTwoPiF), s, c);
    return make_float2(w * c, w * s);
}

// Gray levels of four phases in [0, 2 pi) of grid row `row`, columns col ..
// col + 3 (those inside the grid), into the SLM frame: level
// rint(Phi * lscale) mod levels in FP32, gray = lut[level].  Four aligned
// in-grid bytes go as one 32-bit store.
__device__ __forceinline__ void write_gray4(const HoloDev &H, int row, int col, const float o[4])
{
    uint32_t g[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int l = __float2int_rn(o[j] * H.lscale);
        l = l >= H.levels ? l - H.levels : l;
        g[j] = __ldg(H.lut + l);
    }
    uint8_t *dst = H.slm + (size_t)row * H.slm_pitch + col;
    if (col + 3 < H.P && (reinterpret_cast<uintptr_t>(dst) & 3) == 0) {
        *reinterpret_cast<uint32_t *>(dst) = g[0] | (g[1] << 8) | (g[2] << 16) | (g[3] << 24);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (col + j < H.P) dst[j] = (uint8_t)g[j];
    }
}

// A tile of a pass over all pixels (full iteration or final pass), using the
// separability of the lens-and-prism phase (Eq. 2):
//   e^{i phi_n(x', y')} = C_n(x') R_n(y'),  C_n = e^{i 2 pi (a x' + g x'^2)},
//                                           R_n = e^{i 2 pi (b y' + g y'^2)}.
// Over a rectangle of ROWS x 64 pixels the N spots need ROWS + 64 phasors each
// instead of 64 ROWS.  Back-propagation (Eq. 1) is then
//   S(x', y') = sum_n [w_n a_n e^{i theta_n} R_n(y')] C_n(x'),
// one complex multiply-add per (pixel, spot), and the forward projection
// (Eq. 3) is  V_n = sum_x' conj(C_n(x')) sum_y' e^{i Phi(x', y')} conj(R_n(y')).
template <int THREADS>
__device__ void process_full_tile(const HoloDev &H, const LaunchSlot &sl, int t, int maxN,
                                  unsigned char *smem, double *s_red, int *s_last)
{
    constexpr int ROWS = THREADS / 4;
    constexpr int COLS = kFullCols;
    constexpr int NF = kFactorChunk;
    const TileSmem m = tile_smem<THREADS>(smem, maxN);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int P = H.P, N = H.N, half = P >> 1;
    const int pass = sl.pass;
    const int col_tiles = (P + COLS - 1) / COLS;
    const int y0 = (t / col_tiles) * ROWS, x0 = (t % col_tiles) * COLS;
    const int tx = tid & 15, ty = tid >> 4;   // pixels: rows y0 + 4 ty + i, columns x0 + 4 tx + j
    float2 *sR = m.fac;                 // NF x ROWS
    float2 *sC = m.fac + NF * ROWS;     // NF x COLS, interleaved (col_slot)

    // a tile wholly outside the round pupil: zero partials, and in the final
    // pass phase 0 (gray lut[0]) over its grid pixels
    if (H.aperture != 0) {
        const int ylo = y0 - half, yhi = min(y0 + ROWS, P) - 1 - half;
        const int xlo = x0 - half, xhi = min(x0 + COLS, P) - 1 - half;
        const int64_t dy = ylo > 0 ? ylo : (yhi < 0 ? yhi : 0);   // nearest y' to 0 in the tile
        const int64_t dx = xlo > 0 ? xlo : (xhi < 0 ? xhi : 0);
        if (dx * dx + dy * dy > (int64_t)half * half) {
            for (int n = tid; n < N; n += THREADS) {
                if (pass == kPassFinal) H.part64[(size_t)t * N + n] = make_double2(0.0, 0.0);
                else H.part[(size_t)t * N + n] = make_float2(0.f, 0.f);
            }
            if (pass == kPassFinal) {
                const int rows = min(ROWS, P - y0), cols = min(COLS, P - x0);
                const uint8_t g0 = H.slm ? __ldg(H.lut) : 0;
                for (int f = tid; f < rows * cols; f += THREADS) {
                    const int r = y0 + f / cols, c = x0 + f % cols;
                    if (H.phase_out) H.phase_out[(size_t)r * P + c] = 0.f;
                    if (H.slm) H.slm[(size_t)r * H.slm_pitch + c] = g0;
                }
            }
            finish_tile<THREADS>(H, sl, m.v, s_red, s_last);
            return;
        }
    }

    load_spot_tables<THREADS>(H, m);
    __syncthreads();

    // spot factors of spots n0 .. n0 + nc - 1 into sR, sC; the row factors
    // carry w_n a_n e^{i theta_n} when `weighted`
    auto make_factors = [&](int n0, int nc, bool weighted) {
        for (int f = tid; f < nc * (ROWS + COLS); f += THREADS) {
            if (f < nc * ROWS) {
                const int q = f / ROWS, r = f - q * ROWS;
                const int4 c = m.coef[n0 + q];
                const uint2 bw = m.bw[n0 + q];
                sR[q * ROWS + r] = spot_factor(c.y, c.z, __int_as_float(c.w), y0 + r - half,
                                               weighted ? bw.x : kFixRound,
                                               weighted ? __uint_as_float(bw.y) : 1.f);
            } else {
                const int g = f - nc * ROWS, q = g / COLS, x = g - q * COLS;
                const int4 c = m.coef[n0 + q];
                sC[q * COLS + col_slot(x)] =
                    spot_factor(c.x, c.z, __int_as_float(c.w), x0 + x - half, kFixRound, 1.f);
            }
        }
    };
    auto load_factors = [&](int q, float2 R[4], float2 C[4]) {
        const float4 r01 = *reinterpret_cast<const float4 *>(&sR[q * ROWS + 4 * ty]);
        const float4 r23 = *reinterpret_cast<const float4 *>(&sR[q * ROWS + 4 * ty + 2]);
        const float4 c01 = *reinterpret_cast<const float4 *>(&sC[q * COLS + 2 * tx]);
        const float4 c23 = *reinterpret_cast<const float4 *>(&sC[q * COLS + 32 + 2 * tx]);
        R[0] = make_float2(r01.x, r01.y); R[1] = make_float2(r01.z, r01.w);
        R[2] = make_float2(r23.x, r23.y); R[3] = make_float2(r23.z, r23.w);
        C[0] = make_float2(c01.x, c01.y); C[1] = make_float2(c01.z, c01.w);
        C[2] = make_float2(c23.x, c23.y); C[3] = make_float2(c23.z, c23.w);
    };

    // back-propagation, Eq. 1
    float2 S[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) S[i][j] = make_float2(0.f, 0.f);
    for (int n0 = 0; n0 < N; n0 += NF) {
        const int nc = min(NF, N - n0);
        make_factors(n0, nc, true);
        __syncthreads();
        for (int q = 0; q < nc; ++q) {
            float2 R[4], C[4];
            load_factors(q, R, C);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    S[i][j].x = fmaf(R[i].x, C[j].x, fmaf(-R[i].y, C[j].y, S[i][j].x));
                    S[i][j].y = fmaf(R[i].x, C[j].y, fmaf(R[i].y, C[j].x, S[i][j].y));
                }
        }
        __syncthreads();
    }

    // A e^{i Phi} = A S / |S| (arg 0 = 0), kept in S; zero outside the grid and
    // the pupil so it adds nothing below.  The final pass writes Phi (0
    // outside the pupil) and its gray level.
    const bool vec_out = pass == kPassFinal && H.phase_out && (P & 3) == 0 &&
                         (reinterpret_cast<uintptr_t>(H.phase_out) & 15) == 0;
    const int64_t R2 = (int64_t)half * half;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = y0 + 4 * ty + i;
        const int yq = row - half;
        float o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = x0 + 4 * tx + j;
            const int xq = col - half;
            const int64_t rho2 = (int64_t)xq * xq + (int64_t)yq * yq;
            const bool valid = row < P && col < P && (H.aperture == 0 || rho2 <= R2);
            const float n2 = S[i][j].x * S[i][j].x + S[i][j].y * S[i][j].y;
            if (pass == kPassFinal) {
                float ph = atan2f(S[i][j].y, S[i][j].x);
                ph = ph < 0.f ? ph + kTwoPiF : ph;
                o[j] = (ph >= kTwoPiF || !valid) ? 0.f : ph;
            }
            if (!valid) S[i][j] = make_float2(0.f, 0.f);
            else if (n2 > 0.f) {
                const float rs = rsqrtf(n2) * pupil_amp(H, (float)rho2);
                S[i][j] = make_float2(S[i][j].x * rs, S[i][j].y * rs);
            } else S[i][j] = make_float2(pupil_amp(H, (float)rho2), 0.f);
        }
        if (pass == kPassFinal && row < P) {
            const int col = x0 + 4 * tx;
            if (H.phase_out) {
                float *dst = H.phase_out + (size_t)row * P + col;
                if (vec_out && col + 3 < P) {
                    *reinterpret_cast<float4 *>(dst) = make_float4(o[0], o[1], o[2], o[3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (col + j < P) dst[j] = o[j];
                }
            }
            if (H.slm) write_gray4(H, row, col, o);
        }
    }

    // forward projection, Eq. 3, reduced like the compressed tiles
    float2 *wbuf = m.wbuf + warp * 32 * kWarpRow;
    for (int w0 = 0; w0 < N; w0 += kSpotChunk) {
        const int wc = min(kSpotChunk, N - w0);
        for (int n0 = w0; n0 < w0 + wc; n0 += NF) {
            const int nc = min(NF, w0 + wc - n0);   // NF == kWarpChunk: one transpose round
            make_factors(n0, nc, false);
            __syncthreads();
            for (int q = 0; q < nc; ++q) {
                float2 R[4], C[4];
                load_factors(q, R, C);
                float vr = 0.f, vi = 0.f;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float a = 0.f, b = 0.f;             // sum_i e^{i Phi} conj(R_i)
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        a = fmaf(S[i][j].x, R[i].x, fmaf(S[i][j].y, R[i].y, a));
                        b = fmaf(S[i][j].y, R[i].x, fmaf(-S[i][j].x, R[i].y, b));
                    }
                    vr = fmaf(a, C[j].x, fmaf(b, C[j].y, vr));   // times conj(C_j)
                    vi = fmaf(b, C[j].x, fmaf(-a, C[j].y, vi));
                }
                wbuf[lane * kWarpRow + q] = make_float2(vr, vi);
            }
            __syncwarp();
            warp_transpose_reduce(wbuf, lane, nc, m.part + warp * kSpotChunk + (n0 - w0));
            __syncthreads();
        }
        store_tile_partials<THREADS>(H, pass, t, w0, wc, m.part);
        __syncthreads();
    }
    finish_tile<THREADS>(H, sl, m.v, s_red, s_last);
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

// Dynamic shared memory of the tile processors for THREADS threads and up to
// maxN spots (the layout of TileSmem; the factor buffer only for full passes).
__host__ __device__ constexpr size_t tile_smem_bytes(int threads, int maxN, bool factors)
{
    return (size_t)maxN * (sizeof(int4) + sizeof(uint2) + sizeof(float2)) +
           (size_t)(threads / 32) * kSpotChunk * sizeof(float2) +
           (size_t)(threads / 32) * 32 * kWarpRow * sizeof(float2) +
           (factors ? (size_t)kFactorChunk * (threads / 4 + kFullCols) * sizeof(float2) : 0);
}

}  // namespace cswgs
