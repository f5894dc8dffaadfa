// Full iterations and the final pass on the tensor cores (tcgen05, sm_103a).
//
// The lens-and-prism phase (Eq. 2) is separable, e^{i phi_n(x', y')} =
// C_n(x') R_n(y'), so over a tile of 128 rows x 64 columns both passes are
// dense complex matrix products with the spots as the contracted index:
//   back-propagation (Eq. 1):   S(y, x) = sum_n R'_n(y) C_n(x),
//                               R'_n = w_n a_n e^{i theta_n} R_n          [GEMM 1]
//   forward projection (Eq. 3): Z(n, y) = sum_x conj(C_n(x)) u(y, x),
//                               u = A e^{i Phi} = A S / |S|               [GEMM 2]
//                               V_n  = sum_y conj(R_n(y)) Z(n, y)         [per spot, CUDA cores]
// GEMM 1 is M = 128 rows x N = 64 columns x K = 16 spots per instruction,
// GEMM 2 is M = 128 spots x N = 128 rows x K = 16 columns.  The complex
// products become real ones (re re - im im, re im + im re), and every FP32
// operand is split into two BF16 halves, v = hi + lo, with the product kept as
// hi hi + hi lo + lo hi: 2^-16 relative per product, FP32-class phases.  The
// accumulators (FP32) live in tensor memory; operands are staged in shared
// memory in the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per
// core matrix).  One thread issues the MMAs and commits them to an mbarrier;
// every wait on it is bounded and records a timeout in the launch's status
// word instead of hanging.
#include <cuda_bf16.h>

#include "tile.cuh"

namespace cswgs {
namespace tc {

constexpr int kRows = 128;          // tile rows (GEMM 1 M, GEMM 2 N)
constexpr int kCols = 64;           // tile columns (GEMM 1 N, GEMM 2 K)
constexpr int kThreads = 256;
constexpr int kChunk = 16;          // spots per GEMM 1 instruction (K)
constexpr int kSpotBlock = 128;     // spots per GEMM 2 instruction (M)
constexpr int kTmemCols = 256;      // S (cols 0..127) and then Z (cols 0..255)
constexpr uint32_t kWaitPolls = 1u << 20;

// component tiles (bytes): GEMM 1 operands per stage, GEMM 2 operands
constexpr uint32_t kA1 = kRows * kChunk * 2;        // R' component [128 rows][16 spots]
constexpr uint32_t kB1 = kCols * kChunk * 2;        // C component [64 columns][16 spots]
constexpr uint32_t kStage = 4 * kA1 + 4 * kB1;      // one GEMM 1 stage
constexpr uint32_t kU = kRows * kCols * 2;          // u component [128 rows][64 columns]
constexpr uint32_t kCs = kSpotBlock * kCols * 2;    // C component [128 spots][64 columns]

__host__ __device__ constexpr size_t align1k(size_t x) { return (x + 1023) & ~(size_t)1023; }

// Dynamic shared memory: spot tables, two GEMM 1 stages, u, C for GEMM 2,
// the half sums of the last epilogue (and 1 KB to align the base).
__host__ __device__ constexpr size_t smem_bytes(int maxN)
{
    return 1024 + align1k((size_t)maxN * (sizeof(int4) + sizeof(uint2) + sizeof(float2))) + 2 * (size_t)kStage +
           4 * (size_t)kU + 4 * (size_t)kCs + kSpotBlock * sizeof(float2);
}

__host__ __device__ inline int tiles(int P) { return ((P + kRows - 1) / kRows) * ((P + kCols - 1) / kCols); }

struct Smem {
    int4 *coef;
    uint2 *bw;
    float2 *v;                  // tail scratch (maxN)
    unsigned char *g1[2];       // stages: A components (4 x kA1), then B components (4 x kB1)
    unsigned char *u;           // 4 x kU: u re hi, re lo, im hi, im lo
    unsigned char *cs;          // 4 x kCs: C re hi, re lo, im hi, im lo
    float2 *vh;                 // kSpotBlock half sums
};

__device__ __forceinline__ Smem carve(unsigned char *raw, int maxN)
{
    unsigned char *b = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~(uintptr_t)1023);
    Smem m;
    m.coef = reinterpret_cast<int4 *>(b);
    m.bw = reinterpret_cast<uint2 *>(m.coef + maxN);
    m.v = reinterpret_cast<float2 *>(m.bw + maxN);
    b += align1k((size_t)maxN * (sizeof(int4) + sizeof(uint2) + sizeof(float2)));
    m.g1[0] = b;
    m.g1[1] = b + kStage;
    m.u = b + 2 * kStage;
    m.cs = m.u + 4 * kU;
    m.vh = reinterpret_cast<float2 *>(m.cs + 4 * kCs);
    return m;
}

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row, k) of a [rows][K] BF16 tile in the no-swizzle
// K-major layout: core matrices of 8 rows x 8 elements (16 bytes a row, 128
// bytes each), the K / 8 cores of a row group side by side.
__device__ __forceinline__ uint32_t core_off(int row, int k, int K)
{
    return (uint32_t)((row >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor of a K-major no-swizzle tile: start address,
// leading byte offset (next core matrix along K), stride byte offset (next
// 8-row group), version 1, no swizzle.
__device__ __forceinline__ uint64_t desc(uint32_t start, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((start & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc(int M, int N, int neg_a)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)neg_a << 13) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar)
                 : "memory");
}

// Bounded wait for phase `parity` of an mbarrier; false when it ran out.
__device__ __forceinline__ bool wait(uint32_t mbar, uint32_t parity)
{
    for (uint32_t it = 0; it < kWaitPolls; ++it) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Eight complex values -> the four BF16 component rows (re hi, re lo, im hi,
// im lo), one 16-byte store each, at byte offset `off` of four tiles `stride`
// bytes apart.
__device__ __forceinline__ void put8(unsigned char *base, uint32_t stride, uint32_t off, const float2 *v)
{
    uint32_t w[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float re[2], im[2];
        __nv_bfloat16 rh[2], rl[2], ih[2], il[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            re[e] = v[2 * q + e].x;
            im[e] = v[2 * q + e].y;
            rh[e] = __float2bfloat16_rn(re[e]);
            rl[e] = __float2bfloat16_rn(re[e] - __bfloat162float(rh[e]));
            ih[e] = __float2bfloat16_rn(im[e]);
            il[e] = __float2bfloat16_rn(im[e] - __bfloat162float(ih[e]));
        }
        w[0][q] = (uint32_t)__bfloat16_as_ushort(rh[0]) | ((uint32_t)__bfloat16_as_ushort(rh[1]) << 16);
        w[1][q] = (uint32_t)__bfloat16_as_ushort(rl[0]) | ((uint32_t)__bfloat16_as_ushort(rl[1]) << 16);
        w[2][q] = (uint32_t)__bfloat16_as_ushort(ih[0]) | ((uint32_t)__bfloat16_as_ushort(ih[1]) << 16);
        w[3][q] = (uint32_t)__bfloat16_as_ushort(il[0]) | ((uint32_t)__bfloat16_as_ushort(il[1]) << 16);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
        *reinterpret_cast<uint4 *>(base + c * stride + off) = make_uint4(w[c][0], w[c][1], w[c][2], w[c][3]);
}

// Per-block state that lives across tiles: tensor memory and the barriers.
struct State {
    uint32_t tmem;
    uint32_t mbar[3];     // GEMM 1 stages 0 and 1, GEMM 2
    uint32_t phase[3];
    bool failed;
};

// Issues the 12 MMAs of a complex product with split operands:
//   D_re += Ar Br - Ai Bi,  D_im += Ar Bi + Ai Br   (conj_a = 0)
//   D_re += Ar Br + Ai Bi,  D_im += Ar Bi - Ai Br   (conj_a = 1)
// a[c], b[c]: descriptors of the components re hi, re lo, im hi, im lo.
__device__ __forceinline__ void complex_mma(uint32_t d_re, uint32_t d_im, const uint64_t a[4], const uint64_t b[4],
                                            uint32_t id, uint32_t id_neg, uint32_t acc, int conj_a)
{
    const uint32_t id_ii = conj_a ? id : id_neg;     // the Ai Bi term of D_re
    const uint32_t id_ir = conj_a ? id_neg : id;     // the Ai Br term of D_im
    mma(d_re, a[0], b[0], id, acc);
    mma(d_re, a[0], b[1], id, 1u);
    mma(d_re, a[1], b[0], id, 1u);
    mma(d_re, a[2], b[2], id_ii, 1u);
    mma(d_re, a[2], b[3], id_ii, 1u);
    mma(d_re, a[3], b[2], id_ii, 1u);
    mma(d_im, a[0], b[2], id, acc);
    mma(d_im, a[0], b[3], id, 1u);
    mma(d_im, a[1], b[2], id, 1u);
    mma(d_im, a[2], b[0], id_ir, 1u);
    mma(d_im, a[2], b[1], id_ir, 1u);
    mma(d_im, a[3], b[0], id_ir, 1u);
}

// Waits, on every thread, for the next phase of barrier b.  The outcome is
// voted across the block, so every thread takes the same path afterwards; a
// timed-out wait sets bit 0 of the launch's status word and turns the block's
// remaining tiles into empty ones (nothing waits on a barrier again).
__device__ __forceinline__ void wait_all(State &st, int b, unsigned *status)
{
    bool ok = true;
    if (!st.failed) ok = wait(st.mbar[b], st.phase[b]);
    ok = __syncthreads_and(ok) != 0;
    st.phase[b] ^= 1u;
    if (!ok) {
        if (!st.failed && threadIdx.x == 0) atomicOr(status, 1u);
        st.failed = true;
    }
}

// One tile of a full iteration or the final pass.
__device__ void process_tile(const HoloDev &H, const LaunchSlot &sl, int t, int maxN, unsigned char *raw,
                             double *s_red, int *s_last, State &st, unsigned *status)
{
    const Smem m = carve(raw, maxN);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = H.P, N = H.N, half = P >> 1;
    const int pass = sl.pass;
    const int col_tiles = (P + kCols - 1) / kCols;
    const int y0 = (t / col_tiles) * kRows, x0 = (t % col_tiles) * kCols;

    // a tile wholly outside the round pupil: zero partials; in the final pass
    // phase 0 (gray lut[0]) over its grid pixels.  After a timed-out wait the
    // block does the same for its remaining tiles, so every hologram's tiles
    // still arrive.
    bool empty = st.failed;
    if (H.aperture != 0) {
        const int ylo = y0 - half, yhi = min(y0 + kRows, P) - 1 - half;
        const int xlo = x0 - half, xhi = min(x0 + kCols, P) - 1 - half;
        const int64_t dy = ylo > 0 ? ylo : (yhi < 0 ? yhi : 0);
        const int64_t dx = xlo > 0 ? xlo : (xhi < 0 ? xhi : 0);
        empty |= dx * dx + dy * dy > (int64_t)half * half;
    }
    if (empty) {
        for (int n = tid; n < N; n += kThreads) {
            if (pass == kPassFinal) H.part64[(size_t)t * N + n] = make_double2(0.0, 0.0);
            else H.part[(size_t)t * N + n] = make_float2(0.f, 0.f);
        }
        if (pass == kPassFinal) {
            const int rows = min(kRows, P - y0), cols = min(kCols, P - x0);
            const uint8_t g0 = H.slm ? __ldg(H.lut) : 0;
            for (int f = tid; f < rows * cols; f += kThreads) {
                const int r = y0 + f / cols, c = x0 + f % cols;
                if (H.phase_out) H.phase_out[(size_t)r * P + c] = 0.f;
                if (H.slm) H.slm[(size_t)r * H.slm_pitch + c] = g0;
            }
        }
        finish_tile<kThreads>(H, sl, m.v, s_red, s_last);
        return;
    }

    for (int n = tid; n < N; n += kThreads) {
        m.coef[n] = H.coef[n];
        const SpotState s = H.state[n];
        m.bw[n] = make_uint2(s.theta + kFixRound, __float_as_uint(s.w * s.a0));
    }
    __syncthreads();

    const uint32_t id1 = idesc(kRows, kCols, 0), id1n = idesc(kRows, kCols, 1);
    const uint32_t id2 = idesc(kSpotBlock, kRows, 0), id2n = idesc(kSpotBlock, kRows, 1);
    const uint32_t t_re = st.tmem, t_im1 = st.tmem + kCols, t_im2 = st.tmem + kRows;

    // ---- GEMM 1: S = R' C^T over spot chunks, two stages ----------------------
    const int nchunk = (N + kChunk - 1) / kChunk;
    for (int c = 0; c < nchunk; ++c) {
        const int s = c & 1;
        if (c >= 2) wait_all(st, s, status);
        unsigned char *stg = m.g1[s];
        // 256 row items (row, 8 spots) of R', then 128 column items of C
        for (int i = tid; i < 2 * kRows + 2 * kCols; i += kThreads) {
            float2 v[8];
            if (i < 2 * kRows) {
                const int row = i >> 1, g = i & 1;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int n = c * kChunk + g * 8 + q;
                    if (n < N) {
                        const int4 cf = m.coef[n];
                        const uint2 bw = m.bw[n];
                        v[q] = spot_factor(cf.y, cf.z, __int_as_float(cf.w), y0 + row - half, bw.x,
                                           __uint_as_float(bw.y));
                    } else {
                        v[q] = make_float2(0.f, 0.f);
                    }
                }
                put8(stg, kA1, core_off(row, g * 8, kChunk), v);
            } else {
                const int j = i - 2 * kRows, col = j >> 1, g = j & 1;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int n = c * kChunk + g * 8 + q;
                    if (n < N) {
                        const int4 cf = m.coef[n];
                        v[q] = spot_factor(cf.x, cf.z, __int_as_float(cf.w), x0 + col - half, kFixRound, 1.f);
                    } else {
                        v[q] = make_float2(0.f, 0.f);
                    }
                }
                put8(stg + 4 * kA1, kB1, core_off(col, g * 8, kChunk), v);
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0 && !st.failed) {
            uint64_t a[4], b[4];
            for (int q = 0; q < 4; ++q) {
                a[q] = desc(saddr(stg + q * kA1), 128, 256);
                b[q] = desc(saddr(stg + 4 * kA1 + q * kB1), 128, 256);
            }
            complex_mma(t_re, t_im1, a, b, id1, id1n, c > 0 ? 1u : 0u, 0);
            commit(st.mbar[s]);
        }
    }
    // the last two chunks' commits (every earlier one was waited for above)
    for (int c = max(0, nchunk - 2); c < nchunk; ++c) wait_all(st, c & 1, status);
    fence_after();

    // ---- epilogue 1: u = A S / |S| into GEMM 2's B operand; Phi and gray out --
    {
        const int q = warp & 3, h = warp >> 2;
        const int row = 32 * q + lane, xs = 32 * h;
        const uint32_t lanes = (uint32_t)(32 * q) << 16;
        float sr[32], si[32];
        ld16(t_re + lanes + xs, sr);
        ld16(t_re + lanes + xs + 16, sr + 16);
        ld16(t_im1 + lanes + xs, si);
        ld16(t_im1 + lanes + xs + 16, si + 16);
        ld_wait();
        const int gy = y0 + row, yq = gy - half;
        const int64_t R2 = (int64_t)half * half;
        float o[32];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            float2 u[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int j = 8 * g + e;
                const int gx = x0 + xs + j, xq = gx - half;
                const int64_t rho2 = (int64_t)xq * xq + (int64_t)yq * yq;
                const bool valid = gy < P && gx < P && (H.aperture == 0 || rho2 <= R2);
                const float a = sr[j], b = si[j];
                const float n2 = a * a + b * b;
                if (pass == kPassFinal) {
                    float ph = atan2f(b, a);
                    ph = ph < 0.f ? ph + kTwoPiF : ph;
                    o[j] = (ph >= kTwoPiF || !valid) ? 0.f : ph;
                }
                if (!valid) u[e] = make_float2(0.f, 0.f);
                else if (n2 > 0.f) {
                    const float rs = rsqrtf(n2) * pupil_amp(H, (float)rho2);
                    u[e] = make_float2(a * rs, b * rs);
                } else u[e] = make_float2(pupil_amp(H, (float)rho2), 0.f);
            }
            put8(m.u, kU, core_off(row, xs + 8 * g, kCols), u);
        }
        if (pass == kPassFinal && gy < P) {
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                const int col = x0 + xs + 4 * g;
                if (col >= P) break;
                if (H.phase_out) {
                    float *dst = H.phase_out + (size_t)gy * P + col;
                    if (col + 3 < P && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
                        *reinterpret_cast<float4 *>(dst) = make_float4(o[4 * g], o[4 * g + 1], o[4 * g + 2], o[4 * g + 3]);
                    } else {
                        for (int e = 0; e < 4; ++e)
                            if (col + e < P) dst[e] = o[4 * g + e];
                    }
                }
                if (H.slm) write_gray4(H, gy, col, o + 4 * g);
            }
        }
    }

    // ---- GEMM 2 per block of 128 spots, then V_n = sum_y conj(R_n(y)) Z(n, y) --
    for (int sb = 0; sb * kSpotBlock < N; ++sb) {
        // C of this block's spots over the tile's 64 columns: 128 x 8 items
        for (int i = tid; i < kSpotBlock * (kCols / 8); i += kThreads) {
            const int nl = i >> 3, g = i & 7, n = sb * kSpotBlock + nl;
            float2 v[8];
            if (n < N) {
                const int4 cf = m.coef[n];
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    v[e] = spot_factor(cf.x, cf.z, __int_as_float(cf.w), x0 + 8 * g + e - half, kFixRound, 1.f);
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = make_float2(0.f, 0.f);
            }
            put8(m.cs, kCs, core_off(nl, 8 * g, kCols), v);
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0 && !st.failed) {
            for (int ks = 0; ks < kCols / 16; ++ks) {
                uint64_t a[4], b[4];
                for (int q = 0; q < 4; ++q) {
                    a[q] = desc(saddr(m.cs + q * kCs) + ks * 256, 128, (kCols / 8) * 128);
                    b[q] = desc(saddr(m.u + q * kU) + ks * 256, 128, (kCols / 8) * 128);
                }
                complex_mma(t_re, t_im2, a, b, id2, id2n, ks > 0 ? 1u : 0u, 1);
            }
            commit(st.mbar[2]);
        }
        wait_all(st, 2, status);
        fence_after();
        {
            const int q = warp & 3, h = warp >> 2;
            const int nl = 32 * q + lane, n = sb * kSpotBlock + nl;
            const uint32_t lanes = (uint32_t)(32 * q) << 16;
            int4 cf = make_int4(0, 0, 0, 0);
            if (n < N) cf = m.coef[n];
            float vr = 0.f, vi = 0.f;
            for (int y16 = 0; y16 < 64; y16 += 16) {
                const int ys = 64 * h + y16;
                float zr[16], zi[16];
                ld16(t_re + lanes + ys, zr);
                ld16(t_im2 + lanes + ys, zi);
                ld_wait();
                if (n < N) {
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const float2 r = spot_factor(cf.y, cf.z, __int_as_float(cf.w), y0 + ys + e - half, kFixRound, 1.f);
                        vr = fmaf(r.x, zr[e], fmaf(r.y, zi[e], vr));
                        vi = fmaf(r.x, zi[e], fmaf(-r.y, zr[e], vi));
                    }
                }
            }
            if (h == 1) m.vh[nl] = make_float2(vr, vi);
            fence_before();
            __syncthreads();
            if (h == 0 && n < N) {
                const float2 o2 = m.vh[nl];
                const size_t off = (size_t)t * N + n;
                if (pass == kPassFinal) H.part64[off] = make_double2((double)vr + (double)o2.x, (double)vi + (double)o2.y);
                else H.part[off] = make_float2(vr + o2.x, vi + o2.y);
            }
        }
        __syncthreads();
        fence_after();
    }
    finish_tile<kThreads>(H, sl, m.v, s_red, s_last);
}

}  // namespace tc

__global__ void __launch_bounds__(tc::kThreads, 1)
iter_full_tc_kernel(const HoloDev *__restrict__ holos, const LaunchSlot *__restrict__ slots, int nslots,
                    int total_tiles, int maxN, unsigned *queue)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ double s_red[tc::kThreads / 32];
    __shared__ int s_last, s_item, s_slot;
    __shared__ __align__(8) uint64_t s_mbar[3];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int b = 0; b < 3; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc::saddr(&s_mbar[b])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((tid >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(tc::saddr(&s_tmem)), "r"(tc::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    tc::State st;
    st.tmem = s_tmem;
    for (int b = 0; b < 3; ++b) {
        st.mbar[b] = tc::saddr(&s_mbar[b]);
        st.phase[b] = 0u;
    }
    st.failed = false;
    unsigned *status = queue + 2;

    for (;;) {
        if (tid == 0) {
            int item = (int)atomicAdd(queue, 1u);
            s_item = item;
            if (item < total_tiles) {
                int lo = 0, hi = nslots - 1;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (slots[mid].tile_begin <= item) lo = mid;
                    else hi = mid - 1;
                }
                s_slot = lo;
            }
        }
        __syncthreads();
        const int item = s_item;
        if (item >= total_tiles) break;
        const LaunchSlot sl = slots[s_slot];
        const HoloDev H = holos[sl.holo];
        tc::process_tile(H, sl, item - sl.tile_begin, maxN, smem, s_red, &s_last, st, status);
    }
    tc::fence_before();
    __syncthreads();
    if ((tid >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(st.tmem), "r"(tc::kTmemCols));
    if (tid == 0) {
        unsigned done = atomicAdd(queue + 1, 1u);
        if (done == gridDim.x - 1) {
            queue[0] = 0u;
            queue[1] = 0u;
            __threadfence();
        }
    }
}

int full_tc_tiles(int P) { return tc::tiles(P); }

size_t full_tc_smem(int maxN) { return tc::smem_bytes(maxN); }

int full_tc_max_grid(int maxN, int sm_count)
{
    // the dynamic limit is the block's 227 KB less the kernel's static shared memory
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, iter_full_tc_kernel) != cudaSuccess) return 0;
    const size_t limit = 227 * 1024 - fa.sharedSizeBytes;
    const size_t smem = tc::smem_bytes(maxN);
    if (smem > limit) return 0;
    if (cudaFuncSetAttribute(iter_full_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit) !=
        cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, iter_full_tc_kernel, tc::kThreads, smem) !=
        cudaSuccess)
        return 0;
    // tensor memory: each block holds kTmemCols of the SM's 512 columns
    per_sm = min(per_sm, 512 / tc::kTmemCols);
    return per_sm * sm_count;
}

cudaError_t launch_full_tc(const HoloDev *holos, const LaunchSlot *slots, int nslots, int total_tiles, int maxN,
                           unsigned *queue, int grid, cudaStream_t s)
{
    (void)cudaGetLastError();
    iter_full_tc_kernel<<<grid, tc::kThreads, tc::smem_bytes(maxN), s>>>(holos, slots, nslots, total_tiles, maxN,
                                                                          queue);
    return cudaGetLastError();
}

}  // namespace cswgs
