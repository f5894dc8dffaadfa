// Both passes of an iteration on the tensor cores (tcgen05, sm_103a).
//
// The lens-and-prism phase (Eq. 2) is separable, e^{i phi_n(x', y')} =
// C_n(x') R_n(y'), so over a tile of 128 rows x 64 columns both passes are
// dense complex matrix products with the spots as the contracted index:
//   back-propagation (Eq. 1):   S(y, x) = sum_n R'_n(y) C_n(x),
//                               R'_n = w_n a_n e^{i theta_n} R_n          [GEMM 1]
//   forward projection (Eq. 3): Z(n, y) = sum_x conj(C_n(x)) u(y, x),
//                               u = A e^{i Phi} = A S / |S|               [GEMM 2]
//                               V_n  = sum_y conj(R_n(y)) Z(n, y)         [per spot, CUDA cores]
// A compressed iteration is the same computation with u zero outside the
// subset S_j, so the sums run over S_j as Eqs. 1 and 3 ask.
// The accumulators (FP32) live in tensor memory.
// GEMM 1 sets each pixel's phase: its FP32 operands are split into two BF16
// halves, v = hi + lo, and each real product is kept as hi hi + hi lo + lo hi
// (2^-16 relative per product, FP32-class phases).  It runs its complex
// product as two real ones stacked along N (M = 128 rows, N = 128, K = 16
// spots):
//   [S_re | S_im] = R'_re [C_re | C_im] + R'_im [-C_im | C_re],
// with the two B operands as two 128-row windows of one 192-row tile
// [-C_im | C_re | C_im]: 6 instructions per spot chunk.
// GEMM 2 (the forward projection) is M = 128 spots x N = 128 rows x K = 16
// columns per instruction, real and imaginary parts apart, with split BF16
// operands too (12 instructions per K-step).  The half-precision option
// (compressed launches only) takes single FP16 operands instead (|u|, |C| <=
// 1; 4 instructions per K-step): the sums run over many pixels whose
// rounding errors (2^-12 relative) do not add up coherently.
//
// The operands are factor tables in global memory, laid out block by block
// exactly as the MMAs read them from shared memory (no-swizzle K-major core
// matrices, 8 rows x 16 bytes): C (per 64 columns and 16 spots) and C for
// GEMM 2 (per 16 columns, one K-step, and 128 spots) depend on the spots only
// and are made once per hologram; R' (per 128 rows and 16 spots) carries w and
// theta and is remade before every launch.  A tile streams its blocks into shared memory
// with bulk copies (cp.async.bulk, completion counted on an mbarrier) through
// a ring; a producer warp issues GEMM 1's copies, two issuing warps (GEMM 1,
// GEMM 2) issue the MMAs and commit them to mbarriers, and eight epilogue
// warps run the CUDA-core stages: four turn S into u (epilogue 1), four reduce
// Z to the spot fields (epilogue 2) once per strip of tiles along a row block
// and, in the final pass, write the phase map from S.  Every wait is bounded
// and a timeout is recorded in the launch's status word instead of hanging.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <functional>
#include <vector>
#include <type_traits>

#include "tile.cuh"

namespace cswgs {
namespace tc {

constexpr int kRows = 128;          // tile rows (GEMM 1 M, GEMM 2 N)
constexpr int kCols = 64;           // tile columns (GEMM 2 K; GEMM 1 N is re and im of them)
constexpr int kChunk = 16;          // spots per GEMM 1 instruction (K)
constexpr int kSpotBlock = 128;     // spots per GEMM 2 instruction (M)
constexpr uint32_t kWaitPolls = 1u << 20;   // polls of a bounded wait, unless a launch asks for fewer

// The launch's poll limit (set by thread 0 before the first block barrier).
__shared__ uint32_t s_wait_polls;

// component tiles (bytes): GEMM 1 operands per stage, GEMM 2 operands
constexpr uint32_t kA1 = kRows * kChunk * 2;        // R' component [128 rows][16 spots]
constexpr uint32_t kB1 = 3 * kCols * kChunk * 2;    // stacked C half [-C_im | C_re | C_im][16 spots]
constexpr uint32_t kB1Win = kCols * kChunk * 2;     // byte offset of the [C_re | C_im] window
constexpr uint32_t kStage = 4 * kA1 + 2 * kB1;      // one GEMM 1 stage: R' (4 components), C (hi, lo)
constexpr uint32_t kUc = kRows * 16 * 2;            // u component of one GEMM 2 K-step [128 rows][16 columns]
constexpr uint32_t kUSlot = 4 * kUc;                // u of one K-step (4 components)
constexpr uint32_t kCs = kSpotBlock * kCols * 2;    // C component [128 spots][64 columns]
constexpr uint32_t kCk = kSpotBlock * 16 * 2;       // C component of one GEMM 2 K-step [128 spots][16 columns]

__host__ __device__ inline int tiles(int P) { return ((P + kRows - 1) / kRows) * ((P + kCols - 1) / kCols); }

// Factor tables of one hologram (bytes): R' blocks (row block, spot chunk), C
// blocks (column block, spot chunk), GEMM 2 C blocks (column block, spot block).
__host__ __device__ inline int nchunks(int N) { return (N + kChunk - 1) / kChunk; }
__host__ __device__ inline int nspotblocks(int N) { return (N + kSpotBlock - 1) / kSpotBlock; }
__host__ __device__ inline size_t rw_table_bytes(int P, int N) { return (size_t)((P + kRows - 1) / kRows) * nchunks(N) * 4 * kA1; }
__host__ __device__ inline size_t c_table_bytes(int P, int N) { return (size_t)((P + kCols - 1) / kCols) * nchunks(N) * 2 * kB1; }
__host__ __device__ inline size_t cs_table_bytes(int P, int N)
{
    return (size_t)((P + kCols - 1) / kCols) * nspotblocks(N) * 4 * kCs;
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

// Instruction descriptor, kind::f16: D FP32, A and B both BF16 (bf16 = 1) or
// both FP16 (bf16 = 0), both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc(int M, int N, int neg_a, int bf16 = 1)
{
    return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | ((uint32_t)neg_a << 13) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
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

__device__ __forceinline__ bool try_wait(uint32_t mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
    return ok != 0u;
}

// Bounded wait for phase `parity` of an mbarrier; false when it ran out.  The
// first poll does not wait for the poll limit's shared-memory load.
__device__ __forceinline__ bool wait(uint32_t mbar, uint32_t parity)
{
    if (try_wait(mbar, parity)) return true;
    const uint32_t polls = s_wait_polls;
    for (uint32_t it = 1; it < polls; ++it)
        if (try_wait(mbar, parity)) return true;
    return false;
}

// One bulk copy global -> shared, counted on an mbarrier (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

// The arrival of the issuing thread, announcing `bytes` of copies to come.
__device__ __forceinline__ void expect_tx(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes) : "memory");
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
// bytes apart.  Pairs are converted together (round to nearest): hi = bf16(v),
// lo = bf16(v - hi).
__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 h)
{
    return (uint32_t)__bfloat16_as_ushort(h.x) | ((uint32_t)__bfloat16_as_ushort(h.y) << 16);
}

__device__ __forceinline__ void put8(unsigned char *base, uint32_t stride, uint32_t off, const float2 *v)
{
    uint32_t w[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 a = v[2 * q], b = v[2 * q + 1];
        const __nv_bfloat162 rh = __floats2bfloat162_rn(a.x, b.x), ih = __floats2bfloat162_rn(a.y, b.y);
        const float2 rf = __bfloat1622float2(rh), jf = __bfloat1622float2(ih);
        w[0][q] = bf16x2_bits(rh);
        w[1][q] = bf16x2_bits(__floats2bfloat162_rn(a.x - rf.x, b.x - rf.y));
        w[2][q] = bf16x2_bits(ih);
        w[3][q] = bf16x2_bits(__floats2bfloat162_rn(a.y - jf.x, b.y - jf.y));
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
        *reinterpret_cast<uint4 *>(base + c * stride + off) = make_uint4(w[c][0], w[c][1], w[c][2], w[c][3]);
}

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

// Eight complex values -> FP16 rows of the re and im component tiles
// (`stride` bytes apart), one 16-byte store each (round to nearest).
__device__ __forceinline__ uint32_t h2_bits(__half2 h)
{
    return (uint32_t)__half_as_ushort(__low2half(h)) | ((uint32_t)__half_as_ushort(__high2half(h)) << 16);
}

__device__ __forceinline__ void put8h(unsigned char *base, uint32_t stride, uint32_t off, const float2 *v)
{
    uint32_t wr[4], wi[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        wr[q] = h2_bits(__floats2half2_rn(v[2 * q].x, v[2 * q + 1].x));
        wi[q] = h2_bits(__floats2half2_rn(v[2 * q].y, v[2 * q + 1].y));
    }
    *reinterpret_cast<uint4 *>(base + off) = make_uint4(wr[0], wr[1], wr[2], wr[3]);
    *reinterpret_cast<uint4 *>(base + stride + off) = make_uint4(wi[0], wi[1], wi[2], wi[3]);
}

// Eight complex values of u, split for GEMM 2 and packed (the four BF16
// component rows, or the two FP16 ones), to be stored once their slot is free.
struct Packed8 {
    uint32_t w[4][4];
};

template <bool F16>
__device__ __forceinline__ Packed8 pack8(const float2 *v)
{
    Packed8 p;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 a = v[2 * q], b = v[2 * q + 1];
        if (F16) {
            p.w[0][q] = h2_bits(__floats2half2_rn(a.x, b.x));
            p.w[1][q] = h2_bits(__floats2half2_rn(a.y, b.y));
            p.w[2][q] = p.w[3][q] = 0u;
        } else {
            const __nv_bfloat162 rh = __floats2bfloat162_rn(a.x, b.x), ih = __floats2bfloat162_rn(a.y, b.y);
            const float2 rf = __bfloat1622float2(rh), jf = __bfloat1622float2(ih);
            p.w[0][q] = bf16x2_bits(rh);
            p.w[1][q] = bf16x2_bits(__floats2bfloat162_rn(a.x - rf.x, b.x - rf.y));
            p.w[2][q] = bf16x2_bits(ih);
            p.w[3][q] = bf16x2_bits(__floats2bfloat162_rn(a.y - jf.x, b.y - jf.y));
        }
    }
    return p;
}

// The rows of a Packed8 at byte offset `off` of the component tiles `stride`
// bytes apart: split BF16 re hi, re lo, im hi, im lo; FP16 re, im.
template <bool F16>
__device__ __forceinline__ void store8(unsigned char *base, uint32_t stride, uint32_t off, const Packed8 &p)
{
    if (F16) {
        *reinterpret_cast<uint4 *>(base + off) = make_uint4(p.w[0][0], p.w[0][1], p.w[0][2], p.w[0][3]);
        *reinterpret_cast<uint4 *>(base + stride + off) = make_uint4(p.w[1][0], p.w[1][1], p.w[1][2], p.w[1][3]);
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            *reinterpret_cast<uint4 *>(base + c * stride + off) = make_uint4(p.w[c][0], p.w[c][1], p.w[c][2], p.w[c][3]);
    }
}


// ------------------------------------------------------------- factor tables --
// Items of eight phasors; consecutive threads take consecutive rows of one
// core matrix, so a warp's 16-byte stores fill whole 128-byte lines.

// Eight values -> rows of the two BF16 halves (hi, lo) of a stacked C block:
// hi at base, lo at base + kB1, row offsets re_off, im_off (C_im) and
// neg_off (-C_im); each a 16-byte store.
__device__ __forceinline__ void put8_stacked(unsigned char *base, uint32_t re_off, uint32_t im_off,
                                             uint32_t neg_off, const float2 *v)
{
    uint32_t w[6][4];   // re hi, re lo, im hi, im lo, -im hi, -im lo
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 a = v[2 * q], b = v[2 * q + 1];
        const __nv_bfloat162 rh = __floats2bfloat162_rn(a.x, b.x), ih = __floats2bfloat162_rn(a.y, b.y);
        const float2 rf = __bfloat1622float2(rh), jf = __bfloat1622float2(ih);
        const __nv_bfloat162 rl = __floats2bfloat162_rn(a.x - rf.x, b.x - rf.y);
        const __nv_bfloat162 il = __floats2bfloat162_rn(a.y - jf.x, b.y - jf.y);
        w[0][q] = bf16x2_bits(rh);
        w[1][q] = bf16x2_bits(rl);
        w[2][q] = bf16x2_bits(ih);
        w[3][q] = bf16x2_bits(il);
        w[4][q] = bf16x2_bits(__hneg2(ih));   // the split of -v is -(hi), -(lo): exact
        w[5][q] = bf16x2_bits(__hneg2(il));
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        unsigned char *t = base + h * kB1;
        *reinterpret_cast<uint4 *>(t + re_off) = make_uint4(w[h][0], w[h][1], w[h][2], w[h][3]);
        *reinterpret_cast<uint4 *>(t + im_off) = make_uint4(w[2 + h][0], w[2 + h][1], w[2 + h][2], w[2 + h][3]);
        *reinterpret_cast<uint4 *>(t + neg_off) = make_uint4(w[4 + h][0], w[4 + h][1], w[4 + h][2], w[4 + h][3]);
    }
}

// C (GEMM 1's B: per block of 64 columns and 16 spots, each half a 192-row
// tile [-C_im | C_re | C_im] with row = column within each third) and C for
// GEMM 2 (128 spots x 64 columns per block, stored K-step by K-step: 4 x [the
// components of 128 spots x 16 columns]; split BF16, and for the
// half-precision option also FP16 re and im) of hologram blockIdx.y, from its
// spot coefficients.
__global__ void __launch_bounds__(256) const_tables_kernel(const HoloDev *__restrict__ holos, int count)
{
    const HoloDev H = holos[blockIdx.y];
    if (!H.ctab) return;
    const int P = H.P, N = H.N, half = P >> 1, nc = nchunks(N), nsb = nspotblocks(N);
    const int ncb = (P + kCols - 1) / kCols;
    const int items_c = ncb * nc * 128;                 // (block, 64 columns x 2 groups)
    const int items_cs = ncb * nsb * 1024;              // (block, 128 spots x 8 groups)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < items_c + items_cs; i += gridDim.x * blockDim.x) {
        float2 v[8];
        if (i < items_c) {
            const int blk = i >> 7, j = i & 127;
            const int cb = blk / nc, c = blk % nc;
            const int col = (j & 7) + 8 * (j >> 4), g = (j >> 3) & 1;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int n = c * kChunk + 8 * g + e;
                if (n < N) {
                    const int4 cf = H.coef[n];
                    v[e] = spot_factor(cf.x, cf.z, __int_as_float(cf.w), cb * kCols + col - half, kFixRound, 1.f);
                } else {
                    v[e] = make_float2(0.f, 0.f);
                }
            }
            put8_stacked(H.ctab + (size_t)blk * (2 * kB1), core_off(kCols + col, 8 * g, kChunk),
                         core_off(2 * kCols + col, 8 * g, kChunk), core_off(col, 8 * g, kChunk), v);
        } else {
            const int k = i - items_c, blk = k >> 10, j = k & 1023;
            const int cb = blk / nsb, sb = blk % nsb;
            const int nl = (j & 7) + 8 * (j >> 6), g = (j >> 3) & 7, n = sb * kSpotBlock + nl;
            if (n < N) {
                const int4 cf = H.coef[n];
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    v[e] = spot_factor(cf.x, cf.z, __int_as_float(cf.w), cb * kCols + 8 * g + e - half, kFixRound, 1.f);
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = make_float2(0.f, 0.f);
            }
            // K-step g / 2 of the block, column group g % 2 of the K-step
            const int ks = g >> 1;
            put8(H.cstab + (size_t)blk * (4 * kCs) + (size_t)ks * (4 * kCk), kCk, core_off(nl, 8 * (g & 1), 16), v);
            if (H.cstab16)
                put8h(H.cstab16 + (size_t)blk * (2 * kCs) + (size_t)ks * (2 * kCk), kCk, core_off(nl, 8 * (g & 1), 16),
                      v);
        }
    }
}

// R' = w a e^{i theta} R (GEMM 1's A: 128 rows x 16 spots per block) of the
// hologram of each slot, from its current spot state (rw_tables_kernel below).

// The Mp draws of S_j (Section 3) of the slot's hologram, each setting its
// pixel's bit in the iteration's mask, which is clear before (the tails of the
// last launch that used it cleared it).  Grid: blocks x slots.
__device__ __forceinline__ void scatter_subset(const HoloDev &H, const LaunchSlot &sl)
{
    uint32_t *mask = subset_mask(H, sl.j);
    const SubsetDraw d = subset_draw(H, sl.j);
    const UDiv dP = udiv_of((uint32_t)H.P);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < H.Mp; k += gridDim.x * blockDim.x) {
        const uint32_t m = subset_pixel(H, d, (uint32_t)k);
        uint32_t c;
        const uint32_t r = udiv(m, dP, c);
        atomicOr(mask + (size_t)r * H.mask_words + (c >> 5), 1u << (c & 31));
    }
}

__global__ void __launch_bounds__(256) mask_scatter_kernel(const HoloDev *__restrict__ holos,
                                                           const LaunchSlot *__restrict__ slots)
{
    const LaunchSlot sl = slots[blockIdx.y];
    const HoloDev H = holos[sl.holo];
    if (sl.pass == kPassSubset && H.mask) scatter_subset(H, sl);
}

// The same masks drawn in shared memory: G CTAs per slot (grid G x slots),
// each holding the slot's whole mask and taking 1 / G of the Mp draws, each
// draw an OR in shared memory; the CTA's copy then goes out word by word (G =
// 1: stored whole, zero words included; G > 1: the non-zero words ORed into
// the mask, which is clear before).  P^2 / 8 bytes of shared memory: up to P
// of about 1280.
constexpr int kLocalThreads = 1024;

__global__ void __launch_bounds__(kLocalThreads) mask_local_kernel(const HoloDev *__restrict__ holos,
                                                                   const LaunchSlot *__restrict__ slots)
{
    extern __shared__ __align__(16) uint32_t s_words[];
    const LaunchSlot sl = slots[blockIdx.y];
    const HoloDev H = holos[sl.holo];
    if (sl.pass != kPassSubset || !H.mask) return;
    const uint32_t G = gridDim.x, x = blockIdx.x;
    const int P = H.P, mw = H.mask_words, words = P * mw;
    const int tid = threadIdx.x;
    for (int i = tid; i < words; i += kLocalThreads) s_words[i] = 0u;
    __syncthreads();
    const SubsetDraw d = subset_draw(H, sl.j);
    const UDiv dP = udiv_of((uint32_t)P);
    const uint32_t k0 = (uint32_t)((uint64_t)H.Mp * x / G), k1 = (uint32_t)((uint64_t)H.Mp * (x + 1) / G);
    if (H.aperture == 0 && H.fa == (uint32_t)P && H.fb == (uint32_t)P && H.D == P * P) {
        // the square grid: the permutation's rectangle is the grid, so its
        // final halves (L, R) are the pixel's row and column (subset_pixel
        // without the cycle walk, the pupil map and the division by P)
        const uint32_t D = (uint32_t)H.D;
        for (uint32_t k = k0 + tid; k < k1; k += kLocalThreads) {
            uint32_t kk = k + d.off;
            kk = kk >= D ? kk - D : kk;
            uint32_t R;
            uint32_t L = udiv(kk, dP, R);
            feistel_round(L, R, d.K.k0, (uint32_t)P);
            feistel_round(L, R, d.K.k1, (uint32_t)P);
            feistel_round(L, R, d.K.k2, (uint32_t)P);
            feistel_round(L, R, d.K.k3, (uint32_t)P);
            atomicOr(s_words + L * (uint32_t)mw + (R >> 5), 1u << (R & 31));
        }
    } else {
        for (uint32_t k = k0 + tid; k < k1; k += kLocalThreads) {
            const uint32_t m = subset_pixel(H, d, k);
            uint32_t c;
            const uint32_t r = udiv(m, dP, c);
            atomicOr(s_words + r * (uint32_t)mw + (c >> 5), 1u << (c & 31));
        }
    }
    __syncthreads();
    uint32_t *g = subset_mask(H, sl.j);
    if (G == 1) {
        for (int i = tid; i < words; i += kLocalThreads) g[i] = s_words[i];
    } else {
        for (int i = tid; i < words; i += kLocalThreads) {
            const uint32_t v = s_words[i];
            if (v) atomicOr(g + i, v);
        }
    }
}

__global__ void __launch_bounds__(256) rw_tables_kernel(const HoloDev *__restrict__ holos,
                                                        const LaunchSlot *__restrict__ slots)
{
    // one block (128 rows x 16 spots) per pass of the loop: its 16 spots' row
    // coefficients and state are read once into shared memory
    __shared__ int4 s_cf[kChunk];      // {B, Gh, gl, theta + rounding}
    __shared__ float s_wa[kChunk];     // w a
    const LaunchSlot sl = slots[blockIdx.y];
    const HoloDev H = holos[sl.holo];
    if (!H.rwtab) return;
    const int P = H.P, N = H.N, half = P >> 1, nc = nchunks(N);
    const int blocks = ((P + kRows - 1) / kRows) * nc;   // (128 rows, 16 spots) blocks, 256 threads each
    const int j = threadIdx.x;
    const int row = (j & 7) + 8 * (j >> 4), g = (j >> 3) & 1;
    for (int blk = blockIdx.x; blk < blocks; blk += gridDim.x) {
        const int rb = blk / nc, c = blk % nc;
        __syncthreads();   // the previous block's spots are read
        if (j < kChunk) {
            const int n = c * kChunk + j;
            int4 v = make_int4(0, 0, 0, 0);
            float wa = 0.f;
            if (n < N) {
                const int4 cf = H.coef[n];
                const SpotState st = H.state[n];
                v = make_int4(cf.y, cf.z, cf.w, (int)(st.theta + kFixRound));
                wa = st.w * st.a0;
            }
            s_cf[j] = v;
            s_wa[j] = wa;
        }
        __syncthreads();
        float2 v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int4 cf = s_cf[8 * g + e];
            v[e] = spot_factor(cf.x, cf.y, __int_as_float(cf.z), rb * kRows + row - half, (uint32_t)cf.w,
                               s_wa[8 * g + e]);
        }
        put8(H.rwtab + (size_t)blk * (4 * kA1), kA1, core_off(row, 8 * g, kChunk), v);
    }
}


// ----------------------------------------------------------- warp roles --
// Tiles are pipelined by warp roles: a producer warp (takes the work items and
// loads GEMM 1's operand stages), a GEMM 1 warp, a GEMM 2 warp (one elected
// lane of each issues its bulk copies and MMAs), 4 u warps (epilogue 1) and 4
// V warps (epilogue 2).  The producer runs ahead of the GEMM 1 warp by the
// ring's depth: a tcgen05.mma issue waits for the tensor pipe, so copies
// issued from the MMA warp would start one stage late.
// A work item is a strip: LaunchSlot::strip consecutive tiles of one row block
// of a hologram.  Since V_n = sum_y conj(R_n(y)) Z(n, y) takes the same R_n(y)
// for every tile of a row block, GEMM 2 accumulates Z(n, y) over the strip's
// tiles and the V warps reduce it once per strip; a hologram with more than
// one GEMM 2 spot block (Z holds one) takes strips of one tile.
// Tensor memory holds two S buffers (columns 256..383 and 384..511; tile k
// uses buffer k & 1) and Z (columns 0..255).  GEMM 1 runs ahead into the next
// tile's back-propagation while the u warps turn S into u; the GEMM 2 warp
// streams the tile's C block in meanwhile and follows the u warps K-step by
// K-step; the u warps write a K-step's columns of u as soon as GEMM 2 of the
// previous tile has read them.  The per-hologram tails (Eqs. 4-6, or the
// metrics) run in a small kernel right after the launch, so tiles neither
// fence nor count arrivals.
// Hand-overs, all mbarriers:
//   ready[2]          producer -> GEMM 1, u and V warps: tile k in info slot k & 1
//   full[r], empty[r] GEMM 1 operand ring: copies landed / MMAs done
//   s_full[2]         GEMM 1 of the tile in that S buffer is done
//   s_empty[2]        the u warps have read that S buffer and info slot, the V and
//                     GEMM 1 warps that info slot
//   g2_info           u warps -> GEMM 2 warp: the tile's C blocks and its place in
//                     its strip (or done)
//   u_step[4]         the u warps have written u's columns of one K-step of GEMM 2
//   u_free[4]         GEMM 2 has read them (one phase per tile with products, so
//                     that no wait is two phases short)
//   cs_full           GEMM 2's C block has landed
//   cs_free           the MMAs that read it are done (its buffer is free)
//   z_full            a Z accumulation is done: a strip, or one spot block of a tile
//   z_empty           the V warps have read Z
//   drain             both issuing warps' last commits, before tensor memory is freed
// Every wait is bounded; a timeout ends the loop of the side that saw it and
// sets the status word, and the other side's waits then run out in turn.
namespace ws {

constexpr int kRingMax = 4;
constexpr uint32_t kS0 = 256;       // S buffers at columns 256 and 384, Z at 0
constexpr int kTmemColsWs = 512;
constexpr int kKSteps = kCols / 16; // GEMM 2 K-steps per tile

enum Bar {
    kReady0 = 0,
    kFull0 = 2,
    kEmpty0 = kFull0 + kRingMax,
    kSFull0 = kEmpty0 + kRingMax,
    kSEmpty0 = kSFull0 + 2,
    kUStep0 = kSEmpty0 + 2,       // u's columns of GEMM 2's K-step 0 .. 3 are written
    kUFree0 = kUStep0 + kKSteps,  // ... and GEMM 2 has read them
    kCsFull = kUFree0 + kKSteps,  // GEMM 2's C block has landed
    kCsFree,                      // the MMAs that read it are done
    kZFull,                       // a Z accumulation is done
    kZEmpty,
    kG2Info,    // the u warps have published the next tile's GEMM 2 operands
    kDrain,     // both issuing warps' last commits (2 arrivals)
    kBarsWs
};

// The GEMM 2 warp's work item, published by the u warps when they take up a
// tile with products (a single slot: the next one is written only after the
// GEMM 2 warp has issued that tile's first K-step, so it has read it).
struct G2Info {
    const unsigned char *cstab;   // GEMM 2's C blocks in the launch's format
    int nsb, cb, done, f16;
    int first, last;              // the tile opens / closes its strip's Z accumulation
};

// A published tile: its work item (strip), its tile index in the hologram's
// pass, its place in the strip, and copies of its launch slot and its
// hologram's descriptor (staged by the producer warp so that the other warps
// read them from shared memory).
struct Info {
    int item, empty, done, tile;
    int first, last;   // the first / last tile with products of the strip
    int zero, pad;     // zero: the strip's last tile, and the strip has no products
    LaunchSlot sl;
    HoloDev H;
};


// The epilogue warps: 4 u warps (epilogue 1, warps 0 .. 3) and 4 V warps
// (epilogue 2, warps 4 .. 7), each group one warp per TMEM lane quadrant.
// (Eight warps sharing both epilogues were measured: 5 % slower, and 12 % at
// more than one GEMM 2 spot block, where epilogue 2 of every tile no longer
// overlaps epilogue 1 of the next.)
constexpr int kUWarps = 4, kVWarps = 4;

template <int W>
struct Cfg {
    static_assert(W == kUWarps + kVWarps, "epilogue warps: the u and the V group");
    static constexpr int kEpi = 32 * W;               // epilogue threads
    static constexpr int kThreads = kEpi + 96;        // and the producer, GEMM 1 and GEMM 2 warps
};

// Shared-memory layout of the kernel with US slots of u (one K-step each;
// GEMM 2 of more than one spot block re-reads all of a tile's u, so US = 4):
// the GEMM 1 ring, GEMM 2's C block and u (and 128 bytes to align the base;
// the no-swizzle layouts and the bulk copies need 16).  (Two u slots and a
// fourth ring stage were measured: the epilogue then waits for GEMM 2 to free
// a slot, 7 % slower at N = 100.)
template <int US>
struct Lay {
    static_assert(US == kKSteps, "u slots");
    static constexpr int kRing = 3;
    static constexpr size_t kSmem = 128 + (size_t)kRing * kStage + 4 * (size_t)kCs + (size_t)US * kUSlot;
};

struct SmemWs {
    unsigned char *ring, *cs, *u;
};

template <int US>
__device__ __forceinline__ SmemWs carve_ws(unsigned char *raw)
{
    unsigned char *b = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(raw) + 127) & ~(uintptr_t)127);
    SmemWs m;
    m.ring = b;
    m.cs = m.ring + Lay<US>::kRing * kStage;
    m.u = m.cs + 4 * kCs;
    return m;
}

__device__ __forceinline__ void arrive(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(mbar) : "memory");
}

__device__ __forceinline__ bool wait_newest(uint32_t mbar, uint32_t given) { return wait(mbar, (given - 1u) & 1u); }

// A warp's vote: true when every lane's p is.  The epilogue warps wait each
// on its own; the hand-over barriers keep them within a tile of each other,
// and a wait that runs out in one warp runs out in the others too, since the
// pipeline behind it has stopped.
__device__ __forceinline__ bool warp_and(bool p) { return __all_sync(0xffffffffu, p) != 0; }

// Tile t of hologram H lies wholly outside the round pupil.
__device__ __forceinline__ bool tile_outside(const HoloDev &H, int t)
{
    if (H.aperture == 0) return false;
    const int P = H.P, half = P >> 1, col_tiles = (P + kCols - 1) / kCols;
    const int y0 = (t / col_tiles) * kRows, x0 = (t % col_tiles) * kCols;
    const int ylo = y0 - half, yhi = min(y0 + kRows, P) - 1 - half;
    const int xlo = x0 - half, xhi = min(x0 + kCols, P) - 1 - half;
    const int64_t dy = ylo > 0 ? ylo : (yhi < 0 ? yhi : 0);
    const int64_t dx = xlo > 0 ? xlo : (xhi < 0 ? xhi : 0);
    return dx * dx + dy * dy > (int64_t)half * half;
}

// Barrier i of the block's array, by shared-memory address.
__device__ __forceinline__ uint32_t mbar_at(uint32_t base, int i) { return base + 8u * (uint32_t)i; }

// One elected lane of a converged warp (the issuing lane of a producer or MMA warp).
__device__ __forceinline__ bool elect_one()
{
    uint32_t p;
    asm volatile("{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n selp.u32 %0, 1, 0, e;\n}\n" : "=r"(p));
    return p != 0;
}

// Every lane's bounded wait for phase `parity`, voted across the warp.
__device__ __forceinline__ bool warp_wait(uint32_t mbar, uint32_t parity)
{
    return __all_sync(0xffffffffu, wait(mbar, parity & 1u)) != 0;
}

// An issuing warp's pipeline state, the same in every lane and all scalars.
// GEMM 1 chunks go round the ring in order, so chunk q (counted over the
// block's tiles) is stage q % R's (q / R)-th use (R the ring's depth) and both ring waits
// take their parity from q; the other barriers count their phases.  The whole
// warp runs the loop and waits; one elected lane issues the copies, MMAs,
// commits and arrivals.
struct Ctl {
    uint32_t mb;      // barrier 0
    uint32_t tmem;
    uint32_t ring, cs, u;   // shared addresses of the ring, GEMM 2's C block and u
    uint32_t ql;      // GEMM 1 chunks loaded
    uint32_t qm;      // GEMM 1 chunks multiplied
    uint32_t nz;      // Z accumulations closed
    uint32_t ncs;     // GEMM 2 C blocks loaded
    uint32_t nu;      // u hand-overs taken
};

// GEMM 1's operands of one tile, issued by the producer warp: for each chunk of
// 16 spots, R' of row block rb and the stacked C of column block cb into the
// next ring stage once the GEMM 1 warp's products have released it.
template <int R>
__device__ __forceinline__ bool load_gemm1(Ctl &C, const HoloDev &H, int rb, int cb)
{
    const int nc = nchunks(H.N);
    for (int c = 0; c < nc; ++c) {
        const uint32_t s = C.ql % R;
        if (C.ql >= (uint32_t)R && !warp_wait(mbar_at(C.mb, kEmpty0 + s), C.ql / R - 1u)) return false;
        if (elect_one()) {
            const uint32_t stg = C.ring + s * kStage, full = mbar_at(C.mb, kFull0 + s);
            expect_tx(full, kStage);
            bulk_load(stg, H.rwtab + ((size_t)rb * nc + c) * (4 * kA1), 4 * kA1, full);
            bulk_load(stg + 4 * kA1, H.ctab + ((size_t)cb * nc + c) * (2 * kB1), 2 * kB1, full);
        }
        __syncwarp();
        C.ql++;
    }
    return true;
}

// GEMM 1 of one tile into S buffer j, [S_re | S_im] = R' [C_re | C_im] with
// the complex product stacked along N: per chunk six M128 N128 K16 MMAs (the
// split operands' hi hi, hi lo and lo hi terms of R'_re [C_re | C_im] and
// R'_im [-C_im | C_re]), issued as each ring stage lands.  The stage goes back
// to the producer when its MMAs complete.
template <int R>
__device__ __forceinline__ bool gemm1(Ctl &C, int nc, int j)
{
    const uint32_t id = idesc(kRows, 2 * kCols, 0);
    const uint32_t s_acc = C.tmem + kS0 + 2 * kCols * j;   // [S_re | S_im]
    const uint64_t ring0 = desc(C.ring, 128, 256);
    for (int c = 0; c < nc; ++c) {
        const uint32_t s = C.qm % R;
        if (!warp_wait(mbar_at(C.mb, kFull0 + s), C.qm / R)) return false;
        // A: R' re hi, re lo, im hi, im lo; B: [C_re | C_im] and [-C_im | C_re] windows, hi and lo
        const uint64_t st = ring0 + ((uint64_t)(s * kStage) >> 4);
        const uint64_t arh = st, arl = st + (kA1 >> 4), aih = st + (2 * kA1 >> 4), ail = st + (3 * kA1 >> 4);
        const uint64_t bh = st + (4 * kA1 >> 4), bl = bh + (kB1 >> 4);
        const uint64_t b1h = bh + (kB1Win >> 4), b1l = bl + (kB1Win >> 4);
        if (elect_one()) {
            mma(s_acc, arh, b1h, id, c > 0 ? 1u : 0u);
            mma(s_acc, arh, b1l, id, 1u);
            mma(s_acc, arl, b1h, id, 1u);
            mma(s_acc, aih, bh, id, 1u);
            mma(s_acc, aih, bl, id, 1u);
            mma(s_acc, ail, bh, id, 1u);
            commit(mbar_at(C.mb, kEmpty0 + s));
        }
        __syncwarp();
        C.qm++;
    }
    if (elect_one()) commit(mbar_at(C.mb, kSFull0 + j));   // covers this GEMM 1 and every MMA before it
    __syncwarp();
    return true;
}

// GEMM 2 of one tile: Z = conj(C)^T u, one block of 128 spots at a time, into
// columns 0..255; each block's C (its four K-steps one after the other)
// streams in once the MMAs that read the previous one are done (block 0 while
// u is still being written).  Split BF16 operands (4 components each), or FP16
// re and im for the half-precision option.  The first tile of a strip (and
// each spot block past the first) opens a Z accumulation, once the epilogue
// has read the last one; the last tile of a strip (and each spot block but the
// last) closes it.  After each K-step of the last spot block, u's columns of
// that K-step go back to the epilogue warps.
template <int US>
__device__ __forceinline__ bool gemm2(Ctl &C, const G2Info &g)
{
    const int f16 = g.f16;
    const uint32_t comps = f16 ? 2u : 4u, kbytes = comps * kCk;
    const uint32_t id = idesc(kSpotBlock, kRows, 0, f16 ? 0 : 1), idn = idesc(kSpotBlock, kRows, 1, f16 ? 0 : 1);
    const uint32_t z_re = C.tmem, z_im = C.tmem + kRows;
    const uint64_t cs0 = desc(C.cs, 128, 256);                       // [128 spots][16 columns] per component
    const uint64_t u0 = desc(C.u, 128, 256);                         // [128 rows][16 columns] per component
    for (int sb = 0; sb < g.nsb; ++sb) {
        if (C.ncs > 0 && !warp_wait(mbar_at(C.mb, kCsFree), C.ncs - 1u)) return false;
        if (elect_one()) {
            const uint32_t full = mbar_at(C.mb, kCsFull);
            expect_tx(full, kKSteps * kbytes);
            bulk_load(C.cs, g.cstab + ((size_t)g.cb * g.nsb + sb) * (kKSteps * kbytes), kKSteps * kbytes, full);
        }
        __syncwarp();
        C.ncs++;
        const bool opens = sb > 0 || g.first, closes = sb < g.nsb - 1 || g.last;
        // a new accumulation overwrites Z: the epilogue has read the last one
        if (opens && C.nz > 0 && !warp_wait(mbar_at(C.mb, kZEmpty), C.nz - 1u)) return false;
        if (!warp_wait(mbar_at(C.mb, kCsFull), C.ncs - 1u)) return false;
        fence_after();
        for (int ks = 0; ks < kKSteps; ++ks) {
            // on a tile's first spot block, each K-step waits for its columns of u
            if (sb == 0) {
                if (!warp_wait(mbar_at(C.mb, kUStep0 + ks), C.nu)) return false;
                fence_after();
            }
            const uint32_t acc = (opens && ks == 0) ? 0u : 1u;
            const uint64_t cs = cs0 + ((uint64_t)(ks * kbytes) >> 4);
            const uint64_t us = u0 + ((uint64_t)((ks % US) * kUSlot) >> 4);   // u's slot of this K-step
            if (f16) {
                // conj(C) u: Z_re = C_re u_re + C_im u_im, Z_im = C_re u_im - C_im u_re
                const uint64_t cr = cs, ci = cs + ((uint64_t)kCk >> 4);
                const uint64_t ur = us, ui = us + ((uint64_t)kUc >> 4);
                if (elect_one()) {
                    mma(z_re, cr, ur, id, acc);
                    mma(z_re, ci, ui, id, 1u);
                    mma(z_im, cr, ui, id, acc);
                    mma(z_im, ci, ur, idn, 1u);
                    if (sb == g.nsb - 1) commit(mbar_at(C.mb, kUFree0 + ks));
                }
            } else {
                uint64_t a[4], b[4];
                for (int q = 0; q < 4; ++q) {
                    a[q] = cs + ((uint64_t)(q * kCk) >> 4);
                    b[q] = us + ((uint64_t)(q * kUc) >> 4);
                }
                if (elect_one()) {
                    complex_mma(z_re, z_im, a, b, id, idn, acc, 1);
                    if (sb == g.nsb - 1) commit(mbar_at(C.mb, kUFree0 + ks));
                }
            }
            __syncwarp();
        }
        if (sb == 0) C.nu++;
        if (elect_one()) {
            commit(mbar_at(C.mb, kCsFree));
            if (closes) commit(mbar_at(C.mb, kZFull));
        }
        __syncwarp();
        if (closes) C.nz++;
    }
    return true;
}

// Every MMA of an issuing warp done before tensor memory is freed, and every
// copy of a warp landed before shared memory is; true when all ended in time.
template <int R>
__device__ __forceinline__ bool drain(const Ctl &C, bool mmas)
{
    bool drained = true;
    if (mmas) {
        if (elect_one()) commit(mbar_at(C.mb, kDrain));
        __syncwarp();
        drained = warp_wait(mbar_at(C.mb, kDrain), 0u);
    }
    for (uint32_t s = 0; s < (uint32_t)R; ++s) {
        const uint32_t loads = (C.ql + R - 1u - s) / R;   // chunks q < ql with q % R == s
        if (loads) drained &= warp_wait(mbar_at(C.mb, kFull0 + s), loads - 1u);
    }
    if (C.ncs) drained &= warp_wait(mbar_at(C.mb, kCsFull), C.ncs - 1u);
    return drained;
}

__device__ __forceinline__ Ctl ctl_init(const SmemWs &m, uint32_t mb, uint32_t tmem)
{
    Ctl C;
    C.mb = mb;
    C.tmem = tmem;
    C.ring = saddr(m.ring);
    C.cs = saddr(m.cs);
    C.u = saddr(m.u);
    C.ql = C.qm = C.nz = C.ncs = C.nu = 0u;
    return C;
}

// The GEMM 2 warp: per tile with products, its operands as the epilogue
// publishes them, then GEMM 2 once u is ready.
template <int US>
__device__ __noinline__ void control_gemm2(const SmemWs &m, const G2Info *g2, uint32_t mb, uint32_t tmem,
                                           unsigned *status)
{
    Ctl C = ctl_init(m, mb, tmem);
    bool ok = true;
    for (uint32_t n = 0;; ++n) {
        ok = warp_wait(mbar_at(mb, kG2Info), n);
        if (!ok) break;
        const G2Info g = *g2;
        if (g.done) break;
        ok = gemm2<US>(C, g);
        if (!ok) break;
    }
    const bool drained = drain<Lay<US>::kRing>(C, true);
    if ((!ok || !drained) && (threadIdx.x & 31) == 0) atomicOr(status, 1u);
}

// The GEMM 1 warp: per published tile with products, GEMM 1 into S buffer j
// as the producer's stages land; then it gives info slot j back.
template <int R>
__device__ __noinline__ void control_gemm1(const SmemWs &m, const Info *info, uint32_t mb, uint32_t tmem,
                                           unsigned *status)
{
    Ctl C = ctl_init(m, mb, tmem);
    bool ok = true;
    for (uint32_t k = 0;; ++k) {
        const int j = k & 1;
        ok = warp_wait(mbar_at(mb, kReady0 + j), (k >> 1) & 1u);
        if (!ok) break;
        const int done = info[j].done, empty = info[j].empty, N = info[j].H.N;
        if (done) break;
        if (!empty) {
            fence_after();
            ok = gemm1<R>(C, nchunks(N), j);
        }
        __syncwarp();
        if ((threadIdx.x & 31) == 0) arrive(mbar_at(mb, kSEmpty0 + j));
        if (!ok) break;
    }
    const bool drained = drain<R>(C, true);
    if ((!ok || !drained) && (threadIdx.x & 31) == 0) atomicOr(status, 1u);
}

// The producer warp: takes work items (strips), publishes their tiles one by
// one, and loads GEMM 1's operand stages of each (running up to the ring's
// depth ahead of the MMAs).  The pop of the next item and the global loads of
// the item's slot and descriptor are issued ahead of the waits they would
// otherwise follow.
template <int R>
__device__ __noinline__ void control_load(const HoloDev *__restrict__ holos, const LaunchSlot *__restrict__ slots,
                                           int nslots, int total_tiles, unsigned *queue, const SmemWs &m,
                                           Info *info, uint32_t mb, uint32_t tmem, unsigned *status)
{
    constexpr int kHWords = (int)(sizeof(HoloDev) / 4), kHPer = (kHWords + 31) / 32;
    static_assert(sizeof(HoloDev) % 4 == 0, "word copies");
    Ctl C = ctl_init(m, mb, tmem);
    const int lane = threadIdx.x & 31;
    const bool lane0 = lane == 0;
    bool ok = true;
    int slot = 0;   // a block's items only rise, so their slots are found by scanning forward
    int item = total_tiles;
    if (lane0) item = (int)atomicAdd(queue, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    uint32_t k = 0;   // tiles published
    for (bool stop = false; !stop;) {
        const bool fin = item >= total_tiles || !ok;
        // the next item's pop is in flight while this one is published and multiplied
        int next = total_tiles;
        if (lane0 && !fin) next = (int)atomicAdd(queue, 1u);
        const HoloDev *Hp = nullptr;
        LaunchSlot sl{};
        uint32_t hw[kHPer];
        // the strip: row block rb, column tiles c0 .. c1 - 1, the ones with
        // products cf .. cl (a round pupil is convex: they are contiguous)
        int rb = 0, c0 = 0, c1 = 1, col_tiles = 1, cf = -1, cl = -1;
        if (!fin) {
            while (slot + 1 < nslots && slots[slot + 1].tile_begin <= item) ++slot;
            sl = slots[slot];
            Hp = &holos[sl.holo];
            const uint32_t *src = reinterpret_cast<const uint32_t *>(Hp);
#pragma unroll
            for (int i = 0; i < kHPer; ++i) {
                const int w = lane + 32 * i;
                hw[i] = w < kHWords ? __ldg(src + w) : 0u;
            }
            col_tiles = (Hp->P + kCols - 1) / kCols;
            const int S = max(1, sl.strip), per_row = (col_tiles + S - 1) / S;
            const int s_loc = item - sl.tile_begin;
            rb = s_loc / per_row;
            c0 = (s_loc % per_row) * S;
            c1 = min(c0 + S, col_tiles);
            for (int c = c0; c < c1; ++c)
                if (!tile_outside(*Hp, rb * col_tiles + c)) {
                    if (cf < 0) cf = c;
                    cl = c;
                }
        }
        for (int c = c0; c < c1; ++c) {
            const int j = k & 1;
            // S buffer j and info slot j are free once the epilogue and the GEMM 1
            // warp are done with tile k - 2
            if (k >= 2 && ok) ok = warp_wait(mbar_at(mb, kSEmpty0 + j), (k >> 1) - 1u);
            stop = fin || !ok;
            const bool empty = stop || cf < 0 || c < cf || c > cl;
            if (stop) {
                if (lane0) info[j].done = 1;
            } else {
                if (lane0) {
                    info[j].item = item;
                    info[j].tile = rb * col_tiles + c;
                    info[j].empty = empty ? 1 : 0;
                    info[j].done = 0;
                    info[j].first = c == cf ? 1 : 0;
                    info[j].last = c == cl ? 1 : 0;
                    info[j].zero = (cf < 0 && c == c1 - 1) ? 1 : 0;
                    info[j].sl = sl;
                }
                uint32_t *dst = reinterpret_cast<uint32_t *>(&info[j].H);
#pragma unroll
                for (int i = 0; i < kHPer; ++i) {
                    const int w = lane + 32 * i;
                    if (w < kHWords) dst[w] = hw[i];
                }
            }
            __syncwarp();
            if (lane0) arrive(mbar_at(mb, kReady0 + j));
            ++k;
            if (stop) break;
            if (!empty) ok = load_gemm1<R>(C, *Hp, rb, c);
        }
        item = __shfl_sync(0xffffffffu, next, 0);
    }
    const bool drained = drain<R>(C, false);
    if ((!ok || !drained) && lane0) atomicOr(status, 1u);
}

// The partial V_n = sum_y conj(R_n(y)) Z(n, y) of spot n of a closed Z
// accumulation (a strip at row block y0) over the tile's 128 rows.  R_n(y)
// along the rows by recurrence: its phase is quadratic in y, so R(y + 1) =
// R(y) D(y) and D(y + 1) = D(y) E with the constant E = e^{i (2 pi 2 Gh / 2^32
// + 2 gl)}; R and D are evaluated directly every 8 rows (the product's
// rounding grows with the run length).  Every lane computes (a lane past N
// uses spot N - 1's factors and stores nothing): no divergent branch in the
// row loop.
__device__ __forceinline__ float2 strip_dot(uint32_t z_re, uint32_t z_im, const int4 *coef, int n, int N, int y0,
                                            int half)
{
    const int4 cf = coef[min(n, N - 1)];
    const int32_t tilt = cf.y, Gh = cf.z;
    const float gl = __int_as_float(cf.w);
    float es, ec;
    sincos_fix(kFixRound + 2u * (uint32_t)Gh, fmaf(2.f, gl, -kTwoPiF), es, ec);
    float vr0 = 0.f, vi0 = 0.f, vr1 = 0.f, vi1 = 0.f;
#pragma unroll 1
    for (int ys = 0; ys < kRows; ys += 16) {
        float zr[16], zi[16];
        ld16(z_re + ys, zr);
        ld16(z_im + ys, zi);
        float2 r[16];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int u0 = y0 + ys + 8 * b - half, du = 2 * u0 + 1;
            float2 pr = spot_factor(tilt, Gh, gl, u0, kFixRound, 1.f);
            float ds, dc;
            sincos_fix(kFixRound + (uint32_t)tilt + (uint32_t)Gh * (uint32_t)du, fmaf(gl, (float)du, -kTwoPiF), ds,
                       dc);
            float2 d = make_float2(dc, ds);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                r[8 * b + e] = pr;
                if (e < 7) {
                    pr = make_float2(fmaf(pr.x, d.x, -pr.y * d.y), fmaf(pr.x, d.y, pr.y * d.x));
                    d = make_float2(fmaf(d.x, ec, -d.y * es), fmaf(d.x, es, d.y * ec));
                }
            }
        }
        ld_wait();
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            vr0 = fmaf(r[2 * e].x, zr[2 * e], fmaf(r[2 * e].y, zi[2 * e], vr0));
            vi0 = fmaf(r[2 * e].x, zi[2 * e], fmaf(-r[2 * e].y, zr[2 * e], vi0));
            vr1 = fmaf(r[2 * e + 1].x, zr[2 * e + 1], fmaf(r[2 * e + 1].y, zi[2 * e + 1], vr1));
            vi1 = fmaf(r[2 * e + 1].x, zi[2 * e + 1], fmaf(-r[2 * e + 1].y, zr[2 * e + 1], vi1));
        }
    }
    return make_float2(vr0 + vr1, vi0 + vi1);
}

// The columns xl .. xr of grid row gy that lie in the pupil: the grid's, within
// the round pupil (|x - half|^2 + (gy - half)^2 <= half^2) unless the aperture
// is square; xr < xl for a row outside.
__device__ __forceinline__ void row_span(int P, int aperture, int gy, int &xl, int &xr)
{
    const int half = P >> 1, yq = gy - half;
    const int R2 = half * half, yq2 = yq * yq;   // P <= 32768: squares stay below 2^30
    xl = 0;
    xr = gy < P ? P - 1 : -1;
    if (aperture != 0) {
        const int D = R2 - yq2;
        int wr = -1;
        if (D >= 0) {
            wr = (int)sqrtf((float)D);   // within 1 of floor(sqrt(D))
            if ((wr + 1) * (wr + 1) <= D) ++wr;
            if (wr * wr > D) --wr;
        }
        xl = max(xl, half - wr);
        xr = min(xr, half + wr);
    }
}

// The final pass's phase map Phi = arg S (Eq. 1) and SLM gray levels of one
// tile row (grid row gy, columns x0 .. x0 + 63), from S in tensor memory, K-step
// by K-step: 0 outside the pupil.  Every lane of the warp runs the tensor-memory
// loads (they are warp-collective); a row past the grid stores nothing.
__device__ __forceinline__ void final_phases(const HoloDev &H, uint32_t s_re, uint32_t s_im, int gy, int x0)
{
    const int P = H.P;
    int xl, xr;
    row_span(P, H.aperture, gy, xl, xr);
#pragma unroll 1
    for (int ks = 0; ks < kKSteps; ++ks) {
        const int gx0 = x0 + 16 * ks;
        float sr[16], si[16], o[16];
        __syncwarp();   // converged for the warp-collective loads
        ld16(s_re + 16 * ks, sr);
        ld16(s_im + 16 * ks, si);
        ld_wait();
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
            const int x = gx0 + jj;
            float ph = atan2f(si[jj], sr[jj]);
            ph = ph < 0.f ? ph + kTwoPiF : ph;
            o[jj] = (ph >= kTwoPiF || x < xl || x > xr) ? 0.f : ph;
        }
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int col = gx0 + 4 * g;
            if (gy >= P || col >= P) break;
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

// The u warps (epilogue 1): per tile, u = A S / |S| into GEMM 2's B operand,
// K-step by K-step: K-step ks goes to u's slot ks % US once GEMM 2 has read
// that slot's last K-step (computed first, stored after the wait).  A tile outside the pupil gets, in
// the final pass, phase 0 and gray lut[0] here, and a strip with no tile
// inside the pupil its zero partials.
template <bool F16, int US>
__device__ __forceinline__ void epilogue_u(const SmemWs &m, const Info *info, G2Info *g2, uint32_t mb, uint32_t tmem,
                                           unsigned *status)
{
    constexpr int kT = 32 * kUWarps;
    const int tid = threadIdx.x, lane = tid & 31, q = tid >> 5;   // warps 0 .. 3: TMEM lane quadrant q
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    // phases seen: s_full[j] once per tile with products (low half: j = 0,
    // high half: j = 1); n_p: tiles with products taken up (u_free[ks]
    // completes once per such tile)
    uint32_t n_s = 0u, n_p = 0u;
    bool ok = true;
    for (uint32_t k = 0;; ++k) {
        const int j = k & 1;
        ok = warp_and(wait(mbar_at(mb, kReady0 + j), (k >> 1) & 1u));
        if (!ok) break;
        if (info[j].done) {
            // the GEMM 2 warp has read the last published operands once it has
            // issued that tile's first K-step
            if (n_p > 0u) ok = warp_and(wait_newest(mbar_at(mb, kUFree0), n_p));
            if (ok && tid == 0) {
                g2->done = 1;
                arrive(mbar_at(mb, kG2Info));
            }
            break;
        }
        const int item = info[j].item, empty = info[j].empty, t = info[j].tile;
        const int first = info[j].first, last = info[j].last, zero = info[j].zero;
        const LaunchSlot sl = info[j].sl;
        const HoloDev H = info[j].H;   // by value: global stores below cannot alias it
        const int P = H.P, N = H.N, half = P >> 1, pass = sl.pass;
        const int col_tiles = (P + kCols - 1) / kCols;
        const int y0 = (t / col_tiles) * kRows, x0 = (t % col_tiles) * kCols;
        if (empty) {
            // wholly outside the round pupil: in the final pass phase 0 (gray
            // lut[0]) over its grid pixels; a strip without products has zero
            // partials
            __syncwarp();
            if (lane == 0) arrive(mbar_at(mb, kSEmpty0 + j));
            if (zero) {
                const size_t s_loc = (size_t)(item - sl.tile_begin);
                for (int n = tid; n < N; n += kT) {
                    if (pass == kPassFinal) H.part64[s_loc * N + n] = make_double2(0.0, 0.0);
                    else H.part[s_loc * N + n] = make_float2(0.f, 0.f);
                }
            }
            if (pass == kPassFinal) {
                const int rows = min(kRows, P - y0), cols = min(kCols, P - x0);
                const uint8_t g0 = H.slm ? __ldg(H.lut) : 0;
                for (int f = tid; f < rows * cols; f += kT) {
                    const int r = y0 + f / cols, c = x0 + f % cols;
                    if (H.phase_out) H.phase_out[(size_t)r * P + c] = 0.f;
                    if (H.slm) H.slm[(size_t)r * H.slm_pitch + c] = g0;
                }
            }
            continue;
        }

        // A compressed pass reads the subset mask bits of the tile's columns
        // first (two words: x0 is a multiple of 64), before the waits.
        const int row = 32 * q + lane, gy = y0 + row;
        uint64_t mword = ~0ull;
        if (pass == kPassSubset) {
            const int w0 = x0 >> 5;
            if (gy < P) {
                const uint32_t *mrow = subset_mask(H, sl.j) + (size_t)gy * H.mask_words;
                mword = (uint64_t)__ldg(mrow + w0) | (w0 + 1 < H.mask_words ? (uint64_t)__ldg(mrow + w0 + 1) << 32 : 0ull);
            } else {
                mword = 0ull;
            }
        }
        // the single GEMM 2 operand slot is free once GEMM 2 has issued the
        // previous tile's first K-step
        if (n_p > 0u) {
            ok = warp_and(wait_newest(mbar_at(mb, kUFree0), n_p));
            if (!ok) break;
        }
        if (tid == 0) {
            g2->cstab = F16 ? H.cstab16 : H.cstab;
            g2->nsb = nspotblocks(N);
            g2->cb = t % col_tiles;
            g2->done = 0;
            g2->f16 = F16 ? 1 : 0;
            g2->first = first;
            g2->last = last;
            arrive(mbar_at(mb, kG2Info));
        }
        n_p++;
        n_s += 1u << (16 * j);
        ok = warp_and(wait_newest(mbar_at(mb, kSFull0 + j), (n_s >> (16 * j)) & 0xFFFFu));
        if (!ok) break;
        fence_after();
        {
            const uint32_t s_re = tmem + kS0 + 2 * kCols * j, s_im = s_re + kCols;
            const int yq = gy - half, yq2 = yq * yq;
            int xl, xr;
            row_span(P, H.aperture, gy, xl, xr);
            const float kA = H.kA;
            // the row's 16 columns of each K-step, with the Gaussian beam's
            // amplitude or the uniform one (a uniform branch outside the loop)
            auto ksteps = [&](auto gauss_tag) {
                constexpr bool kGauss = decltype(gauss_tag)::value;
#pragma unroll 1
                for (int ks = 0; ks < kKSteps; ++ks) {
                    const int xs = 16 * ks, gx0 = x0 + xs;
                    // the pixels that carry u: in the row's span and, in a
                    // compressed pass, in S_j (the rest add nothing to Eq. 3's sum)
                    const int lo = max(xl - gx0, 0), hi = min(xr - gx0, 15);
                    uint32_t bits = 0u;
                    if (lo <= hi) bits = (0xFFFFu >> (15 - hi + lo)) << lo;
                    bits &= (uint32_t)(mword >> xs);
                    float sr[16], si[16];
                    ld16(s_re + lanes + xs, sr);
                    ld16(s_im + lanes + xs, si);
                    ld_wait();
                    Packed8 pk[2];
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
                        float2 u[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            // branch-free: the lanes are rows, so a per-pixel branch
                            // (subset membership, the pupil edge) would diverge
                            const int jj = 8 * g + e;
                            const bool valid = ((bits >> jj) & 1u) != 0u;
                            const float a = sr[jj], b = si[jj];
                            const float n2 = a * a + b * b;
                            float amp = 1.f;   // Eq. 3's A
                            if constexpr (kGauss) {
                                const int xq = gx0 + jj - half;
                                amp = exp2f(-kA * (float)(xq * xq + yq2));
                            }
                            const bool lit = n2 > 0.f;
                            const float rs = rsqrtf(n2) * amp;
                            const float ur = lit ? a * rs : amp, ui = lit ? b * rs : 0.f;   // S = 0: phase 0
                            u[e] = make_float2(valid ? ur : 0.f, valid ? ui : 0.f);
                        }
                        pk[g] = pack8<F16>(u);
                    }
                    // u's slot of this K-step is free once GEMM 2 has read its last
                    // K-step (US earlier in GEMM 2's order: of this tile, or of the
                    // previous tile with products); K-step 0's was waited for above
                    // (the condition is the same in every lane of the warp, so
                    // the warp's vote stays matched)
                    const int pks = (ks + kKSteps - US) % kKSteps;
                    const uint32_t pcount = ks >= US ? n_p : n_p - 1u;
                    if (pcount > 0u && !(ks == 0 && US == kKSteps) &&
                        !warp_and(wait_newest(mbar_at(mb, kUFree0 + pks), pcount)))
                        return false;
                    unsigned char *slot = m.u + (ks % US) * kUSlot;
                    store8<F16>(slot, kUc, core_off(row, 0, 16), pk[0]);
                    store8<F16>(slot, kUc, core_off(row, 8, 16), pk[1]);
                    // this K-step's columns of u are in place
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) arrive(mbar_at(mb, kUStep0 + ks));
                }
                return true;
            };
            ok = kA != 0.f ? ksteps(std::true_type{}) : ksteps(std::false_type{});
            if (!ok) break;
        }
        fence_before();
        __syncwarp();
        if (lane == 0) arrive(mbar_at(mb, kSEmpty0 + j));
    }
    if (!ok && lane == 0) atomicOr(status, 1u);
}

// The V warps (epilogue 2): per strip (after the GEMM 2 of its last tile with
// products) and spot block, the strip's partial V_n = sum_y conj(R_n(y))
// Z(n, y), one spot per thread over all 128 rows, while the u warps go on with
// the next tiles.  In the final pass they also write each tile's phase map
// (and gray levels) from S, beside the u warps' work on u.
__device__ __forceinline__ void epilogue_v(const Info *info, uint32_t mb, uint32_t tmem, unsigned *status)
{
    const int tid = threadIdx.x - 32 * kUWarps, lane = tid & 31, q = tid >> 5;   // TMEM lane quadrant q
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    uint32_t n_z = 0u;   // Z accumulations reduced
    uint32_t n_s = 0u;   // tiles with products seen, per S buffer (low half: j = 0, high half: j = 1)
    bool ok = true;
    for (uint32_t k = 0;; ++k) {
        const int j = k & 1;
        ok = warp_and(wait(mbar_at(mb, kReady0 + j), (k >> 1) & 1u));
        if (!ok) break;
        if (info[j].done) break;
        const int item = info[j].item, empty = info[j].empty, t = info[j].tile, last = info[j].last;
        const int tile_begin = info[j].sl.tile_begin, pass = info[j].sl.pass;
        const int P = info[j].H.P, N = info[j].H.N;
        const int4 *coef = info[j].H.coef;
        float2 *part = info[j].H.part;
        double2 *part64 = info[j].H.part64;
        const int y0 = (t / ((P + kCols - 1) / kCols)) * kRows;
        if (!empty) n_s += 1u << (16 * j);
        if (!empty && pass == kPassFinal) {
            // the final pass's phase map, from S beside the u warps (S buffer j
            // goes back once both groups have read it)
            const HoloDev H = info[j].H;
            ok = warp_and(wait_newest(mbar_at(mb, kSFull0 + j), (n_s >> (16 * j)) & 0xFFFFu));
            if (!ok) break;
            fence_after();
            const uint32_t s_re = tmem + kS0 + 2 * kCols * j + lanes;
            final_phases(H, s_re, s_re + kCols, y0 + 32 * q + lane, (t % ((P + kCols - 1) / kCols)) * kCols);
            fence_before();
        }
        // the info slot (and S buffer) is read: it goes back with this group's arrival
        __syncwarp();
        if (lane == 0) arrive(mbar_at(mb, kSEmpty0 + j));
        if (empty || !last) continue;
        const int s_loc = item - tile_begin, half = P >> 1;
        for (int sb = 0; sb * kSpotBlock < N; ++sb) {
            n_z++;
            ok = warp_and(wait_newest(mbar_at(mb, kZFull), n_z));
            if (!ok) break;
            fence_after();
            const int n = sb * kSpotBlock + 32 * q + lane;
            const float2 v = strip_dot(tmem + lanes, tmem + kRows + lanes, coef, n, N, y0, half);
            fence_before();
            __syncwarp();
            if (lane == 0) arrive(mbar_at(mb, kZEmpty));
            if (n < N) {
                const size_t off = (size_t)s_loc * N + n;
                if (pass == kPassFinal) part64[off] = make_double2((double)v.x, (double)v.y);
                else part[off] = make_float2(v.x, v.y);
            }
        }
        if (!ok) break;
    }
    if (!ok && lane == 0) atomicOr(status, 1u);
}

}  // namespace ws

}  // namespace tc

template <int W, bool F16, int US>
__global__ void __launch_bounds__(tc::ws::Cfg<W>::kThreads, 1)
iter_full_tcws_kernel(const HoloDev *__restrict__ holos, const LaunchSlot *__restrict__ slots, int nslots,
                      int total_tiles, unsigned *queue)
{
    using namespace tc::ws;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t s_mbar[kBarsWs];
    __shared__ Info s_info[2];
    __shared__ G2Info s_g2;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5;
    // queue[3] != 0 (a test of the bounded waits): the producer publishes no
    // work item, so every other role's first wait runs out, before any copy
    // or MMA is issued; queue[4] != 0: the poll limit of every wait
    const bool withhold = queue[3] != 0u;
    if (tid == 0) {
        tc::s_wait_polls = queue[4] != 0u ? queue[4] : tc::kWaitPolls;
        for (int b = 0; b < kBarsWs; ++b) {
            // the epilogue's releases arrive once per warp
            // S buffers and info slots go back from the epilogue and the GEMM 1 warp
            const uint32_t cnt = (b == kSEmpty0 || b == kSEmpty0 + 1) ? W + 1
                                 : b == kZEmpty                               ? kVWarps
                                 : (b >= kUStep0 && b < kUStep0 + kKSteps)    ? kUWarps
                                 : b == kDrain                                ? 2
                                                                              : 1;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(tc::saddr(&s_mbar[b])), "r"(cnt));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(tc::saddr(&s_tmem)), "r"(kTmemColsWs));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t mb = tc::saddr(&s_mbar[0]);
    const SmemWs m = carve_ws<US>(smem);
    constexpr int R = Lay<US>::kRing;
    unsigned *status = queue + 2;
    if (warp == W) {
        if (!withhold) control_load<R>(holos, slots, nslots, total_tiles, queue, m, s_info, mb, s_tmem, status);
    } else if (warp == W + 1) {
        control_gemm1<R>(m, s_info, mb, s_tmem, status);
    } else if (warp == W + 2) {
        control_gemm2<US>(m, &s_g2, mb, s_tmem, status);
    } else if (warp < kUWarps) {
        epilogue_u<F16, US>(m, s_info, &s_g2, mb, s_tmem, status);
    } else {
        epilogue_v(s_info, mb, s_tmem, status);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(s_tmem), "r"(kTmemColsWs));
    if (tid == 0) {
        unsigned done = atomicAdd(queue + 1, 1u);
        if (done == gridDim.x - 1) {
            queue[0] = 0u;
            queue[1] = 0u;
            __threadfence();
        }
    }
}

// The per-hologram tails of a warp-specialised launch, one block per slot
// (blockIdx.y == 0): the weighted update (Eqs. 4-6) from the tile partials, or
// the metrics.  The other blocks of a compressed slot clear its subset mask
// for the next draw.
constexpr int kTailThreads = 1024;   // a hologram's tile sums take a whole block's loads in flight

__global__ void __launch_bounds__(kTailThreads) tcws_tails_kernel(const HoloDev *__restrict__ holos,
                                                         const LaunchSlot *__restrict__ slots)
{
    extern __shared__ float2 s_v[];
    __shared__ double s_red[kTailThreads / 32];
    const LaunchSlot sl = slots[blockIdx.x];
    const HoloDev &H = holos[sl.holo];
    if (blockIdx.y > 0) {
        if (sl.pass == kPassSubset && H.mask) {
            uint32_t *mask = subset_mask(H, sl.j);
            const size_t words = (size_t)H.P * H.mask_words;
            for (size_t i = (size_t)(blockIdx.y - 1) * blockDim.x + threadIdx.x; i < words;
                 i += (size_t)(gridDim.y - 1) * blockDim.x)
                mask[i] = 0u;
        }
        return;
    }
    if (sl.pass == kPassFinal) tail_metrics<kTailThreads, true>(H, sl, s_red);
    else tail_update<kTailThreads, true>(H, sl, s_v, s_red);
}

template <int W, bool F16, int US>
static int tcws_max_grid_of(int maxN, int sm_count)
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, iter_full_tcws_kernel<W, F16, US>) != cudaSuccess) return 0;
    const size_t limit = 227 * 1024 - fa.sharedSizeBytes;
    const size_t smem = tc::ws::Lay<US>::kSmem;
    if (smem > limit || (size_t)maxN * sizeof(float2) > 48 * 1024) return 0;
    if (cudaFuncSetAttribute(iter_full_tcws_kernel<W, F16, US>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)limit) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, iter_full_tcws_kernel<W, F16, US>,
                                                      tc::ws::Cfg<W>::kThreads, smem) != cudaSuccess)
        return 0;
    return std::min(per_sm, 1) * sm_count;   // a block holds all 512 tensor-memory columns
}

// Resident blocks of the kernel (both precisions; sets their shared-memory limit).
template <int W>
static int tcws_max_grid(int maxN, int sm_count)
{
    constexpr int K4 = tc::ws::kKSteps;
    return std::min(tcws_max_grid_of<W, false, K4>(maxN, sm_count), tcws_max_grid_of<W, true, K4>(maxN, sm_count));
}

template <int W, bool F16, int US>
static void tcws_launch_one(const HoloDev *holos, const LaunchSlot *slots, int nslots, int total_tiles,
                            unsigned *queue, int grid, cudaStream_t s)
{
    iter_full_tcws_kernel<W, F16, US><<<grid, tc::ws::Cfg<W>::kThreads, tc::ws::Lay<US>::kSmem, s>>>(
        holos, slots, nslots, total_tiles, queue);
}

// The per-hologram tails of a launch whose kernel writes tile partials and no
// tail of its own: one block per slot, plus (compressed launches) blocks that
// clear the subset masks.
cudaError_t launch_tc_tails(const HoloDev *holos, const LaunchSlot *slots, int nslots, int maxN, bool subset,
                            cudaStream_t s)
{
    const dim3 tails((unsigned)nslots, 1u + (subset ? 8u : 0u));
    tcws_tails_kernel<<<tails, kTailThreads, (size_t)maxN * sizeof(float2), s>>>(holos, slots);
    return cudaGetLastError();
}

template <int W>
static cudaError_t tcws_launch(const HoloDev *holos, const LaunchSlot *slots, int nslots, int total_tiles, int maxN,
                               unsigned *queue, int grid, bool subset, int f16, cudaStream_t s)
{
    constexpr int K4 = tc::ws::kKSteps;
    (void)cudaGetLastError();
    if (f16) tcws_launch_one<W, true, K4>(holos, slots, nslots, total_tiles, queue, grid, s);
    else tcws_launch_one<W, false, K4>(holos, slots, nslots, total_tiles, queue, grid, s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_tc_tails(holos, slots, nslots, maxN, subset, s);
}

// epilogue warps of the warp-specialised kernel
constexpr int kWsWarps = 8;

int full_tc_tiles(int P) { return tc::tiles(P); }

// Strip length of a launch: the one that minimises an estimate of its time in
// tile times, (tiles + f items) / grid + S / 2: the work spread over the
// resident blocks, a flush per work item (epilogue 2 and the hand-over of Z,
// f = 1/2 a tile), and the tail left by the last strips (half a strip); or the
// forced length.  A hologram with more than one spot block per GEMM 2 takes
// strips of one tile.
int full_tc_assign_strips(LaunchSlot *slots, int nslots, const int *P, const int *N, int grid, int forced)
{
    using namespace tc;
    grid = std::max(1, grid);
    auto cols = [&](int i) { return (P[i] + kCols - 1) / kCols; };
    auto rows = [&](int i) { return (P[i] + kRows - 1) / kRows; };
    auto strip_of = [&](int i, int S) { return nspotblocks(N[i]) == 1 ? std::min(S, cols(i)) : 1; };
    int smax = 1;
    for (int i = 0; i < nslots; ++i)
        if (nspotblocks(N[i]) == 1) smax = std::max(smax, cols(i));
    // The launch's finish time for strip length S, in tiles: the persistent
    // blocks take the work items in queue order, each the next free block
    // (simulated with a heap of the blocks' finish times); an item costs its
    // tiles plus a hand-over of ~0.15 tile, and 0.1 tile per unit of S stands
    // for the wider spread of holograms (and of their tables in L2) that long
    // strips keep in flight (fitted to strips of 1, 2, 3, 4, 6, 9, 12 and 18 at
    // 64 holograms of P = 1152, where 3 is fastest).
    constexpr double kItemCost = 0.15, kStripCost = 0.1;
    std::vector<double> heap;
    auto finish = [&](int S) {
        heap.assign((size_t)grid, 0.0);   // all zero: a valid min-heap
        auto take = [&](double w) {
            std::pop_heap(heap.begin(), heap.end(), std::greater<double>());
            heap.back() += w + kItemCost;
            std::push_heap(heap.begin(), heap.end(), std::greater<double>());
        };
        for (int i = 0; i < nslots; ++i) {
            const int st = strip_of(i, S), c = cols(i);
            for (int r = 0; r < rows(i); ++r)
                for (int c0 = 0; c0 < c; c0 += st) take((double)std::min(st, c - c0));
        }
        return *std::max_element(heap.begin(), heap.end());
    };
    int best = forced > 0 ? forced : 1;
    double best_cost = 1e300;
    for (int S = 1; S <= smax && forced <= 0; ++S) {
        const double cost = finish(S) + kStripCost * S;
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = S;
        }
    }
    int begin = 0;
    for (int i = 0; i < nslots; ++i) {
        const int st = strip_of(i, best);
        slots[i].strip = st;
        slots[i].tiles = rows(i) * ((cols(i) + st - 1) / st);
        slots[i].tile_begin = begin;
        begin += slots[i].tiles;
    }
    return begin;
}

int full_tc_max_grid(int variant, int maxN, int sm_count)
{
    return variant == kFullTcWs ? tcws_max_grid<kWsWarps>(maxN, sm_count) : 0;
}

void full_tc_table_bytes(int P, int N, size_t *rw, size_t *c, size_t *cs)
{
    *rw = tc::rw_table_bytes(P, N);
    *c = tc::c_table_bytes(P, N);
    *cs = tc::cs_table_bytes(P, N);
}

cudaError_t launch_tc_const_tables(const HoloDev *holos, int count, int sm_count, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    (void)cudaGetLastError();
    dim3 grid((unsigned)std::max(1, 2 * sm_count / std::max(1, count)), (unsigned)count);
    tc::const_tables_kernel<<<grid, 256, 0, s>>>(holos, count);
    return cudaGetLastError();
}

cudaError_t launch_tc_rw_tables(const HoloDev *holos, const LaunchSlot *slots, int nslots, int sm_count,
                                cudaStream_t s)
{
    if (nslots <= 0) return cudaSuccess;
    (void)cudaGetLastError();
    dim3 grid((unsigned)std::max(1, 16 * sm_count / std::max(1, nslots)), (unsigned)nslots);
    tc::rw_tables_kernel<<<grid, 256, 0, s>>>(holos, slots);
    return cudaGetLastError();
}

// The shared-memory form of the mask draw for a launch whose holograms are
// at most maxP pixels a side: the CTAs per slot (about one wave over the
// SMs), or 0 when the mask does not fit a CTA's shared memory or the launch
// has too few holograms for it: every CTA also clears and writes out a whole
// mask, so past 8 CTAs per hologram the global bit sets of
// mask_scatter_kernel (a few hundred thousand draws spread over every SM)
// cost less.
static int mask_local_shape(int maxP, int nslots, int sm_count, size_t *smem)
{
    const int G = std::max(1, sm_count / std::max(1, nslots));
    if (G > 8) return 0;
    *smem = (size_t)maxP * (size_t)mask_words_of(maxP) * 4;
    if (*smem > 200 * 1024) return 0;
    if (cudaFuncSetAttribute(tc::mask_local_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return G;
}

cudaError_t launch_tc_mask_scatter(const HoloDev *holos, const LaunchSlot *slots, int nslots, int maxP, int sm_count,
                                   cudaStream_t s)
{
    if (nslots <= 0) return cudaSuccess;
    (void)cudaGetLastError();
    size_t smem = 0;
    if (const int G = mask_local_shape(maxP, nslots, sm_count, &smem)) {
        tc::mask_local_kernel<<<dim3((unsigned)G, (unsigned)nslots), tc::kLocalThreads, smem, s>>>(holos, slots);
        return cudaGetLastError();
    }
    // a launch of few holograms (or holograms too large for the shared-memory
    // form): four blocks per SM over the launch, the draws' latency spread wide
    dim3 grid((unsigned)std::max(1, 4 * sm_count / std::max(1, nslots)), (unsigned)nslots);
    tc::mask_scatter_kernel<<<grid, 256, 0, s>>>(holos, slots);
    return cudaGetLastError();
}

cudaError_t launch_subset_tc(const HoloDev *holos, const LaunchSlot *slots, int nslots, int total_tiles, int maxN,
                             unsigned *queue, int grid, int f16, cudaStream_t s)
{
    return tcws_launch<kWsWarps>(holos, slots, nslots, total_tiles, maxN, queue, grid, true, f16, s);
}

cudaError_t launch_full_tc(int variant, const HoloDev *holos, const LaunchSlot *slots, int nslots, int total_tiles,
                           int maxN, unsigned *queue, int grid, cudaStream_t s)
{
    if (variant != kFullTcWs) return cudaErrorInvalidValue;
    return tcws_launch<kWsWarps>(holos, slots, nslots, total_tiles, maxN, queue, grid, false, 0, s);
}

}  // namespace cswgs
