// Compressed iterations over the pixels of the subset S_j only, on the CUDA
// cores, with the separable factors of the lens-and-prism phase (Eq. 2):
//   e^{i phi_n(x', y')} = C_n(x') R_n(y'),  C_n = e^{i 2 pi (a x' + g x'^2)},
//                                           R_n = e^{i 2 pi (b y' + g y'^2)}.
// Per pixel m = (y, x) of S_j:
//   back-propagation (Eq. 1):   S_m = sum_n R'_n(y) C_n(x),  R'_n = w_n a_n e^{i theta_n} R_n,
//   forward projection (Eq. 3): V_n = sum_y conj(R_n(y)) Z_n(y),  Z_n(y) = sum_{x in S_j, row y} conj(C_n(x)) u_m,
// u = A S / |S|.  Each (pixel, spot) pair costs one complex multiply-add per
// pass, so a launch costs c times a full one: the work of Eqs. 1 and 3 over
// S_j and nothing else.  A work item is a band of kBand columns and kRowsPer
// rows of one hologram: C_n(x) of the band is made once per item in shared
// memory, R_n(y) once per row.  The lanes of a warp are spots (spot
// lane + 32 i, i < SPL); a warp scan of the row's bit mask lists the row's
// pixels in shared memory, taken in batches of PB: each lane forms its spots'
// share of S for every pixel of the batch, a lane transpose sums the shares
// (lane l ends with pixel p(l)'s total), u goes back to every lane, and the
// forward projection reuses the batch's C values from registers.  The per-hologram tails (Eqs. 4-6) run in
// the tails kernel after the launch.
#include <algorithm>

#include "tile.cuh"

namespace cswgs {
namespace gather {

constexpr int kBand = 128;       // columns per work item (x0 a multiple of 128: four mask words)
constexpr int kRowsPer = 256;    // rows per work item
constexpr int kMaxSpl = 6;       // spots per lane: N <= 192 (more spill registers)
constexpr int kList = kBand + 8; // a warp's pixel list: the row's pixels and PB padding entries

template <int SPL>
struct Cfg {
    static constexpr int kWarps = SPL <= 4 ? 16 : 12;   // one block per SM; 12 warps leave 168 registers a thread
    static constexpr int kThreads = 32 * kWarps;
    static constexpr int kNpad = 32 * SPL;
    static constexpr int kPB = SPL <= 2 ? 8 : (SPL <= 4 ? 4 : 2);   // pixels per batch (registers: PB x SPL C values)
    static constexpr int kLevels = kPB == 8 ? 3 : (kPB == 4 ? 2 : 1);
    // C of the band [kBand][kNpad], the warps' partial fields [kWarps][kNpad],
    // the warps' pixel lists [kWarps][kList]
    static constexpr size_t kSmem = (size_t)kBand * kNpad * sizeof(float2) + (size_t)kWarps * kNpad * sizeof(float2) +
                                    (size_t)kWarps * kList * sizeof(int);
};

__host__ __device__ inline int bands(int P) { return (P + kBand - 1) / kBand; }
__host__ __device__ inline int row_ranges(int P) { return (P + kRowsPer - 1) / kRowsPer; }
__host__ __device__ inline int items(int P) { return bands(P) * row_ranges(P); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Packed FP32 pairs (one 64-bit register, low half first) and the packed
// fused multiply-add d = a * b + c of both halves (fma.rn.f32x2).
using f2p = unsigned long long;
__device__ __forceinline__ f2p pk(float lo, float hi)
{
    return ((f2p)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ float lo_of(f2p v) { return __uint_as_float((unsigned)v); }
__device__ __forceinline__ float hi_of(f2p v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ f2p fma2(f2p a, f2p b, f2p c)
{
    f2p d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// The pixel whose total lane `lane` ends with: bit (L - 1 - l) of p(lane) is
// lane bit (4 - l), for the L = log2(PB) exchange levels l (offsets 16, 8, ...).
template <int L>
__device__ __forceinline__ int pixel_of_lane(int lane)
{
    int p = 0;
#pragma unroll
    for (int l = 0; l < L; ++l) p |= ((lane >> (4 - l)) & 1) << (L - 1 - l);
    return p;
}

// The lane transpose of a batch.  Slot k of a holds this lane's share of pixel
// k ^ p(lane) (the slots of each lane are permuted by its own p); afterwards
// the return value is pixel p(lane)'s sum over all 32 lanes.  At level l the
// partners differ in lane bit 4 - l, hence in bit h = PB / 2^(l+1) of p: a
// lane's slot k + h holds the pixel of its partner's slot k, so every lane
// keeps its first h slots and adds the partner's upper h.
template <int PB, int L>
__device__ __forceinline__ float2 lane_transpose_sum(float2 (&a)[PB])
{
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const int off = 16 >> l, h = PB >> (l + 1);
#pragma unroll
        for (int k = 0; k < h; ++k)
            a[k] = make_float2(a[k].x + __shfl_xor_sync(0xffffffffu, a[k + h].x, off),
                               a[k].y + __shfl_xor_sync(0xffffffffu, a[k + h].y, off));
    }
    float2 v = a[0];
#pragma unroll
    for (int off = 16 >> L; off > 0; off >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    return v;
}

// A lane holding pixel k's sum after lane_transpose_sum.
template <int L>
__device__ __forceinline__ int lane_of_pixel(int k)
{
    int lane = 0;
#pragma unroll
    for (int l = 0; l < L; ++l) lane |= ((k >> (L - 1 - l)) & 1) << (4 - l);
    return lane;
}

template <int SPL>
__device__ void process_item(const HoloDev &H, const LaunchSlot &sl, int item, unsigned char *smem)
{
    using K = Cfg<SPL>;
    constexpr int NP = K::kNpad, PB = K::kPB, L = K::kLevels, kWarps = K::kWarps, kThreads = K::kThreads;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int P = H.P, N = H.N, half = P >> 1;
    const int nb = bands(P);
    const int band = item % nb, rr = item / nb;
    const int x0 = band * kBand, ncols = min(kBand, P - x0);
    const int y_begin = rr * kRowsPer, y_end = min(P, y_begin + kRowsPer);
    float2 *cs = reinterpret_cast<float2 *>(smem);   // [kBand][NP]
    float2 *red = cs + kBand * NP;                   // [kWarps][NP]
    int *list = reinterpret_cast<int *>(red + kWarps * NP) + warp * kList;   // this warp's pixel list

    // C_n(x) of the band (zero for padding spots)
    for (int f = tid; f < ncols * NP; f += kThreads) {
        const int x = f / NP, n = f - x * NP;
        float2 v = make_float2(0.f, 0.f);
        if (n < N) {
            const int4 cf = H.coef[n];
            v = spot_factor(cf.x, cf.z, __int_as_float(cf.w), x0 + x - half, kFixRound, 1.f);
        }
        cs[x * NP + n] = v;
    }
    // this lane's spots: coefficients and W_n = w_n a_n e^{i theta_n}
    int4 cf[SPL];
    float2 W[SPL];
#pragma unroll
    for (int i = 0; i < SPL; ++i) {
        const int n = lane + 32 * i;
        if (n < N) {
            cf[i] = H.coef[n];
            const SpotState st = H.state[n];
            float sn, c;
            sincos_fix(st.theta + kFixRound, -kTwoPiF, sn, c);
            W[i] = make_float2(st.w * st.a0 * c, st.w * st.a0 * sn);
        } else {
            cf[i] = make_int4(0, 0, 0, 0);
            W[i] = make_float2(0.f, 0.f);
        }
    }
    __syncthreads();

    const uint32_t *mask = subset_mask(H, sl.j);
    const int w0 = x0 >> 5;
    const float kA = H.kA;
    float2 vp[SPL];   // this warp's partial V_n of its spots
#pragma unroll
    for (int i = 0; i < SPL; ++i) vp[i] = make_float2(0.f, 0.f);

    // the row's mask word of this lane's four columns (4 lane .. 4 lane + 3 of
    // the band), the next row's loaded while this one is processed
    const int mw = H.mask_words, wl = w0 + (lane >> 3), sh = (lane & 7) * 4;
    auto row_word = [&](int y) -> uint32_t {
        return y < y_end && wl < mw ? __ldg(mask + (size_t)y * mw + wl) : 0u;
    };
    const int p = pixel_of_lane<L>(lane);
    uint32_t next = row_word(y_begin + warp);
    for (int y = y_begin + warp; y < y_end; y += kWarps) {
        const uint32_t nib = (next >> sh) & 0xFu;
        next = row_word(y + kWarps);
        // the row's pixels in column order: an inclusive scan of the lanes' counts
        const int cnt = __popc(nib);
        int incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, off);
            incl += lane >= off ? t : 0;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (total == 0) continue;
        int pos = incl - cnt;
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if ((nib >> t) & 1u) list[pos++] = 4 * lane + t;
        if (lane < PB) list[total + lane] = 0;   // padding entries: column 0 of the band, u = 0
        __syncwarp();
        const int yq = y - half;
        // R_n(y) and R'_n(y) of this lane's spots; the products run on packed
        // pairs: S's share as Re R' (C) and Im R' (C), Z as (C) Re u and (C) Im u
        float2 r[SPL];
        f2p rpx[SPL], rpy[SPL], z1[SPL], z2[SPL];
#pragma unroll
        for (int i = 0; i < SPL; ++i) {
            r[i] = lane + 32 * i < N ? spot_factor(cf[i].y, cf[i].z, __int_as_float(cf[i].w), yq, kFixRound, 1.f)
                                     : make_float2(0.f, 0.f);
            const float2 rp = cmul(r[i], W[i]);
            rpx[i] = pk(rp.x, rp.x);
            rpy[i] = pk(rp.y, rp.y);
            z1[i] = z2[i] = 0ull;
        }
        for (int b = 0; b < total; b += PB) {
            // back-propagation shares of this lane's spots; slot k is pixel b + (k ^ p)
            f2p c[PB][SPL];
            float2 a[PB];
#pragma unroll
            for (int k = 0; k < PB; ++k) {
                const f2p *crow = reinterpret_cast<const f2p *>(cs + list[b + (k ^ p)] * NP + lane);
                f2p ax = 0ull, ay = 0ull;   // sum of Re R' (C), sum of Im R' (C)
#pragma unroll
                for (int i = 0; i < SPL; ++i) {
                    c[k][i] = crow[32 * i];
                    ax = fma2(rpx[i], c[k][i], ax);
                    ay = fma2(rpy[i], c[k][i], ay);
                }
                a[k] = make_float2(lo_of(ax) - hi_of(ay), hi_of(ax) + lo_of(ay));
            }
            // S of pixel b + p, then u = A S / |S| (0 for a padding pixel)
            const float2 S = lane_transpose_sum<PB, L>(a);
            float amp = 1.f;   // Eq. 3's A
            if (kA != 0.f) {
                const int xq = x0 + list[b + p] - half;
                amp = exp2f(-kA * (float)(xq * xq + yq * yq));
            }
            const float n2 = S.x * S.x + S.y * S.y;
            const float rs = rsqrtf(n2) * amp;
            float2 u = n2 > 0.f ? make_float2(S.x * rs, S.y * rs) : make_float2(amp, 0.f);   // S = 0: phase 0
            if (b + p >= total) u = make_float2(0.f, 0.f);
            // forward projection: Z_n(y) += conj(C_n(x)) u; slot k's u is held
            // by the lanes whose p is k ^ p, lane ^ lane_of_pixel(k) among them
#pragma unroll
            for (int k = 0; k < PB; ++k) {
                const int x = lane_of_pixel<L>(k);
                const float ur = k == 0 ? u.x : __shfl_xor_sync(0xffffffffu, u.x, x);
                const float ui = k == 0 ? u.y : __shfl_xor_sync(0xffffffffu, u.y, x);
                const f2p urr = pk(ur, ur), uii = pk(ui, ui);
#pragma unroll
                for (int i = 0; i < SPL; ++i) {
                    z1[i] = fma2(c[k][i], urr, z1[i]);
                    z2[i] = fma2(c[k][i], uii, z2[i]);
                }
            }
        }
        __syncwarp();   // the list is rewritten for the next row
        // V_n += conj(R_n(y)) Z_n(y), Z = sum conj(C) u = (Re C Re u + Im C Im u, Re C Im u - Im C Re u)
#pragma unroll
        for (int i = 0; i < SPL; ++i) {
            const float zx = lo_of(z1[i]) + hi_of(z2[i]), zy = lo_of(z2[i]) - hi_of(z1[i]);
            vp[i].x = fmaf(r[i].x, zx, fmaf(r[i].y, zy, vp[i].x));
            vp[i].y = fmaf(r[i].x, zy, fmaf(-r[i].y, zx, vp[i].y));
        }
    }
    // the item's partial fields: the warps' partials summed through shared memory
#pragma unroll
    for (int i = 0; i < SPL; ++i) red[warp * NP + lane + 32 * i] = vp[i];
    __syncthreads();
    const size_t s_loc = (size_t)(item);
    for (int n = tid; n < N; n += kThreads) {
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            sr += red[w * NP + n].x;
            si += red[w * NP + n].y;
        }
        H.part[s_loc * N + n] = make_float2(sr, si);
    }
    __syncthreads();
}

}  // namespace gather

// Persistent blocks take work items (bands) from the launch's queue.
template <int SPL>
__global__ void __launch_bounds__(gather::Cfg<SPL>::kThreads, 1)
iter_subset_gather_kernel(const HoloDev *__restrict__ holos, const LaunchSlot *__restrict__ slots, int nslots,
                          int total_items, unsigned *queue)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item, s_slot;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) {
            const int item = (int)atomicAdd(queue, 1u);
            s_item = item;
            if (item < total_items) {
                int lo = 0, hi = nslots - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (slots[mid].tile_begin <= item) lo = mid;
                    else hi = mid - 1;
                }
                s_slot = lo;
            }
        }
        __syncthreads();
        const int item = s_item;
        if (item >= total_items) break;
        const LaunchSlot sl = slots[s_slot];
        const HoloDev H = holos[sl.holo];
        gather::process_item<SPL>(H, sl, item - sl.tile_begin, smem);   // ends with __syncthreads()
    }
    if (tid == 0) {
        const unsigned done = atomicAdd(queue + 1, 1u);
        if (done == gridDim.x - 1) {
            queue[0] = 0u;
            queue[1] = 0u;
            __threadfence();
        }
    }
}

#define CSWGS_GATHER_SPL(X) X(1) X(2) X(3) X(4) X(5) X(6)

static int gather_spl(int maxN) { return std::max(1, (maxN + 31) / 32); }

int subset_gather_items(int P) { return gather::items(P); }

int subset_gather_max_grid(int maxN, int sm_count)
{
    const int spl = gather_spl(maxN);
    if (spl > gather::kMaxSpl) return 0;
    int per_sm = 0;
#define X(S)                                                                                                      \
    if (spl == S) {                                                                                               \
        const size_t smem = gather::Cfg<S>::kSmem;                                                                \
        if (cudaFuncSetAttribute(iter_subset_gather_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                 (int)smem) != cudaSuccess ||                                                     \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, iter_subset_gather_kernel<S>,                   \
                                                          gather::Cfg<S>::kThreads,                               \
                                                          smem) != cudaSuccess)                                   \
            return 0;                                                                                             \
    }
    CSWGS_GATHER_SPL(X)
#undef X
    return per_sm * sm_count;
}

cudaError_t launch_subset_gather(const HoloDev *holos, const LaunchSlot *slots, int nslots, int total_items, int maxN,
                                 unsigned *queue, int grid, cudaStream_t s)
{
    const int spl = gather_spl(maxN);
    (void)cudaGetLastError();
#define X(S)                                                                                                   \
    if (spl == S)                                                                                              \
        iter_subset_gather_kernel<S><<<grid, gather::Cfg<S>::kThreads, gather::Cfg<S>::kSmem, s>>>(            \
            holos, slots, nslots, total_items, queue);
    CSWGS_GATHER_SPL(X)
#undef X
    if (spl > gather::kMaxSpl) return cudaErrorInvalidValue;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_tc_tails(holos, slots, nslots, maxN, true, s);
}

}  // namespace cswgs
