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
// lane + 32 i, i < SPL); the pixels of a row come from the subset's bit mask
// in batches of PB: each lane forms its spots' share of S for every pixel of
// the batch, a lane transpose sums the shares (lane l ends with pixel p(l)'s
// total), u goes back to every lane, and the forward projection reuses the
// batch's C values from registers.  The per-hologram tails (Eqs. 4-6) run in
// the tails kernel after the launch.
#include <algorithm>

#include "tile.cuh"

namespace cswgs {
namespace gather {

constexpr int kBand = 128;       // columns per work item (x0 a multiple of 128: four mask words)
constexpr int kRowsPer = 256;    // rows per work item
constexpr int kWarps = 16;
constexpr int kThreads = 32 * kWarps;
constexpr int kMaxSpl = 6;       // spots per lane: N <= 192 (more spill registers)

template <int SPL>
struct Cfg {
    static constexpr int kNpad = 32 * SPL;
    static constexpr int kPB = SPL <= 2 ? 8 : (SPL <= 4 ? 4 : 2);   // pixels per batch (registers: PB x SPL C values)
    static constexpr int kLevels = kPB == 8 ? 3 : (kPB == 4 ? 2 : 1);
    // C of the band [kBand][kNpad], the warps' partial fields [kWarps][kNpad]
    static constexpr size_t kSmem = (size_t)kBand * kNpad * sizeof(float2) + (size_t)kWarps * kNpad * sizeof(float2);
};

__host__ __device__ inline int bands(int P) { return (P + kBand - 1) / kBand; }
__host__ __device__ inline int row_ranges(int P) { return (P + kRowsPer - 1) / kRowsPer; }
__host__ __device__ inline int items(int P) { return bands(P) * row_ranges(P); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// The lane transpose of a batch: a[k] holds this lane's share of pixel k's
// sum; afterwards the return value is pixel p(lane)'s sum over all 32 lanes,
// p(lane) taking bit (L - 1 - l) from lane bit (4 - l) for the L = log2(PB)
// exchange levels l (offsets 16, 8, ...): at each level a lane keeps one half
// of its values and adds the partner's copy of that half.
template <int PB, int L>
__device__ __forceinline__ float2 lane_transpose_sum(float2 (&a)[PB], int lane)
{
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const int off = 16 >> l, h = PB >> (l + 1);
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const float2 send = up ? a[k] : a[k + h];
            const float2 keep = up ? a[k + h] : a[k];
            a[k] = make_float2(keep.x + __shfl_xor_sync(0xffffffffu, send.x, off),
                               keep.y + __shfl_xor_sync(0xffffffffu, send.y, off));
        }
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
    constexpr int NP = K::kNpad, PB = K::kPB, L = K::kLevels;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int P = H.P, N = H.N, half = P >> 1;
    const int nb = bands(P);
    const int band = item % nb, rr = item / nb;
    const int x0 = band * kBand, ncols = min(kBand, P - x0);
    const int y_begin = rr * kRowsPer, y_end = min(P, y_begin + kRowsPer);
    float2 *cs = reinterpret_cast<float2 *>(smem);   // [kBand][NP]
    float2 *red = cs + kBand * NP;                   // [kWarps][NP]

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

    // a row's four mask words of the band, the next row's loaded while this one is processed
    const int mw = H.mask_words;
    auto row_bits = [&](int y, uint64_t &lo, uint64_t &hi) {
        lo = hi = 0ull;
        if (y >= y_end) return;
        const uint32_t *mrow = mask + (size_t)y * mw;
        lo = (uint64_t)__ldg(mrow + w0) | (w0 + 1 < mw ? (uint64_t)__ldg(mrow + w0 + 1) << 32 : 0ull);
        hi = (w0 + 2 < mw ? (uint64_t)__ldg(mrow + w0 + 2) : 0ull) |
             (w0 + 3 < mw ? (uint64_t)__ldg(mrow + w0 + 3) << 32 : 0ull);
    };
    uint64_t next_lo, next_hi;
    row_bits(y_begin + warp, next_lo, next_hi);
    for (int y = y_begin + warp; y < y_end; y += kWarps) {
        uint64_t lo = next_lo, hi = next_hi;
        row_bits(y + kWarps, next_lo, next_hi);
        if ((lo | hi) == 0ull) continue;
        const int yq = y - half;
        // R_n(y) and R'_n(y) of this lane's spots
        float2 r[SPL], rp[SPL], z[SPL];
#pragma unroll
        for (int i = 0; i < SPL; ++i) {
            r[i] = lane + 32 * i < N ? spot_factor(cf[i].y, cf[i].z, __int_as_float(cf[i].w), yq, kFixRound, 1.f)
                                     : make_float2(0.f, 0.f);
            rp[i] = cmul(r[i], W[i]);
            z[i] = make_float2(0.f, 0.f);
        }
        while ((lo | hi) != 0ull) {
            // the next PB pixels of the row (padding pixels repeat the first
            // and carry u = 0)
            int xs[PB];
            int cnt = 0;
#pragma unroll
            for (int k = 0; k < PB; ++k) {
                int b = -1;
                if (lo != 0ull) {
                    b = __ffsll((long long)lo) - 1;
                    lo &= lo - 1ull;
                } else if (hi != 0ull) {
                    b = 64 + __ffsll((long long)hi) - 1;
                    hi &= hi - 1ull;
                }
                xs[k] = b;
                cnt += b >= 0 ? 1 : 0;
            }
#pragma unroll
            for (int k = 1; k < PB; ++k) xs[k] = xs[k] >= 0 ? xs[k] : xs[0];
            // back-propagation shares of this lane's spots
            float2 c[PB][SPL], a[PB];
#pragma unroll
            for (int k = 0; k < PB; ++k) {
                const float2 *crow = cs + xs[k] * NP + lane;
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < SPL; ++i) {
                    c[k][i] = crow[32 * i];
                    acc.x = fmaf(rp[i].x, c[k][i].x, fmaf(-rp[i].y, c[k][i].y, acc.x));
                    acc.y = fmaf(rp[i].x, c[k][i].y, fmaf(rp[i].y, c[k][i].x, acc.y));
                }
                a[k] = acc;
            }
            // S of pixel p(lane), then u = A S / |S| (0 for a padding pixel)
            const float2 S = lane_transpose_sum<PB, L>(a, lane);
            int p = 0;
#pragma unroll
            for (int l = 0; l < L; ++l) p |= ((lane >> (4 - l)) & 1) << (L - 1 - l);
            float amp = 1.f;   // Eq. 3's A
            if (kA != 0.f) {
                int xp = xs[0];   // xs[p] by selects (a lane-dependent index would go to local memory)
#pragma unroll
                for (int k = 1; k < PB; ++k) xp = p == k ? xs[k] : xp;
                const int xq = x0 + xp - half;
                amp = exp2f(-kA * (float)(xq * xq + yq * yq));
            }
            const float n2 = S.x * S.x + S.y * S.y;
            const float rs = rsqrtf(n2) * amp;
            float2 u = n2 > 0.f ? make_float2(S.x * rs, S.y * rs) : make_float2(amp, 0.f);   // S = 0: phase 0
            if (p >= cnt) u = make_float2(0.f, 0.f);
            // forward projection: Z_n(y) += conj(C_n(x)) u
#pragma unroll
            for (int k = 0; k < PB; ++k) {
                const int src = lane_of_pixel<L>(k);
                const float ur = __shfl_sync(0xffffffffu, u.x, src), ui = __shfl_sync(0xffffffffu, u.y, src);
#pragma unroll
                for (int i = 0; i < SPL; ++i) {
                    z[i].x = fmaf(c[k][i].x, ur, fmaf(c[k][i].y, ui, z[i].x));
                    z[i].y = fmaf(c[k][i].x, ui, fmaf(-c[k][i].y, ur, z[i].y));
                }
            }
        }
        // V_n += conj(R_n(y)) Z_n(y)
#pragma unroll
        for (int i = 0; i < SPL; ++i) {
            vp[i].x = fmaf(r[i].x, z[i].x, fmaf(r[i].y, z[i].y, vp[i].x));
            vp[i].y = fmaf(r[i].x, z[i].y, fmaf(-r[i].y, z[i].x, vp[i].y));
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
__global__ void __launch_bounds__(gather::kThreads, 1)
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
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, iter_subset_gather_kernel<S>, gather::kThreads,\
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
        iter_subset_gather_kernel<S><<<grid, gather::kThreads, gather::Cfg<S>::kSmem, s>>>(holos, slots, nslots, \
                                                                                          total_items, queue);
    CSWGS_GATHER_SPL(X)
#undef X
    if (spl > gather::kMaxSpl) return cudaErrorInvalidValue;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_tc_tails(holos, slots, nslots, maxN, true, s);
}

}  // namespace cswgs
