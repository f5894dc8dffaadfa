// A CS-WGS solve for callers that cannot allocate device memory.
//
// Some callers of this library must not call cudaMalloc: a real-time loop
// that feeds a spatial light modulator every frame cannot take an
// allocation's latency or its chance of failing mid-experiment; a host
// program that was given a fixed device-memory budget up front cannot grow
// it; code that runs where the CUDA allocator is off limits to it (an
// allocation would also synchronise the device).  They can still own their
// inputs and outputs.  cswgs_solve_noalloc serves them: it runs the same
// fused FP32 iteration kernel as the plan-based solver, but everything the
// solve needs besides the caller's buffers (spot tables, per-tile partial
// fields, counters, metrics) lives in one fixed array of device memory that
// is part of this library's image.
//
// Costs and rules of that array:
//  - it is kNoAllocScratchBytes on every GPU that loads the library, held
//    until the process exits;
//  - every call uses the same array and leaves its contents behind; the parts
//    that must start at zero (the work queue and the arrival counter) are
//    cleared by each call on its stream;
//  - two calls whose work overlaps on the GPU (other streams, other threads)
//    race on the array and give wrong results: serialise them.
#include <cmath>
#include <cstring>
#include <mutex>

#include "runtime.h"
#include "tile.cuh"

namespace cswgs {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;   // 16 MiB
constexpr int kNoAllocMaxP = 1152;
constexpr int kNoAllocMaxN = 512;
constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocPPT = 4;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

__global__ void __launch_bounds__(kNoAllocThreads, 3)
noalloc_iter_kernel(HoloDev H, LaunchSlot sl, int maxN, unsigned *queue)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_red[kNoAllocThreads / 32];
    __shared__ int s_item, s_last;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= sl.tiles) break;
        if (sl.pass == kPassSubset)
            process_tile<kNoAllocThreads, kNoAllocPPT>(H, sl, item, maxN, smem, s_red, &s_last);
        else
            process_full_tile<kNoAllocThreads>(H, sl, item, maxN, smem, s_red, &s_last);
    }
    if (threadIdx.x == 0) {
        unsigned done = atomicAdd(queue + 1, 1u);
        if (done == gridDim.x - 1) {
            queue[0] = 0u;
            queue[1] = 0u;
            __threadfence();
        }
    }
}

__global__ void noalloc_prep_kernel(HoloDev H)
{
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < H.N; n += gridDim.x * blockDim.x)
        prep_spot(H, n);
}

// Set-up of one device, done by the first call on it: the scratch array's
// device address (in host code its name is only a stand-in), the kernel's
// shared-memory limit and its resident grid.  The set-up belongs to the
// device's current CUDA context: a caller that destroys the primary context
// (cudaDeviceReset) gets a new one, whose first call here runs the set-up
// again instead of using an address of the old context.
struct NoAllocDevice {
    std::mutex mu;
    bool ready = false;
    unsigned long long ctx = 0;   // id of the context the set-up was made in
    unsigned char *base = nullptr;
    int grid = 0;
};
static NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];

// Id of the calling thread's current context (driver entry points looked up
// through the runtime, so the library needs no link to the driver library).
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

static cudaError_t current_context_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        err = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", reinterpret_cast<void **>(&get_current), 12000,
                                               cudaEnableDefault, &q1);
        if (err == cudaSuccess)
            err = cudaGetDriverEntryPointByVersion("cuCtxGetId", reinterpret_cast<void **>(&get_id), 12000,
                                                   cudaEnableDefault, &q2);
        if (err == cudaSuccess && (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess))
            err = cudaErrorNotSupported;
    });
    if (err != cudaSuccess) return err;
    void *ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return cudaErrorDeviceUninitialized;
    if (get_id(ctx, id) != 0) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

static cudaError_t noalloc_setup(NoAllocDevice &d, int device)
{
    unsigned char *base = nullptr;
    cudaError_t err = cudaGetSymbolAddress(reinterpret_cast<void **>(&base), g_noalloc_scratch);
    if (err != cudaSuccess) return err;
    const size_t smem = tile_smem_bytes(kNoAllocThreads, kNoAllocMaxN, true);
    err = cudaFuncSetAttribute(noalloc_iter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0, sms = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, noalloc_iter_kernel, kNoAllocThreads, smem);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (err != cudaSuccess) return err;
    if (per_sm * sms <= 0) return cudaErrorInvalidConfiguration;
    d.base = base;
    d.grid = per_sm * sms;
    return cudaSuccess;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace cswgs

using namespace cswgs;

extern "C" cswgs_status cswgs_solve_noalloc(const double *spots_xyz, const double *amplitudes, int N, int P,
                                            double subset_fraction, int iterations, uint64_t seed,
                                            float *phase_out, double *eu_out, void *stream)
{
    if (!spots_xyz || !phase_out) return set_error(CSWGS_EINVAL, "spots_xyz and phase_out must be device pointers");
    if (P < 2 || (P & 1) || P > kNoAllocMaxP)
        return set_error(CSWGS_EINVAL, "P=%d: the allocation-free solve takes an even P in [2, %d]", P, kNoAllocMaxP);
    if (N < 1 || N > kNoAllocMaxN)
        return set_error(CSWGS_EINVAL, "N=%d: the allocation-free solve takes 1 <= N <= %d", N, kNoAllocMaxN);
    if (!(subset_fraction > 0.0 && subset_fraction <= 1.0))
        return set_error(CSWGS_EINVAL, "subset fraction %g not in (0, 1]", subset_fraction);
    const int M = P * P;
    const int Mp = (int)std::floor(subset_fraction * (double)M);
    if (Mp < 1) return set_error(CSWGS_EINVAL, "subset fraction %g gives an empty subset", subset_fraction);
    if (iterations < 0) return set_error(CSWGS_EINVAL, "iterations=%d < 0", iterations);

    // layout of the scratch array for this size
    const int tp = kNoAllocThreads * kNoAllocPPT;
    const int full_tiles = full_pass_tiles(P, kNoAllocThreads);
    const int sub_tiles = (Mp + tp - 1) / tp;
    // iterations write FP32 tile partials (compressed or full-pixel tiles);
    // only the final pass writes the FP64 ones
    const size_t tiles = (size_t)(sub_tiles > full_tiles ? sub_tiles : full_tiles);
    size_t off = 0;
    const size_t o_queue = off; off += 256;
    const size_t o_counter = off; off += 256;
    const size_t o_coef = off; off += al256(sizeof(int4) * N);
    const size_t o_state = off; off += al256(sizeof(SpotState) * N);
    const size_t o_part = off; off += al256(sizeof(float2) * tiles * N);
    const size_t o_part64 = off; off += al256(sizeof(double2) * (size_t)full_tiles * N);
    const size_t o_metrics = off; off += al256(sizeof(double) * (2 + N));
    if (off > kNoAllocScratchBytes)
        return set_error(CSWGS_EINVAL, "P=%d, N=%d needs %zu scratch bytes; the allocation-free solve has %zu", P, N,
                         off, kNoAllocScratchBytes);

    int device = 0;
    CSWGS_CUDA_TRY(cudaGetDevice(&device));
    if (device < 0 || device >= kNoAllocMaxDevices)
        return set_error(CSWGS_EINVAL, "device %d beyond the %d supported", device, kNoAllocMaxDevices);
    // the caller's current context, or the device's primary context when the
    // thread has none yet (cudaSetDevice binds it and allocates nothing)
    unsigned long long ctx = 0;
    if (current_context_id(&ctx) != cudaSuccess) {
        CSWGS_CUDA_TRY(cudaSetDevice(device));
        CSWGS_CUDA_TRY(current_context_id(&ctx));
    }
    NoAllocDevice &d = g_noalloc_dev[device];
    unsigned char *b = nullptr;
    int dgrid = 0;
    {
        std::lock_guard<std::mutex> lk(d.mu);
        if (!d.ready || d.ctx != ctx) {
            d.ready = false;
            const cudaError_t e = noalloc_setup(d, device);
            if (e != cudaSuccess)
                return set_error(CSWGS_ECUDA, "allocation-free solve set-up on device %d: %s", device,
                                 cudaGetErrorString(e));
            d.ctx = ctx;
            d.ready = true;
        }
        b = d.base;
        dgrid = d.grid;
    }
    HoloDev H;
    std::memset(&H, 0, sizeof H);
    H.P = P;
    H.N = N;
    H.Mp = Mp;
    H.D = M;
    H.fa = H.fb = (uint32_t)P;
    H.norm = (double)M;
    H.seed = seed;
    H.xyz = spots_xyz;
    H.amp = amplitudes;
    H.coef = reinterpret_cast<int4 *>(b + o_coef);
    H.state = reinterpret_cast<SpotState *>(b + o_state);
    H.part = reinterpret_cast<float2 *>(b + o_part);
    H.part64 = reinterpret_cast<double2 *>(b + o_part64);
    H.counter = reinterpret_cast<unsigned *>(b + o_counter);
    H.phase_out = phase_out;
    H.metrics = reinterpret_cast<double *>(b + o_metrics);
    unsigned *queue = reinterpret_cast<unsigned *>(b + o_queue);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CSWGS_CUDA_TRY(cudaMemsetAsync(b, 0, 512, s));   // work queue and arrival counter start at zero
    // launch errors are read with cudaPeekAtLastError, which leaves an error
    // the caller had pending in place (it is reported, not consumed)
    noalloc_prep_kernel<<<(N + 127) / 128, 128, 0, s>>>(H);
    CSWGS_CUDA_TRY(cudaPeekAtLastError());
    const size_t smem = tile_smem_bytes(kNoAllocThreads, N, true);
    // the schedule of cswgs_solve: the last two iterations over all pixels, then the final pass
    const int n_full = iterations < 2 ? iterations : 2;
    for (int L = 0; L <= iterations; ++L) {
        LaunchSlot sl;
        sl.holo = 0;
        sl.pass = L < iterations - n_full ? kPassSubset : (L < iterations ? kPassFull : kPassFinal);
        sl.j = 1 + L;
        sl.count = sl.pass == kPassSubset ? Mp : M;
        sl.tiles = sl.pass == kPassSubset ? sub_tiles : full_tiles;
        sl.tile_begin = 0;
        sl.strip = 1;
        sl.pad = 0;
        const int grid = sl.tiles < dgrid ? sl.tiles : dgrid;
        noalloc_iter_kernel<<<grid, kNoAllocThreads, smem, s>>>(H, sl, N, queue);
        CSWGS_CUDA_TRY(cudaPeekAtLastError());
    }
    if (eu_out)
        CSWGS_CUDA_TRY(cudaMemcpyAsync(eu_out, H.metrics, 2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return CSWGS_OK;
}
