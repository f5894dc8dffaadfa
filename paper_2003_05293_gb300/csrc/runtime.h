// Host runtime of the CS-WGS library: plans, device buffers, FP32 batches
// (launch schedule + CUDA graph), the autotuner and the serving loop.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <cstdarg>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cswgs_internal.h"

namespace cswgs {

cswgs_status set_error(cswgs_status s, const char *fmt, ...);

#define CSWGS_CUDA_TRY(expr)                                                               \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return ::cswgs::set_error(e_ == cudaErrorMemoryAllocation ? CSWGS_ENOMEM       \
                                                                      : CSWGS_ECUDA,       \
                                      "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_),     \
                                      __FILE__, __LINE__);                                 \
    } while (0)

#define CSWGS_TRY(expr)                              \
    do {                                             \
        cswgs_status s_ = (expr);                    \
        if (s_ != CSWGS_OK) return s_;               \
    } while (0)

// Owning device allocation.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cswgs_status ensure(size_t n)
    {
        if (n <= bytes && p) return CSWGS_OK;
        release();
        if (n == 0) n = 256;
        CSWGS_CUDA_TRY(cudaMalloc(&p, n));
        bytes = n;
        return CSWGS_OK;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// One hologram as the runtime sees it (validated copy of a request).
struct HoloSpec {
    int P = 0, N = 0, Mp = 0;
    int iterations = 0, n_full = 2, first_j = 1, final_pass = 1;
    uint64_t seed = 0;
    bool has_amp = false, has_init_w = false, has_init_th = false;
    std::vector<double> xyz, amp, init_w, init_th;
    // pupil (defaults: the square uniform grid) and SLM output (none)
    int aperture = 0, windows = 0;
    double waist = 0.0;
    int D = 0;                       // pupil pixel count
    uint32_t fa = 0, fb = 0;         // subset permutation rectangle
    double norm = 0.0;               // sum of A over the pupil
    const int2 *rows = nullptr;      // device row table of the round aperture (owned by the plan)
    bool has_slm = false;
    cswgs_slm_frame slm{};
};

cswgs_status validate_request(const cswgs_plan_desc &d, const double *xyz, const double *amp, int N,
                              int P, double c, int iterations, int n_full, HoloSpec *out);
// Applies a pupil (validated) to a validated spec: pupil size, subset size
// floor(c D), permutation rectangle, sum of A, row table.
cswgs_status apply_pupil(cswgs_plan_s *p, const cswgs_pupil &pu, double c, HoloSpec *h);
// Applies an SLM frame (validated; NULL: none).
cswgs_status apply_slm(const cswgs_slm_frame *f, HoloSpec *h);
// The pupil and SLM fields of a device hologram record from its spec.
void fill_pupil(HoloDev &H, const HoloSpec &s);

// Number of launches of the FP32 schedule: one per iteration plus the final pass.
int schedule_launches(const HoloSpec &h);
int pass_of(const HoloSpec &h, int L);   // PassKind of launch L, or -1
// Work items of a pass: subset tiles of threads * ppt pixels, or separable
// full-pass tiles (threads / 8 rows x 64 columns).
int pass_tiles(int pass, int P, int Mp, TileShape shape);
// Most work items any pass of this hologram has (size of its partial buffer).
int max_pass_tiles(const HoloSpec &h, TileShape shape);

// An FP32 batch ready to run: device buffers for every hologram, the launch
// schedule (one persistent launch per iteration), and a CUDA graph of it.
struct Fp32Batch {
    cswgs_plan_s *plan = nullptr;
    std::vector<HoloSpec> specs;
    std::vector<HoloDev> holos;           // host mirror of holos_d
    std::vector<size_t> in_off;           // per hologram: offset of its inputs in the staging block
    size_t in_bytes = 0;                  // size of the input block (device + pinned staging)
    DevBuf mem;                           // all per-hologram buffers
    DevBuf holos_d, slots_d, queue_d;
    void *staging = nullptr;              // pinned host copy of the inputs
    std::vector<float *> own_phase;       // internal phase buffers (host outputs), per hologram
    std::vector<int> l_slot0, l_nslots, l_tiles, l_maxN, l_maxP;   // per (step, kernel kind)
    TileShape shape{256, 4, 256};
    int grid[2] = {0, 0};                                     // resident blocks per kernel kind
    int maxN = 0;
    bool timing = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> events;      // launch boundaries (timing)
    double pairs_total = 0.0, pairs_iter = 0.0;
    size_t mask_begin = 0, mask_bytes = 0;   // subset masks (cleared at the start of every run)
    // the next compressed launch's subset masks are drawn on a side stream
    // (two masks per hologram, by the parity of j), beside the tails and the
    // R' tables between launches, when every hologram has the square
    // aperture; a round pupil's draws (a row search each) run on the main
    // stream before the launch
    cudaStream_t side = nullptr;
    cudaEvent_t ev_start = nullptr, ev_tail[2] = {nullptr, nullptr}, ev_scat[2] = {nullptr, nullptr};
    DevBuf copy_jobs;   // host phase maps written out by the copy kernel (cswgs_solve_batch)
    unsigned test_words[2] = {0u, 0u};   // bounded-wait test words last written to the queue
    ~Fp32Batch();
};

cswgs_status batch_build(cswgs_plan_s *p, std::vector<HoloSpec> specs, bool timing,
                         std::unique_ptr<Fp32Batch> *out);
cswgs_status batch_upload_inputs(Fp32Batch *b, cudaStream_t s);
// CSWGS_ETIMEOUT when a bounded wait inside a kernel of the batch ran out (synchronises s)
cswgs_status batch_status(Fp32Batch *b, cudaStream_t s);
cswgs_status batch_set_outputs(Fp32Batch *b, const std::vector<float *> &dev_phase, cudaStream_t s);
cswgs_status batch_enqueue(Fp32Batch *b, cudaStream_t s);   // graph launch (captures on first use)
cswgs_status batch_enqueue_direct(Fp32Batch *b, cudaStream_t s, bool capturing = false);

class Server;

}  // namespace cswgs

struct cswgs_plan_s {
    cswgs_plan_desc desc{};
    int device = 0;
    int sm_count = 0;
    bool pageable_direct = false;   // kernels may write pageable host memory (shared page tables)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::mutex mu;
    std::map<std::string, std::unique_ptr<cswgs::Fp32Batch>> solve_cache;
    std::map<std::string, cswgs::TileShape> tune;
    std::string tune_path;
    // FP64 solver workspace
    cswgs::DevBuf f64_mem;
    // small device scratch for results
    cswgs::DevBuf scratch;
    // row tables of round apertures, per grid side (uploaded once, like the
    // paper's fixed per-pixel arrays)
    std::mutex pupil_mu;
    std::map<int, std::unique_ptr<cswgs::DevBuf>> pupil_rows;
    std::unique_ptr<cswgs::Server> server;
    // test of the tensor-core kernel's bounded waits (cswgs_plan_test_waits)
    unsigned test_withhold = 0u, test_polls = 0u;
};

struct cswgs_batch_s {
    cswgs_plan_s *plan = nullptr;
    std::unique_ptr<cswgs::Fp32Batch> b;
    int count = 0;
    float last_ms = 0.f;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    // host-buffer batches (cswgs_batch_create_host): a stream of their own, the
    // caller's host phase maps of the next run, e and u landing in pinned memory
    bool host = false;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr;          // the last run has read the staged inputs
    double *eu_host = nullptr;            // pinned, 2 per hologram
    std::vector<float *> host_out;        // per hologram: host phase map of the next run, or NULL
    cswgs::DevBuf jobs;                   // map copies of the last run
    ~cswgs_batch_s();
};

namespace cswgs {
// autotuner
TileShape tuned_shape(cswgs_plan_s *p, const std::vector<HoloSpec> &specs);
cswgs_status tune_batch(cswgs_plan_s *p, Fp32Batch *b, double *best_ms);
std::string tune_key(const std::vector<HoloSpec> &specs, bool fp16);
void tune_load(cswgs_plan_s *p);
void tune_save(cswgs_plan_s *p);
}  // namespace cswgs
