/*
 * cswgs.h -- C ABI of the GB300 (sm_103a) CS-WGS hologram library.
 *
 * The library computes phase-only holograms for 3D point clouds with the
 * compressed-sensing weighted Gerchberg-Saxton method (CS-WGS) of Pozzi &
 * Mapelli: back-propagation of the spot fields to the SLM (Eq. 1) with the
 * lens-and-prism spot phases of Eq. 2, forward projection onto the spots
 * (Eq. 3) over a random pixel subset, the weighted update of Eqs. 4-6, a
 * final pass over all pixels, and the efficiency / uniformity metrics (Eq. 7).
 *
 * Conventions for every entry point:
 *  - All functions return a cswgs_status and never throw or abort.  On
 *    failure cswgs_last_error() gives a one-line message (per host thread).
 *  - Input arrays are read during the call only; the caller may free or
 *    reuse them when it returns.  Outputs go to caller-owned memory.
 *  - Spot units (Eq. 2, normalised): spots_xyz holds N triples
 *    (alpha, beta, gamma) of doubles, row-major N x 3.  alpha and beta are the
 *    tilt in cycles across the P-pixel aperture, gamma the defocus in waves at
 *    the aperture edge, so that the phase of spot n at pixel (i, r) is
 *        phi_n = 2 pi [ (alpha x' + beta y') / P + gamma (x'^2 + y'^2) / (P/2)^2 ]
 *    with x' = i - P/2, y' = r - P/2, pixel index m = r * P + i.
 *  - amplitudes: N doubles a_n^0 > 0 (NULL = all 1).
 *  - The phase map is P * P floats, row-major (m = r * P + i), in [0, 2 pi).
 *  - The pupil (cswgs_pupil) is the whole P x P grid with amplitude A = 1
 *    unless a request asks for the paper's round aperture or Gaussian beam.
 *  - A plan is not thread-safe: use one plan per host thread, or the
 *    submit / poll serving calls, which are internally locked.
 *  - Argument checks (each failing with CSWGS_EINVAL): 2 <= P <= max_P and P
 *    even; 1 <= N <= max_N; 0 < subset_fraction <= 1 and
 *    Mp = floor(subset_fraction * D) >= 1, D the pupil's pixel count (P * P
 *    for the square grid); iterations >= 0; finite spot coordinates;
 *    amplitudes finite and > 0; a valid pupil and SLM frame when given.
 */
#ifndef CSWGS_H
#define CSWGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CSWGS_ABI_VERSION 2

typedef struct cswgs_plan_s *cswgs_plan;
typedef struct cswgs_batch_s *cswgs_batch;

typedef enum {
    CSWGS_OK = 0,
    CSWGS_EINVAL = 1,      /* bad argument */
    CSWGS_ENOMEM = 2,      /* device or host allocation failed, or admission refused */
    CSWGS_ECUDA = 3,       /* a CUDA call failed (message in cswgs_last_error) */
    CSWGS_ETIMEOUT = 4,    /* a bounded wait ran out (serving, or a wait inside a kernel) */
    CSWGS_EBUSY = 5,       /* serving: the request is not finished yet */
    CSWGS_ECANCELLED = 6,  /* serving: the request was cancelled */
    CSWGS_ENOTFOUND = 7    /* serving: unknown or already collected ticket */
} cswgs_status;

typedef enum {
    CSWGS_FP64 = 0,             /* plain double-precision kernels (the baseline solver) */
    CSWGS_FP32 = 1,             /* fixed-point phase range reduction + FP32 sincos, FP64 metrics */
    CSWGS_FP32_FP16SINCOS = 2   /* as FP32, with packed half-precision sincos in the compressed
                                   iterations (phasor error ~1e-3 rad; full iterations and final pass FP32) */
} cswgs_precision;

/* --------------------------------------------------------------- pupil --- */

typedef enum {
    CSWGS_APERTURE_SQUARE = 0,  /* every pixel of the P x P grid */
    CSWGS_APERTURE_ROUND = 1    /* Section 4: the round aperture of diameter P, x'^2 + y'^2 <= (P/2)^2 */
} cswgs_aperture;

typedef enum {
    CSWGS_SUBSET_FRESH = 0,     /* a new random order of the pupil's pixels per iteration j (keyed by seed, j) */
    CSWGS_SUBSET_WINDOWS = 1    /* Section 3: one random order made at the start (keyed by seed, 0); iteration
                                   j takes its entries (j-1) Mp .. j Mp - 1, wrapping around after the last */
} cswgs_subset_mode;

/* The light at the SLM and how the subsets are drawn from it (Eq. 3: the
 * forward projection sums A e^{i(Phi - phi_n)} over the pupil's pixels Omega;
 * Section 4: the paper's aperture is round, lit by a Gaussian beam).  An
 * all-zero cswgs_pupil is the default: square grid, A = 1, fresh subsets.
 * With a pupil:
 *  - subsets: Mp = floor(c D) of the D pupil pixels, through a keyed
 *    permutation of [0, D) applied to the pupil's pixels in row-major order;
 *  - iterations and the final pass run over the pupil's pixels only; the
 *    phase map holds 0 outside the pupil (no light falls there);
 *  - the forward projection weighs each pixel by A (Eq. 3);
 *  - e, u: V_n = sum_Omega A e^{i(Phi - phi_n)} / sum_Omega A, so that a
 *    hologram putting all the light into one spot has e = 1. */
typedef struct {
    int aperture;               /* cswgs_aperture */
    int subset_mode;            /* cswgs_subset_mode */
    double beam_waist;          /* Gaussian beam radius in pixels (1/e^2 of the intensity):
                                   A = exp(-(x'^2 + y'^2) / waist^2); 0: uniform A = 1 */
} cswgs_pupil;

/* Headless SLM output (Section 3: the hologram goes straight to the SLM; the
 * phase-to-gray lookup table is uploaded once at start-up).  The final pass
 * writes, for every grid pixel (i, r), the gray value
 *     frame[(offset_y + r) * pitch + offset_x + i] = lut[l],
 *     l = rint(Phi * s) mod levels,  s = (float)(levels / (2 pi)),
 * with the product and the rounding in FP32 (Phi the float phase in
 * [0, 2 pi); pixels outside the pupil have Phi = 0).  Frame pixels outside
 * the P x P grid are not touched.  The structure is copied at the call; the
 * frame and the table must stay valid until the hologram is finished. */
typedef struct {
    uint8_t *frame;             /* device, height rows of `pitch` bytes, caller-owned */
    int width, height;          /* frame size in pixels */
    int pitch;                  /* bytes per frame row, >= width */
    int offset_x, offset_y;     /* frame position of grid pixel (0, 0); the grid must lie inside the frame */
    const uint8_t *lut;         /* device, `levels` gray values: lut[l] for phase 2 pi l / levels */
    int levels;                 /* 2 .. 65536 */
} cswgs_slm_frame;

/* ------------------------------------------------- physical-unit input --- */

/* The optics of Eq. 2: wavelength lambda, focal length f of the lens that
 * images the SLM's Fourier plane, SLM pixel pitch.  All in metres. */
typedef struct {
    double wavelength;
    double focal_length;
    double pixel_pitch;
} cswgs_optics;

/* Spots given in the focal volume (metres: x, y lateral, z axial from the
 * focal plane) -> the normalised units of every solve (alpha, beta cycles
 * across the P-pixel aperture, gamma waves of defocus at its edge):
 *     alpha = x P pitch / (lambda f),  beta = y P pitch / (lambda f)
 * (Eq. 2's tilt: one cycle across the aperture is the first diffraction
 * order, at lambda f / (P pitch) in the focal plane), and
 *     gamma = z (P pitch / 2)^2 / (2 lambda f^2)
 * the paraxial defocus pi z rho^2 / (lambda f^2) at rho = P pitch / 2.  Eq. 2
 * prints 2 pi / (lambda f^2) for the defocus prefactor, twice the paraxial
 * one; the paraxial form is taken.  Host arrays, N x 3 in and out (may be
 * the same array).  Host only: no device work.  CSWGS_EINVAL for
 * non-positive or non-finite optics or coordinates, N < 1, P < 2. */
cswgs_status cswgs_spots_from_physical(const cswgs_optics *optics, const double *xyz_m, int N, int P,
                                       double *spots_out);

/* ---------------------------------------------------------------- plan --- */

typedef struct {
    int device;                 /* CUDA device ordinal */
    int max_P;                  /* largest grid side accepted */
    int max_N;                  /* largest spot count accepted */
    int max_batch;              /* largest batch, and number of serving slots */
    size_t mem_cap_bytes;       /* device bytes the serving loop may hold (0: half the free memory, at most 16 GiB) */
    cswgs_precision precision;
    void *stream;               /* cudaStream_t to run on; NULL: the plan creates its own */
    const char *tune_cache;     /* autotuner JSON cache file; NULL: keep tunings in memory only */
} cswgs_plan_desc;

/* Fills d with defaults: device 0, max_P 2048, max_N 1024, max_batch 64,
 * mem_cap 0, FP32, NULL stream, no tune cache. */
void cswgs_plan_desc_default(cswgs_plan_desc *d);

/* Creates a plan: binds the device, creates or adopts the stream, reads the
 * tune cache.  *out receives an opaque handle owned by the library. */
cswgs_status cswgs_plan_create(cswgs_plan *out, const cswgs_plan_desc *d);

/* Stops the serving loop (cancelling pending requests), frees every device
 * buffer and graph of the plan.  NULL is accepted. */
cswgs_status cswgs_plan_destroy(cswgs_plan p);

/* --------------------------------------------------------------- solve --- */

/* One hologram, synchronous.  The method (Section 2): w_n = 1 and theta_n^0
 * ~ U[0, 2 pi) drawn from `seed` (the random-superposition start, Eq. 1);
 * `iterations` WGS iterations, each a back-propagation (Eq. 1) and forward
 * projection (Eq. 3) over the iteration's pixel set followed by the update of
 * Eqs. 4-6; the pixel set is a random subset S_j of Mp = floor(c P^2)
 * pixels drawn from (seed, j) for all but the last two iterations, which run
 * over all pixels as Section 2 prescribes; then a full back-propagation
 * writes the phase map, and a full forward projection gives
 *   e = sum_n |V_n|^2 (power fraction at the spots) and u by Eq. 7,
 * with V_n = (1/P^2) sum_m e^{i(Phi_m - phi_n(m))}.
 * iterations = 0 gives the random-superposition hologram; c = 1 plain WGS.
 * phase_out: P*P floats, a device pointer (e.g. a torch tensor's data) or,
 * when out_on_host != 0, a host pointer.  e, u: host doubles (either may be
 * NULL).  Blocks until the result is written. */
cswgs_status cswgs_solve(cswgs_plan p, const double *spots_xyz, const double *amplitudes,
                         int N, int P, double subset_fraction, int iterations, uint64_t seed,
                         float *phase_out, int out_on_host, double *e, double *u);

/* Options of cswgs_solve_ex; cswgs_solve_opts_default() gives the
 * cswgs_solve behaviour. */
typedef struct {
    int full_iterations;        /* how many of the last iterations use all pixels (default 2, Section 2) */
    int first_iteration;        /* index j of the first iteration, keying its subset (default 1) */
    int final_pass;             /* 1: full back-propagation + metrics (default); 0: state only */
    const double *init_w;       /* host, N weights to start from, or NULL (all 1) */
    const double *init_theta;   /* host, N spot phases (radians) to start from, or NULL (drawn from seed) */
    double *final_w;            /* host, N: the weights after the last iteration, or NULL */
    double *final_theta;        /* host, N: the spot phases after the last iteration (radians), or NULL */
    double *spot_intensity;     /* host, N: I_n = |V_n|^2 of the final hologram, or NULL */
    cswgs_pupil pupil;          /* aperture, beam and subset reading (default all zero: square, A = 1, fresh) */
    const cswgs_slm_frame *slm; /* gray-level SLM frame written by the final pass, or NULL */
} cswgs_solve_opts;

void cswgs_solve_opts_default(cswgs_solve_opts *o);

/* cswgs_solve with options: resume from or teacher-force a state (init_w,
 * init_theta, first_iteration), choose the schedule (full_iterations), skip
 * the final pass, read back the state, take the paper's round aperture and
 * Gaussian beam (pupil), and write an SLM frame.  With final_pass = 0 the
 * phase map, frame, e and u are not written (phase_out may be NULL).  The
 * FP64 baseline solver takes the default pupil and no SLM frame only. */
cswgs_status cswgs_solve_ex(cswgs_plan p, const double *spots_xyz, const double *amplitudes,
                            int N, int P, double subset_fraction, int iterations, uint64_t seed,
                            const cswgs_solve_opts *opts, float *phase_out, int out_on_host,
                            double *e, double *u);

/* The pixel subset S_j of iteration j (Section 2, CS-WGS; Section 3,
 * "Compressed sensing": pixels taken in a random order): out_device[k] =
 * pi_{seed,j}(k) for 0 <= k < Mp, where pi is the library's keyed
 * permutation of [0, P^2).  out_device: device int32 array of Mp entries,
 * caller-owned.  Runs the same device code the solver uses.  Synchronous. */
cswgs_status cswgs_subset(cswgs_plan p, int P, int64_t Mp, uint64_t seed, int j,
                          int32_t *out_device);

/* The subset S_j of iteration j under a pupil (NULL: the default pupil):
 * *count = Mp = floor(subset_fraction * D) pixel indices m = r * P + i of
 * the pupil's pixels, in the order the solver visits them, written to
 * out_device (device int32, caller-owned, room for D entries).  Same device
 * code as the solver.  Synchronous. */
cswgs_status cswgs_subset_ex(cswgs_plan p, int P, double subset_fraction, uint64_t seed, int j,
                             const cswgs_pupil *pupil, int32_t *out_device, int64_t *count);

/* ------------------------------------------------- batches and graphs --- */

/* One hologram of a batch or a serving request. */
typedef struct {
    const double *spots_xyz;    /* host, N x 3 (copied at the call) */
    const double *amplitudes;   /* host, N, or NULL */
    int N;
    int P;
    double subset_fraction;
    int iterations;
    uint64_t seed;
    int full_iterations;        /* < 0: the default 2 */
    float *phase_out;           /* P*P floats: device pointer, or host when out_on_host; NULL: not written */
    int out_on_host;
    cswgs_pupil pupil;          /* default all zero: square, A = 1, fresh subsets */
    const cswgs_slm_frame *slm; /* gray-level SLM frame written by the final pass, or NULL */
} cswgs_request;

typedef struct {
    cswgs_status status;
    double e;                   /* efficiency */
    double u;                   /* uniformity, Eq. 7 */
    double latency_ms;          /* serving: submit -> result ready; batches: the batch's run time */
    double queue_ms;            /* serving: submit -> admitted */
} cswgs_result;

/* Prepares a batch of `count` holograms (count <= max_batch) to be run many
 * times: copies the inputs to the device, allocates their state and
 * workspace, picks tile shapes (autotuner) and captures the whole hot path
 * (spot preparation, every iteration of every hologram as one persistent
 * launch per iteration, final pass, metrics) into one CUDA graph.  Every
 * request's phase_out must be a device pointer (or NULL).  FP32 plans only. */
cswgs_status cswgs_batch_create(cswgs_plan p, const cswgs_request *reqs, int count,
                                cswgs_batch *out);

/* Launches the batch's graph on the plan's stream and returns (asynchronous). */
cswgs_status cswgs_batch_run(cswgs_batch b);

/* Waits for the last run and copies e, u of each hologram to results[count]. */
cswgs_status cswgs_batch_results(cswgs_batch b, cswgs_result *results);

/* Device time of each kernel launch of the last run, in milliseconds, in
 * launch order (spot preparation, then one entry per iteration launch, then
 * the final pass), measured with CUDA events recorded inside the graph.
 * *count receives the number of launches; ms may be NULL to query it. */
cswgs_status cswgs_batch_kernel_times(cswgs_batch b, float *ms, int cap, int *count);

/* Algorithmic sincos evaluations (pixel-spot phasors; each is one sine and one
 * cosine) of one run of the batch, for throughput accounting: per hologram
 * N * (2 * (I - F) * Mp + 2 * F * M + 2 * M), F = min(full_iterations, I). */
cswgs_status cswgs_batch_pairs(cswgs_batch b, double *pairs_total, double *pairs_iter_launches);

/* Launch shapes of the batch's two iteration kernels, as chosen by the
 * autotuner: for compressed iterations threads per block and pixels per
 * thread; for full iterations and the final pass threads per block of the
 * CUDA-core kernel, or a tensor-core kernel (tiles of 128 x 64 pixels,
 * split-BF16 products accumulated in FP32): 2 = the warp-specialised kernel,
 * pipelined across tiles (8 epilogue warps, a producer warp and two MMA
 * warps); compressed
 * iterations report threads = 1 when they run on that kernel too (u zero
 * outside the subset); and the persistent blocks of each per launch.  Any
 * pointer may be NULL. */
cswgs_status cswgs_batch_tile_shape(cswgs_batch b, int *threads, int *pixels_per_thread, int *full_threads,
                                    int *blocks, int *full_blocks);

cswgs_status cswgs_batch_destroy(cswgs_batch b);

/* Host-buffer batches: the end-to-end form of a batch, for a caller whose
 * spots and phase maps live in host memory and who solves batch after batch
 * (the method is that of cswgs_batch_create; this form only moves the data).
 * As cswgs_batch_create, except that:
 *  - every request with a phase map asks for a host one (out_on_host = 1;
 *    pinned memory is written by cudaMemcpyAsync on the copy engines, which
 *    leave the SMs to the other batch's iterations; pageable memory on a
 *    device that shares the host's page tables by a copy kernel; other memory
 *    by cudaMemcpyAsync);
 *  - the batch runs on a stream of its own (not the plan's): each
 *    cswgs_batch_run queues on it the copy of the staged inputs to the device,
 *    the batch's graph, e and u into a pinned host block and the phase maps to
 *    their host buffers, and returns at once;
 *  - cswgs_batch_results waits for that stream and reports e and u.
 * Two host batches made from one plan overlap on the device: while one copies
 * its phase maps out, the other computes.  A caller who alternates them
 * (update, run one; collect the other's results) keeps the copies off the
 * device's critical path.  Ownership: the host phase maps must stay valid
 * until cswgs_batch_results of the run that writes them returns. */
cswgs_status cswgs_batch_create_host(cswgs_plan p, const cswgs_request *reqs, int count,
                                     cswgs_batch *out);

/* New inputs and outputs for the next run of a host-buffer batch: spots_xyz,
 * amplitudes, seed and phase_out (host, or NULL: not written) of each of the
 * `count` requests are taken; the spots are copied into the batch's pinned
 * staging block at the call (the caller may reuse its arrays on return).
 * N, P, subset_fraction, iterations, full_iterations and the pupil must be
 * those the batch was made with (CSWGS_EINVAL otherwise).  Blocks until the
 * batch's last run has read its staged inputs (the start of that run), not
 * until it finishes.  CSWGS_EINVAL for a batch of cswgs_batch_create. */
cswgs_status cswgs_batch_update(cswgs_batch b, const cswgs_request *reqs, int count);

/* Runs `count` requests (host or device outputs) as one batch, synchronous:
 * the convenience form of create + run + results + destroy, reusing a cached
 * graph when the batch has the same shape as an earlier call. */
cswgs_status cswgs_solve_batch(cswgs_plan p, const cswgs_request *reqs, int count,
                               cswgs_result *results);

/* --------------------------------------------------------------- serving --- */

/* Continuous batching: a host thread of the plan admits queued requests as
 * serving slots and device memory (mem_cap_bytes) allow, keeps each admitted
 * request's state (w, theta, phase map, workspace) on the device, and advances
 * every admitted request by one iteration per persistent launch; requests join
 * and leave between launches.  The serving loop starts on the first submit. */

/* Queues a request (inputs are copied).  *ticket identifies it.  A request
 * whose footprint can never fit mem_cap_bytes fails with CSWGS_ENOMEM. */
cswgs_status cswgs_submit(cswgs_plan p, const cswgs_request *r, uint64_t *ticket);

/* CSWGS_EBUSY while pending; CSWGS_OK with *res filled once finished (the
 * ticket is then released); CSWGS_ECANCELLED / CSWGS_ENOTFOUND otherwise. */
cswgs_status cswgs_poll(cswgs_plan p, uint64_t ticket, cswgs_result *res);

/* As cswgs_poll, but waits up to timeout_s seconds (CSWGS_ETIMEOUT after). */
cswgs_status cswgs_wait(cswgs_plan p, uint64_t ticket, double timeout_s, cswgs_result *res);

/* Cancels a queued or running request; its slot is freed before the next launch. */
cswgs_status cswgs_cancel(cswgs_plan p, uint64_t ticket);

typedef struct {
    uint64_t submitted, completed, cancelled, rejected;
    uint64_t launches;          /* persistent launches issued */
    int active;                 /* requests holding a slot now */
    int queued;                 /* requests waiting for admission */
    size_t bytes_in_use;        /* device bytes held by admitted requests */
    size_t bytes_cap;
    double busy_ms;             /* summed device time of the serving launches */
} cswgs_serve_stats;

cswgs_status cswgs_serve_stats_get(cswgs_plan p, cswgs_serve_stats *s);

/* ------------------------------------------------------ tuning, probes --- */

/* Times the candidate tile shapes (threads per block, pixels per thread) of
 * the FP32 iteration kernel on a synthetic hologram of this size, keeps the
 * fastest for the (P, N) bucket and writes the tune cache if the plan has one.
 * *best_ms (may be NULL) receives the best per-iteration time. */
cswgs_status cswgs_autotune(cswgs_plan p, int P, int N, double subset_fraction, double *best_ms);

/* Measures the device's sincos throughput with a kernel that does nothing but
 * FP32 sine and cosine approximations: *sincos_per_s receives sine-or-cosine
 * results per second, *sm_mhz the SM clock seen during the run. */
cswgs_status cswgs_sincos_peak(cswgs_plan p, double *sincos_per_s, double *sm_mhz);

/* ------------------------------------------------- allocation-free solve --- */

/* The paper has no counterpart of this entry point: it serves callers that
 * cannot allocate device memory (a real-time loop feeding an SLM that cannot
 * take an allocation's latency or its risk of failing, a host with a fixed
 * device-memory budget).  It runs the cswgs_solve method (FP32, the last two
 * iterations over all pixels, the final pass) on the caller's device buffers
 * and calls no cudaMalloc, cudaFree or other allocating routine: its scratch
 * (spot tables, per-tile partial fields, counters) is one 16 MiB array of
 * device memory in the library's image, present on every GPU that loads the
 * library until the process exits.
 *   spots_xyz: device, N x 3 doubles (not checked for finiteness: device data);
 *   amplitudes: device, N doubles, or NULL (all 1);
 *   phase_out: device, P*P floats, written in [0, 2 pi);
 *   eu_out: device, 2 doubles (e, u), or NULL;
 *   stream: cudaStream_t the work is queued on (NULL: the default stream).
 * Limits: P even, 2 <= P <= 1152; 1 <= N <= 512; larger sizes fail with
 * CSWGS_EINVAL and a message.  Runs on the current device and returns once
 * the work is queued: synchronise the stream before reading the outputs.
 * The first call on a device looks up the array's device address and the
 * kernel's launch limits; make that first call before any stream capture.
 * The look-up belongs to the device's CUDA context: after the caller destroys
 * that context (cudaDeviceReset), the next call looks up again, so that call
 * too must come before any stream capture.  Launch errors are read without
 * clearing an error the caller left pending (that error is reported).
 * Every call shares the array and leaves its contents behind (each call
 * clears the parts that must start at zero); calls whose work overlaps on the
 * GPU race on it and must be serialised by the caller. */
cswgs_status cswgs_solve_noalloc(const double *spots_xyz, const double *amplitudes, int N, int P,
                                 double subset_fraction, int iterations, uint64_t seed,
                                 float *phase_out, double *eu_out, void *stream);

/* --------------------------------------------------- test of the waits --- */

/* A test of the tensor-core kernel's bounded waits (the paper has no
 * counterpart: it is the library's own safeguard).  Every wait of that kernel
 * on another of its warps (an mbarrier) gives up after a bounded number of
 * polls, records the time-out in the launch's status word and lets the
 * kernel end, so that a stalled hand-over returns CSWGS_ETIMEOUT instead of
 * hanging the GPU.  With withhold_first_item != 0, every later FP32 solve or
 * batch run of this plan launches the kernel with its producer warp holding
 * back the first work item: every other warp's first wait runs out, before
 * any bulk copy or MMA is issued, and the solve reports CSWGS_ETIMEOUT (its
 * outputs are undefined).  wait_polls != 0 sets the poll limit of every wait
 * (0: the default, 2^20).  Both 0 (the default) turn the test off; the plan
 * then solves as before.  Not for the serving loop. */
cswgs_status cswgs_plan_test_waits(cswgs_plan p, int withhold_first_item, unsigned wait_polls);

/* ---------------------------------------------------------------- misc --- */

int cswgs_abi_version(void);
const char *cswgs_status_string(cswgs_status s);
const char *cswgs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CSWGS_H */
