// Internal declarations shared by the kernels and the host runtime of the
// CS-WGS library.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/cswgs.h"

namespace cswgs {

// Pass kinds of one persistent launch, per hologram slot.
enum PassKind : int {
    kPassSubset = 0,   // one CS iteration over the subset S_j, then the update (Eqs. 1, 3-6)
    kPassFull = 1,     // one WGS iteration over all pixels, then the update
    kPassFinal = 2     // full back-propagation -> phase map, full projection -> e, u (Eq. 7)
};

// Per-spot state of the FP32 solver.
struct SpotState {
    uint32_t theta;   // theta_n in fixed-point turns
    float w;          // weight w_n (Eq. 4)
    float a0;         // target amplitude a_n^0
    float pad;
};

// One hologram's device buffers (FP32 solver).  All pointers are device.
// The pupil fields describe the square uniform grid when a hologram asks for
// no other pupil: D = P^2, fa = fb = P, aperture 0, kA 0, norm = P^2.
struct HoloDev {
    int P, N;
    int Mp;                 // subset size floor(c D)
    int D;                  // pupil pixel count
    uint64_t seed;
    const double *xyz;      // N x 3 inputs
    const double *amp;      // N or nullptr
    const double *init_w;   // N or nullptr: start weights
    const double *init_th;  // N or nullptr: start phases (radians)
    int4 *coef;             // N fixed-point spot coefficients (SpotFix)
    SpotState *state;       // N
    float2 *part;           // tiles x N per-tile partial fields (iterations)
    double2 *part64;        // tiles x N per-tile partial fields (final pass)
    unsigned *counter;      // tiles finished in the current pass
    float *phase_out;       // M or nullptr
    double *metrics;        // 2 + N: e, u, I_0 .. I_{N-1}
    // pupil (Section 4; Eq. 3's A) and the subset reading (Section 3)
    const int2 *rows;       // round aperture: P + 1 entries {first pupil index of row r, its first column}
    uint32_t fa, fb;        // rectangle fa x fb >= D of the subset permutation
    int aperture;           // cswgs_aperture
    int windows;            // 1: windows of one permutation; 0: a new permutation per iteration
    float kA;               // A = exp2(-kA rho^2); 0: uniform
    int pad1;
    double norm;            // sum of A over the pupil (metrics normalisation)
    // SLM frame written by the final pass (nullptr: none)
    uint8_t *slm;           // frame address of grid pixel (0, 0)
    const uint8_t *lut;     // levels gray values
    int slm_pitch;          // bytes per frame row
    int levels;
    float lscale;           // (float)(levels / (2 pi))
    int pad2;
    // factor tables of the tensor-core full passes (nullptr: not used)
    unsigned char *rwtab;   // R' = w a e^{i theta} R blocks, remade before every full pass
    unsigned char *ctab;    // C blocks (GEMM 1 operand), made once
    unsigned char *cstab;   // C blocks for GEMM 2 (split BF16), made once
    unsigned char *cstab16; // the same in FP16 for the half-precision option (nullptr: not made)
    // subset mask of compressed passes on the tensor cores (nullptr: not used):
    // P rows of mask_words words, bit c % 32 of word c / 32 for pixel column c.
    // Iteration j uses the mask at word offset (j & 1) * mask_stride: two masks
    // (one is drawn while the other is in use), or one when mask_stride is 0.
    uint32_t *mask;
    int mask_words;
    int mask_stride;
};

// One hologram's share of one persistent launch.
struct LaunchSlot {
    int holo;         // index into the HoloDev array
    int pass;         // PassKind
    int j;            // iteration index (subset key) for kPassSubset
    int tile_begin;   // first work item of this slot in the launch
    int tiles;        // work items of this slot
    int count;        // pixels of the pass (Mp or M)
    int strip;        // tensor-core kernel: tiles of one row block per work item (1 elsewhere)
    int pad;
};

// Tile shapes of the two FP32 iteration kernels.
struct TileShape {
    int threads;        // compressed iterations: threads per block, or kSubsetTc
    int ppt;            // compressed iterations: pixels per thread
    int full_threads;   // full iterations and final pass: threads per block, or kFullTcWs
    int fp16 = 0;       // compressed iterations use the half-precision sincos
    int strip = 0;      // tensor-core launches: tiles per work item (0: chosen per launch)
};

// full_threads value that selects the tensor-core kernel for full iterations
// and the final pass (kernels_tc.cu, 128 x 64-pixel tiles; warp-specialised
// and pipelined across tiles: 4 u and 4 V epilogue warps, a producer warp and
// two MMA warps; the tails in a kernel of their own)
constexpr int kFullTcWs = 2;
inline bool is_full_tc(int full_threads) { return full_threads == kFullTcWs; }

// threads value that runs the compressed iterations on the warp-specialised
// tensor-core kernel: every pixel through both products, u zero outside the
// subset S_j (a bit mask made before each launch), so the sums are those of
// Eqs. 1 and 3 over S_j
constexpr int kSubsetTc = 1;

// The two iteration kernels: compressed-iteration tiles, separable full-pass tiles.
enum LaunchKind : int { kLaunchSubset = 0, kLaunchFull = 1 };

// threads value that runs the compressed iterations on the subset-only gather
// kernel (kernels_gather.cu): the pixels of S_j only, on the CUDA cores, each
// pair one complex multiply-add per pass with the separable factors of Eq. 2;
// spots up to 192
constexpr int kSubsetGather = 3;

// Whether a batch needs the tensor-core factor tables, whether a launch of a
// kind runs on a tensor-core kernel (R' tables before it), and whether its
// compressed launches read the subset bit masks.
inline bool uses_tc(TileShape s) { return is_full_tc(s.full_threads) || s.threads == kSubsetTc; }
inline bool launch_uses_tc(TileShape s, int kind)
{
    return kind == kLaunchSubset ? s.threads == kSubsetTc : is_full_tc(s.full_threads);
}
inline bool uses_masks(TileShape s) { return s.threads == kSubsetTc || s.threads == kSubsetGather; }
inline int mask_words_of(int P) { return (P + 31) / 32; }

// Kernel launchers (kernels_fp32.cu).
cudaError_t launch_prep_fp32(const HoloDev *holos, int count, int maxN, cudaStream_t s);
cudaError_t launch_iter_fp32(TileShape shape, int kind, const HoloDev *holos, const LaunchSlot *slots,
                             int nslots, int total_tiles, int maxN, unsigned *queue,
                             int grid, cudaStream_t s);
int iter_fp32_max_grid(TileShape shape, int kind, int maxN, int sm_count);
bool tile_shape_supported(TileShape shape);
size_t iter_fp32_smem(TileShape shape, int kind, int maxN);
cudaError_t launch_subset_kernel(int P, int64_t Mp, uint64_t seed, int j, int32_t *out,
                                 cudaStream_t s);
// Tensor-core full-pass kernel (kernels_tc.cu).
int full_tc_tiles(int P);
int full_tc_max_grid(int variant, int maxN, int sm_count);
cudaError_t launch_full_tc(int variant, const HoloDev *holos, const LaunchSlot *slots, int nslots, int total_tiles,
                           int maxN, unsigned *queue, int grid, cudaStream_t s);
cudaError_t launch_subset_tc(const HoloDev *holos, const LaunchSlot *slots, int nslots, int total_tiles, int maxN,
                             unsigned *queue, int grid, int f16, cudaStream_t s);
void full_tc_table_bytes(int P, int N, size_t *rw, size_t *c, size_t *cs);   // cs: split BF16 (FP16: half)
cudaError_t launch_tc_const_tables(const HoloDev *holos, int count, int sm_count, cudaStream_t s);
cudaError_t launch_tc_rw_tables(const HoloDev *holos, const LaunchSlot *slots, int nslots, int sm_count,
                                cudaStream_t s);
// subset masks of a launch's compressed slots (holograms at most maxP pixels a side)
cudaError_t launch_tc_mask_scatter(const HoloDev *holos, const LaunchSlot *slots, int nslots, int maxP, int sm_count,
                                   cudaStream_t s);
cudaError_t launch_tc_tails(const HoloDev *holos, const LaunchSlot *slots, int nslots, int maxN, bool subset,
                            cudaStream_t s);
// Subset-only gather kernel (kernels_gather.cu): work items per hologram,
// resident blocks (0: N too large), launch (the kernel and the tails).
int subset_gather_items(int P);
int subset_gather_max_grid(int maxN, int sm_count);
cudaError_t launch_subset_gather(const HoloDev *holos, const LaunchSlot *slots, int nslots, int total_items, int maxN,
                                 unsigned *queue, int grid, cudaStream_t s);
// Work items of a tensor-core launch: chooses the strip length (tiles of one
// row block per work item, 1 for holograms of more than one GEMM 2 spot
// block; `forced` > 0 takes that length) and rewrites each slot's strip, tiles
// and tile_begin; P[i], N[i] are slot i's hologram sizes.  Returns the
// launch's work items.
int full_tc_assign_strips(LaunchSlot *slots, int nslots, const int *P, const int *N, int grid, int forced);

// Either full-pass kernel, by tile shape (runtime.cu).
bool shape_supported(TileShape shape);
int shape_max_grid(TileShape shape, int kind, int maxN, int sm_count);
int shape_full_tiles(int P, TileShape shape);
TileShape full_fallback(TileShape shape, int maxN, int sm_count);
cudaError_t shape_launch(TileShape shape, int kind, const HoloDev *holos, const LaunchSlot *slots, int nslots,
                         int total_tiles, int maxN, unsigned *queue, int grid, cudaStream_t s);

cudaError_t launch_subset_ex_kernel(const HoloDev &H, int j, int32_t *out, cudaStream_t s);
cudaError_t launch_sincos_probe(float *sink, long long *cycles, int iters, int blocks,
                                int threads, cudaStream_t s);

// FP64 baseline solver (kernels_fp64.cu): one hologram, plain kernels.
struct Fp64Work {
    double *xyz, *amp, *init_w, *init_th;
    double *coef;        // N x 3: turns per pixel (a, b, g)
    double *w, *theta;   // N
    double *phi;         // M
    int32_t *pix;        // Mp
    double2 *part;       // chunks x N
    double *metrics;     // 2 + N
    int chunks;
};
cudaError_t fp64_solve(const Fp64Work &wk, int P, int N, int Mp, int iterations, int n_full,
                       int first_j, uint64_t seed, int final_pass, float *phase_out,
                       cudaStream_t s);

}  // namespace cswgs
