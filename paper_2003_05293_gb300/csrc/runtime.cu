// Host runtime: validation, FP32 batches (buffers, launch schedule, CUDA
// graph, kernel timing) and the FP64 baseline driver.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "runtime.h"
#include "tile.cuh"

namespace cswgs {

static thread_local std::string g_last_error;

cswgs_status set_error(cswgs_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

const char *last_error() { return g_last_error.c_str(); }

static bool finite_all(const double *a, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

cswgs_status validate_request(const cswgs_plan_desc &d, const double *xyz, const double *amp, int N,
                              int P, double c, int iterations, int n_full, HoloSpec *out)
{
    if (P < 2 || (P & 1) || P > d.max_P)
        return set_error(CSWGS_EINVAL, "P=%d: need an even grid side in [2, %d]", P, d.max_P);
    if (N < 1 || N > d.max_N) return set_error(CSWGS_EINVAL, "N=%d: need 1 <= N <= %d", N, d.max_N);
    if (!(c > 0.0 && c <= 1.0)) return set_error(CSWGS_EINVAL, "subset fraction %g not in (0, 1]", c);
    const int64_t M = (int64_t)P * P;
    const int64_t Mp = (int64_t)std::floor(c * (double)M);
    if (Mp < 1) return set_error(CSWGS_EINVAL, "subset fraction %g gives an empty subset at P=%d", c, P);
    if (iterations < 0) return set_error(CSWGS_EINVAL, "iterations=%d < 0", iterations);
    if (!xyz) return set_error(CSWGS_EINVAL, "spots_xyz is NULL");
    if (!finite_all(xyz, (size_t)N * 3)) return set_error(CSWGS_EINVAL, "non-finite spot coordinate");
    if (amp) {
        for (int n = 0; n < N; ++n)
            if (!std::isfinite(amp[n]) || !(amp[n] > 0.0))
                return set_error(CSWGS_EINVAL, "amplitude %d is %g: need finite and > 0", n, amp[n]);
    }
    out->P = P;
    out->N = N;
    out->Mp = (int)Mp;
    out->D = (int)M;
    out->fa = out->fb = (uint32_t)P;
    out->norm = (double)M;
    out->iterations = iterations;
    out->n_full = n_full < 0 ? 2 : n_full;
    out->xyz.assign(xyz, xyz + (size_t)N * 3);
    out->has_amp = amp != nullptr;
    if (amp) out->amp.assign(amp, amp + N);
    return CSWGS_OK;
}

// Row r of the round aperture (y' = r - P/2): columns with x'^2 + y'^2 <=
// (P/2)^2, i.e. |x'| <= h = isqrt((P/2)^2 - y'^2), clipped to x' <= P/2 - 1.
static void round_row(int P, int r, int *first_col, int *count)
{
    const int64_t half = P / 2, y = r - half;
    const int64_t rem = half * half - y * y;
    int64_t h = (int64_t)std::sqrt((double)rem);
    while (h * h > rem) --h;
    while ((h + 1) * (h + 1) <= rem) ++h;
    const int64_t hi = std::min<int64_t>(h, half - 1);
    *first_col = (int)(half - h);
    *count = (int)(hi + h + 1);
}

cswgs_status apply_pupil(cswgs_plan_s *p, const cswgs_pupil &pu, double c, HoloSpec *h)
{
    if (pu.aperture != CSWGS_APERTURE_SQUARE && pu.aperture != CSWGS_APERTURE_ROUND)
        return set_error(CSWGS_EINVAL, "unknown aperture %d", pu.aperture);
    if (pu.subset_mode != CSWGS_SUBSET_FRESH && pu.subset_mode != CSWGS_SUBSET_WINDOWS)
        return set_error(CSWGS_EINVAL, "unknown subset mode %d", pu.subset_mode);
    if (!std::isfinite(pu.beam_waist) || pu.beam_waist < 0.0)
        return set_error(CSWGS_EINVAL, "beam waist %g: need finite and >= 0 (0 = uniform)", pu.beam_waist);
    const int P = h->P, half = P / 2;
    h->aperture = pu.aperture;
    h->windows = pu.subset_mode;
    h->waist = pu.beam_waist;
    // the amplitude is separable: A = ex(x') ex(y')
    std::vector<double> ex(P, 1.0), pre(P + 1, 0.0);
    if (h->waist > 0.0)
        for (int i = 0; i < P; ++i) {
            const double x = (double)(i - half);
            ex[i] = std::exp(-x * x / (h->waist * h->waist));
        }
    for (int i = 0; i < P; ++i) pre[i + 1] = pre[i] + ex[i];
    int64_t D = 0;
    double norm = 0.0;
    std::vector<int2> rows;
    if (h->aperture == CSWGS_APERTURE_ROUND) {
        rows.resize(P + 1);
        for (int r = 0; r < P; ++r) {
            int c0 = 0, cnt = 0;
            round_row(P, r, &c0, &cnt);
            rows[r] = make_int2((int)D, c0);
            D += cnt;
            norm += ex[r] * (pre[c0 + cnt] - pre[c0]);
        }
        rows[P] = make_int2((int)D, 0);
    } else {
        D = (int64_t)P * P;
        norm = pre[P] * pre[P];
    }
    const int64_t Mp = (int64_t)std::floor(c * (double)D);
    if (Mp < 1) return set_error(CSWGS_EINVAL, "subset fraction %g gives an empty subset of %lld pupil pixels", c,
                                 (long long)D);
    h->D = (int)D;
    h->Mp = (int)Mp;
    h->norm = norm;
    permute_rect_of((uint32_t)D, &h->fa, &h->fb);
    h->rows = nullptr;
    if (h->aperture == CSWGS_APERTURE_ROUND) {
        std::lock_guard<std::mutex> lk(p->pupil_mu);
        auto &slot = p->pupil_rows[P];
        if (!slot) {
            auto buf = std::make_unique<DevBuf>();
            CSWGS_TRY(buf->ensure(sizeof(int2) * rows.size()));
            CSWGS_CUDA_TRY(cudaSetDevice(p->device));
            CSWGS_CUDA_TRY(cudaMemcpy(buf->p, rows.data(), sizeof(int2) * rows.size(), cudaMemcpyHostToDevice));
            slot = std::move(buf);
        }
        h->rows = slot->as<int2>();
    }
    return CSWGS_OK;
}

cswgs_status apply_slm(const cswgs_slm_frame *f, HoloSpec *h)
{
    h->has_slm = false;
    if (!f) return CSWGS_OK;
    if (!f->frame || !f->lut) return set_error(CSWGS_EINVAL, "SLM frame: NULL frame or lookup table");
    if (f->levels < 2 || f->levels > 65536) return set_error(CSWGS_EINVAL, "SLM frame: %d levels", f->levels);
    if (f->width < 1 || f->height < 1 || f->pitch < f->width)
        return set_error(CSWGS_EINVAL, "SLM frame: %d x %d pixels, pitch %d", f->width, f->height, f->pitch);
    if (f->offset_x < 0 || f->offset_y < 0 || (int64_t)f->offset_x + h->P > f->width ||
        (int64_t)f->offset_y + h->P > f->height)
        return set_error(CSWGS_EINVAL, "SLM frame: the %d x %d grid at (%d, %d) leaves the %d x %d frame", h->P,
                         h->P, f->offset_x, f->offset_y, f->width, f->height);
    h->has_slm = true;
    h->slm = *f;
    return CSWGS_OK;
}

void fill_pupil(HoloDev &H, const HoloSpec &s)
{
    H.D = s.D;
    H.fa = s.fa;
    H.fb = s.fb;
    H.aperture = s.aperture;
    H.windows = s.windows;
    H.kA = s.waist > 0.0 ? (float)(1.4426950408889634 / (s.waist * s.waist)) : 0.f;
    H.norm = s.norm;
    H.rows = s.rows;
    if (s.has_slm) {
        H.slm = s.slm.frame + (size_t)s.slm.offset_y * s.slm.pitch + s.slm.offset_x;
        H.lut = s.slm.lut;
        H.slm_pitch = s.slm.pitch;
        H.levels = s.slm.levels;
        H.lscale = (float)((double)s.slm.levels / kTwoPi);
    } else {
        H.slm = nullptr;
        H.lut = nullptr;
        H.slm_pitch = 0;
        H.levels = 0;
        H.lscale = 0.f;
    }
}

int schedule_launches(const HoloSpec &h) { return h.iterations + (h.final_pass ? 1 : 0); }

int pass_of(const HoloSpec &h, int L)
{
    if (L < h.iterations) {
        int F = h.n_full < h.iterations ? h.n_full : h.iterations;
        return L >= h.iterations - F ? kPassFull : kPassSubset;
    }
    if (L == h.iterations && h.final_pass) return kPassFinal;
    return -1;
}

static int pass_count(const HoloSpec &h, int pass)
{
    return pass == kPassSubset ? h.Mp : h.D;
}

bool shape_supported(TileShape shape)
{
    // the CUDA-core kernels the shape names, with stand-ins for the tensor-core ones
    TileShape cuda_core = shape;
    if (shape.threads == kSubsetTc || shape.threads == kSubsetGather) {
        cuda_core.threads = 256;
        cuda_core.ppt = 4;
    }
    if (is_full_tc(shape.full_threads)) cuda_core.full_threads = 256;
    return tile_shape_supported(cuda_core);
}

int shape_max_grid(TileShape shape, int kind, int maxN, int sm_count)
{
    if (kind == kLaunchFull && is_full_tc(shape.full_threads))
        return full_tc_max_grid(shape.full_threads, maxN, sm_count);
    if (kind == kLaunchSubset && shape.threads == kSubsetTc) return full_tc_max_grid(kFullTcWs, maxN, sm_count);
    if (kind == kLaunchSubset && shape.threads == kSubsetGather) return subset_gather_max_grid(maxN, sm_count);
    return iter_fp32_max_grid(shape, kind, maxN, sm_count);
}

int shape_full_tiles(int P, TileShape shape)
{
    return is_full_tc(shape.full_threads) ? full_tc_tiles(P) : full_pass_tiles(P, shape.full_threads);
}

cudaError_t shape_launch(TileShape shape, int kind, const HoloDev *holos, const LaunchSlot *slots, int nslots,
                         int total_tiles, int maxN, unsigned *queue, int grid, cudaStream_t s)
{
    if (kind == kLaunchFull && is_full_tc(shape.full_threads))
        return launch_full_tc(shape.full_threads, holos, slots, nslots, total_tiles, maxN, queue, grid, s);
    if (kind == kLaunchSubset && shape.threads == kSubsetTc)
        return launch_subset_tc(holos, slots, nslots, total_tiles, maxN, queue, grid, shape.fp16, s);
    if (kind == kLaunchSubset && shape.threads == kSubsetGather)
        return launch_subset_gather(holos, slots, nslots, total_tiles, maxN, queue, grid, s);
    return launch_iter_fp32(shape, kind, holos, slots, nslots, total_tiles, maxN, queue, grid, s);
}

TileShape full_fallback(TileShape shape, int maxN, int sm_count)
{
    // past the tensor-core kernel's spot limit the CUDA-core kernels take over
    if (shape.full_threads == kFullTcWs && full_tc_max_grid(kFullTcWs, maxN, sm_count) <= 0)
        shape.full_threads = 256;
    if ((shape.threads == kSubsetTc && full_tc_max_grid(kFullTcWs, maxN, sm_count) <= 0) ||
        (shape.threads == kSubsetGather && subset_gather_max_grid(maxN, sm_count) <= 0)) {
        shape.threads = 256;
        shape.ppt = 4;
    }
    return shape;
}

int pass_tiles(int pass, int P, int Mp, TileShape shape)
{
    if (pass != kPassSubset) return shape_full_tiles(P, shape);
    if (shape.threads == kSubsetTc) return full_tc_tiles(P);
    if (shape.threads == kSubsetGather) return subset_gather_items(P);
    const int tp = shape.threads * shape.ppt;
    return (Mp + tp - 1) / tp;
}

int max_pass_tiles(const HoloSpec &h, TileShape shape)
{
    return std::max(pass_tiles(kPassSubset, h.P, h.Mp, shape), pass_tiles(kPassFull, h.P, h.Mp, shape));
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

Fp32Batch::~Fp32Batch()
{
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto e : events) cudaEventDestroy(e);
    for (cudaEvent_t e : {ev_start, ev_tail[0], ev_tail[1], ev_scat[0], ev_scat[1]})
        if (e) cudaEventDestroy(e);
    if (side) cudaStreamDestroy(side);
    if (staging) cudaFreeHost(staging);
}

// Builds the device side of a batch with a given tile shape.
static cswgs_status batch_build_shape(cswgs_plan_s *p, std::vector<HoloSpec> specs, TileShape shape,
                                      bool timing, bool host_out, std::unique_ptr<Fp32Batch> *out)
{
    auto b = std::make_unique<Fp32Batch>();
    b->plan = p;
    b->specs = std::move(specs);
    {
        int mN = 1;
        for (auto &s : b->specs) mN = std::max(mN, s.N);
        shape = full_fallback(shape, mN, p->sm_count);
    }
    b->shape = shape;
    b->timing = timing;
    const int count = (int)b->specs.size();

    // inputs block (mirrored in pinned staging)
    size_t in = 0;
    b->in_off.resize(count);
    for (int h = 0; h < count; ++h) {
        const HoloSpec &s = b->specs[h];
        b->in_off[h] = in;
        in += align256(sizeof(double) * 3 * s.N);
        if (s.has_amp) in += align256(sizeof(double) * s.N);
        if (s.has_init_w) in += align256(sizeof(double) * s.N);
        if (s.has_init_th) in += align256(sizeof(double) * s.N);
    }
    b->in_bytes = in;
    // work buffers
    size_t work = in;
    std::vector<size_t> w_off(count);
    b->maxN = 0;
    for (int h = 0; h < count; ++h) {
        const HoloSpec &s = b->specs[h];
        const int M = s.P * s.P;
        const int tiles_it = max_pass_tiles(s, shape);
        const int tiles_full = pass_tiles(kPassFull, s.P, s.Mp, shape);
        w_off[h] = work;
        work += align256(sizeof(int4) * s.N);                                   // coef
        work += align256(sizeof(SpotState) * s.N);                              // state
        work += align256(sizeof(float2) * (size_t)tiles_it * s.N);              // part
        work += align256(sizeof(double2) * (size_t)(s.final_pass ? tiles_full : 1) * s.N);  // part64
        work += 256;                                                            // counter
        work += align256(sizeof(double) * (2 + s.N));                           // metrics
        if (host_out) work += align256(sizeof(float) * (size_t)M);              // own phase
        if (uses_tc(shape)) {                                                    // tensor-core factor tables
            size_t rw, c, cs;
            full_tc_table_bytes(s.P, s.N, &rw, &c, &cs);
            work += align256(rw) + align256(c) + align256(cs);
            if (shape.fp16 && shape.threads == kSubsetTc) work += align256(cs / 2);   // FP16 C for GEMM 2
        }
        b->maxN = std::max(b->maxN, s.N);
    }
    // subset masks of compressed passes on the tensor cores or the gather
    // kernel, one block for all
    std::vector<size_t> m_off(count, 0);
    b->mask_begin = work;
    if (uses_masks(shape))
        for (int h = 0; h < count; ++h) {
            m_off[h] = work;
            work += align256(2 * sizeof(uint32_t) * (size_t)b->specs[h].P * mask_words_of(b->specs[h].P));
        }
    b->mask_bytes = work - b->mask_begin;
    CSWGS_TRY(b->mem.ensure(work));
    CSWGS_CUDA_TRY(cudaMallocHost(&b->staging, std::max<size_t>(in, 256)));

    char *base = b->mem.as<char>();
    char *stg = static_cast<char *>(b->staging);
    b->holos.resize(count);
    b->own_phase.assign(count, nullptr);
    for (int h = 0; h < count; ++h) {
        const HoloSpec &s = b->specs[h];
        HoloDev &H = b->holos[h];
        std::memset(&H, 0, sizeof H);
        H.P = s.P;
        H.N = s.N;
        H.Mp = s.Mp;
        H.seed = s.seed;
        fill_pupil(H, s);
        size_t o = b->in_off[h];
        H.xyz = reinterpret_cast<const double *>(base + o);
        std::memcpy(stg + o, s.xyz.data(), sizeof(double) * 3 * s.N);
        o += align256(sizeof(double) * 3 * s.N);
        if (s.has_amp) {
            H.amp = reinterpret_cast<const double *>(base + o);
            std::memcpy(stg + o, s.amp.data(), sizeof(double) * s.N);
            o += align256(sizeof(double) * s.N);
        }
        if (s.has_init_w) {
            H.init_w = reinterpret_cast<const double *>(base + o);
            std::memcpy(stg + o, s.init_w.data(), sizeof(double) * s.N);
            o += align256(sizeof(double) * s.N);
        }
        if (s.has_init_th) {
            H.init_th = reinterpret_cast<const double *>(base + o);
            std::memcpy(stg + o, s.init_th.data(), sizeof(double) * s.N);
            o += align256(sizeof(double) * s.N);
        }
        const int M = s.P * s.P;
        const int tiles_it = max_pass_tiles(s, shape);
        const int tiles_full = pass_tiles(kPassFull, s.P, s.Mp, shape);
        size_t w = w_off[h];
        H.coef = reinterpret_cast<int4 *>(base + w);
        w += align256(sizeof(int4) * s.N);
        H.state = reinterpret_cast<SpotState *>(base + w);
        w += align256(sizeof(SpotState) * s.N);
        H.part = reinterpret_cast<float2 *>(base + w);
        w += align256(sizeof(float2) * (size_t)tiles_it * s.N);
        H.part64 = reinterpret_cast<double2 *>(base + w);
        w += align256(sizeof(double2) * (size_t)(s.final_pass ? tiles_full : 1) * s.N);
        H.counter = reinterpret_cast<unsigned *>(base + w);
        w += 256;
        H.metrics = reinterpret_cast<double *>(base + w);
        w += align256(sizeof(double) * (2 + s.N));
        if (host_out) {
            b->own_phase[h] = reinterpret_cast<float *>(base + w);
            w += align256(sizeof(float) * (size_t)M);
        }
        H.phase_out = b->own_phase[h];
        if (uses_masks(shape)) {
            H.mask = reinterpret_cast<uint32_t *>(base + m_off[h]);
            H.mask_words = mask_words_of(s.P);
            H.mask_stride = s.P * H.mask_words;
        }
        if (uses_tc(shape)) {
            size_t rw, c, cs;
            full_tc_table_bytes(s.P, s.N, &rw, &c, &cs);
            H.rwtab = reinterpret_cast<unsigned char *>(base + w);
            w += align256(rw);
            H.ctab = reinterpret_cast<unsigned char *>(base + w);
            w += align256(c);
            H.cstab = reinterpret_cast<unsigned char *>(base + w);
            w += align256(cs);
            if (shape.fp16 && shape.threads == kSubsetTc) {
                H.cstab16 = reinterpret_cast<unsigned char *>(base + w);
                w += align256(cs / 2);
            }
        }
    }

    for (int kind = 0; kind < 2; ++kind) {
        b->grid[kind] = shape_max_grid(shape, kind, b->maxN, p->sm_count);
        if (b->grid[kind] <= 0)
            return set_error(CSWGS_ECUDA, "tile shape %dx%d / %d cannot be resident with N=%d", shape.threads,
                             shape.ppt, shape.full_threads, b->maxN);
    }
    // launch schedule: step L advances every hologram that still has work, with
    // one launch of each kernel kind that has slots in it
    int L_max = 0;
    for (auto &s : b->specs) L_max = std::max(L_max, schedule_launches(s));
    // heavier tiles first: order holograms by N (tile cost) descending; among
    // holograms of equal N every other step runs backwards, so that a launch
    // starts on the holograms whose factor tables the previous launch read
    // last (still in L2)
    std::vector<int> order(count);
    for (int h = 0; h < count; ++h) order[h] = h;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int c) { return b->specs[a].N > b->specs[c].N; });
    std::vector<int> order_back(order);
    std::stable_sort(order_back.begin(), order_back.end(), [&](int a, int c) {
        return b->specs[a].N != b->specs[c].N ? b->specs[a].N > b->specs[c].N : a > c;
    });
    std::vector<LaunchSlot> slots;
    double pairs_total = 0.0, pairs_iter = 0.0;
    for (int L = 0; L < L_max; ++L) {
        for (int kind = 0; kind < 2; ++kind) {
            int first = (int)slots.size(), tiles = 0, mN = 0, mP = 0;
            for (int h : (L & 1) ? order_back : order) {
                const HoloSpec &s = b->specs[h];
                int pass = pass_of(s, L);
                if (pass < 0 || (pass == kPassSubset) != (kind == kLaunchSubset)) continue;
                LaunchSlot sl;
                sl.holo = h;
                sl.pass = pass;
                sl.j = s.first_j + L;
                sl.count = pass_count(s, pass);
                sl.tiles = pass_tiles(pass, s.P, s.Mp, shape);
                sl.tile_begin = tiles;
                sl.strip = 1;
                sl.pad = 0;
                tiles += sl.tiles;
                mN = std::max(mN, s.N);
                mP = std::max(mP, s.P);
                slots.push_back(sl);
                double pr = 2.0 * (double)s.N * (double)sl.count;
                pairs_total += pr;
                if (pass != kPassFinal) pairs_iter += pr;
            }
            if (tiles > 0 && launch_uses_tc(shape, kind)) {
                // the tensor-core kernel takes strips of tiles along a row block
                std::vector<int> sP, sN;
                for (size_t i = first; i < slots.size(); ++i) {
                    sP.push_back(b->specs[slots[i].holo].P);
                    sN.push_back(b->specs[slots[i].holo].N);
                }
                tiles = full_tc_assign_strips(slots.data() + first, (int)slots.size() - first, sP.data(), sN.data(),
                                              b->grid[kind], shape.strip);
            }
            b->l_slot0.push_back(first);
            b->l_nslots.push_back((int)slots.size() - first);
            b->l_tiles.push_back(tiles);
            b->l_maxN.push_back(mN);
            b->l_maxP.push_back(mP);
        }
    }
    b->pairs_total = pairs_total;
    b->pairs_iter = pairs_iter;
    CSWGS_TRY(b->holos_d.ensure(sizeof(HoloDev) * count));
    CSWGS_TRY(b->slots_d.ensure(sizeof(LaunchSlot) * std::max<size_t>(1, slots.size())));
    CSWGS_TRY(b->queue_d.ensure(256));
    CSWGS_CUDA_TRY(cudaMemcpy(b->holos_d.p, b->holos.data(), sizeof(HoloDev) * count, cudaMemcpyHostToDevice));
    if (!slots.empty())
        CSWGS_CUDA_TRY(cudaMemcpy(b->slots_d.p, slots.data(), sizeof(LaunchSlot) * slots.size(),
                                  cudaMemcpyHostToDevice));
    CSWGS_CUDA_TRY(cudaMemset(b->queue_d.p, 0, 256));
    CSWGS_CUDA_TRY(cudaMemset(b->mem.p, 0, work));
    if (timing) {
        b->events.resize(L_max + 2);   // before the preparation, before each step, after the last
        for (auto &e : b->events) CSWGS_CUDA_TRY(cudaEventCreate(&e));
    }
    bool square = true;
    for (const HoloDev &H : b->holos) square = square && H.aperture == 0;
    if (uses_masks(shape) && square) {
        CSWGS_CUDA_TRY(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
        for (cudaEvent_t *e : {&b->ev_start, &b->ev_tail[0], &b->ev_tail[1], &b->ev_scat[0], &b->ev_scat[1]})
            CSWGS_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    *out = std::move(b);
    return CSWGS_OK;
}

cswgs_status batch_build(cswgs_plan_s *p, std::vector<HoloSpec> specs, bool timing,
                         std::unique_ptr<Fp32Batch> *out)
{
    TileShape shape = tuned_shape(p, specs);
    return batch_build_shape(p, std::move(specs), shape, timing, false, out);
}

cswgs_status batch_build_host(cswgs_plan_s *p, std::vector<HoloSpec> specs, bool timing,
                              bool host_out, std::unique_ptr<Fp32Batch> *out)
{
    TileShape shape = tuned_shape(p, specs);
    return batch_build_shape(p, std::move(specs), shape, timing, host_out, out);
}

cswgs_status batch_build_with(cswgs_plan_s *p, std::vector<HoloSpec> specs, TileShape shape,
                              std::unique_ptr<Fp32Batch> *out)
{
    return batch_build_shape(p, std::move(specs), shape, true, false, out);
}

// Re-stages the inputs of hologram h from its spec (after the spec changed).
void batch_restage(Fp32Batch *b, int h)
{
    const HoloSpec &s = b->specs[h];
    char *stg = static_cast<char *>(b->staging);
    size_t o = b->in_off[h];
    std::memcpy(stg + o, s.xyz.data(), sizeof(double) * 3 * s.N);
    o += align256(sizeof(double) * 3 * s.N);
    if (s.has_amp) {
        std::memcpy(stg + o, s.amp.data(), sizeof(double) * s.N);
        o += align256(sizeof(double) * s.N);
    }
    if (s.has_init_w) {
        std::memcpy(stg + o, s.init_w.data(), sizeof(double) * s.N);
        o += align256(sizeof(double) * s.N);
    }
    if (s.has_init_th) {
        std::memcpy(stg + o, s.init_th.data(), sizeof(double) * s.N);
        o += align256(sizeof(double) * s.N);
    }
}

cswgs_status batch_status(Fp32Batch *b, cudaStream_t s)
{
    unsigned st = 0;
    CSWGS_CUDA_TRY(cudaMemcpyAsync(&st, b->queue_d.as<unsigned>() + 2, sizeof st, cudaMemcpyDeviceToHost, s));
    CSWGS_CUDA_TRY(cudaStreamSynchronize(s));
    if (st) return set_error(CSWGS_ETIMEOUT, "a bounded wait inside the tensor-core kernel ran out (status %u)", st);
    return CSWGS_OK;
}

cswgs_status batch_upload_inputs(Fp32Batch *b, cudaStream_t s)
{
    if (b->in_bytes)
        CSWGS_CUDA_TRY(cudaMemcpyAsync(b->mem.p, b->staging, b->in_bytes, cudaMemcpyHostToDevice, s));
    return CSWGS_OK;
}

cswgs_status batch_set_outputs(Fp32Batch *b, const std::vector<float *> &dev_phase, cudaStream_t s)
{
    bool changed = false;
    for (size_t h = 0; h < b->holos.size(); ++h) {
        float *want = h < dev_phase.size() && dev_phase[h] ? dev_phase[h] : b->own_phase[h];
        if (b->holos[h].phase_out != want) {
            b->holos[h].phase_out = want;
            changed = true;
        }
    }
    if (changed)
        CSWGS_CUDA_TRY(cudaMemcpyAsync(b->holos_d.p, b->holos.data(), sizeof(HoloDev) * b->holos.size(),
                                       cudaMemcpyHostToDevice, s));
    return CSWGS_OK;
}

cswgs_status batch_enqueue_direct(Fp32Batch *b, cudaStream_t s, bool capturing)
{
    // inside a stream capture the timing events become event-record nodes
    const unsigned evflag = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    const HoloDev *holos = b->holos_d.as<HoloDev>();
    const LaunchSlot *slots = b->slots_d.as<LaunchSlot>();
    unsigned *queue = b->queue_d.as<unsigned>();
    const int count = (int)b->holos.size();
    // work queue, blocks done, status word (a bounded wait inside a kernel that ran out)
    CSWGS_CUDA_TRY(cudaMemsetAsync(queue, 0, 3 * sizeof(unsigned), s));
    if (b->mask_bytes) CSWGS_CUDA_TRY(cudaMemsetAsync(b->mem.as<char>() + b->mask_begin, 0, b->mask_bytes, s));
    if (b->timing) CSWGS_CUDA_TRY(cudaEventRecordWithFlags(b->events[0], s, evflag));
    CSWGS_CUDA_TRY(launch_prep_fp32(holos, count, b->maxN, s));
    if (uses_tc(b->shape)) CSWGS_CUDA_TRY(launch_tc_const_tables(holos, count, b->plan->sm_count, s));
    const size_t steps = b->l_tiles.size() / 2;
    // Compressed launches on the tensor cores draw their subset masks on the
    // side stream, one step ahead: the draw of step L + 1 is queued beside the
    // launch of step L, after the tails of step L - 1 have cleared that mask
    // (each hologram advances one iteration per step, so it alternates its two
    // masks); it runs as the launch's blocks leave, beside its tails and the
    // next R' tables.
    const bool side_masks = b->side && uses_masks(b->shape);
    auto masked = [&](size_t L) { return L < steps && b->l_tiles[2 * L + kLaunchSubset] > 0; };
    bool tail_rec[2] = {false, false};
    auto draw = [&](size_t L) -> cswgs_status {
        if (tail_rec[L & 1]) CSWGS_CUDA_TRY(cudaStreamWaitEvent(b->side, b->ev_tail[L & 1], 0));
        const size_t i = 2 * L + kLaunchSubset;
        CSWGS_CUDA_TRY(launch_tc_mask_scatter(holos, slots + b->l_slot0[i], b->l_nslots[i], b->l_maxP[i],
                                              b->plan->sm_count, b->side));
        CSWGS_CUDA_TRY(cudaEventRecordWithFlags(b->ev_scat[L & 1], b->side, 0));
        return CSWGS_OK;
    };
    if (side_masks) {
        CSWGS_CUDA_TRY(cudaEventRecordWithFlags(b->ev_start, s, 0));   // the masks are clear
        CSWGS_CUDA_TRY(cudaStreamWaitEvent(b->side, b->ev_start, 0));
        if (masked(0)) CSWGS_TRY(draw(0));
    }
    for (size_t L = 0; L < steps; ++L) {
        if (b->timing) CSWGS_CUDA_TRY(cudaEventRecordWithFlags(b->events[L + 1], s, evflag));
        for (int kind = 0; kind < 2; ++kind) {
            const size_t i = 2 * L + kind;
            const int tiles = b->l_tiles[i];
            if (tiles == 0) continue;
            const int grid = std::min(b->grid[kind], tiles);
            const bool side_draw = side_masks && kind == kLaunchSubset;
            if (kind == kLaunchSubset && uses_masks(b->shape) && !side_draw)
                CSWGS_CUDA_TRY(launch_tc_mask_scatter(holos, slots + b->l_slot0[i], b->l_nslots[i], b->l_maxP[i],
                                                      b->plan->sm_count, s));
            if (launch_uses_tc(b->shape, kind))
                CSWGS_CUDA_TRY(launch_tc_rw_tables(holos, slots + b->l_slot0[i], b->l_nslots[i], b->plan->sm_count, s));
            if (side_draw) CSWGS_CUDA_TRY(cudaStreamWaitEvent(s, b->ev_scat[L & 1], 0));
            CSWGS_CUDA_TRY(shape_launch(b->shape, kind, holos, slots + b->l_slot0[i], b->l_nslots[i], tiles,
                                        b->l_maxN[i], queue, grid, s));
            if (side_draw) {
                CSWGS_CUDA_TRY(cudaEventRecordWithFlags(b->ev_tail[L & 1], s, 0));
                tail_rec[L & 1] = true;
                if (masked(L + 1)) CSWGS_TRY(draw(L + 1));
            }
        }
    }
    if (b->timing) CSWGS_CUDA_TRY(cudaEventRecordWithFlags(b->events[steps + 1], s, evflag));
    return CSWGS_OK;
}

cswgs_status batch_enqueue(Fp32Batch *b, cudaStream_t s)
{
    if (!b->exec) {
        cudaStream_t cap;
        CSWGS_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cap);
            CSWGS_CUDA_TRY(e);
        }
        cswgs_status st = batch_enqueue_direct(b, cap, true);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (st != CSWGS_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        CSWGS_CUDA_TRY(e);
        b->graph = g;
        CSWGS_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
    }
    // the plan's bounded-wait test words (queue[3], queue[4]), when they changed
    const unsigned want[2] = {b->plan->test_withhold, b->plan->test_polls};
    if (want[0] != b->test_words[0] || want[1] != b->test_words[1]) {
        CSWGS_CUDA_TRY(cudaMemcpyAsync(b->queue_d.as<unsigned>() + 3, want, sizeof want, cudaMemcpyHostToDevice, s));
        CSWGS_CUDA_TRY(cudaStreamSynchronize(s));   // `want` lives on this stack frame
        b->test_words[0] = want[0];
        b->test_words[1] = want[1];
    }
    CSWGS_CUDA_TRY(cudaGraphLaunch(b->exec, s));
    return CSWGS_OK;
}

}  // namespace cswgs
