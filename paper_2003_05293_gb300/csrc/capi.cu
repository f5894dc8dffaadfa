// C ABI entry points (include/cswgs.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "runtime.h"
#include "serve.h"

namespace cswgs {
const char *last_error();
cswgs_status batch_build_host(cswgs_plan_s *p, std::vector<HoloSpec> specs, bool timing, bool host_out,
                              std::unique_ptr<Fp32Batch> *out);
void batch_restage(Fp32Batch *b, int h);
cswgs_status tune_single(cswgs_plan_s *p, int P, int N, double c, double *best_ms);

static std::string shape_key(const std::vector<HoloSpec> &v, bool host_out)
{
    std::string k = host_out ? "H" : "D";
    char buf[160];
    for (auto &s : v) {
        snprintf(buf, sizeof buf, "|%d,%d,%d,%d,%d,%d,%d,%d%d%d,%d%d", s.P, s.N, s.Mp, s.iterations, s.n_full,
                 s.first_j, s.final_pass, (int)s.has_amp, (int)s.has_init_w, (int)s.has_init_th, s.aperture,
                 s.windows);
        k += buf;
    }
    return k;
}

// FP64 baseline: one hologram on the plan's stream.
static cswgs_status solve_fp64(cswgs_plan_s *p, const HoloSpec &h, float *phase_out, int out_on_host,
                               double *e, double *u, double *final_w, double *final_theta,
                               double *spot_intensity)
{
    const int N = h.N, P = h.P;
    const int64_t M = (int64_t)P * P;
    const int chunks = (int)((M + 4095) / 4096);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0;
    size_t o_xyz = off; off += al(sizeof(double) * 3 * N);
    size_t o_amp = off; off += al(sizeof(double) * N);
    size_t o_iw = off; off += al(sizeof(double) * N);
    size_t o_it = off; off += al(sizeof(double) * N);
    size_t o_coef = off; off += al(sizeof(double) * 3 * N);
    size_t o_w = off; off += al(sizeof(double) * N);
    size_t o_th = off; off += al(sizeof(double) * N);
    size_t o_phi = off; off += al(sizeof(double) * M);
    size_t o_pix = off; off += al(sizeof(int32_t) * std::max(h.Mp, 1));
    size_t o_part = off; off += al(sizeof(double2) * (size_t)chunks * N);
    size_t o_met = off; off += al(sizeof(double) * (2 + N));
    size_t o_out = off; off += out_on_host ? al(sizeof(float) * M) : 0;
    CSWGS_TRY(p->f64_mem.ensure(off));
    char *b = p->f64_mem.as<char>();
    Fp64Work wk;
    wk.xyz = reinterpret_cast<double *>(b + o_xyz);
    wk.amp = h.has_amp ? reinterpret_cast<double *>(b + o_amp) : nullptr;
    wk.init_w = h.has_init_w ? reinterpret_cast<double *>(b + o_iw) : nullptr;
    wk.init_th = h.has_init_th ? reinterpret_cast<double *>(b + o_it) : nullptr;
    wk.coef = reinterpret_cast<double *>(b + o_coef);
    wk.w = reinterpret_cast<double *>(b + o_w);
    wk.theta = reinterpret_cast<double *>(b + o_th);
    wk.phi = reinterpret_cast<double *>(b + o_phi);
    wk.pix = reinterpret_cast<int32_t *>(b + o_pix);
    wk.part = reinterpret_cast<double2 *>(b + o_part);
    wk.metrics = reinterpret_cast<double *>(b + o_met);
    wk.chunks = chunks;
    cudaStream_t s = p->stream;
    CSWGS_CUDA_TRY(cudaMemcpyAsync(wk.xyz, h.xyz.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s));
    if (wk.amp) CSWGS_CUDA_TRY(cudaMemcpyAsync(wk.amp, h.amp.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
    if (wk.init_w) CSWGS_CUDA_TRY(cudaMemcpyAsync(wk.init_w, h.init_w.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
    if (wk.init_th) CSWGS_CUDA_TRY(cudaMemcpyAsync(wk.init_th, h.init_th.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
    float *dev_out = out_on_host ? reinterpret_cast<float *>(b + o_out) : phase_out;
    CSWGS_CUDA_TRY(fp64_solve(wk, P, N, h.Mp, h.iterations, std::min(h.n_full, h.iterations), h.first_j,
                              h.seed, h.final_pass, phase_out ? dev_out : nullptr, s));
    std::vector<double> met(2 + N);
    if (h.final_pass) {
        CSWGS_CUDA_TRY(cudaMemcpyAsync(met.data(), wk.metrics, sizeof(double) * (2 + N), cudaMemcpyDeviceToHost, s));
        if (out_on_host && phase_out)
            CSWGS_CUDA_TRY(cudaMemcpyAsync(phase_out, dev_out, sizeof(float) * M, cudaMemcpyDeviceToHost, s));
    }
    if (final_w) CSWGS_CUDA_TRY(cudaMemcpyAsync(final_w, wk.w, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
    std::vector<double> th(N);
    if (final_theta) CSWGS_CUDA_TRY(cudaMemcpyAsync(th.data(), wk.theta, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
    CSWGS_CUDA_TRY(cudaStreamSynchronize(s));
    if (final_theta)
        for (int n = 0; n < N; ++n) final_theta[n] = std::remainder(th[n], 2.0 * M_PI);
    if (h.final_pass) {
        if (e) *e = met[0];
        if (u) *u = met[1];
        if (spot_intensity) std::memcpy(spot_intensity, met.data() + 2, sizeof(double) * N);
    }
    return CSWGS_OK;
}

// Host phase maps go out through a copy kernel where the GPU can write the
// host buffer itself: pinned memory through its mapped device address, or
// pageable memory on a device that shares the host's page tables.  Each warp
// stores 512 contiguous bytes, which the link to host memory takes at a far
// higher rate than a copy-engine transfer of the same map.  Other buffers
// (and any not 16-byte aligned) are copied by cudaMemcpyAsync.
struct MapCopy {
    const float *src;
    float *dst;
    size_t n;
};

__global__ void __launch_bounds__(256) copy_maps_kernel(const MapCopy *__restrict__ jobs)
{
    const MapCopy j = jobs[blockIdx.y];
    const size_t n4 = j.n / 4, step = (size_t)gridDim.x * blockDim.x;
    const float4 *s4 = reinterpret_cast<const float4 *>(j.src);
    float4 *d4 = reinterpret_cast<float4 *>(j.dst);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += step) d4[i] = __ldcs(s4 + i);
    for (size_t i = 4 * n4 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < j.n; i += step) j.dst[i] = j.src[i];
}

static float *host_direct(const cswgs_plan_s *p, float *h)
{
    if (reinterpret_cast<uintptr_t>(h) & 15) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeHost) return static_cast<float *>(a.devicePointer);
    if (a.type == cudaMemoryTypeUnregistered && p->pageable_direct) return h;
    return nullptr;
}

static bool is_pinned(const float *h)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// Writes the maps of `jobs` out (one launch), on stream s after the solve.
static cswgs_status copy_maps(cswgs_plan_s *p, DevBuf &buf, const std::vector<MapCopy> &jobs, cudaStream_t s)
{
    if (jobs.empty()) return CSWGS_OK;
    CSWGS_TRY(buf.ensure(sizeof(MapCopy) * jobs.size()));
    CSWGS_CUDA_TRY(cudaMemcpyAsync(buf.p, jobs.data(), sizeof(MapCopy) * jobs.size(), cudaMemcpyHostToDevice, s));
    const int n = (int)jobs.size();
    const dim3 grid((unsigned)std::max(1, 4 * p->sm_count / n), (unsigned)n);
    copy_maps_kernel<<<grid, 256, 0, s>>>(static_cast<const MapCopy *>(buf.p));
    CSWGS_CUDA_TRY(cudaGetLastError());
    return CSWGS_OK;
}

// FP32 solver: one hologram through a cached single-hologram batch.
static cswgs_status solve_fp32(cswgs_plan_s *p, HoloSpec h, float *phase_out, int out_on_host,
                               double *e, double *u, double *final_w, double *final_theta,
                               double *spot_intensity)
{
    const int N = h.N;
    std::vector<HoloSpec> v{h};
    const bool host_out = out_on_host && phase_out;
    std::string key = shape_key(v, host_out);
    Fp32Batch *b = nullptr;
    auto it = p->solve_cache.find(key);
    if (it == p->solve_cache.end()) {
        std::unique_ptr<Fp32Batch> nb;
        CSWGS_TRY(batch_build_host(p, v, false, host_out, &nb));
        b = nb.get();
        p->solve_cache[key] = std::move(nb);
    } else {
        b = it->second.get();
        b->specs[0] = std::move(h);
        b->holos[0].seed = b->specs[0].seed;
        fill_pupil(b->holos[0], b->specs[0]);
        batch_restage(b, 0);
        // the seed, the beam and the SLM frame live in the device hologram record
        CSWGS_CUDA_TRY(cudaMemcpyAsync(b->holos_d.p, b->holos.data(), sizeof(HoloDev), cudaMemcpyHostToDevice,
                                       p->stream));
    }
    cudaStream_t s = p->stream;
    CSWGS_TRY(batch_upload_inputs(b, s));
    std::vector<float *> outs{host_out ? nullptr : phase_out};
    CSWGS_TRY(batch_set_outputs(b, outs, s));
    CSWGS_TRY(batch_enqueue(b, s));
    const HoloDev &H = b->holos[0];
    std::vector<double> met(2 + N);
    std::vector<SpotState> st(N);
    if (b->specs[0].final_pass) {
        CSWGS_CUDA_TRY(cudaMemcpyAsync(met.data(), H.metrics, sizeof(double) * (2 + N), cudaMemcpyDeviceToHost, s));
        if (host_out) {
            const size_t n = (size_t)H.P * H.P;
            if (float *d = host_direct(p, phase_out))
                CSWGS_TRY(copy_maps(p, b->copy_jobs, {MapCopy{b->own_phase[0], d, n}}, s));
            else
                CSWGS_CUDA_TRY(cudaMemcpyAsync(phase_out, b->own_phase[0], sizeof(float) * n, cudaMemcpyDeviceToHost, s));
        }
    }
    if (final_w || final_theta)
        CSWGS_CUDA_TRY(cudaMemcpyAsync(st.data(), H.state, sizeof(SpotState) * N, cudaMemcpyDeviceToHost, s));
    CSWGS_TRY(batch_status(b, s));
    for (int n = 0; n < N; ++n) {
        if (final_w) final_w[n] = (double)st[n].w;
        if (final_theta) final_theta[n] = (double)(int32_t)st[n].theta * (2.0 * M_PI / 4294967296.0);
    }
    if (b->specs[0].final_pass) {
        if (e) *e = met[0];
        if (u) *u = met[1];
        if (spot_intensity) std::memcpy(spot_intensity, met.data() + 2, sizeof(double) * N);
    }
    return CSWGS_OK;
}

static cswgs_status set_device(cswgs_plan_s *p)
{
    CSWGS_CUDA_TRY(cudaSetDevice(p->device));
    return CSWGS_OK;
}

// e and u of every hologram of a batch into one host block (pinned memory,
// written through its device address): one launch instead of a copy per
// hologram.
__global__ void eu_gather_kernel(const HoloDev *__restrict__ holos, int count, double *dst)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        dst[2 * i] = holos[i].metrics[0];
        dst[2 * i + 1] = holos[i].metrics[1];
    }
}

// A request of a host-buffer batch's update must keep the batch's shape.
static bool same_shape(const HoloSpec &a, const HoloSpec &b)
{
    return a.P == b.P && a.N == b.N && a.Mp == b.Mp && a.iterations == b.iterations && a.n_full == b.n_full &&
           a.has_amp == b.has_amp && a.aperture == b.aperture && a.windows == b.windows && a.waist == b.waist &&
           a.has_slm == b.has_slm;
}

}  // namespace cswgs

cswgs_batch_s::~cswgs_batch_s()
{
    if (stream) cudaStreamSynchronize(stream);
    b.reset();
    if (ev_in) cudaEventDestroy(ev_in);
    if (eu_host) cudaFreeHost(eu_host);
    if (stream) cudaStreamDestroy(stream);
}

using namespace cswgs;

extern "C" {

int cswgs_abi_version(void) { return CSWGS_ABI_VERSION; }

const char *cswgs_status_string(cswgs_status s)
{
    switch (s) {
    case CSWGS_OK: return "ok";
    case CSWGS_EINVAL: return "invalid argument";
    case CSWGS_ENOMEM: return "out of memory";
    case CSWGS_ECUDA: return "CUDA error";
    case CSWGS_ETIMEOUT: return "timed out";
    case CSWGS_EBUSY: return "busy";
    case CSWGS_ECANCELLED: return "cancelled";
    case CSWGS_ENOTFOUND: return "not found";
    }
    return "unknown status";
}

const char *cswgs_last_error(void) { return cswgs::last_error(); }

void cswgs_plan_desc_default(cswgs_plan_desc *d)
{
    if (!d) return;
    std::memset(d, 0, sizeof *d);
    d->device = 0;
    d->max_P = 2048;
    d->max_N = 1024;
    d->max_batch = 64;
    d->mem_cap_bytes = 0;
    d->precision = CSWGS_FP32;
    d->stream = nullptr;
    d->tune_cache = nullptr;
}

void cswgs_solve_opts_default(cswgs_solve_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->full_iterations = 2;
    o->first_iteration = 1;
    o->final_pass = 1;
}

cswgs_status cswgs_spots_from_physical(const cswgs_optics *optics, const double *xyz_m, int N, int P,
                                       double *spots_out)
{
    if (!optics || !xyz_m || !spots_out) return set_error(CSWGS_EINVAL, "NULL optics, spots or output");
    if (N < 1 || P < 2) return set_error(CSWGS_EINVAL, "N=%d, P=%d", N, P);
    const double lam = optics->wavelength, f = optics->focal_length, pitch = optics->pixel_pitch;
    if (!(std::isfinite(lam) && lam > 0.0 && std::isfinite(f) && f > 0.0 && std::isfinite(pitch) && pitch > 0.0))
        return set_error(CSWGS_EINVAL, "optics: wavelength %g, focal length %g, pitch %g must be finite and > 0",
                         lam, f, pitch);
    const double aperture = (double)P * pitch;            // metres across the P-pixel aperture
    const double tilt = aperture / (lam * f);              // cycles per metre in the focal plane
    const double edge = 0.5 * aperture;
    const double defocus = edge * edge / (2.0 * lam * f * f);   // waves at the edge per metre of z
    for (int n = 0; n < N; ++n) {
        const double x = xyz_m[3 * n], y = xyz_m[3 * n + 1], z = xyz_m[3 * n + 2];
        if (!(std::isfinite(x) && std::isfinite(y) && std::isfinite(z)))
            return set_error(CSWGS_EINVAL, "spot %d: non-finite coordinate", n);
        spots_out[3 * n] = x * tilt;
        spots_out[3 * n + 1] = y * tilt;
        spots_out[3 * n + 2] = z * defocus;
    }
    return CSWGS_OK;
}

cswgs_status cswgs_plan_create(cswgs_plan *out, const cswgs_plan_desc *d)
{
    if (!out || !d) return set_error(CSWGS_EINVAL, "NULL plan or descriptor");
    *out = nullptr;
    if (d->max_P < 2 || d->max_P > 32768 || d->max_N < 1 || d->max_N > 4096 || d->max_batch < 1 ||
        d->max_batch > 4096)
        return set_error(CSWGS_EINVAL, "plan limits out of range (max_P %d, max_N %d, max_batch %d)", d->max_P,
                         d->max_N, d->max_batch);
    if (d->precision != CSWGS_FP64 && d->precision != CSWGS_FP32 && d->precision != CSWGS_FP32_FP16SINCOS)
        return set_error(CSWGS_EINVAL, "unknown precision %d", (int)d->precision);
    int ndev = 0;
    CSWGS_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (d->device < 0 || d->device >= ndev) return set_error(CSWGS_EINVAL, "device %d of %d", d->device, ndev);
    auto *p = new (std::nothrow) cswgs_plan_s();
    if (!p) return set_error(CSWGS_ENOMEM, "host allocation");
    p->desc = *d;
    p->desc.tune_cache = nullptr;
    p->device = d->device;
    if (d->tune_cache) p->tune_path = d->tune_cache;
    cswgs_status st = set_device(p);
    if (st == CSWGS_OK) {
        cudaError_t e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
        if (e != cudaSuccess) st = set_error(CSWGS_ECUDA, "device attribute: %s", cudaGetErrorString(e));
        int pageable = 0, shared_tables = 0;
        if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, p->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&shared_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, p->device) !=
                cudaSuccess)
            (void)cudaGetLastError();
        p->pageable_direct = pageable != 0 && shared_tables != 0;
    }
    if (st == CSWGS_OK) {
        if (d->stream) {
            p->stream = static_cast<cudaStream_t>(d->stream);
        } else {
            cudaError_t e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) st = set_error(CSWGS_ECUDA, "stream: %s", cudaGetErrorString(e));
            p->own_stream = true;
        }
    }
    if (st != CSWGS_OK) {
        delete p;
        return st;
    }
    tune_load(p);
    *out = p;
    return CSWGS_OK;
}

cswgs_status cswgs_plan_destroy(cswgs_plan p)
{
    if (!p) return CSWGS_OK;
    cudaSetDevice(p->device);
    p->server.reset();
    cudaStreamSynchronize(p->stream);
    p->solve_cache.clear();
    p->f64_mem.release();
    p->scratch.release();
    if (p->own_stream) cudaStreamDestroy(p->stream);
    delete p;
    return CSWGS_OK;
}

cswgs_status cswgs_solve_ex(cswgs_plan p, const double *spots_xyz, const double *amplitudes, int N, int P,
                            double subset_fraction, int iterations, uint64_t seed, const cswgs_solve_opts *opts,
                            float *phase_out, int out_on_host, double *e, double *u)
{
    if (!p) return set_error(CSWGS_EINVAL, "NULL plan");
    cswgs_solve_opts o;
    cswgs_solve_opts_default(&o);
    if (opts) o = *opts;
    if (o.full_iterations < 0) o.full_iterations = 2;
    if (o.first_iteration < 0) return set_error(CSWGS_EINVAL, "first_iteration %d < 0", o.first_iteration);
    HoloSpec h;
    CSWGS_TRY(validate_request(p->desc, spots_xyz, amplitudes, N, P, subset_fraction, iterations,
                               o.full_iterations, &h));
    CSWGS_TRY(apply_pupil(p, o.pupil, subset_fraction, &h));
    CSWGS_TRY(apply_slm(o.slm, &h));
    if (p->desc.precision == CSWGS_FP64 && (h.aperture || h.windows || h.waist > 0.0 || h.has_slm))
        return set_error(CSWGS_EINVAL, "the FP64 baseline solver takes the default pupil and no SLM frame");
    h.seed = seed;
    h.first_j = o.first_iteration;
    h.final_pass = o.final_pass ? 1 : 0;
    if (o.init_w) {
        for (int n = 0; n < N; ++n)
            if (!std::isfinite(o.init_w[n]) || !(o.init_w[n] > 0.0))
                return set_error(CSWGS_EINVAL, "init_w[%d] = %g: need finite and > 0", n, o.init_w[n]);
        h.has_init_w = true;
        h.init_w.assign(o.init_w, o.init_w + N);
    }
    if (o.init_theta) {
        for (int n = 0; n < N; ++n)
            if (!std::isfinite(o.init_theta[n])) return set_error(CSWGS_EINVAL, "init_theta[%d] not finite", n);
        h.has_init_th = true;
        h.init_th.assign(o.init_theta, o.init_theta + N);
    }
    std::lock_guard<std::mutex> lk(p->mu);
    CSWGS_TRY(set_device(p));
    if (p->desc.precision == CSWGS_FP64)
        return solve_fp64(p, h, phase_out, out_on_host, e, u, o.final_w, o.final_theta, o.spot_intensity);
    return solve_fp32(p, std::move(h), phase_out, out_on_host, e, u, o.final_w, o.final_theta,
                      o.spot_intensity);
}

cswgs_status cswgs_solve(cswgs_plan p, const double *spots_xyz, const double *amplitudes, int N, int P,
                         double subset_fraction, int iterations, uint64_t seed, float *phase_out,
                         int out_on_host, double *e, double *u)
{
    return cswgs_solve_ex(p, spots_xyz, amplitudes, N, P, subset_fraction, iterations, seed, nullptr, phase_out,
                          out_on_host, e, u);
}

cswgs_status cswgs_subset(cswgs_plan p, int P, int64_t Mp, uint64_t seed, int j, int32_t *out_device)
{
    if (!p || !out_device) return set_error(CSWGS_EINVAL, "NULL plan or output");
    if (P < 2 || (P & 1) || P > p->desc.max_P) return set_error(CSWGS_EINVAL, "P=%d out of range", P);
    if (Mp < 0 || Mp > (int64_t)P * P) return set_error(CSWGS_EINVAL, "Mp=%lld not in [0, P^2]", (long long)Mp);
    if (j < 0) return set_error(CSWGS_EINVAL, "j=%d < 0", j);
    std::lock_guard<std::mutex> lk(p->mu);
    CSWGS_TRY(set_device(p));
    if (Mp == 0) return CSWGS_OK;
    CSWGS_CUDA_TRY(launch_subset_kernel(P, Mp, seed, j, out_device, p->stream));
    CSWGS_CUDA_TRY(cudaStreamSynchronize(p->stream));
    return CSWGS_OK;
}

cswgs_status cswgs_subset_ex(cswgs_plan p, int P, double subset_fraction, uint64_t seed, int j,
                             const cswgs_pupil *pupil, int32_t *out_device, int64_t *count)
{
    if (!p || !out_device) return set_error(CSWGS_EINVAL, "NULL plan or output");
    if (P < 2 || (P & 1) || P > p->desc.max_P) return set_error(CSWGS_EINVAL, "P=%d out of range", P);
    if (!(subset_fraction > 0.0 && subset_fraction <= 1.0))
        return set_error(CSWGS_EINVAL, "subset fraction %g not in (0, 1]", subset_fraction);
    if (j < 0) return set_error(CSWGS_EINVAL, "j=%d < 0", j);
    HoloSpec h;
    h.P = P;
    cswgs_pupil pu{};
    if (pupil) pu = *pupil;
    CSWGS_TRY(apply_pupil(p, pu, subset_fraction, &h));
    if (count) *count = h.Mp;
    HoloDev H;
    std::memset(&H, 0, sizeof H);
    H.P = P;
    H.Mp = h.Mp;
    H.seed = seed;
    fill_pupil(H, h);
    std::lock_guard<std::mutex> lk(p->mu);
    CSWGS_TRY(set_device(p));
    CSWGS_CUDA_TRY(launch_subset_ex_kernel(H, j, out_device, p->stream));
    CSWGS_CUDA_TRY(cudaStreamSynchronize(p->stream));
    return CSWGS_OK;
}

static cswgs_status specs_from_requests(cswgs_plan p, const cswgs_request *reqs, int count,
                                        std::vector<HoloSpec> *out)
{
    if (!reqs || count < 1) return set_error(CSWGS_EINVAL, "empty batch");
    if (count > p->desc.max_batch)
        return set_error(CSWGS_EINVAL, "batch of %d exceeds max_batch %d", count, p->desc.max_batch);
    out->clear();
    for (int i = 0; i < count; ++i) {
        const cswgs_request &r = reqs[i];
        HoloSpec h;
        cswgs_status st = validate_request(p->desc, r.spots_xyz, r.amplitudes, r.N, r.P, r.subset_fraction,
                                           r.iterations, r.full_iterations, &h);
        if (st == CSWGS_OK) st = apply_pupil(p, r.pupil, r.subset_fraction, &h);
        if (st == CSWGS_OK) st = apply_slm(r.slm, &h);
        if (st == CSWGS_OK && p->desc.precision == CSWGS_FP64 &&
            (h.aperture || h.windows || h.waist > 0.0 || h.has_slm))
            st = set_error(CSWGS_EINVAL, "the FP64 baseline solver takes the default pupil and no SLM frame");
        if (st != CSWGS_OK) return set_error(st, "request %d: %s", i, cswgs::last_error());
        h.seed = r.seed;
        out->push_back(std::move(h));
    }
    return CSWGS_OK;
}

cswgs_status cswgs_batch_create(cswgs_plan p, const cswgs_request *reqs, int count, cswgs_batch *out)
{
    if (!p || !out) return set_error(CSWGS_EINVAL, "NULL plan or output");
    *out = nullptr;
    if (p->desc.precision == CSWGS_FP64)
        return set_error(CSWGS_EINVAL, "graph batches run the FP32 solver; this plan is FP64");
    std::vector<HoloSpec> specs;
    CSWGS_TRY(specs_from_requests(p, reqs, count, &specs));
    for (int i = 0; i < count; ++i)
        if (reqs[i].out_on_host && reqs[i].phase_out)
            return set_error(CSWGS_EINVAL, "request %d: graph batches write device outputs only", i);
    std::lock_guard<std::mutex> lk(p->mu);
    CSWGS_TRY(set_device(p));
    auto *bb = new (std::nothrow) cswgs_batch_s();
    if (!bb) return set_error(CSWGS_ENOMEM, "host allocation");
    bb->plan = p;
    bb->count = count;
    cswgs_status st = batch_build(p, std::move(specs), true, &bb->b);
    if (st == CSWGS_OK) st = batch_upload_inputs(bb->b.get(), p->stream);
    std::vector<float *> outs(count);
    for (int i = 0; i < count; ++i) outs[i] = reqs[i].phase_out;
    if (st == CSWGS_OK) st = batch_set_outputs(bb->b.get(), outs, p->stream);
    if (st == CSWGS_OK) {
        cudaError_t e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) st = set_error(CSWGS_ECUDA, "%s", cudaGetErrorString(e));
    }
    if (st != CSWGS_OK) {
        delete bb;
        return st;
    }
    *out = bb;
    return CSWGS_OK;
}

cswgs_status cswgs_batch_run(cswgs_batch b)
{
    if (!b) return set_error(CSWGS_EINVAL, "NULL batch");
    cswgs_plan_s *p = b->plan;
    std::lock_guard<std::mutex> lk(p->mu);
    CSWGS_TRY(set_device(p));
    if (!b->host) return batch_enqueue(b->b.get(), p->stream);
    // host-buffer batch, all on its own stream: staged inputs in, the graph,
    // e and u out, the phase maps out
    Fp32Batch *fb = b->b.get();
    cudaStream_t s = b->stream;
    CSWGS_TRY(batch_upload_inputs(fb, s));
    CSWGS_CUDA_TRY(cudaEventRecord(b->ev_in, s));
    CSWGS_TRY(batch_enqueue(fb, s));
    eu_gather_kernel<<<1, 128, 0, s>>>(fb->holos_d.as<HoloDev>(), b->count, b->eu_host);
    CSWGS_CUDA_TRY(cudaGetLastError());
    // pinned maps go out on the copy engines: host batches are meant to
    // alternate, and the engines leave the SMs to the other batch's
    // iterations (the copy kernel would share them); pageable maps the GPU can
    // write go through the copy kernel
    std::vector<MapCopy> jobs;
    for (int i = 0; i < b->count; ++i) {
        float *dst = b->host_out[i];
        if (!dst) continue;
        const size_t n = (size_t)fb->specs[i].P * fb->specs[i].P;
        float *d = is_pinned(dst) ? nullptr : host_direct(p, dst);
        if (d)
            jobs.push_back(MapCopy{fb->own_phase[i], d, n});
        else
            CSWGS_CUDA_TRY(cudaMemcpyAsync(dst, fb->own_phase[i], sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    }
    return copy_maps(p, b->jobs, jobs, s);
}

static cswgs_status host_batch_fill(cswgs_batch b, const cswgs_request *reqs, std::vector<HoloSpec> &specs,
                                    bool first)
{
    Fp32Batch *fb = b->b.get();
    bool changed = false;
    for (int i = 0; i < b->count; ++i) {
        if (!first) {
            if (!same_shape(specs[i], fb->specs[i]) || (reqs[i].out_on_host == 0 && reqs[i].phase_out))
                return set_error(CSWGS_EINVAL, "request %d: a host batch's update keeps each hologram's shape "
                                               "(N, P, c, iterations, pupil) and takes host phase maps only", i);
            fb->specs[i].xyz = std::move(specs[i].xyz);
            fb->specs[i].amp = std::move(specs[i].amp);
            fb->specs[i].seed = specs[i].seed;
            if (fb->holos[i].seed != fb->specs[i].seed) {
                fb->holos[i].seed = fb->specs[i].seed;
                changed = true;
            }
            batch_restage(fb, i);
        }
        b->host_out[i] = reqs[i].phase_out;
    }
    if (changed)
        CSWGS_CUDA_TRY(cudaMemcpyAsync(fb->holos_d.p, fb->holos.data(), sizeof(HoloDev) * b->count,
                                       cudaMemcpyHostToDevice, b->stream));
    return CSWGS_OK;
}

cswgs_status cswgs_batch_create_host(cswgs_plan p, const cswgs_request *reqs, int count, cswgs_batch *out)
{
    if (!p || !out) return set_error(CSWGS_EINVAL, "NULL plan or output");
    *out = nullptr;
    if (p->desc.precision == CSWGS_FP64)
        return set_error(CSWGS_EINVAL, "graph batches run the FP32 solver; this plan is FP64");
    std::vector<HoloSpec> specs;
    CSWGS_TRY(specs_from_requests(p, reqs, count, &specs));
    for (int i = 0; i < count; ++i)
        if (!reqs[i].out_on_host && reqs[i].phase_out)
            return set_error(CSWGS_EINVAL, "request %d: a host batch writes host phase maps only", i);
    std::lock_guard<std::mutex> lk(p->mu);
    CSWGS_TRY(set_device(p));
    auto *bb = new (std::nothrow) cswgs_batch_s();
    if (!bb) return set_error(CSWGS_ENOMEM, "host allocation");
    bb->plan = p;
    bb->count = count;
    bb->host = true;
    bb->host_out.assign(count, nullptr);
    cswgs_status st = batch_build_host(p, specs, true, true, &bb->b);
    auto cuda = [&](cudaError_t e, const char *what) {
        if (st == CSWGS_OK && e != cudaSuccess)
            st = set_error(e == cudaErrorMemoryAllocation ? CSWGS_ENOMEM : CSWGS_ECUDA, "%s: %s", what,
                           cudaGetErrorString(e));
    };
    if (st == CSWGS_OK) cuda(cudaStreamCreateWithFlags(&bb->stream, cudaStreamNonBlocking), "stream");
    if (st == CSWGS_OK) cuda(cudaEventCreateWithFlags(&bb->ev_in, cudaEventDisableTiming), "event");
    if (st == CSWGS_OK)
        cuda(cudaMallocHost(reinterpret_cast<void **>(&bb->eu_host), sizeof(double) * 2 * count), "pinned e, u");
    if (st == CSWGS_OK) st = host_batch_fill(bb, reqs, specs, true);
    if (st == CSWGS_OK) st = batch_set_outputs(bb->b.get(), std::vector<float *>(count, nullptr), bb->stream);
    if (st == CSWGS_OK) cuda(cudaStreamSynchronize(bb->stream), "set-up");
    if (st != CSWGS_OK) {
        delete bb;
        return st;
    }
    *out = bb;
    return CSWGS_OK;
}

cswgs_status cswgs_batch_update(cswgs_batch b, const cswgs_request *reqs, int count)
{
    if (!b || !reqs) return set_error(CSWGS_EINVAL, "NULL batch or requests");
    if (!b->host) return set_error(CSWGS_EINVAL, "cswgs_batch_update takes a batch of cswgs_batch_create_host");
    if (count != b->count) return set_error(CSWGS_EINVAL, "update of %d holograms for a batch of %d", count, b->count);
    cswgs_plan_s *p = b->plan;
    std::vector<HoloSpec> specs;
    CSWGS_TRY(specs_from_requests(p, reqs, count, &specs));
    std::lock_guard<std::mutex> lk(p->mu);
    CSWGS_TRY(set_device(p));
    // the staging block is rewritten: the last run must have copied it in
    CSWGS_CUDA_TRY(cudaEventSynchronize(b->ev_in));
    return host_batch_fill(b, reqs, specs, false);
}

cswgs_status cswgs_batch_results(cswgs_batch b, cswgs_result *results)
{
    if (!b || !results) return set_error(CSWGS_EINVAL, "NULL batch or results");
    cswgs_plan_s *p = b->plan;
    std::lock_guard<std::mutex> lk(p->mu);
    CSWGS_TRY(set_device(p));
    Fp32Batch *fb = b->b.get();
    if (b->host) {
        CSWGS_TRY(batch_status(fb, b->stream));   // synchronises the batch's stream
        float ms = 0.f;
        if (fb->timing) cudaEventElapsedTime(&ms, fb->events.front(), fb->events.back());
        for (int i = 0; i < b->count; ++i) {
            results[i].status = CSWGS_OK;
            results[i].e = b->eu_host[2 * i];
            results[i].u = b->eu_host[2 * i + 1];
            results[i].latency_ms = ms;
            results[i].queue_ms = 0.0;
        }
        return CSWGS_OK;
    }
    std::vector<double> eu(2 * b->count);
    for (int i = 0; i < b->count; ++i)
        CSWGS_CUDA_TRY(cudaMemcpyAsync(&eu[2 * i], fb->holos[i].metrics, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                       p->stream));
    CSWGS_TRY(batch_status(fb, p->stream));
    float ms = 0.f;
    if (fb->timing) cudaEventElapsedTime(&ms, fb->events.front(), fb->events.back());
    for (int i = 0; i < b->count; ++i) {
        results[i].status = CSWGS_OK;
        results[i].e = eu[2 * i];
        results[i].u = eu[2 * i + 1];
        results[i].latency_ms = ms;
        results[i].queue_ms = 0.0;
    }
    return CSWGS_OK;
}

cswgs_status cswgs_batch_kernel_times(cswgs_batch b, float *ms, int cap, int *count)
{
    if (!b || !count) return set_error(CSWGS_EINVAL, "NULL batch or count");
    Fp32Batch *fb = b->b.get();
    const int n = (int)fb->events.size() - 1;
    *count = n;
    if (!ms) return CSWGS_OK;
    cswgs_plan_s *p = b->plan;
    std::lock_guard<std::mutex> lk(p->mu);
    CSWGS_TRY(set_device(p));
    CSWGS_CUDA_TRY(cudaEventSynchronize(fb->events.back()));
    for (int i = 0; i < n && i < cap; ++i) CSWGS_CUDA_TRY(cudaEventElapsedTime(&ms[i], fb->events[i], fb->events[i + 1]));
    return CSWGS_OK;
}

cswgs_status cswgs_batch_pairs(cswgs_batch b, double *pairs_total, double *pairs_iter_launches)
{
    if (!b) return set_error(CSWGS_EINVAL, "NULL batch");
    if (pairs_total) *pairs_total = b->b->pairs_total;
    if (pairs_iter_launches) *pairs_iter_launches = b->b->pairs_iter;
    return CSWGS_OK;
}

cswgs_status cswgs_batch_tile_shape(cswgs_batch b, int *threads, int *pixels_per_thread, int *full_threads,
                                    int *blocks, int *full_blocks)
{
    if (!b) return set_error(CSWGS_EINVAL, "NULL batch");
    if (threads) *threads = b->b->shape.threads;
    if (pixels_per_thread) *pixels_per_thread = b->b->shape.ppt;
    if (full_threads) *full_threads = b->b->shape.full_threads;
    if (blocks) *blocks = b->b->grid[kLaunchSubset];
    if (full_blocks) *full_blocks = b->b->grid[kLaunchFull];
    return CSWGS_OK;
}

cswgs_status cswgs_batch_destroy(cswgs_batch b)
{
    if (!b) return CSWGS_OK;
    cswgs_plan_s *p = b->plan;
    {
        std::lock_guard<std::mutex> lk(p->mu);
        cudaSetDevice(p->device);
        cudaStreamSynchronize(b->host ? b->stream : p->stream);
        delete b;
    }
    return CSWGS_OK;
}

cswgs_status cswgs_solve_batch(cswgs_plan p, const cswgs_request *reqs, int count, cswgs_result *results)
{
    if (!p || !results) return set_error(CSWGS_EINVAL, "NULL plan or results");
    std::vector<HoloSpec> specs;
    CSWGS_TRY(specs_from_requests(p, reqs, count, &specs));
    std::lock_guard<std::mutex> lk(p->mu);
    CSWGS_TRY(set_device(p));
    if (p->desc.precision == CSWGS_FP64) {
        for (int i = 0; i < count; ++i) {
            cudaEvent_t a, c;
            cudaEventCreate(&a);
            cudaEventCreate(&c);
            cudaEventRecord(a, p->stream);
            cswgs_status st = solve_fp64(p, specs[i], reqs[i].phase_out, reqs[i].out_on_host, &results[i].e,
                                         &results[i].u, nullptr, nullptr, nullptr);
            cudaEventRecord(c, p->stream);
            cudaEventSynchronize(c);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, c);
            cudaEventDestroy(a);
            cudaEventDestroy(c);
            results[i].status = st;
            results[i].latency_ms = ms;
            results[i].queue_ms = 0.0;
            if (st != CSWGS_OK) return st;
        }
        return CSWGS_OK;
    }
    // FP32: one cached batch per shape, inputs and outputs refreshed per call
    bool host_out = false;
    for (int i = 0; i < count; ++i) host_out |= reqs[i].out_on_host && reqs[i].phase_out;
    std::string key = "B" + shape_key(specs, host_out);
    Fp32Batch *b = nullptr;
    auto it = p->solve_cache.find(key);
    if (it == p->solve_cache.end()) {
        std::unique_ptr<Fp32Batch> nb;
        CSWGS_TRY(batch_build_host(p, specs, true, host_out, &nb));
        b = nb.get();
        p->solve_cache[key] = std::move(nb);
    } else {
        b = it->second.get();
        bool changed = false;
        for (int i = 0; i < count; ++i) {
            b->specs[i].xyz = specs[i].xyz;
            b->specs[i].amp = specs[i].amp;
            b->specs[i].seed = specs[i].seed;
            b->specs[i].waist = specs[i].waist;
            b->specs[i].norm = specs[i].norm;
            b->specs[i].has_slm = specs[i].has_slm;
            b->specs[i].slm = specs[i].slm;
            HoloDev H = b->holos[i];
            H.seed = specs[i].seed;
            fill_pupil(H, b->specs[i]);
            if (std::memcmp(&H, &b->holos[i], sizeof H) != 0) {
                b->holos[i] = H;
                changed = true;
            }
            batch_restage(b, i);
        }
        if (changed)
            CSWGS_CUDA_TRY(cudaMemcpyAsync(b->holos_d.p, b->holos.data(), sizeof(HoloDev) * count,
                                           cudaMemcpyHostToDevice, p->stream));
    }
    cudaStream_t s = p->stream;
    CSWGS_TRY(batch_upload_inputs(b, s));
    std::vector<float *> outs(count);
    for (int i = 0; i < count; ++i) outs[i] = (reqs[i].out_on_host ? nullptr : reqs[i].phase_out);
    CSWGS_TRY(batch_set_outputs(b, outs, s));
    CSWGS_TRY(batch_enqueue(b, s));
    std::vector<double> eu(2 * count);
    std::vector<MapCopy> jobs;
    for (int i = 0; i < count; ++i) {
        CSWGS_CUDA_TRY(cudaMemcpyAsync(&eu[2 * i], b->holos[i].metrics, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (reqs[i].out_on_host && reqs[i].phase_out) {
            const size_t n = (size_t)specs[i].P * specs[i].P;
            if (float *d = host_direct(p, reqs[i].phase_out))
                jobs.push_back(MapCopy{b->own_phase[i], d, n});
            else
                CSWGS_CUDA_TRY(cudaMemcpyAsync(reqs[i].phase_out, b->own_phase[i], sizeof(float) * n,
                                               cudaMemcpyDeviceToHost, s));
        }
    }
    CSWGS_TRY(copy_maps(p, b->copy_jobs, jobs, s));
    CSWGS_TRY(batch_status(b, s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->events.front(), b->events.back());
    for (int i = 0; i < count; ++i) {
        results[i].status = CSWGS_OK;
        results[i].e = eu[2 * i];
        results[i].u = eu[2 * i + 1];
        results[i].latency_ms = ms;
        results[i].queue_ms = 0.0;
    }
    return CSWGS_OK;
}

cswgs_status cswgs_plan_test_waits(cswgs_plan p, int withhold_first_item, unsigned wait_polls)
{
    if (!p) return set_error(CSWGS_EINVAL, "NULL plan");
    std::lock_guard<std::mutex> lk(p->mu);
    p->test_withhold = withhold_first_item ? 1u : 0u;
    p->test_polls = wait_polls;
    return CSWGS_OK;
}

cswgs_status cswgs_autotune(cswgs_plan p, int P, int N, double subset_fraction, double *best_ms)
{
    if (!p) return set_error(CSWGS_EINVAL, "NULL plan");
    if (P < 2 || (P & 1) || P > p->desc.max_P || N < 1 || N > p->desc.max_N ||
        !(subset_fraction > 0.0 && subset_fraction <= 1.0))
        return set_error(CSWGS_EINVAL, "autotune: bad size (P %d, N %d, c %g)", P, N, subset_fraction);
    std::lock_guard<std::mutex> lk(p->mu);
    CSWGS_TRY(set_device(p));
    return tune_single(p, P, N, subset_fraction, best_ms);
}

cswgs_status cswgs_sincos_peak(cswgs_plan p, double *sincos_per_s, double *sm_mhz)
{
    if (!p) return set_error(CSWGS_EINVAL, "NULL plan");
    std::lock_guard<std::mutex> lk(p->mu);
    CSWGS_TRY(set_device(p));
    const int threads = 256, iters = 4096;
    const int blocks = p->sm_count * 4;   // one resident wave
    CSWGS_TRY(p->scratch.ensure(4096));
    float *sink = p->scratch.as<float>();
    long long *cyc = reinterpret_cast<long long *>(p->scratch.as<char>() + 256);
    cudaEvent_t a, c;
    CSWGS_CUDA_TRY(cudaEventCreate(&a));
    CSWGS_CUDA_TRY(cudaEventCreate(&c));
    CSWGS_CUDA_TRY(launch_sincos_probe(sink, cyc, iters, blocks, threads, p->stream));  // warm-up
    CSWGS_CUDA_TRY(cudaMemsetAsync(cyc, 0, sizeof(long long), p->stream));
    CSWGS_CUDA_TRY(cudaEventRecord(a, p->stream));
    CSWGS_CUDA_TRY(launch_sincos_probe(sink, cyc, iters, blocks, threads, p->stream));
    CSWGS_CUDA_TRY(cudaEventRecord(c, p->stream));
    CSWGS_CUDA_TRY(cudaEventSynchronize(c));
    float ms = 0.f;
    CSWGS_CUDA_TRY(cudaEventElapsedTime(&ms, a, c));
    long long cycles = 0;
    CSWGS_CUDA_TRY(cudaMemcpy(&cycles, cyc, sizeof cycles, cudaMemcpyDeviceToHost));
    cudaEventDestroy(a);
    cudaEventDestroy(c);
    const double ops = (double)blocks * threads * iters * 8.0 * 2.0;
    if (sincos_per_s) *sincos_per_s = ops / (ms * 1e-3);
    if (sm_mhz) *sm_mhz = (double)cycles / (ms * 1e-3) / 1e6;
    return CSWGS_OK;
}

}  // extern "C"
