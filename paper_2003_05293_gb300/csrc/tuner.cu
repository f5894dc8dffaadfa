// Autotuner of the FP32 iteration kernels' tile shapes (compressed
// iterations: threads per block and pixels per thread; full passes: threads
// per block).  Key: (largest P rounded up to 128, work-weighted spot
// count rounded up to a power of two, batch size rounded up to a power of
// two, subset fraction c as the nearest power of two: a compressed launch on
// the CUDA cores costs c times a full one, on the tensor cores about as much
// as a full one, so the winner changes with c).  Each candidate runs a
// synthetic batch of that key's size (one compressed iteration, one full
// iteration, the final pass); the fastest compressed-iteration shape and the
// fastest full-pass shape win.  Results live in the plan and, when the plan
// names a cache file, in a small JSON file.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>

#include "runtime.h"

namespace cswgs {

cswgs_status batch_build_with(cswgs_plan_s *p, std::vector<HoloSpec> specs, TileShape shape,
                              std::unique_ptr<Fp32Batch> *out);

static int pow2_ceil(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

struct TuneKey {
    int P, N, B;
    int cexp;   // c = 2^-cexp (0 .. 16)
};

// The subset fraction of a batch, weighted by each hologram's compressed
// work (pixels x spots x compressed iterations); 1 when none has any.
static double batch_c(const std::vector<HoloSpec> &specs)
{
    double wsum = 0.0, cw = 0.0;
    for (auto &s : specs) {
        const int F = std::min(s.n_full, s.iterations);
        const double M = (double)s.P * s.P, D = s.D > 0 ? (double)s.D : M;
        const double w = M * s.N * (double)(s.iterations - F), c = (double)s.Mp / D;
        wsum += w;
        cw += w * c;
    }
    return wsum > 0.0 ? cw / wsum : 1.0;
}

static TuneKey key_of(const std::vector<HoloSpec> &specs)
{
    int P = 0;
    double wsum = 0.0, nw = 0.0;
    for (auto &s : specs) {
        P = std::max(P, s.P);
        double w = (double)s.P * s.P * s.N;
        wsum += w;
        nw += w * s.N;
    }
    int N = wsum > 0 ? (int)std::lround(nw / wsum) : 1;
    TuneKey k;
    k.P = ((P + 127) / 128) * 128;
    k.N = std::max(16, pow2_ceil(N));
    k.B = pow2_ceil((int)specs.size());
    const double c = batch_c(specs);
    k.cexp = std::min(16, std::max(0, (int)std::lround(-std::log2(std::max(c, 1e-9)))));
    return k;
}

std::string tune_key(const std::vector<HoloSpec> &specs, bool fp16)
{
    TuneKey k = key_of(specs);
    char buf[64];
    snprintf(buf, sizeof buf, "P%d_N%d_B%d_c%d%s", k.P, k.N, k.B, k.cexp, fp16 ? "_H" : "");
    return buf;
}

// Candidates: compressed-iteration kernel (threads, pixels per thread, the
// masked tensor-core pass, or the subset-only gather kernel) and full-pass
// kernel (threads, or a tensor-core kernel); the two kinds run as separate launches, so each is tuned on its
// own launches.
static const int kSubCandidates[][2] = {{128, 2}, {128, 4}, {128, 8}, {256, 2},  {256, 4},
                                        {256, 8}, {512, 1}, {512, 2}, {512, 4}, {kSubsetTc, 1},
                                        {kSubsetGather, 1}};
static const int kFullCandidates[] = {128, 256, 512, kFullTcWs};

static std::vector<HoloSpec> synthetic(const TuneKey &k, double c)
{
    std::vector<HoloSpec> v;
    for (int b = 0; b < k.B; ++b) {
        HoloSpec s;
        s.P = std::min(k.P, 4096);
        s.N = k.N;
        s.Mp = std::max(1, (int)std::floor(c * (double)s.P * s.P));
        s.D = s.P * s.P;   // the square uniform pupil
        s.fa = s.fb = (uint32_t)s.P;
        s.norm = (double)s.D;
        s.iterations = 2;
        s.n_full = 1;
        s.first_j = 1;
        s.final_pass = 1;
        s.seed = 0x5EEDull + (uint64_t)b;
        s.xyz.resize(3 * (size_t)s.N);
        uint64_t x = 12345 + (uint64_t)b;
        for (auto &q : s.xyz) {
            x = x * 6364136223846793005ull + 1442695040888963407ull;
            q = ((double)(x >> 11) * 0x1.0p-53 - 0.5) * (s.P / 2.0);
        }
        v.push_back(std::move(s));
    }
    return v;
}

// Best-of-two device times of the synthetic schedule's three steps: a
// compressed iteration, a full iteration and the final pass.
static cswgs_status time_steps(cswgs_plan_s *p, const std::vector<HoloSpec> &specs, TileShape sh, double t[3])
{
    std::unique_ptr<Fp32Batch> b;
    CSWGS_TRY(batch_build_with(p, specs, sh, &b));
    CSWGS_TRY(batch_upload_inputs(b.get(), p->stream));
    for (int i = 0; i < 3; ++i) t[i] = 1e30;
    for (int rep = 0; rep < 3; ++rep) {
        CSWGS_TRY(batch_enqueue_direct(b.get(), p->stream));
        CSWGS_CUDA_TRY(cudaStreamSynchronize(p->stream));
        if (rep == 0) continue;   // warm-up
        for (int i = 0; i < 3; ++i) {
            float ms = 0.f;
            CSWGS_CUDA_TRY(cudaEventElapsedTime(&ms, b->events[1 + i], b->events[2 + i]));
            t[i] = std::min(t[i], (double)ms);
        }
    }
    return CSWGS_OK;
}

static cswgs_status tune_for(cswgs_plan_s *p, const TuneKey &k, double c, double wsub, double wfull,
                             TileShape *best_shape, double *best_ms)
{
    std::vector<HoloSpec> specs = synthetic(k, c);
    const int fp16 = p->desc.precision == CSWGS_FP32_FP16SINCOS ? 1 : 0;
    TileShape best{256, 4, 256, fp16};
    double best_sub = 1e30, best_full = 1e30, t[3];
    for (const auto &cand : kSubCandidates) {
        TileShape sh{cand[0], cand[1], best.full_threads, fp16};
        if (!shape_supported(sh)) continue;
        if (shape_max_grid(sh, kLaunchSubset, k.N, p->sm_count) <= 0) continue;
        CSWGS_TRY(time_steps(p, specs, sh, t));
        if (t[0] < best_sub) {
            best_sub = t[0];
            best.threads = cand[0];
            best.ppt = cand[1];
        }
    }
    for (int ft : kFullCandidates) {
        TileShape sh{best.threads, best.ppt, ft, fp16};
        if (shape_max_grid(sh, kLaunchFull, k.N, p->sm_count) <= 0) continue;
        CSWGS_TRY(time_steps(p, specs, sh, t));
        const double tf = wfull * t[1] + t[2];
        if (tf < best_full) {
            best_full = tf;
            best.full_threads = ft;
        }
    }
    *best_shape = best;
    if (best_ms) *best_ms = wsub * best_sub + best_full;
    return CSWGS_OK;
}

TileShape tuned_shape(cswgs_plan_s *p, const std::vector<HoloSpec> &specs)
{
    const bool fp16 = p->desc.precision == CSWGS_FP32_FP16SINCOS;
    std::string key = tune_key(specs, fp16);
    auto it = p->tune.find(key);
    if (it != p->tune.end()) return it->second;
    // tune now, with the schedule's own mix of compressed and full iterations
    double wsub = 0.0, wfull = 0.0;
    for (auto &s : specs) {
        int F = std::min(s.n_full, s.iterations);
        wsub += s.iterations - F;
        wfull += F;
    }
    const double c = std::ldexp(1.0, -key_of(specs).cexp);   // the key's c: one tuning per bucket
    if (!specs.empty()) {
        wsub /= specs.size();
        wfull /= specs.size();
    }
    TileShape sh{256, 4, 256, fp16 ? 1 : 0};
    double ms = 0.0;
    if (tune_for(p, key_of(specs), c, wsub, wfull, &sh, &ms) == CSWGS_OK) {
        p->tune[key] = sh;
        tune_save(p);
    }
    return sh;
}

cswgs_status tune_single(cswgs_plan_s *p, int P, int N, double c, double *best_ms)
{
    HoloSpec s;
    s.P = P;
    s.N = N;
    s.Mp = std::max(1, (int)std::floor(c * (double)P * P));
    s.iterations = 30;
    s.n_full = 2;
    std::vector<HoloSpec> v{s};
    TuneKey k = key_of(v);
    TileShape sh;
    CSWGS_TRY(tune_for(p, k, c, 28.0, 2.0, &sh, best_ms));
    p->tune[tune_key(v, p->desc.precision == CSWGS_FP32_FP16SINCOS)] = sh;
    tune_save(p);
    return CSWGS_OK;
}

void tune_load(cswgs_plan_s *p)
{
    if (p->tune_path.empty()) return;
    std::ifstream f(p->tune_path);
    if (!f) return;
    std::stringstream ss;
    ss << f.rdbuf();
    std::string s = ss.str();
    // entries look like "P1152_N128_B64_c3": [256, 4, 128] or, with a strip
    // length for the tensor-core launches, [1, 1, 2, 6]
    size_t pos = 0;
    while ((pos = s.find('"', pos)) != std::string::npos) {
        size_t end = s.find('"', pos + 1);
        if (end == std::string::npos) break;
        std::string key = s.substr(pos + 1, end - pos - 1);
        pos = end + 1;
        if (key.empty() || key[0] != 'P') continue;
        const int fp16 = key.size() > 2 && key.compare(key.size() - 2, 2, "_H") == 0 ? 1 : 0;
        int t = 0, k = 0, f = 0, st = 0;
        const int got = sscanf(s.c_str() + pos, " : [ %d , %d , %d , %d ]", &t, &k, &f, &st);
        if (got < 3) continue;
        if (got < 4 || st < 0 || st > 4096) st = 0;
        if (shape_supported(TileShape{t, k, f, fp16, st})) p->tune[key] = TileShape{t, k, f, fp16, st};
    }
}

void tune_save(cswgs_plan_s *p)
{
    if (p->tune_path.empty()) return;
    std::string tmp = p->tune_path + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n  \"format\": \"cswgs-tune-3\",\n  \"entries\": {");
    bool first = true;
    for (auto &kv : p->tune) {
        fprintf(f, "%s\n    \"%s\": [%d, %d, %d, %d]", first ? "" : ",", kv.first.c_str(), kv.second.threads,
                kv.second.ppt, kv.second.full_threads, kv.second.strip);
        first = false;
    }
    fprintf(f, "\n  }\n}\n");
    fclose(f);
    rename(tmp.c_str(), p->tune_path.c_str());
}

}  // namespace cswgs
