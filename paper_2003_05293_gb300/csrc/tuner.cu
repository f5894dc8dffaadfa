// Autotuner of the FP32 iteration kernel's tile shape (threads per block,
// pixels per thread).  Key: (largest P rounded up to 128, work-weighted spot
// count rounded up to a power of two, batch size rounded up to a power of
// two).  Each candidate runs a synthetic batch of that key's size (one
// compressed iteration, one full iteration, the final pass) and the shape with
// the least schedule-weighted time wins.  Results live in the plan and,
// when the plan names a cache file, in a small JSON file.
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
};

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
    return k;
}

std::string tune_key(const std::vector<HoloSpec> &specs)
{
    TuneKey k = key_of(specs);
    char buf[64];
    snprintf(buf, sizeof buf, "P%d_N%d_B%d", k.P, k.N, k.B);
    return buf;
}

static const TileShape kCandidates[] = {{128, 4}, {128, 8}, {256, 2}, {256, 4}, {256, 8},
                                        {512, 2}, {512, 4}};

static std::vector<HoloSpec> synthetic(const TuneKey &k, double c)
{
    std::vector<HoloSpec> v;
    for (int b = 0; b < k.B; ++b) {
        HoloSpec s;
        s.P = std::min(k.P, 4096);
        s.N = k.N;
        s.Mp = std::max(1, (int)std::floor(c * (double)s.P * s.P));
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

static cswgs_status time_shape(cswgs_plan_s *p, const std::vector<HoloSpec> &specs, TileShape sh,
                               double weight_sub, double weight_full, double *ms_out)
{
    std::unique_ptr<Fp32Batch> b;
    CSWGS_TRY(batch_build_with(p, specs, sh, &b));
    CSWGS_TRY(batch_upload_inputs(b.get(), p->stream));
    double best = 1e30;
    for (int rep = 0; rep < 3; ++rep) {
        CSWGS_TRY(batch_enqueue_direct(b.get(), p->stream));
        CSWGS_CUDA_TRY(cudaStreamSynchronize(p->stream));
        float t_sub = 0.f, t_full = 0.f, t_fin = 0.f;
        CSWGS_CUDA_TRY(cudaEventElapsedTime(&t_sub, b->events[1], b->events[2]));
        CSWGS_CUDA_TRY(cudaEventElapsedTime(&t_full, b->events[2], b->events[3]));
        CSWGS_CUDA_TRY(cudaEventElapsedTime(&t_fin, b->events[3], b->events[4]));
        double t = weight_sub * t_sub + weight_full * t_full + t_fin;
        if (rep > 0) best = std::min(best, t);   // first run warms up
    }
    *ms_out = best;
    return CSWGS_OK;
}

static cswgs_status tune_for(cswgs_plan_s *p, const TuneKey &k, double c, double wsub, double wfull,
                             TileShape *best_shape, double *best_ms)
{
    std::vector<HoloSpec> specs = synthetic(k, c);
    double best = 1e30;
    TileShape bs{256, 4};
    for (const TileShape &sh : kCandidates) {
        if (iter_fp32_max_grid(sh, k.N, p->sm_count) <= 0) continue;
        double ms;
        cswgs_status st = time_shape(p, specs, sh, wsub, wfull, &ms);
        if (st != CSWGS_OK) return st;
        if (ms < best) {
            best = ms;
            bs = sh;
        }
    }
    *best_shape = bs;
    if (best_ms) *best_ms = best;
    return CSWGS_OK;
}

TileShape tuned_shape(cswgs_plan_s *p, const std::vector<HoloSpec> &specs)
{
    std::string key = tune_key(specs);
    auto it = p->tune.find(key);
    if (it != p->tune.end()) return it->second;
    // tune now, with the schedule's own mix of compressed and full iterations
    double wsub = 0.0, wfull = 0.0, c = 0.125;
    for (auto &s : specs) {
        int F = std::min(s.n_full, s.iterations);
        wsub += s.iterations - F;
        wfull += F;
        c = (double)s.Mp / ((double)s.P * s.P);
    }
    if (!specs.empty()) {
        wsub /= specs.size();
        wfull /= specs.size();
    }
    TileShape sh{256, 4};
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
    p->tune[tune_key(v)] = sh;
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
    // entries look like "P1152_N128_B64": [256, 4]
    size_t pos = 0;
    while ((pos = s.find('"', pos)) != std::string::npos) {
        size_t end = s.find('"', pos + 1);
        if (end == std::string::npos) break;
        std::string key = s.substr(pos + 1, end - pos - 1);
        pos = end + 1;
        if (key.empty() || key[0] != 'P') continue;
        int t = 0, k = 0;
        if (sscanf(s.c_str() + pos, " : [ %d , %d ]", &t, &k) == 2 && tile_shape_supported(TileShape{t, k}))
            p->tune[key] = TileShape{t, k};
    }
}

void tune_save(cswgs_plan_s *p)
{
    if (p->tune_path.empty()) return;
    std::string tmp = p->tune_path + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n  \"format\": \"cswgs-tune-1\",\n  \"entries\": {");
    bool first = true;
    for (auto &kv : p->tune) {
        fprintf(f, "%s\n    \"%s\": [%d, %d]", first ? "" : ",", kv.first.c_str(), kv.second.threads,
                kv.second.ppt);
        first = false;
    }
    fprintf(f, "\n  }\n}\n");
    fclose(f);
    rename(tmp.c_str(), p->tune_path.c_str());
}

}  // namespace cswgs
