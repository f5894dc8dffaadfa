// Continuous-batching server: requests of any (P, N, c, I) share one
// persistent FP32 launch per iteration.  Each launch advances every admitted
// request by one step of its own schedule (compressed iteration, full
// iteration or final pass); requests are admitted between launches as serving
// slots and arena memory free up, and leave when their final pass is done.
// Two launches are kept in flight so host bookkeeping overlaps the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "serve.h"

namespace cswgs {

static double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// ------------------------------------------------------------------ arena --

cswgs_status Arena::init(size_t bytes)
{
    bytes = al256(bytes);
    CSWGS_TRY(mem_.ensure(bytes));
    cap_ = bytes;
    used_ = 0;
    free_.clear();
    taken_.clear();
    free_[0] = bytes;
    return CSWGS_OK;
}

bool Arena::alloc(size_t bytes, size_t *off)
{
    bytes = al256(bytes);
    if (used_ + bytes > cap_) return false;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
        if (it->second >= bytes) {
            size_t o = it->first, sz = it->second;
            free_.erase(it);
            if (sz > bytes) free_[o + bytes] = sz - bytes;
            taken_[o] = bytes;
            used_ += bytes;
            *off = o;
            return true;
        }
    }
    return false;
}

void Arena::free(size_t off)
{
    auto t = taken_.find(off);
    if (t == taken_.end()) return;
    size_t sz = t->second;
    taken_.erase(t);
    used_ -= sz;
    auto it = free_.emplace(off, sz).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        free_.erase(nx);
    }
    if (it != free_.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            free_.erase(it);
        }
    }
}

// ----------------------------------------------------------------- server --

Server::Server(cswgs_plan_s *p) : p_(p) {}

Server::~Server()
{
    {
        std::lock_guard<std::mutex> lk(mu_);
        stop_ = true;
    }
    cv_.notify_all();
    if (th_.joinable()) th_.join();
    cudaSetDevice(p_->device);
    if (stream_) cudaStreamSynchronize(stream_);
    for (int i = 0; i < 2; ++i) {
        if (slots_h_[i]) cudaFreeHost(slots_h_[i]);
        if (holos_h_[i]) cudaFreeHost(holos_h_[i]);
        if (launch_ev_[i]) cudaEventDestroy(launch_ev_[i]);
        if (start_ev_[i]) cudaEventDestroy(start_ev_[i]);
    }
    if (met_h_) cudaFreeHost(met_h_);
    if (status_h_) cudaFreeHost(status_h_);
    if (in_h_) cudaFreeHost(in_h_);
    if (stream_) cudaStreamDestroy(stream_);
}

cswgs_status Server::start()
{
    if (started_) return CSWGS_OK;
    CSWGS_CUDA_TRY(cudaSetDevice(p_->device));
    size_t cap = p_->desc.mem_cap_bytes;
    if (cap == 0) {
        size_t fr = 0, tot = 0;
        CSWGS_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        cap = std::min(fr / 2, (size_t)16 << 30);
    }
    CSWGS_TRY(arena_.init(cap));
    const int B = p_->desc.max_batch;
    CSWGS_TRY(holos_d_.ensure(sizeof(HoloDev) * B * 2));   // slots, then the prep list
    CSWGS_TRY(slots_d_.ensure(sizeof(LaunchSlot) * B * 2));
    CSWGS_TRY(queue_d_.ensure(256));
    CSWGS_CUDA_TRY(cudaMemset(queue_d_.p, 0, 256));
    master_.assign(B, HoloDev{});
    CSWGS_CUDA_TRY(cudaMallocHost(&met_h_, sizeof(double) * 4 * B));
    CSWGS_CUDA_TRY(cudaMallocHost(&status_h_, 2 * sizeof(unsigned)));
    status_h_[0] = status_h_[1] = 0u;
    CSWGS_CUDA_TRY(cudaMallocHost(&in_h_, sizeof(double) * 4 * (size_t)p_->desc.max_N * B));
    for (int i = 0; i < 2; ++i) {
        CSWGS_CUDA_TRY(cudaMallocHost(&holos_h_[i], sizeof(HoloDev) * B));
        std::memset(holos_h_[i], 0, sizeof(HoloDev) * B);
        CSWGS_CUDA_TRY(cudaMallocHost(&slots_h_[i], sizeof(LaunchSlot) * B + sizeof(HoloDev) * B));
        CSWGS_CUDA_TRY(cudaEventCreate(&launch_ev_[i]));
        CSWGS_CUDA_TRY(cudaEventCreate(&start_ev_[i]));
    }
    CSWGS_CUDA_TRY(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
    active_.resize(B);
    st_.bytes_cap = arena_.capacity();
    started_ = true;
    th_ = std::thread([this] { loop(); });
    return CSWGS_OK;
}

size_t Server::footprint(const HoloSpec &s) const
{
    const size_t M = (size_t)s.P * s.P;
    const size_t tiles = (size_t)max_pass_tiles(s, shape_);
    size_t b = 0;
    b += al256(sizeof(double) * 3 * s.N) + (s.has_amp ? al256(sizeof(double) * s.N) : 0);
    b += al256(sizeof(int4) * s.N) + al256(sizeof(SpotState) * s.N);
    b += al256(sizeof(float2) * tiles * s.N) + al256(sizeof(double2) * tiles * s.N);
    b += 256 + al256(sizeof(double) * (2 + s.N));
    b += al256(sizeof(float) * M);   // phase map (the caller's device buffer is used when given)
    if (uses_tc(shape_)) {
        size_t rw, c, cs;
        full_tc_table_bytes(s.P, s.N, &rw, &c, &cs);
        b += al256(rw) + al256(c) + al256(cs);
        if (shape_.fp16 && shape_.threads == kSubsetTc) b += al256(cs / 2);
    }
    if (uses_masks(shape_)) b += al256(sizeof(uint32_t) * (size_t)s.P * mask_words_of(s.P));
    return b;
}

// Lays the request's buffers out in its arena block and fills its HoloDev.
void Server::place(Req &r)
{
    const HoloSpec &s = r.spec;
    const size_t tiles = (size_t)max_pass_tiles(s, shape_);
    char *b = arena_.base() + r.off;
    size_t o = 0;
    HoloDev &H = r.dev;
    std::memset(&H, 0, sizeof H);
    H.P = s.P;
    H.N = s.N;
    H.Mp = s.Mp;
    H.seed = s.seed;
    fill_pupil(H, s);
    // inputs go through this slot's pinned staging area (free again once the
    // slot is, i.e. after the request's last launch has completed)
    double *stg = in_h_ + (size_t)r.slot * 4 * p_->desc.max_N;
    std::memcpy(stg, s.xyz.data(), sizeof(double) * 3 * s.N);
    double *xyz = reinterpret_cast<double *>(b + o);
    o += al256(sizeof(double) * 3 * s.N);
    H.xyz = xyz;
    note(cudaMemcpyAsync(xyz, stg, sizeof(double) * 3 * s.N, cudaMemcpyHostToDevice, stream_));
    if (s.has_amp) {
        std::memcpy(stg + 3 * s.N, s.amp.data(), sizeof(double) * s.N);
        double *a = reinterpret_cast<double *>(b + o);
        o += al256(sizeof(double) * s.N);
        H.amp = a;
        note(cudaMemcpyAsync(a, stg + 3 * s.N, sizeof(double) * s.N, cudaMemcpyHostToDevice, stream_));
    }
    H.coef = reinterpret_cast<int4 *>(b + o);
    o += al256(sizeof(int4) * s.N);
    H.state = reinterpret_cast<SpotState *>(b + o);
    o += al256(sizeof(SpotState) * s.N);
    H.part = reinterpret_cast<float2 *>(b + o);
    o += al256(sizeof(float2) * tiles * s.N);
    H.part64 = reinterpret_cast<double2 *>(b + o);
    o += al256(sizeof(double2) * tiles * s.N);
    H.counter = reinterpret_cast<unsigned *>(b + o);
    o += 256;
    H.metrics = reinterpret_cast<double *>(b + o);
    o += al256(sizeof(double) * (2 + s.N));
    float *own = reinterpret_cast<float *>(b + o);
    o += al256(sizeof(float) * (size_t)s.P * s.P);
    H.phase_out = r.phase_dev ? r.phase_dev : own;
    if (uses_tc(shape_)) {
        size_t rw, c, cs;
        full_tc_table_bytes(s.P, s.N, &rw, &c, &cs);
        H.rwtab = reinterpret_cast<unsigned char *>(b + o);
        o += al256(rw);
        H.ctab = reinterpret_cast<unsigned char *>(b + o);
        o += al256(c);
        H.cstab = reinterpret_cast<unsigned char *>(b + o);
        o += al256(cs);
        if (shape_.fp16 && shape_.threads == kSubsetTc) {
            H.cstab16 = reinterpret_cast<unsigned char *>(b + o);
            o += al256(cs / 2);
        }
    }
    if (uses_masks(shape_)) {
        // the subset mask starts clear (each compressed launch's tails clear it again)
        H.mask = reinterpret_cast<uint32_t *>(b + o);
        H.mask_words = mask_words_of(s.P);
        H.mask_stride = 0;   // one mask: serving draws it in the launch's own table kernel
        const size_t bytes = sizeof(uint32_t) * (size_t)s.P * H.mask_words;
        o += al256(bytes);
        note(cudaMemsetAsync(H.mask, 0, bytes, stream_));
    }
}

cswgs_status Server::submit(const cswgs_request &q, uint64_t *ticket)
{
    auto r = std::make_unique<Req>();
    CSWGS_TRY(validate_request(p_->desc, q.spots_xyz, q.amplitudes, q.N, q.P, q.subset_fraction, q.iterations,
                               q.full_iterations, &r->spec));
    CSWGS_TRY(apply_pupil(p_, q.pupil, q.subset_fraction, &r->spec));
    CSWGS_TRY(apply_slm(q.slm, &r->spec));
    r->spec.seed = q.seed;
    if (q.phase_out) {
        if (q.out_on_host) r->phase_host = q.phase_out;
        else r->phase_dev = q.phase_out;
    }
    std::lock_guard<std::mutex> lk(mu_);
    if (!shape_set_) {
        // tile shape of every serving launch, tuned for a full set of slots like this request
        std::vector<HoloSpec> v(std::min(p_->desc.max_batch, 64), r->spec);
        {
            std::lock_guard<std::mutex> pk(p_->mu);
            cudaSetDevice(p_->device);
            shape_ = tuned_shape(p_, v);
            // past a tensor-core kernel's spot limit the next one down takes over
            shape_ = full_fallback(shape_, p_->desc.max_N, p_->sm_count);
        }
        shape_set_ = true;
        CSWGS_TRY(start());
    }
    size_t need = footprint(r->spec);
    if (need > arena_.capacity()) {
        st_.rejected++;
        return set_error(CSWGS_ENOMEM, "request needs %zu device bytes; the serving cap is %zu", need,
                         arena_.capacity());
    }
    r->bytes = need;
    r->ticket = next_ticket_++;
    r->t_submit = now_s();
    *ticket = r->ticket;
    known_[r->ticket] = true;
    queue_.push_back(std::move(r));
    st_.submitted++;
    cv_.notify_all();
    return CSWGS_OK;
}

void Server::finish(Req &r, cswgs_status st)
{
    cswgs_result res{};
    res.status = st;
    res.e = r.met.size() >= 2 ? r.met[0] : NAN;
    res.u = r.met.size() >= 2 ? r.met[1] : NAN;
    res.latency_ms = (now_s() - r.t_submit) * 1e3;
    res.queue_ms = r.t_admit > 0 ? (r.t_admit - r.t_submit) * 1e3 : res.latency_ms;
    done_[r.ticket] = res;
    if (st == CSWGS_OK) st_.completed++;
    else if (st == CSWGS_ECANCELLED) st_.cancelled++;
    done_cv_.notify_all();
}

void Server::loop()
{
    cudaSetDevice(p_->device);
    const int B = p_->desc.max_batch;
    HoloDev *holos = holos_d_.as<HoloDev>();
    HoloDev *prep_d = holos + B;
    unsigned *queue = queue_d_.as<unsigned>();
    std::unique_lock<std::mutex> lk(mu_);
    int64_t inflight_prev = -1;   // serial of the previous launch, not yet waited for
    std::map<std::pair<int, int>, int> grid_for;   // (kernel kind, max N) -> resident blocks
    // a failed CUDA call is kept: every request finished after it reports CSWGS_ECUDA
    auto chk = [this](cudaError_t e) { note(e); };
    while (true) {
        if (stop_) {
            // the plan is going away: everything pending is cancelled
            for (auto &q : queue_) q->cancelled = true;
            for (auto &a : active_)
                if (a) a->cancelled = true;
            for (int s = 0; s < B; ++s)
                if (active_[s]) retiring_.push_back(std::move(active_[s]));
        }
        // retire cancelled requests whose last launch is complete
        for (auto it = retiring_.begin(); it != retiring_.end();) {
            if ((*it)->last_launch <= completed_serial_) {
                arena_.free((*it)->off);
                finish(**it, CSWGS_ECANCELLED);
                it = retiring_.erase(it);
            } else {
                ++it;
            }
        }
        // admission: FIFO while a slot and arena memory are free
        int nprep = 0;
        LaunchSlot *sbuf = slots_h_[serial_ & 1];
        HoloDev *prep_h = reinterpret_cast<HoloDev *>(sbuf + B);
        while (!queue_.empty()) {
            Req &q = *queue_.front();
            if (q.cancelled) {
                finish(q, CSWGS_ECANCELLED);
                queue_.pop_front();
                continue;
            }
            int slot = -1;
            for (int s = 0; s < B; ++s)
                if (!active_[s]) { slot = s; break; }
            size_t off = 0;
            if (slot < 0 || !arena_.alloc(q.bytes, &off)) break;
            std::unique_ptr<Req> r = std::move(queue_.front());
            queue_.pop_front();
            r->off = off;
            r->slot = slot;
            r->t_admit = now_s();
            place(*r);
            master_[slot] = r->dev;
            prep_h[nprep++] = r->dev;
            active_[slot] = std::move(r);
        }
        int nactive = 0;
        bool has_work = false;
        for (auto &a : active_) {
            if (!a || a->cancelled) continue;
            ++nactive;
            has_work |= pass_of(a->spec, a->L) >= 0;
        }
        st_.active = nactive;
        st_.queued = (int)queue_.size();
        st_.bytes_in_use = arena_.in_use();

        // results of every launch up to completed_serial_
        auto complete = [&]() {
            for (int s = 0; s < B; ++s) {
                Req *r = active_[s].get();
                if (!r || !r->finishing || r->last_launch > completed_serial_) continue;
                const double *m = met_h_ + (size_t)(r->last_launch & 1) * 2 * B + 2 * s;
                r->met.assign(m, m + 2);
                cswgs_status st = cuda_err_ != cudaSuccess ? CSWGS_ECUDA
                                  : status_h_[r->last_launch & 1] ? CSWGS_ETIMEOUT : CSWGS_OK;
                if (r->phase_host) {
                    cudaError_t e = cudaMemcpy(r->phase_host, r->dev.phase_out,
                                               sizeof(float) * (size_t)r->spec.P * r->spec.P,
                                               cudaMemcpyDeviceToHost);
                    if (e != cudaSuccess) st = CSWGS_ECUDA;
                }
                arena_.free(r->off);
                finish(*r, st);
                active_[s].reset();
            }
        };
        auto wait_prev = [&]() {
            if (inflight_prev < 0) return;
            const int64_t w = inflight_prev;
            lk.unlock();
            chk(cudaEventSynchronize(launch_ev_[w & 1]));
            float ms = 0.f;
            chk(cudaEventElapsedTime(&ms, start_ev_[w & 1], launch_ev_[w & 1]));
            lk.lock();
            st_.busy_ms += ms;
            completed_serial_ = w;
            inflight_prev = -1;
        };

        if (!has_work) {
            // nothing to launch: drain the launch in flight, or sleep
            if (inflight_prev >= 0) {
                wait_prev();
                complete();
                for (int s = 0; s < B; ++s)
                    if (active_[s] && active_[s]->cancelled) retiring_.push_back(std::move(active_[s]));
                continue;
            }
            if (stop_ && retiring_.empty() && queue_.empty()) break;
            cv_.wait_for(lk, std::chrono::milliseconds(stop_ ? 1 : 20));
            continue;
        }
        // build launch `serial_`: one slot per request with work left, heaviest
        // first; compressed-iteration slots first, then full-pass slots, each
        // group run by its own kernel
        std::vector<Req *> order;
        for (auto &a : active_)
            if (a && !a->cancelled && pass_of(a->spec, a->L) >= 0) order.push_back(a.get());
        std::stable_sort(order.begin(), order.end(), [](Req *a, Req *b) { return a->spec.N > b->spec.N; });
        int nslots = 0, group_slots[2] = {0, 0}, group_tiles[2] = {0, 0}, group_maxN[2] = {0, 0},
            group_maxP[2] = {0, 0};
        std::vector<Req *> finishing;
        for (int kind = 0; kind < 2; ++kind) {
            for (Req *r : order) {
                const int pass = pass_of(r->spec, r->L);
                if ((pass == kPassSubset) != (kind == kLaunchSubset)) continue;
                LaunchSlot &sl = sbuf[nslots++];
                sl.holo = r->slot;
                sl.pass = pass;
                sl.j = r->spec.first_j + r->L;
                sl.count = pass == kPassSubset ? r->spec.Mp : r->spec.D;
                sl.tiles = pass_tiles(pass, r->spec.P, r->spec.Mp, shape_);
                sl.tile_begin = group_tiles[kind];
                sl.strip = 1;
                sl.pad = 0;
                group_tiles[kind] += sl.tiles;
                group_slots[kind]++;
                group_maxN[kind] = std::max(group_maxN[kind], r->spec.N);
                group_maxP[kind] = std::max(group_maxP[kind], r->spec.P);
                if (pass == kPassFinal) finishing.push_back(r);
            }
        }
        // the tensor-core kernel takes strips of tiles along a row block
        for (int kind = 0, first = 0; kind < 2; first += group_slots[kind], ++kind) {
            if (group_tiles[kind] == 0 || !launch_uses_tc(shape_, kind)) continue;
            auto key = std::make_pair(kind, group_maxN[kind]);
            auto g = grid_for.find(key);
            if (g == grid_for.end())
                g = grid_for.emplace(key, shape_max_grid(shape_, kind, group_maxN[kind], p_->sm_count)).first;
            std::vector<int> sP, sN;
            for (int i = first; i < first + group_slots[kind]; ++i) {
                sP.push_back(master_[sbuf[i].holo].P);
                sN.push_back(master_[sbuf[i].holo].N);
            }
            group_tiles[kind] = full_tc_assign_strips(sbuf + first, group_slots[kind], sP.data(), sN.data(),
                                                      std::max(1, g->second), shape_.strip);
        }
        const int64_t serial = serial_++;
        HoloDev *hbuf = holos_h_[serial & 1];
        std::memcpy(hbuf, master_.data(), sizeof(HoloDev) * B);
        LaunchSlot *sd = slots_d_.as<LaunchSlot>() + (serial & 1) * B;
        chk(cudaMemcpyAsync(holos, hbuf, sizeof(HoloDev) * B, cudaMemcpyHostToDevice, stream_));
        if (nprep) {
            chk(cudaMemcpyAsync(prep_d, prep_h, sizeof(HoloDev) * nprep, cudaMemcpyHostToDevice, stream_));
            int pmax = 0;
            for (int i = 0; i < nprep; ++i) pmax = std::max(pmax, prep_h[i].N);
            chk(launch_prep_fp32(prep_d, nprep, pmax, stream_));
            if (uses_tc(shape_)) chk(launch_tc_const_tables(prep_d, nprep, p_->sm_count, stream_));
        }
        chk(cudaMemcpyAsync(sd, sbuf, sizeof(LaunchSlot) * nslots, cudaMemcpyHostToDevice, stream_));
        chk(cudaEventRecord(start_ev_[serial & 1], stream_));
        for (int kind = 0, first = 0; kind < 2; first += group_slots[kind], ++kind) {
            if (group_tiles[kind] == 0) continue;
            auto key = std::make_pair(kind, group_maxN[kind]);
            auto g = grid_for.find(key);
            if (g == grid_for.end())
                g = grid_for.emplace(key, shape_max_grid(shape_, kind, group_maxN[kind], p_->sm_count)).first;
            if (kind == kLaunchSubset && uses_masks(shape_))
                chk(launch_tc_mask_scatter(holos, sd + first, group_slots[kind], group_maxP[kind], p_->sm_count,
                                           stream_));
            if (launch_uses_tc(shape_, kind))
                chk(launch_tc_rw_tables(holos, sd + first, group_slots[kind], p_->sm_count, stream_));
            chk(shape_launch(shape_, kind, holos, sd + first, group_slots[kind], group_tiles[kind], group_maxN[kind],
                             queue, std::min(g->second, group_tiles[kind]), stream_));
        }
        double *mh = met_h_ + (size_t)(serial & 1) * 2 * B;
        for (Req *r : finishing) {
            chk(cudaMemcpyAsync(mh + 2 * r->slot, r->dev.metrics, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream_));
            r->finishing = true;
        }
        // the launches' status word (a timed-out wait inside a kernel sets it)
        chk(cudaMemcpyAsync(status_h_ + (serial & 1), queue + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, stream_));
        chk(cudaEventRecord(launch_ev_[serial & 1], stream_));
        for (Req *r : order) {          // only the requests that took part advance
            r->L++;
            r->last_launch = serial;
        }
        st_.launches++;
        // wait for the previous launch while this one runs, then collect its results
        wait_prev();
        inflight_prev = serial;
        complete();
        // cancelled requests leave their slot now; memory is freed once idle
        for (int s = 0; s < B; ++s)
            if (active_[s] && active_[s]->cancelled) retiring_.push_back(std::move(active_[s]));
    }
}

cswgs_status Server::poll(uint64_t ticket, cswgs_result *res, double timeout_s, bool wait)
{
    std::unique_lock<std::mutex> lk(mu_);
    auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (true) {
        auto it = done_.find(ticket);
        if (it != done_.end()) {
            if (res) *res = it->second;
            cswgs_status st = it->second.status;
            done_.erase(it);
            known_.erase(ticket);
            return st == CSWGS_OK ? CSWGS_OK : (st == CSWGS_ECANCELLED ? CSWGS_ECANCELLED : st);
        }
        if (!known_.count(ticket)) return set_error(CSWGS_ENOTFOUND, "ticket %llu unknown", (unsigned long long)ticket);
        if (!wait) return CSWGS_EBUSY;
        if (done_cv_.wait_until(lk, deadline) == std::cv_status::timeout && !done_.count(ticket))
            return set_error(CSWGS_ETIMEOUT, "ticket %llu not finished after %g s", (unsigned long long)ticket,
                             timeout_s);
    }
}

cswgs_status Server::cancel(uint64_t ticket)
{
    std::lock_guard<std::mutex> lk(mu_);
    if (!known_.count(ticket) || done_.count(ticket))
        return set_error(CSWGS_ENOTFOUND, "ticket %llu not pending", (unsigned long long)ticket);
    for (auto &q : queue_)
        if (q->ticket == ticket) { q->cancelled = true; cv_.notify_all(); return CSWGS_OK; }
    for (auto &a : active_)
        if (a && a->ticket == ticket) { a->cancelled = true; return CSWGS_OK; }
    return set_error(CSWGS_ENOTFOUND, "ticket %llu not pending", (unsigned long long)ticket);
}

void Server::stats(cswgs_serve_stats *s)
{
    std::lock_guard<std::mutex> lk(mu_);
    *s = st_;
    s->bytes_cap = arena_.capacity();
    s->bytes_in_use = arena_.in_use();
}

}  // namespace cswgs

using namespace cswgs;

extern "C" {

cswgs_status cswgs_submit(cswgs_plan p, const cswgs_request *r, uint64_t *ticket)
{
    if (!p || !r || !ticket) return set_error(CSWGS_EINVAL, "NULL plan, request or ticket");
    if (p->desc.precision == CSWGS_FP64)
        return set_error(CSWGS_EINVAL, "the serving loop runs the FP32 solver; this plan is FP64");
    {
        std::lock_guard<std::mutex> lk(p->mu);
        if (!p->server) p->server = std::make_unique<Server>(p);
    }
    return p->server->submit(*r, ticket);
}

cswgs_status cswgs_poll(cswgs_plan p, uint64_t ticket, cswgs_result *res)
{
    if (!p) return set_error(CSWGS_EINVAL, "NULL plan");
    if (!p->server) return set_error(CSWGS_ENOTFOUND, "no request was submitted to this plan");
    return p->server->poll(ticket, res, 0.0, false);
}

cswgs_status cswgs_wait(cswgs_plan p, uint64_t ticket, double timeout_s, cswgs_result *res)
{
    if (!p) return set_error(CSWGS_EINVAL, "NULL plan");
    if (!p->server) return set_error(CSWGS_ENOTFOUND, "no request was submitted to this plan");
    if (!(timeout_s >= 0.0)) return set_error(CSWGS_EINVAL, "timeout %g", timeout_s);
    return p->server->poll(ticket, res, timeout_s, true);
}

cswgs_status cswgs_cancel(cswgs_plan p, uint64_t ticket)
{
    if (!p) return set_error(CSWGS_EINVAL, "NULL plan");
    if (!p->server) return set_error(CSWGS_ENOTFOUND, "no request was submitted to this plan");
    return p->server->cancel(ticket);
}

cswgs_status cswgs_serve_stats_get(cswgs_plan p, cswgs_serve_stats *s)
{
    if (!p || !s) return set_error(CSWGS_EINVAL, "NULL plan or stats");
    std::memset(s, 0, sizeof *s);
    if (p->server) p->server->stats(s);
    return CSWGS_OK;
}

}  // extern "C"
