// Continuous-batching server of the CS-WGS library.
#pragma once

#include "runtime.h"

namespace cswgs {

// First-fit allocator over one device allocation (the serving arena).
class Arena {
public:
    cswgs_status init(size_t bytes);
    bool alloc(size_t bytes, size_t *off);
    void free(size_t off);
    size_t capacity() const { return cap_; }
    size_t in_use() const { return used_; }
    char *base() const { return static_cast<char *>(mem_.p); }
    void set_capacity_for_test(size_t bytes) { cap_ = bytes; }

private:
    DevBuf mem_;
    size_t cap_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;   // offset -> size
    std::map<size_t, size_t> taken_;  // offset -> size
};

class Server {
public:
    explicit Server(cswgs_plan_s *p);
    ~Server();
    cswgs_status start();
    cswgs_status submit(const cswgs_request &r, uint64_t *ticket);
    cswgs_status poll(uint64_t ticket, cswgs_result *res, double timeout_s, bool wait);
    cswgs_status cancel(uint64_t ticket);
    void stats(cswgs_serve_stats *s);

private:
    struct Req {
        uint64_t ticket = 0;
        HoloSpec spec;
        float *phase_dev = nullptr;      // caller's device output
        float *phase_host = nullptr;     // caller's host output
        double t_submit = 0, t_admit = 0;
        // device side
        size_t off = 0, bytes = 0;
        HoloDev dev{};
        int slot = -1;
        int L = 0;                       // next launch index of this request's schedule
        int64_t last_launch = -1;        // serial of the last launch that used it
        bool cancelled = false;
        bool finishing = false;          // final pass issued
        std::vector<double> met;         // host copy of e, u
    };
    void loop();
    size_t footprint(const HoloSpec &s) const;
    void place(Req &r);
    void finish(Req &r, cswgs_status st);

    cswgs_plan_s *p_;
    cudaStream_t stream_ = nullptr;
    Arena arena_;
    TileShape shape_{256, 4};
    bool shape_set_ = false;
    std::thread th_;
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    bool stop_ = false, started_ = false;
    uint64_t next_ticket_ = 1;
    std::deque<std::unique_ptr<Req>> queue_;
    std::vector<std::unique_ptr<Req>> active_;     // by slot (nullptr = free)
    std::vector<std::unique_ptr<Req>> retiring_;   // cancelled, waiting for in-flight launches
    std::unordered_map<uint64_t, cswgs_result> done_;
    std::unordered_map<uint64_t, bool> known_;
    DevBuf holos_d_, slots_d_, queue_d_;
    std::vector<HoloDev> master_;                   // slot table (host copy)
    HoloDev *holos_h_[2] = {nullptr, nullptr};      // pinned, double-buffered copies of master_
    LaunchSlot *slots_h_[2] = {nullptr, nullptr};   // pinned, double-buffered (slots, then prep list)
    double *met_h_ = nullptr;                       // pinned: e, u per slot, double-buffered
    unsigned *status_h_ = nullptr;                  // pinned: the launches' status word, double-buffered
    cudaError_t cuda_err_ = cudaSuccess;            // first failed CUDA call of the loop (sticky)
    void note(cudaError_t e)
    {
        if (e != cudaSuccess && cuda_err_ == cudaSuccess) cuda_err_ = e;
    }
    double *in_h_ = nullptr;                        // pinned: per-slot input staging (N x 4 doubles)
    cudaEvent_t launch_ev_[2] = {nullptr, nullptr};
    cudaEvent_t start_ev_[2] = {nullptr, nullptr};
    int64_t serial_ = 0, completed_serial_ = -1;
    cswgs_serve_stats st_{};
};

}  // namespace cswgs
