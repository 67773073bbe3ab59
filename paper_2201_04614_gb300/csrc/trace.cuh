// trace.cuh -- optional CUDA-event tracing of the library's own launches.
//
// When enabled, every kernel launch of the library is bracketed by two
// CUDA events recorded on the launch stream; vsz_trace_read() waits for them
// and reports each launch's device time.  Meant for eager execution (events
// recorded while a stream is being captured into a graph do not time it).
#pragma once

#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "vsz.h"

namespace vsz {

struct TraceRec {
    const char* name;
    cudaEvent_t a, b;
    int32_t ndim;
    uint32_t block;
    uint64_t n;
};

class Tracer {
public:
    static Tracer& get() {
        static Tracer t;
        return t;
    }
    bool on() const { return on_; }
    void enable(bool v) {
        std::lock_guard<std::mutex> lk(mu_);
        on_ = v;
    }
    cudaEvent_t take() {
        std::lock_guard<std::mutex> lk(mu_);
        if (!pool_.empty()) {
            cudaEvent_t e = pool_.back();
            pool_.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) e = nullptr;
        return e;
    }
    void push(const TraceRec& r) {
        std::lock_guard<std::mutex> lk(mu_);
        pending_.push_back(r);
    }
    // Waits for the recorded launches, writes up to max records, clears.
    int read(vsz_trace_record* out, int max) {
        std::vector<TraceRec> recs;
        {
            std::lock_guard<std::mutex> lk(mu_);
            recs.swap(pending_);
        }
        int k = 0;
        for (const TraceRec& r : recs) {
            float ms = -1.0f;
            if (r.a && r.b && cudaEventSynchronize(r.b) == cudaSuccess) {
                if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) ms = -1.0f;
            }
            if (out && k < max) {
                vsz_trace_record& o = out[k];
                std::memset(&o, 0, sizeof o);
                std::strncpy(o.name, r.name, sizeof(o.name) - 1);
                o.ndim = r.ndim;
                o.block = r.block;
                o.n = r.n;
                o.ms = ms;
            }
            ++k;
        }
        std::lock_guard<std::mutex> lk(mu_);
        for (const TraceRec& r : recs) {
            if (r.a) pool_.push_back(r.a);
            if (r.b) pool_.push_back(r.b);
        }
        return k;
    }

    // Tracing off; drops the pending records and destroys every event.
    void shutdown() {
        std::lock_guard<std::mutex> lk(mu_);
        on_ = false;
        for (const TraceRec& r : pending_) {
            if (r.a) cudaEventDestroy(r.a);
            if (r.b) cudaEventDestroy(r.b);
        }
        pending_.clear();
        for (cudaEvent_t e : pool_) cudaEventDestroy(e);
        pool_.clear();
    }

private:
    std::mutex mu_;
    bool on_ = false;
    std::vector<TraceRec> pending_;
    std::vector<cudaEvent_t> pool_;
};

// RAII bracket around one launch.
class TraceScope {
public:
    TraceScope(const char* name, cudaStream_t s, int32_t nd = 0, uint32_t b = 0, uint64_t n = 0) : s_(s) {
        Tracer& t = Tracer::get();
        active_ = t.on();
        if (!active_) return;
        r_ = TraceRec{name, t.take(), t.take(), nd, b, n};
        if (r_.a) cudaEventRecord(r_.a, s_);
    }
    ~TraceScope() {
        if (!active_) return;
        if (r_.b) cudaEventRecord(r_.b, s_);
        Tracer::get().push(r_);
    }

private:
    cudaStream_t s_;
    bool active_ = false;
    TraceRec r_{};
};

}  // namespace vsz
