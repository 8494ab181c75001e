// Per-stage launch timing: CUDA event pairs recorded on the launching stream around each
// launch while a profiler is active, resolved (elapsed time) when the counters are read.
#include "tddft_internal.h"

#include <vector>

namespace tddft {

struct Profiler {
    struct Rec {
        cudaEvent_t a, b;
        int stage;
        double flops, bytes;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    long long launches[ST_COUNT] = {};
    double ms[ST_COUNT] = {}, flops[ST_COUNT] = {}, bytes[ST_COUNT] = {};

    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        check(cudaEventCreate(&e), "cudaEventCreate");
        return e;
    }
    void resolve() {
        for (Rec &r : pending) {
            check(cudaEventSynchronize(r.b), "cudaEventSynchronize");
            float t = 0.f;
            check(cudaEventElapsedTime(&t, r.a, r.b), "cudaEventElapsedTime");
            launches[r.stage] += 1;
            ms[r.stage] += t;
            flops[r.stage] += r.flops;
            bytes[r.stage] += r.bytes;
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        pending.clear();
    }
    void reset() {
        resolve();
        for (int i = 0; i < ST_COUNT; ++i) launches[i] = 0, ms[i] = flops[i] = bytes[i] = 0.0;
    }
    ~Profiler() {
        for (Rec &r : pending) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
};

Profiler *&active_profiler() {
    static thread_local Profiler *p = nullptr;
    return p;
}

long long &active_wait_limit() {
    static thread_local long long w = DEFAULT_WAIT_LIMIT;
    return w;
}

const char *stage_name(int s) {
    static const char *names[ST_COUNT] = {"gemm", "response_density", "potential_integrals",
                                          "fft_poisson_fxc", "trace", "vector", "small_fp64"};
    return (s >= 0 && s < ST_COUNT) ? names[s] : "?";
}

ProfScope::ProfScope(cudaStream_t s, int stg, double f, double b)
    : p(active_profiler()), st(s), stage(stg), flops(f), bytes(b), ev0(nullptr) {
    if (!p) return;
    cudaEvent_t e = p->get();
    check(cudaEventRecord(e, st), "cudaEventRecord");
    ev0 = e;
}

ProfScope::~ProfScope() {
    if (!p || !ev0) return;
    cudaEvent_t e = p->get();
    if (cudaEventRecord(e, st) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    p->pending.push_back({static_cast<cudaEvent_t>(ev0), e, stage, flops, bytes});
}

Profiler *profiler_new() { return new Profiler(); }
void profiler_delete(Profiler *p) { delete p; }
void profiler_read(Profiler *p, long long *launches, double *ms, double *flops, double *bytes) {
    p->resolve();
    for (int i = 0; i < ST_COUNT; ++i) {
        launches[i] = p->launches[i];
        ms[i] = p->ms[i];
        flops[i] = p->flops[i];
        bytes[i] = p->bytes[i];
    }
}
void profiler_reset(Profiler *p) { p->reset(); }

}  // namespace tddft
