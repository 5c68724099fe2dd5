// Optional kernel trace: CUDA events recorded on the launching stream around
// every kernel the library issues, summed per kernel kind on request.  Off by
// default; when off, the hooks return at once.
#include <mutex>
#include <vector>

#include "common.cuh"

namespace mgct {

namespace {
struct Rec {
    int kind;
    int tag;
    cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
thread_local cudaEvent_t t_pending = nullptr;
thread_local int t_tag = -1;

cudaEvent_t get_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void recycle_all() {
    for (auto &r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
}
}  // namespace

void trace_begin(int, cudaStream_t s) {
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    t_pending = get_event();
    if (t_pending) cudaEventRecord(t_pending, s);
}

void trace_end(int kind, cudaStream_t s) {
    if (!g_on || !t_pending) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t e = get_event();
    if (!e) return;
    cudaEventRecord(e, s);
    g_recs.push_back({kind, t_tag, t_pending, e});
    t_pending = nullptr;
}

void trace_tag(int tag) { t_tag = tag; }

}  // namespace mgct

using namespace mgct;

extern "C" {

int mgct_trace_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    recycle_all();
    g_on = on != 0;
    return MGCT_OK;
}

static int trace_sum(int tag, double *ms, uint64_t *launches, int nkinds) {
    if (!ms || !launches || nkinds < 1) return set_error(MGCT_EINVAL, "ms and launches must not be NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    for (int k = 0; k < nkinds; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    for (auto &r : g_recs) {
        MGCT_TRY(check_cuda(cudaEventSynchronize(r.b), "trace event sync"));
        float t = 0.0f;
        MGCT_TRY(check_cuda(cudaEventElapsedTime(&t, r.a, r.b), "trace elapsed time"));
        if (r.kind >= 0 && r.kind < nkinds && (tag < 0 || r.tag == tag)) {
            ms[r.kind] += t;
            launches[r.kind] += 1;
        }
    }
    return MGCT_OK;
}

int mgct_trace_read(double *ms, uint64_t *launches, int nkinds) { return trace_sum(-1, ms, launches, nkinds); }

int mgct_trace_read_level(int level, double *ms, uint64_t *launches, int nkinds) {
    if (level < 0) return set_error(MGCT_EINVAL, "level must be >= 0");
    return trace_sum(level, ms, launches, nkinds);
}

}  // extern "C"
