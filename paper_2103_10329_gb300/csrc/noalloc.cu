// Residual projection that allocates nothing: the scratch that
// mgct_project takes from the geometry handle (the x-major copy of the
// volume and the per-block partial sums of |r|^2) lives here in one
// file-scope device array instead, of a fixed size.
//
// Who needs it: callers whose device memory belongs to someone else -- an
// imaging pipeline or framework that hands every buffer out of its own pool
// or caching allocator and does not let plug-ins call cudaMalloc/cudaFree, or
// a process whose device-memory budget is fixed at start-up -- can still run
// the projector with its residual norm, passing only inputs and outputs.
//
// The array is part of the library's device module: every GPU on which the
// module is loaded holds it (NOALLOC_BYTES) until the process exits, whether
// or not it is used.  Under lazy module loading (the CUDA default) the module,
// and with it the array, is loaded on the first use of the library's device
// code on that device -- at the latest by this entry point's first call, whose
// cudaGetSymbolAddress loads it.  A caller whose device-memory budget is fixed
// later should make one call (any size within the limits) at start-up.
#include <mutex>

#include "common.cuh"
#include "project.cuh"

namespace mgct {
namespace {

constexpr size_t NOALLOC_MAX_VOXELS = (size_t)128 * 128 * 128;  // largest volume: 128^3
constexpr size_t NOALLOC_MAX_PARTIALS = (size_t)1 << 18;        // projector blocks per call
constexpr size_t NOALLOC_VOL_BYTES = NOALLOC_MAX_VOXELS * sizeof(float);
constexpr size_t NOALLOC_BYTES = NOALLOC_VOL_BYTES + NOALLOC_MAX_PARTIALS * sizeof(double);

// The scratch itself.  Host code must not take its address directly: on the
// host this name is only a stand-in, so the device address is fetched with
// cudaGetSymbolAddress once per device (below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES] = {};
unsigned long long g_ctx[MAX_DEVICES] = {};  // id of the context the address belongs to

// Identity of the calling thread's current context (cuCtxGetCurrent +
// cuCtxGetId, reached through the runtime's driver entry points so that the
// library needs no link against libcuda); 0 when the driver cannot say.
unsigned long long current_context_id() {
    typedef int (*get_current_t)(void **);
    typedef int (*get_id_t)(void *, unsigned long long *);
    static get_current_t get_current = nullptr;
    static get_id_t get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess && f1 && f2) {
            get_current = reinterpret_cast<get_current_t>(f1);
            get_id = reinterpret_cast<get_id_t>(f2);
        } else {
            cudaGetLastError();
        }
    }
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of the scratch in the current device's current context.
// It is looked up (cudaGetSymbolAddress) on the first call made in a context
// and cached under that context's id; a context created anew on the same
// device (after cudaDeviceReset, or a released and re-created primary
// context) loads the module again, so its address is looked up again.  When
// the context's id cannot be read (no context is current on this thread yet,
// or the driver lacks the call) the address is looked up on that call.
int scratch_address(void **out) {
    int dev = 0;
    MGCT_TRY(check_cuda(cudaGetDevice(&dev), "cudaGetDevice"));
    if (dev < 0 || dev >= MAX_DEVICES) return set_error(MGCT_EINVAL, "device ordinal out of range");
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev] || ctx == 0 || g_ctx[dev] != ctx) {
        void *p = nullptr;
        MGCT_TRY(check_cuda(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(static scratch)"));
        if (!p) return set_error(MGCT_ECUDA, "cudaGetSymbolAddress returned NULL");
        g_addr[dev] = p;
        g_ctx[dev] = ctx;
    }
    *out = g_addr[dev];
    return MGCT_OK;
}

}  // namespace
}  // namespace mgct

using namespace mgct;

extern "C" {

size_t mgct_project_residual_static_bytes(void) { return NOALLOC_BYTES; }

int mgct_project_residual_static(const mgct_geom *g, int level, int view0, int nviews, int stride,
                                 const float *vol, float *out, const float *b, double *sumsq,
                                 mgct_stream stream) {
    MGCT_TRY(validate_level(g, level));
    MGCT_TRY(validate_views(g, view0, nviews, stride));
    MGCT_TRY(check_ptr(vol, "vol"));
    MGCT_TRY(check_ptr(out, "out", nviews == 0));
    MGCT_TRY(check_ptr(b, "b", nviews == 0));
    MGCT_TRY(check_ptr(sumsq, "sumsq"));
    const LevelInfo &L = g->lev[level];
    const size_t nvox = (size_t)L.n * L.n * L.n;
    if (nvox > NOALLOC_MAX_VOXELS)
        return set_error(MGCT_ESHAPE, "mgct_project_residual_static: volume of " + std::to_string(L.n) +
                                          "^3 voxels exceeds the static scratch (at most 128^3 voxels)");
    const size_t blocks = project_blocks(L.nu, L.nv, nviews);
    if (blocks > NOALLOC_MAX_PARTIALS)
        return set_error(MGCT_ESHAPE, "mgct_project_residual_static: " + std::to_string(blocks) +
                                          " projector blocks exceed the static scratch (at most 262144; "
                                          "use fewer views per call)");
    void *base = nullptr;
    MGCT_TRY(scratch_address(&base));
    float *volT = static_cast<float *>(base);
    double *part = reinterpret_cast<double *>(static_cast<unsigned char *>(base) + NOALLOC_VOL_BYTES);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (nviews == 0) return check_cuda(cudaMemsetAsync(sumsq, 0, sizeof(double), s), "memset");
    // every scratch word read below is written first by this call: the
    // transposed volume in full, one partial per projector block
    MGCT_TRY(launch_transpose_xy<float>(L.n, vol, volT, s));
    int nb = 0;
    EpiResidual<float> e{out, b, part, L.nu, L.nv, nviews};
    MGCT_TRY(launch_project<float>(g, level, view0, nviews, stride, vol, volT, e, s, &nb));
    return launch_sum_partials(part, nb, 1, sumsq, s);
}

}  // extern "C"
