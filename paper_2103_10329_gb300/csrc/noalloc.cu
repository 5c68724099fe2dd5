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
// The array is part of the library image: every GPU that loads libmgct holds
// it (NOALLOC_BYTES) until the process exits, whether or not it is used.
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

// Device address of the scratch on the current device, looked up on the
// first call made with that device current.
int scratch_address(void **out) {
    int dev = 0;
    MGCT_TRY(check_cuda(cudaGetDevice(&dev), "cudaGetDevice"));
    if (dev < 0 || dev >= MAX_DEVICES) return set_error(MGCT_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        MGCT_TRY(check_cuda(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(static scratch)"));
        if (!p) return set_error(MGCT_ECUDA, "cudaGetSymbolAddress returned NULL");
        g_addr[dev] = p;
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
