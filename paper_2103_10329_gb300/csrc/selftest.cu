// Self-check of the failure path of the library's bounded device waits.
// The tensor-core convolutions wait on mbarriers for their MMAs with
// mbar_wait_bounded; this runs that same routine on an mbarrier that nothing
// ever arrives on, so the wait must expire, be reported, and leave the
// context usable.  Nothing faults and nothing hangs: the wait is bounded by
// the SM clock.
#include "common.cuh"
#include "conv3d_tc.cuh"

namespace mgct {

__device__ int g_wait_expired;  // the self-check's result (no allocation)

__global__ void k_wait_expires(long long limit) {
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // phase 0 never completes: no thread arrives
    const bool done = mbar_wait_bounded(&mbar, 0u, limit);
    if (threadIdx.x == 0) g_wait_expired = done ? 0 : 1;
}

}  // namespace mgct

using namespace mgct;

extern "C" int mgct_check_bounded_wait(double seconds, int *expired, mgct_stream stream) {
    if (!expired) return set_error(MGCT_EINVAL, "expired must not be NULL");
    if (!(seconds > 0.0 && seconds <= 10.0)) return set_error(MGCT_EINVAL, "seconds must be in (0, 10]");
    *expired = 0;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, khz = 0;
    MGCT_TRY(check_cuda(cudaGetDevice(&dev), "device"));
    MGCT_TRY(check_cuda(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev), "clock rate"));
    const long long limit = (long long)(seconds * (double)khz * 1e3);
    const int zero = 0;
    MGCT_TRY(check_cuda(cudaMemcpyToSymbolAsync(g_wait_expired, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s),
                        "clear flag"));
    MGCT_KERNEL(KK_OTHER, s, k_wait_expires<<<1, 32, 0, s>>>(limit));
    int st = check_cuda(cudaMemcpyFromSymbolAsync(expired, g_wait_expired, sizeof(int), 0, cudaMemcpyDeviceToHost, s),
                        "read flag");
    if (!st) st = check_cuda(cudaStreamSynchronize(s), "bounded wait");
    return st;
}
