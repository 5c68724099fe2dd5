// Microbenchmarks of the two on-chip peaks the projector and back-projector
// are measured against: the FP32 FMA rate and the shared-memory (L1 data
// path) load bandwidth.  Each kernel keeps every SM busy with independent
// work and writes its result only under a condition that never holds, so the
// compiler keeps the work; nothing is allocated (the sink is a static
// device word).
#include "common.cuh"

namespace mgct {

__device__ float g_peak_sink;

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;   // independent FMA chains per thread
constexpr int PK_UNROLL = 16;  // FMAs per chain per loop trip

__global__ void __launch_bounds__(PK_THREADS) k_fma_peak(int iters, float seed) {
    float a[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) a[c] = seed + (float)(threadIdx.x + c);
    const float m = 0.9999999f, k = 1e-7f;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < PK_CHAINS; ++c) a[c] = fmaf(a[c], m, k);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += a[c];
    if (s == -1.0f) g_peak_sink = s;
}

constexpr int PK_SLOTS = 1024;  // float4 slots of shared memory (16 KB)
constexpr int PK_LOADS = 8;     // 16-byte loads per thread per loop trip

__global__ void __launch_bounds__(PK_THREADS) k_lds_peak(int iters) {
    __shared__ float4 buf[PK_SLOTS];
    for (int i = threadIdx.x; i < PK_SLOTS; i += PK_THREADS)
        buf[i] = make_float4((float)i, (float)(i + 1), (float)(i + 2), (float)(i + 3));
    __syncthreads();
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    int idx = threadIdx.x;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
        // a warp's 32 loads cover 512 contiguous bytes: no bank conflicts
#pragma unroll
        for (int u = 0; u < PK_LOADS; ++u) {
            const float4 v = buf[(idx + u * 32) & (PK_SLOTS - 1)];
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        idx = (idx + PK_THREADS) & (PK_SLOTS - 1);
    }
    if (acc.x + acc.y + acc.z + acc.w == -1.0f) g_peak_sink = acc.x;
}

// Median of `reps` CUDA-event timings (ms) of `launch` on stream s.
template <typename F>
static int time_median(F launch, int reps, cudaStream_t s, float *ms) {
    cudaEvent_t e0, e1;
    MGCT_TRY(check_cuda(cudaEventCreate(&e0), "event"));
    int st = check_cuda(cudaEventCreate(&e1), "event");
    float t[16];
    for (int r = 0; r < reps && !st; ++r) {
        st = check_cuda(cudaEventRecord(e0, s), "record");
        if (!st) st = launch();
        if (!st) st = check_cuda(cudaEventRecord(e1, s), "record");
        if (!st) st = check_cuda(cudaEventSynchronize(e1), "synchronize");
        if (!st) st = check_cuda(cudaEventElapsedTime(&t[r], e0, e1), "elapsed");
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    for (int i = 1; i < reps; ++i)
        for (int j = i; j > 0 && t[j] < t[j - 1]; --j) {
            const float x = t[j];
            t[j] = t[j - 1];
            t[j - 1] = x;
        }
    *ms = t[reps / 2];
    return MGCT_OK;
}

}  // namespace mgct

using namespace mgct;

extern "C" int mgct_measure_onchip_peaks(double *fp32_tflops, double *lds_gbs, mgct_stream stream) {
    if (!fp32_tflops || !lds_gbs) return set_error(MGCT_EINVAL, "outputs must not be NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    MGCT_TRY(check_cuda(cudaGetDevice(&dev), "device"));
    MGCT_TRY(check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count"));
    const int blocks = 8 * sms;  // 64 resident warps per SM
    const int fma_iters = 2048, lds_iters = 4096;
    float ms = 0.0f;
    // one untimed launch of each first (module load, clocks)
    MGCT_KERNEL(KK_OTHER, s, k_fma_peak<<<blocks, PK_THREADS, 0, s>>>(fma_iters, 1.0f));
    MGCT_KERNEL(KK_OTHER, s, k_lds_peak<<<blocks, PK_THREADS, 0, s>>>(lds_iters));
    MGCT_TRY(time_median(
        [&]() -> int {
            MGCT_KERNEL(KK_OTHER, s, k_fma_peak<<<blocks, PK_THREADS, 0, s>>>(fma_iters, 1.0f));
            return MGCT_OK;
        },
        5, s, &ms));
    const double flops = 2.0 * PK_CHAINS * PK_UNROLL * (double)fma_iters * blocks * PK_THREADS;
    *fp32_tflops = flops / (ms * 1e-3) / 1e12;
    MGCT_TRY(time_median(
        [&]() -> int {
            MGCT_KERNEL(KK_OTHER, s, k_lds_peak<<<blocks, PK_THREADS, 0, s>>>(lds_iters));
            return MGCT_OK;
        },
        5, s, &ms));
    const double bytes = 16.0 * PK_LOADS * (double)lds_iters * blocks * PK_THREADS;
    *lds_gbs = bytes / (ms * 1e-3) / 1e9;
    return MGCT_OK;
}
