// Learned preconditioner correction: a small 3D convolutional network applied
// to the preconditioned Landweber step (the paper's Sec. 3 discussion asks
// for more effective preconditioning kernels than Eq. 5; the network learns
// a correction on top of it).  Architecture: four 3x3x3 convolutions at full
// resolution with 16, 32 and 64 hidden channels (ReLU) and one linear output
// channel; its input is the step alpha d scaled to unit RMS, x = alpha d / s,
// and the corrected step is d' = s (x + f(x)).  Training minimises the mean
// of (x + f(x) - t)^2 with t = e / s, e the error of the current estimate, by
// Adam on float32 master weights.  The convolutions -- forward, backward
// data and the weight gradient -- run on the tcgen05 tensor cores
// (conv3d_tc.cuh) with float32 accumulation and BF16 activations.
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "common.cuh"
#include "conv3d_tc.cuh"

namespace mgct {

// Layer shapes (padded to multiples of 16 channels): input 1 real channel,
// output 1 real channel.
constexpr int NL = 4;
constexpr int LCIN[NL] = {16, 16, 32, 64};
constexpr int LCOUT[NL] = {16, 32, 64, 16};
constexpr int LCIN_REAL[NL] = {1, 16, 32, 64};
constexpr int LCOUT_REAL[NL] = {16, 32, 64, 1};

inline size_t wcount(int l) { return (size_t)27 * LCOUT[l] * LCIN[l]; }

}  // namespace mgct

struct mgct_net {
    float *w[mgct::NL], *b[mgct::NL];      // float32 master weights [27][COUT][CIN], bias [COUT]
    float *mw[mgct::NL], *vw[mgct::NL];    // Adam moments
    float *mb[mgct::NL], *vb[mgct::NL];
    float *gw[mgct::NL], *gb[mgct::NL];    // gradients of the last forward_backward
    __nv_bfloat16 *wf[mgct::NL];           // bf16 forward weights
    __nv_bfloat16 *wt[mgct::NL];           // bf16 backward-data weights [26 - tap][CIN][COUT]
    double *loss;                          // device scalar of the last forward_backward
    int *err;                              // device word: a convolution's bounded wait expired
    int64_t step;
};

namespace mgct {

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
__global__ void k_pack_weights(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wf,
                               __nv_bfloat16 *__restrict__ wt, int cout, int cin) {
    const int n = 27 * cout * cin;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ci = i % cin, co = (i / cin) % cout, tap = i / (cin * cout);
        const __nv_bfloat16 v = __float2bfloat16_rn(w[i]);
        wf[i] = v;
        wt[((size_t)(26 - tap) * cin + ci) * cout + co] = v;
    }
}

// x (float32 [nvox]) scaled by 1/s into channel 0 of a 16-channel bf16 tensor;
// s = sqrt(sumsq / nnorm) from a device scalar (or 1 when sumsq == NULL);
// nnorm is the voxel count of the whole volume the sum was taken over (a
// z-slab of it may be processed here).
__global__ void k_net_input(const float *__restrict__ x, const double *__restrict__ sumsq, double nnorm, int nvox,
                            __nv_bfloat16 *__restrict__ x0, float *__restrict__ xs) {
    const float inv = sumsq ? (float)(1.0 / fmax(sqrt(sumsq[0] / nnorm), 1e-30)) : 1.0f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nvox; p += gridDim.x * blockDim.x) {
        const float v = x[p] * inv;
        if (xs) xs[p] = v;
        uint4 z = make_uint4(0, 0, 0, 0);
        __nv_bfloat16 *e = reinterpret_cast<__nv_bfloat16 *>(&z);
        e[0] = __float2bfloat16_rn(v);
        uint4 *dst = reinterpret_cast<uint4 *>(x0 + (size_t)p * 16);
        dst[0] = z;
        dst[1] = make_uint4(0, 0, 0, 0);
    }
}

// out = s (x + y)  (the corrected step in the caller's units)
// (NaN everywhere when a convolution of this pass failed, so that the
// learned step's line search rejects it)
__global__ void k_net_output(const float *__restrict__ x, const float *__restrict__ y, const double *__restrict__ sumsq,
                             double nnorm, int nvox, const int *__restrict__ err, float *__restrict__ out) {
    const float s = *err ? __int_as_float(0x7fc00000) : (float)fmax(sqrt(sumsq[0] / nnorm), 1e-30);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nvox; p += gridDim.x * blockDim.x)
        out[p] = s * (x[p] + y[p]);
}

// loss partials and the output gradient: r = x + y - t; dL/dy = 2 r / N
// (a NaN loss when a convolution of the forward pass failed)
__global__ void k_mse(const float *__restrict__ x, const float *__restrict__ y, const float *__restrict__ t, int nvox,
                      const int *__restrict__ err, __nv_bfloat16 *__restrict__ gy, double *__restrict__ part) {
    __shared__ double red[256];
    double s = *err ? __longlong_as_double(0x7ff8000000000000ll) : 0.0;
    const float sc = 2.0f / (float)nvox;
    const double inv_n = 1.0 / (double)nvox;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nvox; p += gridDim.x * blockDim.x) {
        const float r = x[p] + y[p] - t[p];
        s += (double)r * (double)r * inv_n;
        uint4 z = make_uint4(0, 0, 0, 0);
        __nv_bfloat16 *e = reinterpret_cast<__nv_bfloat16 *>(&z);
        e[0] = __float2bfloat16_rn(sc * r);
        uint4 *dst = reinterpret_cast<uint4 *>(gy + (size_t)p * 16);
        dst[0] = z;
        dst[1] = make_uint4(0, 0, 0, 0);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// per-block channel sums of a bf16 [nvox][C] tensor (bias gradients), in a
// fixed order: thread t sums channel t % C over voxel lane t / C, then the
// lanes of each channel are added in lane order.
__global__ void k_channel_sums(const __nv_bfloat16 *__restrict__ g, int nvox, int C, float *__restrict__ part) {
    __shared__ float sm[256];
    const int lanes = blockDim.x / C;
    const int c = threadIdx.x % C, ln = threadIdx.x / C;
    float s = 0.0f;
    if (ln < lanes)
        for (int p = blockIdx.x * lanes + ln; p < nvox; p += gridDim.x * lanes) s += __bfloat162float(g[(size_t)p * C + c]);
    sm[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < C) {
        float t = 0.0f;
        for (int l = 0; l < lanes; ++l) t += sm[l * C + threadIdx.x];
        part[(size_t)blockIdx.x * C + threadIdx.x] = t;
    }
}

// sum of partials [nb][n] in block order -> out[n]
__global__ void k_sum_rows(const float *__restrict__ part, int nb, int n, float *__restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int b = 0; b < nb; ++b) s += part[(size_t)b * n + i];
        out[i] = s;
    }
}

// wgrad partials [27][nb][cout*cin] -> [27][cout*cin]
__global__ void k_sum_wgrad(const float *__restrict__ part, int nb, int m, float *__restrict__ out) {
    const int n = 27 * m;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int tap = i / m, e = i % m;
        float s = 0.0f;
        for (int b = 0; b < nb; ++b) s += part[((size_t)tap * nb + b) * m + e];
        out[i] = s;
    }
}

__global__ void k_adam(int n, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                       const int *__restrict__ live) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (live && !live[i]) continue;  // padding entries stay zero
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ---------------------------------------------------------------------------
// launch helpers (dispatch over the fixed layer shapes)
// ---------------------------------------------------------------------------
#include <cudaTypedefs.h>

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against libcuda), or NULL where the driver does not provide it
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess && f)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        else
            cudaGetLastError();
    }
    return fn;
}

// One tensor map per 8-channel chunk of a channels-last bf16 activation
// [B][D][H][W][CIN]: dimensions (8 channels, W, H, D, B), box (8, 10, 18,
// TZ + 2, 1) -- one chunk plane of a haloed brick -- zero fill outside.
// False where the encoder is missing or refuses (the caller then launches
// the cp.async kernel).
static bool conv_maps(const ConvArgs &a, int cin, ConvMaps *m) {
    auto enc = tensor_map_encoder();
    if (!enc || cin > 64 || cin % 8 || reinterpret_cast<uintptr_t>(a.in) % 16) return false;
    const cuuint64_t e = 2;  // bytes per element
    const cuuint64_t dims[5] = {8, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.D, (cuuint64_t)a.B};
    const cuuint64_t strides[4] = {cin * e, (cuuint64_t)a.W * cin * e, (cuuint64_t)a.H * a.W * cin * e,
                                   (cuuint64_t)a.D * a.H * a.W * cin * e};
    const cuuint32_t box[5] = {8, BK_XB, BK_YB, BK_ZB, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    for (int c = 0; c < cin / 8; ++c) {
        void *addr = const_cast<__nv_bfloat16 *>(a.in + c * 8);
        if (enc(&m->m[c], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, addr, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

#ifndef MGCT_CONV_WS
#define MGCT_CONV_WS 1
#endif

// persistent launch of the warp-specialised kernel (k_conv_ws): one block
// per SM times the blocks that fit; false if it does not apply
template <int CIN, int COUT, bool RELU, bool OUT_F32>
static bool conv_fwd_ws(const ConvArgs &a, int *err, cudaStream_t s, int *st) {
    using C = WsCfg<CIN, COUT>;
    ConvMaps maps;
    if (!MGCT_CONV_WS || !conv_maps(a, CIN, &maps)) return false;
    auto kern = k_conv_ws<CIN, COUT, RELU, OUT_F32>;
    static int per_sm = 0, nsm = 0;  // per instantiation
    if (!per_sm) {
        int dev = 0, occ = 0;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM) != cudaSuccess ||
            cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, WS_THREADS, C::SMEM) != cudaSuccess ||
            occ < 1) {
            cudaGetLastError();
            return false;
        }
        per_sm = std::min(occ, (int)(512 / C::NCOLS));
    }
    const int ntiles = brick_tiles(a.B, a.D, a.H, a.W).ntiles;
    *st = MGCT_OK;
    if (ntiles == 0) return true;
    const int grid = std::min(ntiles, nsm * per_sm);
    *st = [&]() -> int {
        MGCT_KERNEL(KK_CONV, s, kern<<<grid, WS_THREADS, C::SMEM, s>>>(a, maps, err));
        return MGCT_OK;
    }();
    return true;
}

// persistent launch of the brick kernel: one block per SM times the blocks
// that fit (shared memory, and the 512 tensor-memory columns of an SM)
template <int CIN, int COUT, bool RELU, bool OUT_F32>
static int conv_fwd_t(const ConvArgs &a, int *err, cudaStream_t s) {
    int st = MGCT_OK;
    if (conv_fwd_ws<CIN, COUT, RELU, OUT_F32>(a, err, s, &st)) return st;
    using C = BrickCfg<CIN, COUT>;
    auto kern = k_conv_brick_tc<CIN, COUT, RELU, OUT_F32>;
    static int per_sm = 0, nsm = 0;  // per instantiation
    if (!per_sm) {
        MGCT_TRY(check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM),
                            "conv smem"));
        int dev = 0, occ = 0;
        MGCT_TRY(check_cuda(cudaGetDevice(&dev), "conv device"));
        MGCT_TRY(check_cuda(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "conv SMs"));
        MGCT_TRY(check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 128, C::SMEM), "conv occupancy"));
        if (occ < 1) return set_error(MGCT_ECUDA, "convolution does not fit on an SM");
        per_sm = std::min(occ, (int)(512 / C::NCOLS));
    }
    const int ntiles = brick_tiles(a.B, a.D, a.H, a.W).ntiles;
    if (ntiles == 0) return MGCT_OK;
    const int grid = std::min(ntiles, nsm * per_sm);
    MGCT_KERNEL(KK_CONV, s, kern<<<grid, 128, C::SMEM, s>>>(a, err));
    return MGCT_OK;
}

static int conv_forward(int l, const ConvArgs &a, int *err, cudaStream_t s) {
    switch (l) {
        case 0: return conv_fwd_t<16, 16, true, false>(a, err, s);
        case 1: return conv_fwd_t<16, 32, true, false>(a, err, s);
        case 2: return conv_fwd_t<32, 64, true, false>(a, err, s);
        default: return conv_fwd_t<64, 16, false, true>(a, err, s);
    }
}

// backward data of layer l: forward shape (CIN' = COUT_l, COUT' = CIN_l)
static int conv_bwd_data(int l, const ConvArgs &a, int *err, cudaStream_t s) {
    switch (l) {
        case 1: return conv_fwd_t<32, 16, false, false>(a, err, s);
        case 2: return conv_fwd_t<64, 32, false, false>(a, err, s);
        case 3: return conv_fwd_t<16, 64, false, false>(a, err, s);
        default: return set_error(MGCT_EINVAL, "no data gradient for the input layer");
    }
}

constexpr int WG_PARTS = 152;  // most blocks per tap of the weight gradient (partial sums kept)
constexpr int NET_HALO = 4;    // planes each side a slab needs: four 3x3x3 layers

// weight gradient on tcgen05: persistent blocks, (SMs / tap groups) per tap
// group, capped at WG_PARTS; returns the number of partial sums per tap
template <int CIN, int COUT>
static int conv_wgrad_t(const __nv_bfloat16 *in, const __nv_bfloat16 *gout, float *part, int B, int D, int H, int W,
                        int *err, int *nparts, cudaStream_t s) {
    using C = WgCfg<CIN, COUT>;
    auto kern = k_conv_wgrad_tc<CIN, COUT, true>;
    static int nsm = 0;  // per instantiation
    if (!nsm) {
        MGCT_TRY(check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM),
                            "wgrad smem"));
        int dev = 0;
        MGCT_TRY(check_cuda(cudaGetDevice(&dev), "wgrad device"));
        MGCT_TRY(check_cuda(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "wgrad SMs"));
    }
    const int G = std::max(1, std::min(WG_PARTS, nsm / C::TG));
    *nparts = G;
    WgArgs a{in, gout, part, B, D, H, W};
    MGCT_KERNEL(KK_CONV, s, kern<<<dim3(G, C::TG), 128, C::SMEM, s>>>(a, err));
    return MGCT_OK;
}

static int conv_wgrad(int l, const __nv_bfloat16 *in, const __nv_bfloat16 *gout, float *part, int B, int D, int H,
                      int W, int *err, int *nparts, cudaStream_t s) {
    switch (l) {
        case 0: return conv_wgrad_t<16, 16>(in, gout, part, B, D, H, W, err, nparts, s);
        case 1: return conv_wgrad_t<16, 32>(in, gout, part, B, D, H, W, err, nparts, s);
        case 2: return conv_wgrad_t<32, 64>(in, gout, part, B, D, H, W, err, nparts, s);
        default: return conv_wgrad_t<64, 16>(in, gout, part, B, D, H, W, err, nparts, s);
    }
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
struct NetSpace {
    __nv_bfloat16 *x0, *act[NL];  // act[l] = output of layer l (l < 3), bf16
    float *xs, *y;                // scaled input, network output (float32)
    __nv_bfloat16 *g[NL];         // gradient wrt the input of layer l+1 ... (g[l]: [nvox][LCOUT[l]])
    float *wpart, *bpart;
    double *lpart, *sumsq;
};

static size_t carve_net(int64_t nvox, bool training, char *base, NetSpace *sp) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        off = (off + 255) & ~(size_t)255;
        char *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    NetSpace s;
    std::memset(&s, 0, sizeof(s));
    s.x0 = reinterpret_cast<__nv_bfloat16 *>(take((size_t)nvox * 16 * 2));
    for (int l = 0; l < NL - 1; ++l) s.act[l] = reinterpret_cast<__nv_bfloat16 *>(take((size_t)nvox * LCOUT[l] * 2));
    s.xs = reinterpret_cast<float *>(take((size_t)nvox * 4));
    s.y = reinterpret_cast<float *>(take((size_t)nvox * 4));
    s.sumsq = reinterpret_cast<double *>(take(64));
    s.lpart = reinterpret_cast<double *>(take(1024 * 8));
    if (training) {
        for (int l = 0; l < NL; ++l) s.g[l] = reinterpret_cast<__nv_bfloat16 *>(take((size_t)nvox * LCOUT[l] * 2));
        size_t mw = 0;
        for (int l = 0; l < NL; ++l) mw = std::max(mw, wcount(l));
        s.wpart = reinterpret_cast<float *>(take((size_t)WG_PARTS * mw * 4));
        s.bpart = reinterpret_cast<float *>(take((size_t)1024 * 64 * 4));
    }
    if (sp) *sp = s;
    return off + 256;
}

static int net_sumsq(const float *x, int nvox, double *out, double *lpart, cudaStream_t s);

}  // namespace mgct

using namespace mgct;

extern "C" {

size_t mgct_net_param_count(void) {
    size_t n = 0;
    for (int l = 0; l < NL; ++l) n += (size_t)27 * LCOUT_REAL[l] * LCIN_REAL[l] + LCOUT_REAL[l];
    return n;
}

size_t mgct_net_workspace_bytes(int64_t nvox, int training) {
    if (nvox <= 0) return 0;
    return carve_net(nvox, training != 0, nullptr, nullptr);
}

void mgct_net_destroy(mgct_net *net) {
    if (!net) return;
    for (int l = 0; l < NL; ++l) {
        void *ps[] = {net->w[l], net->b[l], net->mw[l], net->vw[l], net->mb[l], net->vb[l], net->gw[l], net->gb[l],
                      net->wf[l], net->wt[l]};
        for (void *p : ps)
            if (p) cudaFree(p);
    }
    if (net->loss) cudaFree(net->loss);
    if (net->err) cudaFree(net->err);
    delete net;
}

// Parameters are exchanged as float32, layer by layer: the real weights
// [27][cout_real][cin_real] (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)) then the
// real biases [cout_real].
int mgct_net_set_params(mgct_net *net, const float *host, size_t count) {
    if (!net || !host) return set_error(MGCT_EINVAL, "net and params must not be NULL");
    if (count != mgct_net_param_count()) return set_error(MGCT_ESHAPE, "wrong parameter count");
    size_t off = 0;
    for (int l = 0; l < NL; ++l) {
        std::vector<float> w(wcount(l), 0.0f), b(LCOUT[l], 0.0f);
        for (int tap = 0; tap < 27; ++tap)
            for (int co = 0; co < LCOUT_REAL[l]; ++co)
                for (int ci = 0; ci < LCIN_REAL[l]; ++ci)
                    w[((size_t)tap * LCOUT[l] + co) * LCIN[l] + ci] = host[off++];
        for (int co = 0; co < LCOUT_REAL[l]; ++co) b[co] = host[off++];
        MGCT_TRY(check_cuda(cudaMemcpy(net->w[l], w.data(), w.size() * 4, cudaMemcpyHostToDevice), "set params"));
        MGCT_TRY(check_cuda(cudaMemcpy(net->b[l], b.data(), b.size() * 4, cudaMemcpyHostToDevice), "set params"));
        k_pack_weights<<<64, 256>>>(net->w[l], net->wf[l], net->wt[l], LCOUT[l], LCIN[l]);
        count_launch();
        MGCT_LAUNCH_CHECK("pack weights");
    }
    return check_cuda(cudaDeviceSynchronize(), "set params");
}

static int get_tensors(const mgct_net *net, float *const *src_w, float *const *src_b, float *host) {
    size_t off = 0;
    for (int l = 0; l < NL; ++l) {
        std::vector<float> w(wcount(l)), b(LCOUT[l]);
        MGCT_TRY(check_cuda(cudaMemcpy(w.data(), src_w[l], w.size() * 4, cudaMemcpyDeviceToHost), "get params"));
        MGCT_TRY(check_cuda(cudaMemcpy(b.data(), src_b[l], b.size() * 4, cudaMemcpyDeviceToHost), "get params"));
        for (int tap = 0; tap < 27; ++tap)
            for (int co = 0; co < LCOUT_REAL[l]; ++co)
                for (int ci = 0; ci < LCIN_REAL[l]; ++ci) host[off++] = w[((size_t)tap * LCOUT[l] + co) * LCIN[l] + ci];
        for (int co = 0; co < LCOUT_REAL[l]; ++co) host[off++] = b[co];
    }
    return MGCT_OK;
}

int mgct_net_get_params(const mgct_net *net, float *host, size_t count) {
    if (!net || !host) return set_error(MGCT_EINVAL, "net and params must not be NULL");
    if (count != mgct_net_param_count()) return set_error(MGCT_ESHAPE, "wrong parameter count");
    return get_tensors(net, net->w, net->b, host);
}

int mgct_net_get_grads(const mgct_net *net, float *host, size_t count) {
    if (!net || !host) return set_error(MGCT_EINVAL, "net and grads must not be NULL");
    if (count != mgct_net_param_count()) return set_error(MGCT_ESHAPE, "wrong parameter count");
    MGCT_TRY(check_cuda(cudaDeviceSynchronize(), "get grads"));
    return get_tensors(net, net->gw, net->gb, host);
}

int mgct_net_create(uint64_t seed, mgct_net **out) {
    if (!out) return set_error(MGCT_EINVAL, "out must not be NULL");
    *out = nullptr;
    mgct_net *net = new mgct_net();
    std::memset(net, 0, sizeof(*net));
    int st = MGCT_OK;
    for (int l = 0; l < NL && !st; ++l) {
        const size_t nw = wcount(l) * 4, nb = (size_t)LCOUT[l] * 4;
        float **fl[] = {&net->w[l], &net->mw[l], &net->vw[l], &net->gw[l]};
        for (float **p : fl)
            if (!st) st = check_cuda(cudaMalloc(p, nw), "net alloc");
        float **fb[] = {&net->b[l], &net->mb[l], &net->vb[l], &net->gb[l]};
        for (float **p : fb)
            if (!st) st = check_cuda(cudaMalloc(p, nb), "net alloc");
        if (!st) st = check_cuda(cudaMalloc(&net->wf[l], wcount(l) * 2), "net alloc");
        if (!st) st = check_cuda(cudaMalloc(&net->wt[l], wcount(l) * 2), "net alloc");
        if (!st) {
            cudaMemset(net->mw[l], 0, nw);
            cudaMemset(net->vw[l], 0, nw);
            cudaMemset(net->gw[l], 0, nw);
            cudaMemset(net->mb[l], 0, nb);
            cudaMemset(net->vb[l], 0, nb);
            cudaMemset(net->gb[l], 0, nb);
        }
    }
    if (!st) st = check_cuda(cudaMalloc(&net->loss, 8), "net alloc");
    if (!st) st = check_cuda(cudaMalloc(&net->err, sizeof(int)), "net alloc");
    if (!st) st = check_cuda(cudaMemset(net->err, 0, sizeof(int)), "net alloc");
    if (st) {
        mgct_net_destroy(net);
        return st;
    }
    // He-normal initialisation (fan-in 27 cin_real), zero biases; the output
    // layer starts at zero so that the initial correction is none.
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    std::vector<float> params(mgct_net_param_count());
    size_t off = 0;
    for (int l = 0; l < NL; ++l) {
        const double sd = l == NL - 1 ? 0.0 : std::sqrt(2.0 / (27.0 * LCIN_REAL[l]));
        for (size_t i = 0; i < (size_t)27 * LCOUT_REAL[l] * LCIN_REAL[l]; ++i) params[off++] = (float)(sd * nd(rng));
        for (int co = 0; co < LCOUT_REAL[l]; ++co) params[off++] = 0.0f;
    }
    st = mgct_net_set_params(net, params.data(), params.size());
    if (st) {
        mgct_net_destroy(net);
        return st;
    }
    net->step = 0;
    *out = net;
    return MGCT_OK;
}

// forward pass on [B][D][H][W] voxels; x float32 [nvox]; scale: when
// `normalise`, x is divided by its RMS (computed here).  Leaves the
// activations in the workspace.
// ss: device sum of squares of the whole volume (x is scaled by 1 / RMS with
// RMS = sqrt(ss / nnorm)), or NULL for no scaling.
static int net_forward(const mgct_net *net, int B, int D, int H, int W, const float *x, const double *ss,
                       double nnorm, const NetSpace &sp, cudaStream_t s) {
    const int nvox = B * D * H * W;
    MGCT_KERNEL(KK_CONV, s, k_net_input<<<std::min((nvox + 255) / 256, 152 * 32), 256, 0, s>>>(x, ss, nnorm, nvox, sp.x0, sp.xs));
    const __nv_bfloat16 *cur = sp.x0;
    for (int l = 0; l < NL; ++l) {
        ConvArgs a;
        a.in = cur;
        a.w = net->wf[l];
        a.bias = net->b[l];
        a.mask = nullptr;
        a.B = B;
        a.D = D;
        a.H = H;
        a.W = W;
        a.nvox = nvox;
        if (l < NL - 1) {
            a.out = sp.act[l];
            a.out_ch = LCOUT[l];
            a.out_stride = LCOUT[l];
        } else {
            a.out = sp.y;
            a.out_ch = 1;
            a.out_stride = 1;
        }
        MGCT_TRY(conv_forward(l, a, net->err, s));
        if (l < NL - 1) cur = sp.act[l];
    }
    return MGCT_OK;
}

}  // extern "C"

namespace mgct {

__global__ void k_sumsq_f(const float *__restrict__ x, int n, double *__restrict__ part) {
    __shared__ double red[256];
    double s = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) s += (double)x[p] * x[p];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

static int net_sumsq(const float *x, int nvox, double *out, double *lpart, cudaStream_t s) {
    const int nb = std::min(1024, (nvox + 255) / 256);
    MGCT_KERNEL(KK_REDUCE, s, k_sumsq_f<<<nb, 256, 0, s>>>(x, nvox, lpart));
    return launch_sum_partials(lpart, nb, 1, out, s);
}

}  // namespace mgct

extern "C" {

int mgct_net_apply(const mgct_net *net, int B, int D, int H, int W, const float *dir, float *out, void *ws,
                   size_t ws_bytes, mgct_stream stream) {
    if (!net) return set_error(MGCT_EINVAL, "net is NULL");
    MGCT_TRY(check_ptr(dir, "dir"));
    MGCT_TRY(check_ptr(out, "out"));
    MGCT_TRY(check_ptr(ws, "workspace"));
    if (B < 1 || D < 1 || H < 1 || W < 1 || (int64_t)B * D * H * W > ((int64_t)1 << 31) - 1)
        return set_error(MGCT_ESHAPE, "bad volume dimensions");
    const int64_t nvox = (int64_t)B * D * H * W, plane = (int64_t)H * W;
    if (reinterpret_cast<uintptr_t>(ws) % 256) return set_error(MGCT_EALIGN, "net workspace must be 256-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    NetSpace sp;
    if (ws_bytes >= mgct_net_workspace_bytes(nvox, 0)) {
        carve_net(nvox, false, static_cast<char *>(ws), &sp);
        MGCT_TRY(net_sumsq(dir, (int)nvox, sp.sumsq, sp.lpart, s));
        MGCT_TRY(net_forward(net, B, D, H, W, dir, sp.sumsq, (double)nvox, sp, s));
        MGCT_KERNEL(KK_CONV, s, k_net_output<<<std::min((int)((nvox + 255) / 256), 152 * 32), 256, 0, s>>>(
                                    sp.xs, sp.y, sp.sumsq, (double)nvox, (int)nvox, net->err, out));
        return MGCT_OK;
    }
    // z-slabs of S planes, each computed on S + 2 NET_HALO planes: the four
    // 3x3x3 layers see NET_HALO planes on each side, so the slab's own planes
    // are exact (at the volume's faces the zero padding is the volume's own)
    int S = 0;
    for (int t = D; t >= 1; t = t > 64 ? t - t / 8 : t - 1)
        if (mgct_net_workspace_bytes(std::min<int64_t>(t + 2 * NET_HALO, D) * plane, 0) <= ws_bytes) {
            S = t;
            break;
        }
    if (S < 1) return set_error(MGCT_ENOMEM, "net workspace too small for one slab");
    carve_net(std::min<int64_t>(S + 2 * NET_HALO, D) * plane, false, static_cast<char *>(ws), &sp);
    MGCT_TRY(net_sumsq(dir, (int)nvox, sp.sumsq, sp.lpart, s));
    for (int b = 0; b < B; ++b) {
        for (int z0 = 0; z0 < D; z0 += S) {
            const int z1 = std::min(D, z0 + S);
            const int zs = std::max(0, z0 - NET_HALO), ze = std::min(D, z1 + NET_HALO);
            const int64_t base = ((int64_t)b * D + zs) * plane;
            MGCT_TRY(net_forward(net, 1, ze - zs, H, W, dir + base, sp.sumsq, (double)nvox, sp, s));
            const int64_t off = (int64_t)(z0 - zs) * plane, cnt = (int64_t)(z1 - z0) * plane;
            MGCT_KERNEL(KK_CONV, s, k_net_output<<<std::min((int)((cnt + 255) / 256), 152 * 32), 256, 0, s>>>(
                                        sp.xs + off, sp.y + off, sp.sumsq, (double)nvox, (int)cnt, net->err,
                                        out + ((int64_t)b * D + z0) * plane));
        }
    }
    return MGCT_OK;
}

int mgct_net_forward_backward(mgct_net *net, int B, int D, int H, int W, const float *x, const float *t, void *ws,
                              size_t ws_bytes, double *loss, mgct_stream stream) {
    if (!net) return set_error(MGCT_EINVAL, "net is NULL");
    MGCT_TRY(check_ptr(x, "x"));
    MGCT_TRY(check_ptr(t, "t"));
    MGCT_TRY(check_ptr(ws, "workspace"));
    if (B < 1 || D < 1 || H < 1 || W < 1 || (int64_t)B * D * H * W > ((int64_t)1 << 31) - 1)
        return set_error(MGCT_ESHAPE, "bad volume dimensions");
    const int nvox = B * D * H * W;
    if (reinterpret_cast<uintptr_t>(ws) % 256 || ws_bytes < mgct_net_workspace_bytes(nvox, 1))
        return set_error(MGCT_ENOMEM, "net workspace too small or misaligned");
    NetSpace sp;
    carve_net(nvox, true, static_cast<char *>(ws), &sp);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // x and t are already in scaled units
    MGCT_TRY(net_forward(net, B, D, H, W, x, nullptr, 1.0, sp, s));
    const int nb = std::min(1024, (nvox + 255) / 256);
    MGCT_KERNEL(KK_CONV, s, k_mse<<<nb, 256, 0, s>>>(sp.xs, sp.y, t, nvox, net->err, sp.g[NL - 1], sp.lpart));
    MGCT_TRY(launch_sum_partials(sp.lpart, nb, 1, net->loss, s));
    // backward through the layers; g[l] = dL/d(output of layer l)
    for (int l = NL - 1; l >= 0; --l) {
        const __nv_bfloat16 *lin = l == 0 ? sp.x0 : sp.act[l - 1];
        int nparts = 0;
        MGCT_TRY(conv_wgrad(l, lin, sp.g[l], sp.wpart, B, D, H, W, net->err, &nparts, s));
        const int m = LCOUT[l] * LCIN[l];
        MGCT_KERNEL(KK_CONV, s, k_sum_wgrad<<<(27 * m + 255) / 256, 256, 0, s>>>(sp.wpart, nparts, m, net->gw[l]));
        const int cb = std::min(1024, (nvox + 255) / 256);
        MGCT_KERNEL(KK_CONV, s, k_channel_sums<<<cb, 256, 0, s>>>(sp.g[l], nvox, LCOUT[l], sp.bpart));
        MGCT_KERNEL(KK_CONV, s, k_sum_rows<<<1, 64, 0, s>>>(sp.bpart, cb, LCOUT[l], net->gb[l]));
        if (l > 0) {
            ConvArgs a;
            a.in = sp.g[l];
            a.w = net->wt[l];
            a.bias = nullptr;
            a.mask = sp.act[l - 1];  // ReLU of the previous layer
            a.out = sp.g[l - 1];
            a.B = B;
            a.D = D;
            a.H = H;
            a.W = W;
            a.nvox = nvox;
            a.out_ch = LCIN[l];
            a.out_stride = LCIN[l];
            MGCT_TRY(conv_bwd_data(l, a, net->err, s));
        }
    }
    if (loss) MGCT_TRY(check_cuda(cudaMemcpyAsync(loss, net->loss, 8, cudaMemcpyDeviceToDevice, s), "loss copy"));
    return MGCT_OK;
}

int mgct_net_check(const mgct_net *net, mgct_stream stream) {
    if (!net) return set_error(MGCT_EINVAL, "net is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int flag = 0;
    MGCT_TRY(check_cuda(cudaMemcpyAsync(&flag, net->err, sizeof(int), cudaMemcpyDeviceToHost, s), "net check"));
    MGCT_TRY(check_cuda(cudaStreamSynchronize(s), "net check"));
    if (!flag) return MGCT_OK;
    MGCT_TRY(check_cuda(cudaMemsetAsync(net->err, 0, sizeof(int), s), "net check"));
    return set_error(MGCT_ETIMEOUT, "a tensor-core convolution gave up waiting for its MMAs");
}

int mgct_net_adam_step(mgct_net *net, double lr, mgct_stream stream) {
    if (!net) return set_error(MGCT_EINVAL, "net is NULL");
    if (!(lr >= 0.0)) return set_error(MGCT_EINVAL, "lr must be >= 0");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    net->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)net->step));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)net->step));
    for (int l = 0; l < NL; ++l) {
        const int nw = (int)wcount(l);
        MGCT_KERNEL(KK_UPDATE, s, k_adam<<<(nw + 255) / 256, 256, 0, s>>>(nw, net->w[l], net->gw[l], net->mw[l], net->vw[l], (float)lr, b1, b2, eps, c1, c2, nullptr));
        MGCT_KERNEL(KK_UPDATE, s, k_adam<<<1, 64, 0, s>>>(LCOUT[l], net->b[l], net->gb[l], net->mb[l], net->vb[l], (float)lr, b1, b2, eps, c1, c2, nullptr));
        MGCT_KERNEL(KK_UPDATE, s, k_pack_weights<<<64, 256, 0, s>>>(net->w[l], net->wf[l], net->wt[l], LCOUT[l], LCIN[l]));
    }
    return MGCT_OK;
}

}  // extern "C"
