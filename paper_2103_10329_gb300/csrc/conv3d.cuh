// 3x3x3 convolutions (stride 1, zero padding 1) as implicit GEMMs on the
// BF16 tensor cores with float32 accumulation -- the layers of the learned
// preconditioner correction.  Activations are channels-last, [voxel][C]
// with voxel = ((b D + z) H + y) W + x; weights are [tap][Cout][Cin] with
// tap = (dz+1)*9 + (dy+1)*3 + (dx+1).
//
//   forward:      out[p][co]  = sum_{tap,ci} in[p + tap][ci] w[tap][co][ci] + bias[co]
//   backward data: gin[p][ci] = sum_{tap,co} gout[p - tap][co] w[tap][co][ci]
//                 = the forward with weights wT[26 - tap][ci][co]
//   weight grad:  dw[tap][co][ci] = sum_p gout[p][co] in[p + tap][ci]
//
// This header holds the shared argument block and the weight gradient
// (mma.sync m16n8k16, bf16 x bf16 -> f32); the forward and backward-data
// convolutions run on tcgen05 (conv3d_tc.cuh).
#pragma once

#include "common.cuh"

namespace mgct {

struct ConvArgs {
    const __nv_bfloat16 *in;   // [nvox][CIN]
    const __nv_bfloat16 *w;    // [27][COUT][CIN]
    const float *bias;         // [COUT] or NULL
    void *out;                 // [nvox][out_stride] (bf16) or [nvox] (float, channel 0 only)
    const __nv_bfloat16 *mask; // [nvox][COUT] or NULL: zero the output where mask <= 0
    int B, D, H, W;
    int nvox;
    int out_ch;                // output channels written (<= COUT)
    int out_stride;            // channels per voxel in out (bf16 output)
};

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld_u32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ void decode_voxel(int p, int W, int H, int D, int &b, int &z, int &y, int &x) {
    x = p % W;
    int t = p / W;
    y = t % H;
    t /= H;
    z = t % D;
    b = t / D;
}

constexpr int CV_M = 128;  // voxels per block (4 warps x 2 m16 tiles)

// Weight gradient, one tap per blockIdx.y; each block loops over voxel tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... and writes its partial
// part[tap][blockIdx.x][COUT][CIN] (float32); a second pass sums the
// partials in block order.  GEMM: M = COUT (rows of gout^T), N = CIN, K =
// voxels; the tiles are staged transposed ([channel][voxel]) so that the
// fragments' k-pairs are contiguous.
template <int CIN, int COUT>
__global__ void __launch_bounds__(128) k_conv_wgrad(const __nv_bfloat16 *__restrict__ in,
                                                   const __nv_bfloat16 *__restrict__ gout, float *__restrict__ part,
                                                   int B, int D, int H, int W, int nvox) {
    constexpr int KP = CV_M + 8;
    __shared__ __align__(16) __nv_bfloat16 Xs[CIN][KP];   // in at p + tap, transposed
    static_assert(COUT % 16 == 0 && CIN % 16 == 0, "channel padding");
    __shared__ __align__(16) __nv_bfloat16 Gs[COUT][KP];  // gout at p, transposed
    constexpr int MT = COUT / 16;                         // m16 tiles
    constexpr int NT = CIN / 8;
    constexpr int TILES = MT * NT;
    constexpr int PER_WARP = (TILES + 3) / 4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int tap = blockIdx.y;
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    float acc[PER_WARP][4];
#pragma unroll
    for (int i = 0; i < PER_WARP; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = 0.0f;
    const int ntiles = (nvox + CV_M - 1) / CV_M;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int p0 = tile * CV_M;
        __syncthreads();
        for (int idx = tid; idx < CV_M * (CIN / 8); idx += 128) {
            const int r = idx / (CIN / 8), ch = idx % (CIN / 8);
            const int p = p0 + r;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (p < nvox) {
                int b, z, y, x;
                decode_voxel(p, W, H, D, b, z, y, x);
                z += dz;
                y += dy;
                x += dx;
                if ((unsigned)z < (unsigned)D && (unsigned)y < (unsigned)H && (unsigned)x < (unsigned)W) {
                    const size_t q = (((size_t)b * D + z) * H + y) * W + x;
                    v = *reinterpret_cast<const uint4 *>(in + q * CIN + ch * 8);
                }
            }
            const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) Xs[ch * 8 + j][r] = e[j];
        }
        for (int idx = tid; idx < CV_M * (COUT / 8); idx += 128) {
            const int r = idx / (COUT / 8), ch = idx % (COUT / 8);
            const int p = p0 + r;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (p < nvox) v = *reinterpret_cast<const uint4 *>(gout + (size_t)p * COUT + ch * 8);
            const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) Gs[ch * 8 + j][r] = e[j];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < PER_WARP; ++i) {
            const int tl = warp * PER_WARP + i;
            if (tl >= TILES) break;
            const int mt = tl / NT, nt = tl % NT;
#pragma unroll
            for (int kc = 0; kc < CV_M / 16; ++kc) {
                uint32_t af[4], bf[2];
                af[0] = ld_u32(&Gs[mt * 16 + g][kc * 16 + 2 * t4]);
                af[1] = ld_u32(&Gs[mt * 16 + g + 8][kc * 16 + 2 * t4]);
                af[2] = ld_u32(&Gs[mt * 16 + g][kc * 16 + 2 * t4 + 8]);
                af[3] = ld_u32(&Gs[mt * 16 + g + 8][kc * 16 + 2 * t4 + 8]);
                bf[0] = ld_u32(&Xs[nt * 8 + g][kc * 16 + 2 * t4]);
                bf[1] = ld_u32(&Xs[nt * 8 + g][kc * 16 + 2 * t4 + 8]);
                mma_bf16_16816(acc[i], af, bf);
            }
        }
    }
    float *o = part + ((size_t)tap * gridDim.x + blockIdx.x) * COUT * CIN;
#pragma unroll
    for (int i = 0; i < PER_WARP; ++i) {
        const int tl = warp * PER_WARP + i;
        if (tl >= TILES) break;
        const int mt = tl / NT, nt = tl % NT;
#pragma unroll
        for (int hr = 0; hr < 2; ++hr)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int co = mt * 16 + g + hr * 8, ci = nt * 8 + 2 * t4 + j;
                o[co * CIN + ci] = acc[i][hr * 2 + j];
            }
    }
}

}  // namespace mgct
