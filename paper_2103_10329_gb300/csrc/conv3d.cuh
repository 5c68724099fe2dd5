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
// This header holds the convolutions' argument block; all three run on
// tcgen05 (conv3d_tc.cuh).
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

}  // namespace mgct
