// 3x3x3 convolution forward (and, with transposed flipped weights, backward
// data) on the 5th-generation tensor cores: tcgen05.mma of kind::f16 with
// BF16 operands staged in shared memory and the float32 accumulator in tensor
// memory, read back with tcgen05.ld for the epilogue.  The implicit GEMM has
// rows = output voxels, columns = Cout, k = 27 taps x Cin; the layout of the
// operands and the pipeline are described at k_conv_brick_tc below.
#pragma once

#include <cuda.h>

#include "conv3d.cuh"

namespace mgct {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    // start address, leading / stride byte offsets (all >> 4), descriptor
    // version 1 (bits 46-47), no swizzle (bits 61-63 = 0)
    return (uint64_t)((addr >> 4) & 0x3fff) | ((uint64_t)((lbo >> 4) & 0x3fff) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fff) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: D float32, A and B bf16, both K-major.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for the completion of the phase with this parity: gives up
// after `limit` SM clock cycles (the default, 2^31, is about a second at
// 2 GHz) and returns false, so that a block whose MMAs never complete reports
// it instead of hanging.
constexpr long long MBAR_WAIT_CYCLES = 1LL << 31;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t parity,
                                                  long long limit = MBAR_WAIT_CYCLES) {
    const long long t0 = clock64();
    while (!mbar_try_wait(mbar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) in a K-major core-matrix tile with `kc`
// core columns (kc = K / 8).
__device__ __forceinline__ uint32_t core_off(int row, int k8, int kc) {
    return (uint32_t)(((row >> 3) * kc + k8) * 128 + (row & 7) * 16);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    // 16-byte global -> shared copy; src-size 0 writes zeros (the padding)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// Haloed-brick implicit GEMM.
//
// An output tile is TZ x 16 x 8 voxels (z, y, x); each of its z planes is one
// M = 128 MMA row block (row r = voxel (y0 + r / 8, x0 + r % 8)).  The block
// copies the tile's input brick -- (TZ + 2) x 18 x 10 voxels with the halo,
// zero outside the volume -- into shared memory ONCE, stored per 8-channel
// chunk as rows of 16 bytes in (z, y, x) order.  Because 8 consecutive x
// rows are 8 consecutive 16-byte rows, every shifted window the 27 taps need
// is itself a K-major core-matrix operand: the tap only moves the descriptor's
// start address by ((dz * 18 + dy) * 10 + dx) * 16 bytes; the stride byte
// offset (next 8 rows = next y) is 10 * 16 bytes and the leading byte offset
// (next 8 channels) is the chunk plane.  The weights of all 27 taps stay in
// shared memory for the life of the (persistent) block.
//
// Channels are consumed in units of CU = min(Cin, 32); a tile is NU = Cin/CU
// units.  Two brick buffers and two accumulator slots in tensor memory: the
// copy of unit k + 1 and the epilogue of tile j - 1 overlap the MMAs of unit
// k (tile j).  tcgen05.commit of unit k arrives on mbar[k & 1]; unit k is the
// (k >> 1)-th arrival there, so its completion is the phase of parity
// (k >> 1) & 1.  Every wait is bounded: on expiry the block sets *err, drains
// what it issued, frees its tensor memory and returns.
// ---------------------------------------------------------------------------
constexpr int BK_TZ = 2, BK_TY = 16, BK_TX = 8;
constexpr int BK_ZB = BK_TZ + 2, BK_YB = BK_TY + 2, BK_XB = BK_TX + 2;
constexpr int BK_ROWS = BK_ZB * BK_YB * BK_XB;  // 720 brick voxels
constexpr uint32_t BK_CSTR = BK_ROWS * 16;      // bytes per 8-channel chunk plane

template <int CIN, int COUT>
struct BrickCfg {
    static constexpr int CU = CIN < 32 ? CIN : 32;   // channels per unit
    static constexpr int NU = CIN / CU;              // units per tile
    static constexpr int CC = CU / 8;                // chunks per unit
    static constexpr int KC = CIN / 8;               // chunks per weight row
    static constexpr uint32_t W_BYTES = 27u * COUT * CIN * 2;
    static constexpr uint32_t BRICK_BYTES = CC * BK_CSTR;
    static constexpr uint32_t SMEM = W_BYTES + 2 * BRICK_BYTES + 1024;  // + alignment slack
    static constexpr uint32_t ACC_COLS = BK_TZ * COUT;                   // one accumulator slot
    static constexpr uint32_t NCOLS = 2 * ACC_COLS < 32 ? 32 : 2 * ACC_COLS;
};

struct BrickTiles {
    int ntx, nty, ntz, ntiles;
};

__host__ __device__ inline BrickTiles brick_tiles(int B, int D, int H, int W) {
    BrickTiles t;
    t.ntx = (W + BK_TX - 1) / BK_TX;
    t.nty = (H + BK_TY - 1) / BK_TY;
    t.ntz = (D + BK_TZ - 1) / BK_TZ;
    t.ntiles = B * t.ntz * t.nty * t.ntx;
    return t;
}

template <int CIN, int COUT, bool RELU, bool OUT_F32>
__global__ void __launch_bounds__(128) k_conv_brick_tc(ConvArgs a, int *err) {
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 256, "tcgen05 shape");
    using C = BrickCfg<CIN, COUT>;
    constexpr uint32_t IDESC = tc_idesc_bf16(128, COUT);
    extern __shared__ unsigned char dsm[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
    const uint32_t w_s = smem_u32(base);
    const uint32_t brick_s = w_s + C::W_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const BrickTiles T = brick_tiles(a.B, a.D, a.H, a.W);
    const int my_tiles = blockIdx.x < T.ntiles ? (T.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int total = my_tiles * C::NU;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(C::NCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // tile j of this block -> origin (b, z0, y0, x0)
    auto tile_origin = [&](int j, int &b, int &z0, int &y0, int &x0) {
        int t = blockIdx.x + j * gridDim.x;
        x0 = (t % T.ntx) * BK_TX;
        t /= T.ntx;
        y0 = (t % T.nty) * BK_TY;
        t /= T.nty;
        z0 = (t % T.ntz) * BK_TZ;
        b = t / T.ntz;
    };
    // copy unit k (tile k / NU, channels (k % NU) * CU ..) into brick buffer k & 1
    auto load_unit = [&](int k) {
        int b, z0, y0, x0;
        tile_origin(k / C::NU, b, z0, y0, x0);
        const int c0 = (k % C::NU) * C::CU;
        const uint32_t dst = brick_s + (k & 1) * C::BRICK_BYTES;
        for (int idx = tid; idx < BK_ROWS * C::CC; idx += 128) {
            const int row = idx / C::CC, ch = idx % C::CC;
            const int xx = row % BK_XB, yy = (row / BK_XB) % BK_YB, zz = row / (BK_XB * BK_YB);
            const int z = z0 - 1 + zz, y = y0 - 1 + yy, x = x0 - 1 + xx;
            const bool valid =
                (unsigned)z < (unsigned)a.D && (unsigned)y < (unsigned)a.H && (unsigned)x < (unsigned)a.W;
            const size_t q = valid ? (((size_t)b * a.D + z) * a.H + y) * a.W + x : 0;
            cp_async16(dst + ch * BK_CSTR + row * 16, a.in + q * CIN + c0 + ch * 8, valid);
        }
    };
    // MMAs of unit k into accumulator slot (k / NU) & 1
    auto issue_unit = [&](int k) {
        const int u = k % C::NU;
        const uint32_t acc0 = tmem + ((k / C::NU) & 1) * C::ACC_COLS;
        const uint64_t adesc0 = tc_smem_desc(brick_s + (k & 1) * C::BRICK_BYTES, BK_CSTR, BK_XB * 16);
        const uint64_t bdesc0 = tc_smem_desc(w_s + u * C::CC * 128, 128, C::KC * 128);
#pragma unroll
        for (int zz = 0; zz < BK_TZ; ++zz) {
#pragma unroll
            for (int tap = 0; tap < 27; ++tap) {
                const uint32_t aoff = (((zz + tap / 9) * BK_YB + (tap / 3) % 3) * BK_XB + tap % 3) * 16;
#pragma unroll
                for (int c = 0; c < C::CU / 16; ++c) {
                    const uint64_t ad = adesc0 + ((aoff + c * 2 * BK_CSTR) >> 4);
                    const uint64_t bd = bdesc0 + ((tap * COUT * CIN * 2 + c * 256) >> 4);
                    tc_mma(acc0 + zz * COUT, ad, bd, IDESC, (u > 0 || tap > 0 || c > 0) ? 1u : 0u);
                }
            }
        }
        tc_commit(&mbar[k & 1]);
    };
    // accumulator slot of tile j -> bias, activation, mask, store
    auto epilogue = [&](int j) {
        int b, z0, y0, x0;
        tile_origin(j, b, z0, y0, x0);
        const int y = y0 + warp * 4 + (lane >> 3), x = x0 + (lane & 7);
        const bool vec = !OUT_F32 && a.out_ch == COUT && (a.out_stride & 7) == 0;
#pragma unroll
        for (int zz = 0; zz < BK_TZ; ++zz) {
            const int z = z0 + zz;
            const bool inside = z < a.D && y < a.H && x < a.W;
            const size_t p = inside ? (((size_t)b * a.D + z) * a.H + y) * a.W + x : 0;
#pragma unroll
            for (int c0 = 0; c0 < (OUT_F32 ? 16 : COUT); c0 += 16) {
                float v[16];
                tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (j & 1) * C::ACC_COLS + zz * COUT + c0, v);
                if (!inside) continue;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    float t = v[i] + (a.bias ? a.bias[c0 + i] : 0.0f);
                    if (RELU) t = fmaxf(t, 0.0f);
                    v[i] = t;
                }
                if (a.mask) {
                    const uint4 *mp = reinterpret_cast<const uint4 *>(a.mask + p * COUT + c0);
                    uint4 m4[2] = {mp[0], mp[1]};
                    const __nv_bfloat16 *m = reinterpret_cast<const __nv_bfloat16 *>(m4);
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (!(__bfloat162float(m[i]) > 0.0f)) v[i] = 0.0f;
                }
                if (OUT_F32) {
                    static_cast<float *>(a.out)[p] = v[0];
                } else if (vec) {
                    uint4 o[2];
                    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(o);
#pragma unroll
                    for (int i = 0; i < 8; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
                    uint4 *op = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(a.out) + p * a.out_stride + c0);
                    op[0] = o[0];
                    op[1] = o[1];
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (c0 + i < a.out_ch)
                            static_cast<__nv_bfloat16 *>(a.out)[p * a.out_stride + c0 + i] = __float2bfloat16_rn(v[i]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    };

    bool ok = true;
    int done = -1;    // last unit whose MMAs are known complete
    int issued = 0;   // units whose MMAs have been issued
    if (total > 0) {
        // all 27 taps' weights, in the K-major core-matrix layout, with unit 0
        for (int idx = tid; idx < 27 * COUT * C::KC; idx += 128) {
            const int k8 = idx % C::KC, co = (idx / C::KC) % COUT, tap = idx / (C::KC * COUT);
            cp_async16(w_s + tap * COUT * CIN * 2 + core_off(co, k8, C::KC), a.w + ((size_t)tap * COUT + co) * CIN + k8 * 8,
                       true);
        }
        load_unit(0);
        cp_async_commit();
    }
    for (int k = 0; k < total; ++k) {
        cp_async_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        ok = __syncthreads_and(ok);
        if (!ok) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            issue_unit(k);
        }
        issued = k + 1;
        if (k >= 1) {
            // warp-uniform outcome: the epilogue's tcgen05.ld is warp-collective
            ok = __all_sync(0xffffffffu, ok && mbar_wait_bounded(&mbar[(k - 1) & 1], (uint32_t)(((k - 1) >> 1) & 1)));
            if (ok) done = k - 1;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (k + 1 < total) {
            load_unit(k + 1);
            cp_async_commit();
        }
        if (ok && k % C::NU == 0 && k >= 1) epilogue(k / C::NU - 1);
    }
    if (ok && total > 0) {
        if (__all_sync(0xffffffffu, mbar_wait_bounded(&mbar[(total - 1) & 1], (uint32_t)(((total - 1) >> 1) & 1)))) {
            done = total - 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            epilogue(my_tiles - 1);
        } else {
            ok = false;
        }
    }
    cp_async_wait<0>();
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        // the MMAs issued after the last completed unit must end before the
        // tensor memory is freed; completions arrive in issue order
        const int last = issued - 1;
        if (tid == 0 && last > done) mbar_wait_bounded(&mbar[last & 1], (uint32_t)((last >> 1) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::NCOLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Warp-specialised form of the haloed-brick implicit GEMM (same tiles, same
// operand layout, same epilogue as k_conv_brick_tc).
//
//   warp 0      producer: one lane loads each unit's brick with the tensor
//               memory accelerator -- per 8-channel chunk one 5-D box
//               (8 channels, 10 x, 18 y, 4 z, 1 volume) of a tensor map over
//               that chunk's channels, zero-filled outside the volume, which
//               is the convolution's padding -- into a ring of S stages;
//   warp 1      MMA issuer: one lane issues the unit's tcgen05.mma (27 taps x
//               TZ planes, K = 16 channels each) once its stage is full,
//               commits the stage back to the producer and, at a tile's last
//               unit, the accumulator slot to the epilogue;
//   warps 2..5  epilogue: read an accumulator slot from tensor memory (warp w
//               owns lanes 32 (w % 4) ..), add bias, activate, mask, store,
//               and hand the slot back.
// Units are 16 channels (CU), so a 110 KB weight set still leaves room for
// five stages.  Barriers: full[s] (expect-tx by the producer, completed by
// the copy), empty[s] and accf[slot] (tcgen05.commit), acce[slot] (128
// epilogue arrivals).  Unit k uses stage k % S, whose (k / S)-th phase it is;
// tile j uses slot j & 1, its (j >> 1)-th phase.  Every wait is bounded: a
// role whose wait expires sets the block's flag and *err and stops; before
// the tensor memory is freed the issuer waits for its last MMAs and the
// producer for its outstanding copies.
// ---------------------------------------------------------------------------
constexpr int WS_THREADS = 192;
#ifndef MGCT_CONV_TAPOUTER
#define MGCT_CONV_TAPOUTER 1
#endif
constexpr uint32_t WS_SMEM_MAX = 232448;  // 227 KB per block

struct ConvMaps {
    CUtensorMap m[8];  // one per 8-channel chunk of the input (Cin <= 64)
};

template <int CIN, int COUT>
struct WsCfg {
    static constexpr int CU = 16;          // channels per unit
    static constexpr int NU = CIN / CU;    // units per tile
    static constexpr int CC = CU / 8;      // chunks per unit
    static constexpr int KC = CIN / 8;     // chunks per weight row
    static constexpr uint32_t W_BYTES = 27u * COUT * CIN * 2;
    static constexpr uint32_t BRICK_BYTES = CC * BK_CSTR;
    static constexpr int S_FIT = (int)((WS_SMEM_MAX - W_BYTES - 1024 - 256) / BRICK_BYTES);
    static constexpr int S = S_FIT < 6 ? S_FIT : 6;  // stages
    static constexpr uint32_t SMEM = W_BYTES + S * BRICK_BYTES + 1024;  // + alignment slack
    static constexpr uint32_t ACC_COLS = BK_TZ * COUT;
    static constexpr uint32_t NCOLS = 2 * ACC_COLS < 32 ? 32 : 2 * ACC_COLS;
};

__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
// 5-D tiled copy global -> shared (coordinates innermost first), completing
// `bytes` of the barrier's expected transaction count
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            int c4, uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(mbar))
        : "memory");
}

template <int CIN, int COUT, bool RELU, bool OUT_F32>
__global__ void __launch_bounds__(WS_THREADS) k_conv_ws(ConvArgs a, const __grid_constant__ ConvMaps maps, int *err) {
    static_assert(CIN % 16 == 0 && CIN <= 64 && COUT % 16 == 0 && COUT <= 256, "tcgen05 shape");
    using C = WsCfg<CIN, COUT>;
    static_assert(C::S >= 2, "at least two stages");
    constexpr uint32_t IDESC = tc_idesc_bf16(128, COUT);
    extern __shared__ unsigned char dsm[];
    __shared__ __align__(8) uint64_t full[C::S], empty[C::S], accf[2], acce[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int fail;
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
    const uint32_t w_s = smem_u32(base);
    const uint32_t brick_s = w_s + C::W_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const BrickTiles T = brick_tiles(a.B, a.D, a.H, a.W);
    const int my_tiles = blockIdx.x < T.ntiles ? (T.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int total = my_tiles * C::NU;
    volatile int *vfail = &fail;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(C::NCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < C::S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&accf[q], 1);
            mbar_init(&acce[q], 128);
        }
        fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // all 27 taps' weights, in the K-major core-matrix layout
    if (total > 0) {
        for (int idx = tid; idx < 27 * COUT * C::KC; idx += WS_THREADS) {
            const int k8 = idx % C::KC, co = (idx / C::KC) % COUT, tap = idx / (C::KC * COUT);
            cp_async16(w_s + tap * COUT * CIN * 2 + core_off(co, k8, C::KC),
                       a.w + ((size_t)tap * COUT + co) * CIN + k8 * 8, true);
        }
        cp_async_commit();
    }
    cp_async_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    auto tile_origin = [&](int j, int &b, int &z0, int &y0, int &x0) {
        int t = blockIdx.x + j * gridDim.x;
        x0 = (t % T.ntx) * BK_TX;
        t /= T.ntx;
        y0 = (t % T.nty) * BK_TY;
        t /= T.nty;
        z0 = (t % T.ntz) * BK_TZ;
        b = t / T.ntz;
    };
    auto give_up = [&]() {
        *vfail = 1;
        atomicExch(err, 1);
    };

    if (warp == 0) {
        // ---------------- producer ----------------
        if (lane == 0) {
            int issued = 0;
            for (int k = 0; k < total; ++k) {
                const int s = k % C::S;
                if (k >= C::S && !mbar_wait_bounded(&empty[s], (uint32_t)((k / C::S - 1) & 1))) {
                    give_up();
                    break;
                }
                if (*vfail) break;
                int b, z0, y0, x0;
                tile_origin(k / C::NU, b, z0, y0, x0);
                const int ch0 = (k % C::NU) * C::CC;
                mbar_expect_tx(&full[s], C::BRICK_BYTES);
#pragma unroll
                for (int cc = 0; cc < C::CC; ++cc)
                    tma_load_5d(brick_s + s * C::BRICK_BYTES + cc * BK_CSTR, &maps.m[ch0 + cc], 0, x0 - 1, y0 - 1,
                                z0 - 1, b, &full[s]);
                issued = k + 1;
            }
            // copies still in flight must land before the block exits
            for (int k = issued - C::S > 0 ? issued - C::S : 0; k < issued; ++k)
                mbar_wait_bounded(&full[k % C::S], (uint32_t)((k / C::S) & 1));
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int issued = 0;
            for (int k = 0; k < total; ++k) {
                const int s = k % C::S, j = k / C::NU, u = k % C::NU, slot = j & 1;
                if (u == 0 && j >= 2 && !mbar_wait_bounded(&acce[slot], (uint32_t)(((j >> 1) - 1) & 1))) {
                    give_up();
                    break;
                }
                if (!mbar_wait_bounded(&full[s], (uint32_t)((k / C::S) & 1))) {
                    give_up();
                    break;
                }
                if (*vfail) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc0 = tmem + slot * C::ACC_COLS;
                const uint64_t adesc0 = tc_smem_desc(brick_s + s * C::BRICK_BYTES, BK_CSTR, BK_XB * 16);
                const uint64_t bdesc0 = tc_smem_desc(w_s + u * C::CC * 128, 128, C::KC * 128);
#pragma unroll
                for (int o = 0; o < BK_TZ * 27; ++o) {
                    // MGCT_CONV_TAPOUTER: the planes' accumulators alternate, tap by tap
                    const int zz = MGCT_CONV_TAPOUTER ? o % BK_TZ : o / 27;
                    const int tap = MGCT_CONV_TAPOUTER ? o / BK_TZ : o % 27;
                    const uint32_t aoff = (((zz + tap / 9) * BK_YB + (tap / 3) % 3) * BK_XB + tap % 3) * 16;
                    const uint64_t ad = adesc0 + (aoff >> 4);
                    const uint64_t bd = bdesc0 + ((tap * COUT * CIN * 2) >> 4);
                    tc_mma(acc0 + zz * COUT, ad, bd, IDESC, (u > 0 || tap > 0) ? 1u : 0u);
                }
                tc_commit(&empty[s]);
                if (u == C::NU - 1) tc_commit(&accf[slot]);
                issued = k + 1;
            }
            // the MMAs issued must end before the tensor memory is freed;
            // completions arrive in issue order
            if (issued > 0) mbar_wait_bounded(&empty[(issued - 1) % C::S], (uint32_t)(((issued - 1) / C::S) & 1));
        }
    } else {
        // ---------------- epilogue ----------------
        const int ew = warp & 3;  // tensor-memory lane quarter of this warp
        const bool vec = !OUT_F32 && a.out_ch == COUT && (a.out_stride & 7) == 0;
        for (int j = 0; j < my_tiles; ++j) {
            const int slot = j & 1;
            const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&accf[slot], (uint32_t)((j >> 1) & 1)));
            // warp-uniform: the tensor-memory loads below are warp-collective
            if (__any_sync(0xffffffffu, !ok || *vfail)) {
                if (!ok && lane == 0) give_up();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int b, z0, y0, x0;
            tile_origin(j, b, z0, y0, x0);
            const int y = y0 + ew * 4 + (lane >> 3), x = x0 + (lane & 7);
#pragma unroll
            for (int zz = 0; zz < BK_TZ; ++zz) {
                const int z = z0 + zz;
                const bool inside = z < a.D && y < a.H && x < a.W;
                const size_t p = inside ? (((size_t)b * a.D + z) * a.H + y) * a.W + x : 0;
#pragma unroll
                for (int c0 = 0; c0 < (OUT_F32 ? 16 : COUT); c0 += 16) {
                    float v[16];
                    tc_ld16(tmem + ((uint32_t)(ew * 32) << 16) + slot * C::ACC_COLS + zz * COUT + c0, v);
                    if (!inside) continue;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        float t = v[i] + (a.bias ? a.bias[c0 + i] : 0.0f);
                        if (RELU) t = fmaxf(t, 0.0f);
                        v[i] = t;
                    }
                    if (a.mask) {
                        const uint4 *mp = reinterpret_cast<const uint4 *>(a.mask + p * COUT + c0);
                        uint4 m4[2] = {mp[0], mp[1]};
                        const __nv_bfloat16 *m = reinterpret_cast<const __nv_bfloat16 *>(m4);
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (!(__bfloat162float(m[i]) > 0.0f)) v[i] = 0.0f;
                    }
                    if (OUT_F32) {
                        static_cast<float *>(a.out)[p] = v[0];
                    } else if (vec) {
                        uint4 o[2];
                        __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(o);
#pragma unroll
                        for (int i = 0; i < 8; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
                        uint4 *op =
                            reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(a.out) + p * a.out_stride + c0);
                        op[0] = o[0];
                        op[1] = o[1];
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (c0 + i < a.out_ch)
                                static_cast<__nv_bfloat16 *>(a.out)[p * a.out_stride + c0 + i] =
                                    __float2bfloat16_rn(v[i]);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&acce[slot]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::NCOLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Weight gradient on tcgen05: dw[tap][co][ci] = sum_p gout[p][co] in[p + tap][ci].
//
// Per tap it is a GEMM D[co][ci] with K = voxels.  The output tile's gout
// rows (256 voxels, 2 x 16 x 8) and its haloed input brick are copied into
// shared memory as 16-byte rows of 8 channels, voxels in (z, y, x) order --
// which is the MN-major core-matrix layout for this GEMM (8 channels x 8
// consecutive x voxels per core matrix): the leading byte offset steps the
// channel chunk, the stride byte offset the next y row (K).  As in the
// forward, a tap only moves the input operand's start address in the brick.
// M = 128 rows with Cout of them real: the rows beyond Cout read whatever
// lies further on in shared memory (the allocation covers them) and land in
// tensor-memory lanes that are never read.  The accumulators of a group of
// taps (taps x Cin columns <= 512) stay in tensor memory over the block's
// voxel tiles (split-K); the block writes its partial sums, which a
// fixed-order pass adds.  Double-buffered tiles, bounded waits as in the
// forward.
// ---------------------------------------------------------------------------
template <int CIN, int COUT>
struct WgCfg {
    static constexpr int TPG = (512 / CIN) < 27 ? (512 / CIN) : 27;  // taps per group
    static constexpr int TG = (27 + TPG - 1) / TPG;                  // tap groups
    static constexpr int CCI = CIN / 8, CCO = COUT / 8;
    static constexpr uint32_t A_CS = 256 * 16;                       // gout chunk plane
    static constexpr uint32_t A_BYTES = CCO * A_CS;
    static constexpr uint32_t B_BYTES = CCI * BK_CSTR;
    // the 16 row groups of the second gout buffer's operand must stay inside
    static constexpr uint32_t REACH = A_BYTES + 17 * A_CS;
    static constexpr uint32_t USED = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr uint32_t SMEM = (USED > REACH ? USED : REACH) + 1024;
    static constexpr uint32_t NCOLS = 512;
};

struct WgArgs {
    const __nv_bfloat16 *in;    // [nvox][CIN]
    const __nv_bfloat16 *gout;  // [nvox][COUT]
    float *part;                // [27][gridDim.x][COUT][CIN]
    int B, D, H, W;
};

template <int CIN, int COUT, bool KLBO = true>
__global__ void __launch_bounds__(128) k_conv_wgrad_tc(WgArgs a, int *err) {
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 128 && CIN <= 256, "tcgen05 shape");
    using C = WgCfg<CIN, COUT>;
    constexpr uint32_t IDESC = tc_idesc_bf16(128, CIN) | (1u << 15) | (1u << 16);  // A and B MN-major
    extern __shared__ unsigned char dsm[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
    const uint32_t a_s = smem_u32(base);
    const uint32_t b_s = a_s + 2 * C::A_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x, g = blockIdx.x;
    const int tap0 = blockIdx.y * C::TPG;
    const int ntap = min(C::TPG, 27 - tap0);
    const BrickTiles T = brick_tiles(a.B, a.D, a.H, a.W);
    const int my_tiles = g < T.ntiles ? (T.ntiles - 1 - g) / G + 1 : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(C::NCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    auto tile_origin = [&](int j, int &b, int &z0, int &y0, int &x0) {
        int t = g + j * G;
        x0 = (t % T.ntx) * BK_TX;
        t /= T.ntx;
        y0 = (t % T.nty) * BK_TY;
        t /= T.nty;
        z0 = (t % T.ntz) * BK_TZ;
        b = t / T.ntz;
    };
    auto load_tile = [&](int j) {
        int b, z0, y0, x0;
        tile_origin(j, b, z0, y0, x0);
        const uint32_t ad = a_s + (j & 1) * C::A_BYTES, bd = b_s + (j & 1) * C::B_BYTES;
        // gout rows of the tile's own voxels (zero outside the volume)
        for (int idx = tid; idx < 256 * C::CCO; idx += 128) {
            const int r = idx / C::CCO, ch = idx % C::CCO;
            const int z = z0 + r / 128, y = y0 + (r / 8) % 16, x = x0 + r % 8;
            const bool valid = z < a.D && y < a.H && x < a.W;
            const size_t q = valid ? (((size_t)b * a.D + z) * a.H + y) * a.W + x : 0;
            cp_async16(ad + ch * C::A_CS + r * 16, a.gout + q * COUT + ch * 8, valid);
        }
        // the input brick with its one-voxel halo (zero outside the volume)
        for (int idx = tid; idx < BK_ROWS * C::CCI; idx += 128) {
            const int row = idx / C::CCI, ch = idx % C::CCI;
            const int xx = row % BK_XB, yy = (row / BK_XB) % BK_YB, zz = row / (BK_XB * BK_YB);
            const int z = z0 - 1 + zz, y = y0 - 1 + yy, x = x0 - 1 + xx;
            const bool valid =
                (unsigned)z < (unsigned)a.D && (unsigned)y < (unsigned)a.H && (unsigned)x < (unsigned)a.W;
            const size_t q = valid ? (((size_t)b * a.D + z) * a.H + y) * a.W + x : 0;
            cp_async16(bd + ch * BK_CSTR + row * 16, a.in + q * CIN + ch * 8, valid);
        }
    };
    auto issue_tile = [&](int j) {
        // MN-major operands: the leading byte offset steps K (the next 8 voxels,
        // here the next y row), the stride byte offset steps M / N (the next
        // 8 channels)
        const uint64_t ad0 = KLBO ? tc_smem_desc(a_s + (j & 1) * C::A_BYTES, 128, C::A_CS)
                                  : tc_smem_desc(a_s + (j & 1) * C::A_BYTES, C::A_CS, 128);
        const uint64_t bd0 = KLBO ? tc_smem_desc(b_s + (j & 1) * C::B_BYTES, BK_XB * 16, BK_CSTR)
                                  : tc_smem_desc(b_s + (j & 1) * C::B_BYTES, BK_CSTR, BK_XB * 16);
        for (int t = 0; t < ntap; ++t) {
            const int tap = tap0 + t;
            const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
            const uint32_t dcol = tmem + t * CIN;
#pragma unroll
            for (int zz = 0; zz < BK_TZ; ++zz)
#pragma unroll
                for (int yp = 0; yp < BK_TY / 2; ++yp) {
                    const uint32_t aoff = (zz * 128 + yp * 16) * 16;
                    const uint32_t boff = (((zz + dz) * BK_YB + 2 * yp + dy) * BK_XB + dx) * 16;
                    tc_mma(dcol, ad0 + (aoff >> 4), bd0 + (boff >> 4), IDESC,
                           (j > 0 || zz > 0 || yp > 0) ? 1u : 0u);
                }
        }
        tc_commit(&mbar[j & 1]);
    };

    bool ok = true;
    int done = -1, issued = 0;
    if (my_tiles > 0) {
        load_tile(0);
        cp_async_commit();
    }
    for (int j = 0; j < my_tiles; ++j) {
        cp_async_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        ok = __syncthreads_and(ok);
        if (!ok) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            issue_tile(j);
        }
        issued = j + 1;
        if (j >= 1) {
            ok = __all_sync(0xffffffffu, ok && mbar_wait_bounded(&mbar[(j - 1) & 1], (uint32_t)(((j - 1) >> 1) & 1)));
            if (ok) done = j - 1;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (j + 1 < my_tiles) {
            load_tile(j + 1);
            cp_async_commit();
        }
    }
    if (ok && my_tiles > 0) {
        if (__all_sync(0xffffffffu, mbar_wait_bounded(&mbar[(my_tiles - 1) & 1], (uint32_t)(((my_tiles - 1) >> 1) & 1))))
            done = my_tiles - 1;
        else
            ok = false;
    }
    cp_async_wait<0>();
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const int co = warp * 32 + lane;
        for (int t = 0; t < ntap; ++t) {
            float *o = a.part + ((size_t)(tap0 + t) * G + g) * COUT * CIN;
#pragma unroll
            for (int c0 = 0; c0 < CIN; c0 += 16) {
                float v[16];
                tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + t * CIN + c0, v);
                if (co < COUT) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) o[(size_t)co * CIN + c0 + i] = my_tiles > 0 ? v[i] : 0.0f;
                }
            }
        }
    } else {
        if (tid == 0) atomicExch(err, 1);
        const int last = issued - 1;
        if (tid == 0 && last > done) mbar_wait_bounded(&mbar[last & 1], (uint32_t)((last >> 1) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::NCOLS) : "memory");
    }
}

}  // namespace mgct
