// Streaming volume and sinogram kernels: transpose and the projector's quad
// copies, the Eq. 5 preconditioner, restriction and prolongation (Alg. 1),
// the Landweber update with soft thresholding, and deterministic float64
// reductions.  All are bound by HBM bandwidth; each reads and writes its
// arrays once with coalesced accesses.
#include <type_traits>

#include "common.cuh"

namespace mgct {

// ---------------------------------------------------------------------------
// vol [z][y][x] -> volT [z][x][y], 32x32 tiles through shared memory
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_transpose_xy(int n, const T *__restrict__ in, T *__restrict__ out) {
    __shared__ T tile[32][33];
    const int z = blockIdx.z;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const size_t slab = (size_t)z * n * n;
    for (int dy = threadIdx.y; dy < 32; dy += 8) {
        int x = x0 + threadIdx.x, y = y0 + dy;
        if (x < n && y < n) tile[dy][threadIdx.x] = in[slab + (size_t)y * n + x];
    }
    __syncthreads();
    for (int dx = threadIdx.y; dx < 32; dx += 8) {
        int y = y0 + threadIdx.x, x = x0 + dx;
        if (x < n && y < n) out[slab + (size_t)x * n + y] = tile[threadIdx.x][dx];
    }
}

template <typename T>
int launch_transpose_xy(int n, const T *in, T *out, cudaStream_t s) {
    dim3 grid((n + 31) / 32, (n + 31) / 32, n);
    MGCT_KERNEL(KK_TRANSPOSE, s, k_transpose_xy<T><<<grid, dim3(32, 8), 0, s>>>(n, in, out));
    return MGCT_OK;
}
template int launch_transpose_xy<float>(int, const float *, float *, cudaStream_t);
template int launch_transpose_xy<__nv_bfloat16>(int, const __nv_bfloat16 *, __nv_bfloat16 *, cudaStream_t);
template int launch_transpose_xy<__half>(int, const __half *, __half *, cudaStream_t);


// two float32 values rounded to 16 bits, packed low then high
__device__ __forceinline__ uint32_t pack2(float lo, float hi, __nv_bfloat16) {
    const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return a | (b << 16);
}
__device__ __forceinline__ uint32_t pack2(float lo, float hi, __half) {
    const uint32_t a = __half_as_ushort(__float2half_rn(lo));
    const uint32_t b = __half_as_ushort(__float2half_rn(hi));
    return a | (b << 16);
}

// ---------------------------------------------------------------------------
// Quad copies: dst[zq][i][bq] = (V(jz, jb), V(jz, jb + 1), V(jz + 1, jb),
// V(jz + 1, jb + 1)) of plane i, jz = zq - QD_PAD, jb = bq - QD_PAD, zero
// outside the volume.  Reads coalesced along b (each value four times, from
// cache); one 16- or 8-byte store per entry.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 make_quad(float a, float b, float c, float d, float) { return make_float4(a, b, c, d); }
template <typename T>
__device__ __forceinline__ uint2 make_quad(float a, float b, float c, float d, T) {
    return make_uint2(pack2(a, b, T()), pack2(c, d, T()));
}

template <typename T, typename QE, typename SRC>
__global__ void __launch_bounds__(128) k_build_quads(int n, const SRC *__restrict__ src, QE *__restrict__ dst) {
    const int side = quad_side(n);
    const int bq = blockIdx.x * 128 + threadIdx.x;
    if (bq >= side) return;
    const int i = blockIdx.y, zq = blockIdx.z;
    const int jz = zq - QD_PAD, jb = bq - QD_PAD;
    auto V = [&](int z, int b) -> float {
        return ((unsigned)z < (unsigned)n && (unsigned)b < (unsigned)n) ? to_f32(__ldg(src + ((size_t)z * n + i) * n + b))
                                                                       : 0.0f;
    };
    dst[((size_t)zq * n + i) * side + bq] = make_quad(V(jz, jb), V(jz, jb + 1), V(jz + 1, jb), V(jz + 1, jb + 1), T());
}

template <typename T, typename SRC>
int launch_build_quads(int n, const SRC *src, void *dst, cudaStream_t s) {
    using QE = typename std::conditional<std::is_same<T, float>::value, float4, uint2>::type;
    dim3 grid((quad_side(n) + 127) / 128, n, quad_side(n));
    MGCT_KERNEL(KK_TRANSPOSE, s, k_build_quads<T, QE, SRC><<<grid, 128, 0, s>>>(n, src, static_cast<QE *>(dst)));
    return MGCT_OK;
}
template int launch_build_quads<float, float>(int, const float *, void *, cudaStream_t);
template int launch_build_quads<__nv_bfloat16, float>(int, const float *, void *, cudaStream_t);
template int launch_build_quads<__half, float>(int, const float *, void *, cudaStream_t);
template int launch_build_quads<__nv_bfloat16, __nv_bfloat16>(int, const __nv_bfloat16 *, void *, cudaStream_t);
template int launch_build_quads<__half, __half>(int, const __half *, void *, cudaStream_t);

// ---------------------------------------------------------------------------
// z-fastest quad copies (the column projector's input): dst[i][bq][zq] holds
// the footprint of plane i at corner (jz, jb) = (zq, bq) - QD_PAD as two
// pairs along z, (V(jz, jb), V(jz + 1, jb)) and (V(jz, jb + 1),
// V(jz + 1, jb + 1)), zero outside the volume.  A block transposes one plane's (z, b) tile of src [z][i][b]
// through shared memory: 33 x 33 source values (the tile and its +1
// neighbours) read along b, entries written along z.
// ---------------------------------------------------------------------------
constexpr int ZQ_T = 32;
template <typename T, typename QE, typename SRC>
__global__ void __launch_bounds__(256) k_build_zquads(int n, const SRC *__restrict__ src, QE *__restrict__ dst) {
    __shared__ float tile[ZQ_T + 1][ZQ_T + 1];  // [z][b], stride 33: conflict-free both ways
    const int side = quad_side(n);
    const int zq0 = blockIdx.x * ZQ_T, bq0 = blockIdx.y * ZQ_T, i = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int r = ty; r <= ZQ_T; r += 8) {
        const int jz = zq0 + r - QD_PAD;
        for (int c = tx; c <= ZQ_T; c += 32) {
            const int jb = bq0 + c - QD_PAD;
            tile[r][c] = ((unsigned)jz < (unsigned)n && (unsigned)jb < (unsigned)n)
                             ? to_f32(__ldg(src + ((size_t)jz * n + i) * n + jb))
                             : 0.0f;
        }
    }
    __syncthreads();
    const int zq = zq0 + tx;
    if (zq >= side) return;
    for (int c = ty; c < ZQ_T; c += 8) {
        const int bq = bq0 + c;
        if (bq >= side) break;
        dst[((size_t)i * side + bq) * side + zq] =
            make_quad(tile[tx][c], tile[tx + 1][c], tile[tx][c + 1], tile[tx + 1][c + 1], T());
    }
}

template <typename T, typename SRC>
int launch_build_zquads(int n, const SRC *src, void *dst, cudaStream_t s) {
    using QE = typename std::conditional<std::is_same<T, float>::value, float4, uint2>::type;
    const int side = quad_side(n);
    dim3 grid((side + ZQ_T - 1) / ZQ_T, (side + ZQ_T - 1) / ZQ_T, n);
    MGCT_KERNEL(KK_TRANSPOSE, s,
                k_build_zquads<T, QE, SRC><<<grid, dim3(32, 8), 0, s>>>(n, src, static_cast<QE *>(dst)));
    return MGCT_OK;
}
template int launch_build_zquads<float, float>(int, const float *, void *, cudaStream_t);
template int launch_build_zquads<__nv_bfloat16, float>(int, const float *, void *, cudaStream_t);
template int launch_build_zquads<__half, float>(int, const float *, void *, cudaStream_t);
template int launch_build_zquads<__nv_bfloat16, __nv_bfloat16>(int, const __nv_bfloat16 *, void *, cudaStream_t);
template int launch_build_zquads<__half, __half>(int, const __half *, void *, cudaStream_t);

// float32 z-fastest pairs (V(jz, jb), V(jz, jb + 1)), same tiling
template <typename SRC>
__global__ void __launch_bounds__(256) k_build_zpairs(int n, const SRC *__restrict__ src, float2 *__restrict__ dst) {
    __shared__ float tile[ZQ_T][ZQ_T + 1];  // [z][b]: the tile and the +1 neighbour along b
    const int side = quad_side(n);
    const int zq0 = blockIdx.x * ZQ_T, bq0 = blockIdx.y * ZQ_T, i = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < ZQ_T; r += 8) {
        const int jz = zq0 + r - QD_PAD;
        for (int c = tx; c <= ZQ_T; c += 32) {
            const int jb = bq0 + c - QD_PAD;
            tile[r][c] = ((unsigned)jz < (unsigned)n && (unsigned)jb < (unsigned)n)
                             ? to_f32(__ldg(src + ((size_t)jz * n + i) * n + jb))
                             : 0.0f;
        }
    }
    __syncthreads();
    const int zq = zq0 + tx;
    if (zq >= side) return;
    for (int c = ty; c < ZQ_T; c += 8) {
        const int bq = bq0 + c;
        if (bq >= side) break;
        dst[((size_t)i * side + bq) * side + zq] = make_float2(tile[tx][c], tile[tx][c + 1]);
    }
}

template <typename SRC>
int launch_build_zpairs(int n, const SRC *src, void *dst, cudaStream_t s) {
    const int side = quad_side(n);
    dim3 grid((side + ZQ_T - 1) / ZQ_T, (side + ZQ_T - 1) / ZQ_T, n);
    MGCT_KERNEL(KK_TRANSPOSE, s,
                k_build_zpairs<SRC><<<grid, dim3(32, 8), 0, s>>>(n, src, static_cast<float2 *>(dst)));
    return MGCT_OK;
}
template int launch_build_zpairs<float>(int, const float *, void *, cudaStream_t);


// ---------------------------------------------------------------------------
// Eq. 5 stencil: out = p * in, zero padding.  Block = 32 x 8 columns; each
// thread walks ZB planes along z with three rolling halo planes in shared
// memory, so every input element is read from HBM about once.
// ---------------------------------------------------------------------------
struct Stencil27 {
    float c[27];  // [dz][dy][dx]
};

constexpr int ST_BX = 32, ST_BY = 8, ST_ZB = 16;

__global__ void __launch_bounds__(ST_BX *ST_BY)
    k_precondition_generic(int n, Stencil27 K, const float *__restrict__ in, float *__restrict__ out) {
    __shared__ float pl[3][ST_BY + 2][ST_BX + 2];
    const int x0 = blockIdx.x * ST_BX, y0 = blockIdx.y * ST_BY, z0 = blockIdx.z * ST_ZB;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + ty * ST_BX;
    const size_t nn = (size_t)n * n;
    auto load_plane = [&](int slot, int z) {
        for (int t = tid; t < (ST_BY + 2) * (ST_BX + 2); t += ST_BX * ST_BY) {
            int ly = t / (ST_BX + 2), lx = t % (ST_BX + 2);
            int x = x0 + lx - 1, y = y0 + ly - 1;
            float v = 0.0f;
            if (z >= 0 && z < n && x >= 0 && x < n && y >= 0 && y < n) v = __ldg(in + z * nn + (size_t)y * n + x);
            pl[slot][ly][lx] = v;
        }
    };
    load_plane(0, z0 - 1);
    load_plane(1, z0);
    const int zend = min(n, z0 + ST_ZB);
    for (int z = z0; z < zend; ++z) {
        const int sm = (z - z0) % 3, s0 = (z - z0 + 1) % 3, sp = (z - z0 + 2) % 3;
        // slots: sm holds z-1, s0 holds z, sp receives z+1
        load_plane(sp, z + 1);
        __syncthreads();
        const int x = x0 + tx, y = y0 + ty;
        if (x < n && y < n) {
            float acc = 0.0f;
            const int sl[3] = {sm, s0, sp};
#pragma unroll
            for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx)
                        acc = fmaf(K.c[(dz * 3 + dy) * 3 + dx], pl[sl[dz]][ty + dy][tx + dx], acc);
            out[z * nn + (size_t)y * n + x] = acc;
        }
        __syncthreads();
    }
}

static Stencil27 eq5_stencil(int slice_axis) {
    // Eq. 5, the printed order: three 3x3 matrices (outer index = slice)
    static const float P[3][3][3] = {{{-1, -1, -1}, {-1, 0, -1}, {-1, -1, -1}},
                                     {{-8, -4, -8}, {-4, 64, -4}, {-8, -4, -8}},
                                     {{-1, -1, -1}, {-1, 0, -1}, {-1, -1, -1}}};
    Stencil27 K;
    for (int dz = 0; dz < 3; ++dz)
        for (int dy = 0; dy < 3; ++dy)
            for (int dx = 0; dx < 3; ++dx) {
                float v;
                if (slice_axis == 2) v = P[dz][dy][dx];
                else if (slice_axis == 0) v = P[dx][dz][dy];
                else v = P[dy][dz][dx];
                K.c[(dz * 3 + dy) * 3 + dx] = v / 64.0f;
            }
    return K;
}

// ---------------------------------------------------------------------------
// Eq. 5 with its slices along z (the default reading), as an HBM stream.
// The two outer slices are the same 3x3 matrix (-1 everywhere but a 0 centre)
// and the middle one is (-8 corners, -4 edges, 64 centre), all over 64, so
// with, in one z plane, c = the centre, e = the sum of the 4 edge and k =
// of the 4 corner neighbours,
//   a(z) = -(e + k) / 64,   b(z) = c - e / 16 - k / 8,
//   out(z) = a(z - 1) + b(z) + a(z + 1).
// A block owns a 128 x 8 column of the volume over PZ_ZB planes; the planes
// (with a one-voxel x/y halo, zero outside) stream through a PZ_ST-deep ring
// of shared-memory slots by cp.async, each is read from shared memory once
// (a float4 per thread and row, the x neighbours by lane shuffles), and a, b
// roll in registers.  Every input element is read from HBM about once.
// ---------------------------------------------------------------------------
constexpr int PZ_TX = 128, PZ_TY = 8, PZ_ZB = 32, PZ_ST = 4, PZ_W = 136;  // slot row: x0-1 at column 3

__device__ __forceinline__ uint32_t sh_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cpa4(float *dst, const float *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sh_addr(dst)), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cpa16(float *dst, const float *src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sh_addr(dst)), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__global__ void __launch_bounds__(PZ_TX / 4 * PZ_TY) k_precondition_z(int n, const float *__restrict__ in,
                                                                      float *__restrict__ out) {
    __shared__ __align__(16) float pl[PZ_ST][PZ_TY + 2][PZ_W];
    const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 5;
    const int x0 = blockIdx.x * PZ_TX, y0 = blockIdx.y * PZ_TY, z0 = blockIdx.z * PZ_ZB;
    const int zend = min(n, z0 + PZ_ZB);
    const int P = zend - z0 + 2;  // planes z0 - 1 .. zend
    const size_t nn = (size_t)n * n;
    const bool vec = (n & 3) == 0;
    auto load = [&](int q) {  // plane z0 - 1 + q into slot q % PZ_ST
        const int p = z0 - 1 + q;
        float(*dst)[PZ_W] = pl[q % PZ_ST];
        const bool zok = p >= 0 && p < n;
        const float *src = in + (zok ? (size_t)p * nn : 0);
        if (vec) {
            for (int e = tid; e < (PZ_TY + 2) * (PZ_TX / 4); e += PZ_TX / 4 * PZ_TY) {
                const int ly = e / (PZ_TX / 4), c4 = e % (PZ_TX / 4);
                const int y = y0 + ly - 1, x = x0 + 4 * c4;
                const bool ok = zok && y >= 0 && y < n && x < n;
                cpa16(&dst[ly][4 + 4 * c4], ok ? src + (size_t)y * n + x : in, ok ? 16 : 0);
            }
            for (int e = tid; e < (PZ_TY + 2) * 2; e += PZ_TX / 4 * PZ_TY) {
                const int ly = e >> 1, side = e & 1;
                const int y = y0 + ly - 1, x = side ? x0 + PZ_TX : x0 - 1;
                const bool ok = zok && y >= 0 && y < n && x >= 0 && x < n;
                cpa4(&dst[ly][side ? 4 + PZ_TX : 3], ok ? src + (size_t)y * n + x : in, ok);
            }
        } else {
            for (int e = tid; e < (PZ_TY + 2) * (PZ_TX + 2); e += PZ_TX / 4 * PZ_TY) {
                const int ly = e / (PZ_TX + 2), lx = e % (PZ_TX + 2);
                const int y = y0 + ly - 1, x = x0 + lx - 1;
                const bool ok = zok && y >= 0 && y < n && x >= 0 && x < n;
                cpa4(&dst[ly][lx + 3], ok ? src + (size_t)y * n + x : in, ok);
            }
        }
    };
    // PZ_ST - 1 groups in flight from the start (empty ones past the end), so
    // that plane q has landed when at most PZ_ST - 2 groups are pending
    for (int q = 0; q < PZ_ST - 1; ++q) {
        if (q < P) load(q);
        cpa_commit();
    }
    const int y = y0 + ty, xb = x0 + 4 * lane;
    float A2[4] = {0.f, 0.f, 0.f, 0.f}, A1[4] = {0.f, 0.f, 0.f, 0.f}, B1[4] = {0.f, 0.f, 0.f, 0.f};
    for (int q = 0; q < P; ++q) {
        asm volatile("cp.async.wait_group %0;" ::"n"(PZ_ST - 2) : "memory");
        __syncthreads();  // plane q visible; every thread is past plane q - 1, whose slot is refilled next
        if (q + PZ_ST - 1 < P) load(q + PZ_ST - 1);
        cpa_commit();
        const float(*S)[PZ_W] = pl[q % PZ_ST];
        float lr[3][4], cc[3][4];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float4 v = *reinterpret_cast<const float4 *>(&S[ty + r][4 + 4 * lane]);
            float left = __shfl_up_sync(0xffffffffu, v.w, 1), right = __shfl_down_sync(0xffffffffu, v.x, 1);
            if (lane == 0) left = S[ty + r][3];
            if (lane == 31) right = S[ty + r][4 + PZ_TX];
            const float e[6] = {left, v.x, v.y, v.z, v.w, right};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                lr[r][j] = e[j] + e[j + 2];
                cc[r][j] = e[j + 1];
            }
        }
        float a[4], b[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float k = lr[0][j] + lr[2][j];
            const float ed = (cc[0][j] + cc[2][j]) + lr[1][j];
            a[j] = -(ed + k) * (1.0f / 64.0f);
            b[j] = cc[1][j] - ed * (1.0f / 16.0f) - k * (1.0f / 8.0f);
        }
        if (q >= 2 && y < n) {
            const int z = z0 + q - 2;
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) o[j] = A2[j] + B1[j] + a[j];
            float *dst = out + (size_t)z * nn + (size_t)y * n + xb;
            if (vec) {
                if (xb < n) *reinterpret_cast<float4 *>(dst) = make_float4(o[0], o[1], o[2], o[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (xb + j < n) dst[j] = o[j];
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            A2[j] = A1[j];
            A1[j] = a[j];
            B1[j] = b[j];
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

int launch_precondition(int n, int slice_axis, const float *in, float *out, cudaStream_t s, const float *custom) {
    if (custom) {
        Stencil27 K;
        for (int i = 0; i < 27; ++i) K.c[i] = custom[i];
        dim3 grid((n + ST_BX - 1) / ST_BX, (n + ST_BY - 1) / ST_BY, (n + ST_ZB - 1) / ST_ZB);
        MGCT_KERNEL(KK_PRECONDITION, s, k_precondition_generic<<<grid, dim3(ST_BX, ST_BY), 0, s>>>(n, K, in, out));
        return MGCT_OK;
    }
    if (slice_axis == 2) {
        dim3 grid((n + PZ_TX - 1) / PZ_TX, (n + PZ_TY - 1) / PZ_TY, (n + PZ_ZB - 1) / PZ_ZB);
        MGCT_KERNEL(KK_PRECONDITION, s, k_precondition_z<<<grid, PZ_TX / 4 * PZ_TY, 0, s>>>(n, in, out));
        return MGCT_OK;
    }
    dim3 grid((n + ST_BX - 1) / ST_BX, (n + ST_BY - 1) / ST_BY, (n + ST_ZB - 1) / ST_ZB);
    MGCT_KERNEL(KK_PRECONDITION, s,
                k_precondition_generic<<<grid, dim3(ST_BX, ST_BY), 0, s>>>(n, eq5_stencil(slice_axis), in, out));
    return MGCT_OK;
}

// ---------------------------------------------------------------------------
// Restriction (2x2x2 mean of mu, 2x2 mean of b) and prolongation
// ---------------------------------------------------------------------------
__global__ void k_restrict_volume(int nc, const float2 *__restrict__ in, float *__restrict__ out) {
    const size_t total = (size_t)nc * nc * nc;
    const int nf2 = nc;  // fine row length in float2 units
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        int x = (int)(t % nc);
        int y = (int)((t / nc) % nc);
        int z = (int)(t / ((size_t)nc * nc));
        float s = 0.0f;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                float2 v = __ldg(in + ((size_t)(2 * z + dz) * (2 * nc) + (2 * y + dy)) * nf2 + x);
                s += v.x + v.y;
            }
        out[t] = 0.125f * s;
    }
}

__global__ void k_restrict_sino(int k, int nvc, int nuc, const float2 *__restrict__ in, float *__restrict__ out) {
    const size_t total = (size_t)k * nvc * nuc;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        int u = (int)(t % nuc);
        size_t rest = t / nuc;
        int v = (int)(rest % nvc);
        size_t view = rest / nvc;
        const float2 *row = in + (view * (2 * nvc) + 2 * v) * nuc;
        float2 a = __ldg(row + u), b = __ldg(row + nuc + u);
        out[t] = 0.25f * ((a.x + a.y) + (b.x + b.y));
    }
}

// fine[2n]^3 += P(new - old): per axis the fine cell 2i takes 3/4 of coarse i
// and 1/4 of coarse i-1, the cell 2i+1 3/4 of i and 1/4 of i+1 (clamped).
// Thread = one coarse cell (i, j, k) and its 2 x 2 x 2 fine cells: the 27
// coarse differences around it are read once (through L1) and the weights
// applied axis by axis; the fine cells are four float2 read-modify-writes.
__global__ void __launch_bounds__(128) k_prolong_add(int nc, const float *__restrict__ cn,
                                                     const float *__restrict__ co, float *__restrict__ fine) {
    const int nf = 2 * nc;
    const int i = blockIdx.x * 128 + threadIdx.x;
    if (i >= nc) return;
    const int j = blockIdx.y, k = blockIdx.z;
    const int xs[3] = {max(i - 1, 0), i, min(i + 1, nc - 1)};
    const int ys[3] = {max(j - 1, 0), j, min(j + 1, nc - 1)};
    const int zs[3] = {max(k - 1, 0), k, min(k + 1, nc - 1)};
    // the fine cells first, so that their loads overlap the coarse ones
    float2 *f[2][2];
    float2 fv[2][2];
#pragma unroll
    for (int pz = 0; pz < 2; ++pz)
#pragma unroll
        for (int py = 0; py < 2; ++py) {
            f[pz][py] = reinterpret_cast<float2 *>(fine + ((size_t)(2 * k + pz) * nf + (2 * j + py)) * nf) + i;
            fv[pz][py] = *f[pz][py];
        }
    // along x: ex = fine 2i, ox = fine 2i + 1, per coarse (z, y) row
    float ex[3][3], ox[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const size_t row = ((size_t)zs[a] * nc + ys[b]) * nc;
            const float dm = __ldg(cn + row + xs[0]) - __ldg(co + row + xs[0]);
            const float d0 = __ldg(cn + row + xs[1]) - __ldg(co + row + xs[1]);
            const float dp = __ldg(cn + row + xs[2]) - __ldg(co + row + xs[2]);
            ex[a][b] = fmaf(0.75f, d0, 0.25f * dm);
            ox[a][b] = fmaf(0.75f, d0, 0.25f * dp);
        }
    // along y, then z
#pragma unroll
    for (int pz = 0; pz < 2; ++pz)
#pragma unroll
        for (int py = 0; py < 2; ++py) {
            float vx[2];
#pragma unroll
            for (int px = 0; px < 2; ++px) {
                float yz[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float *r = px ? ox[a] : ex[a];
                    yz[a] = fmaf(0.75f, r[1], 0.25f * r[py ? 2 : 0]);
                }
                vx[px] = fmaf(0.75f, yz[1], 0.25f * yz[pz ? 2 : 0]);
            }
            *f[pz][py] = make_float2(fv[pz][py].x + vx[0], fv[pz][py].y + vx[1]);
        }
}

static int grid_for(size_t total, int threads = 256) {
    size_t b = (total + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    if (b < 1) b = 1;
    return (int)b;
}

int launch_restrict_volume(int n_fine, const float *in, float *out, cudaStream_t s) {
    int nc = n_fine / 2;
    MGCT_KERNEL(KK_GRID, s, k_restrict_volume<<<grid_for((size_t)nc * nc * nc), 256, 0, s>>>(nc, reinterpret_cast<const float2 *>(in), out));
    return MGCT_OK;
}

int launch_restrict_sino(int k, int nv, int nu, const float *in, float *out, cudaStream_t s) {
    MGCT_KERNEL(KK_GRID, s, k_restrict_sino<<<grid_for((size_t)k * (nv / 2) * (nu / 2)), 256, 0, s>>>(
        k, nv / 2, nu / 2, reinterpret_cast<const float2 *>(in), out));
    return MGCT_OK;
}

int launch_prolong_add(int nc, const float *cn, const float *co, float *fine, cudaStream_t s) {
    const int nf = 2 * nc;
    if (nc < 1) return MGCT_OK;
    (void)nf;
    dim3 grid((nc + 127) / 128, nc, nc);
    MGCT_KERNEL(KK_GRID, s, k_prolong_add<<<grid, 128, 0, s>>>(nc, cn, co, fine));
    return MGCT_OK;
}

// ---------------------------------------------------------------------------
// Alg. 1 BilateralFilter: out(p) = sum_q w x(q) / sum_q w over the window
// |q - p|_inf <= r inside the volume, w = exp(-|q - p|^2 / 2 ss^2 -
// (x(q) - x(p))^2 / 2 sr^2) (one __expf per neighbour; the self weight is 1).
// Thread = voxel; the window's values come through L1.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bilateral(int n, const float *__restrict__ in, float *__restrict__ out,
                                                   float inv2ss, float inv2sr, int r) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
    if (x >= n || y >= n) return;
    const size_t nn = (size_t)n * n;
    const float c = __ldg(in + z * nn + (size_t)y * n + x);
    float num = 0.0f, den = 0.0f;
    for (int dz = -r; dz <= r; ++dz) {
        const int zz = z + dz;
        if ((unsigned)zz >= (unsigned)n) continue;
        for (int dy = -r; dy <= r; ++dy) {
            const int yy = y + dy;
            if ((unsigned)yy >= (unsigned)n) continue;
            const float *row = in + zz * nn + (size_t)yy * n;
            const float dzy = (float)(dz * dz + dy * dy);
            for (int dx = -r; dx <= r; ++dx) {
                const int xx = x + dx;
                if ((unsigned)xx >= (unsigned)n) continue;
                const float v = __ldg(row + xx), d = v - c;
                const float w = __expf(-(dzy + (float)(dx * dx)) * inv2ss - d * d * inv2sr);
                num = fmaf(w, v, num);
                den += w;
            }
        }
    }
    out[z * nn + (size_t)y * n + x] = num / den;
}

int launch_bilateral(int n, const float *in, float *out, double sigma_s, double sigma_r, int radius, cudaStream_t s) {
    dim3 grid((n + 31) / 32, (n + 7) / 8, n);
    MGCT_KERNEL(KK_UPDATE, s, k_bilateral<<<grid, dim3(32, 8), 0, s>>>(n, in, out, (float)(0.5 / (sigma_s * sigma_s)),
                                                                         (float)(0.5 / (sigma_r * sigma_r)), radius));
    return MGCT_OK;
}

// ---------------------------------------------------------------------------
// Deterministic float64 reductions: one block sums the partials in a fixed
// order (strided per thread, then a fixed tree).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_sum_partials(const double *__restrict__ part, int count, int nvals,
                                                       double *__restrict__ out) {
    __shared__ double red[1024];
    for (int c = 0; c < nvals; ++c) {
        double s = 0.0;
        for (int i = threadIdx.x; i < count; i += 1024) s += part[(size_t)i * nvals + c];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = 512; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[c] = red[0];
        __syncthreads();
    }
}

int launch_sum_partials(const double *part, int count, int nvals, double *out, cudaStream_t s) {
    MGCT_KERNEL(KK_REDUCE, s, k_sum_partials<<<1, 1024, 0, s>>>(part, count, nvals, out));
    return MGCT_OK;
}

// ---------------------------------------------------------------------------
// Line-search step size and the update mu <- S_lambda(mu + alpha d)
// sums = {<r, A d>, |A d|^2}; r2 = |r|^2.  stats (device) receives
// {alpha, r2, r2_pred, nonfinite}.
// ---------------------------------------------------------------------------
__global__ void k_step_size(const double *__restrict__ sums, const double *__restrict__ r2, double fixed_alpha,
                            double *__restrict__ stats) {
    double num = sums[0], den = sums[1];
    double rr = r2 ? r2[0] : 0.0;
    double alpha, nonfinite = 0.0;
    if (!isfinite(num) || !isfinite(den) || !isfinite(rr)) {
        // a non-finite residual or direction: no step
        alpha = 0.0;
        nonfinite = 1.0;
    } else {
        if (fixed_alpha > 0.0) alpha = fixed_alpha;
        else alpha = den > 0.0 ? num / den : 0.0;
        if (!isfinite(alpha)) {
            alpha = 0.0;
            nonfinite = 1.0;
        }
    }
    stats[0] = alpha;
    stats[1] = rr;
    stats[2] = rr - 2.0 * alpha * num + alpha * alpha * den;
    stats[3] = nonfinite;
}

int launch_step_size(const double *sums, const double *r2, double fixed_alpha, double *stats, cudaStream_t s) {
    MGCT_KERNEL(KK_REDUCE, s, k_step_size<<<1, 1, 0, s>>>(sums, r2, fixed_alpha, stats));
    return MGCT_OK;
}

__global__ void k_update(size_t count, float *__restrict__ mu, const float *__restrict__ d,
                         const double *__restrict__ alpha_p, float lam) {
    const float alpha = (float)alpha_p[0];
    // alpha = 0 (no descent, or a non-finite step replaced by 0): leave mu
    // untouched, even where d is not finite
    if (alpha == 0.0f) return;
    const size_t n4 = count / 4;
    float4 *mu4 = reinterpret_cast<float4 *>(mu);
    const float4 *d4 = reinterpret_cast<const float4 *>(d);
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n4; t += (size_t)gridDim.x * blockDim.x) {
        float4 m = mu4[t], dv = __ldg(d4 + t);
        float v[4] = {fmaf(alpha, dv.x, m.x), fmaf(alpha, dv.y, m.y), fmaf(alpha, dv.z, m.z), fmaf(alpha, dv.w, m.w)};
        if (lam > 0.0f) {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = copysignf(fmaxf(fabsf(v[q]) - lam, 0.0f), v[q]);
        }
        mu4[t] = make_float4(v[0], v[1], v[2], v[3]);
    }
    for (size_t t = 4 * n4 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x) {
        float v = fmaf(alpha, d[t], mu[t]);
        if (lam > 0.0f) v = copysignf(fmaxf(fabsf(v) - lam, 0.0f), v);
        mu[t] = v;
    }
}

int launch_update(size_t count, float *mu, const float *d, const double *alpha, float lam, cudaStream_t s) {
    MGCT_KERNEL(KK_UPDATE, s, k_update<<<grid_for(count / 4 + 1), 256, 0, s>>>(count, mu, d, alpha, lam));
    return MGCT_OK;
}

// ---------------------------------------------------------------------------
// OS-EMTR voxel update (Eq. 3): mu += num / den where den > 1e-12 max(den).
// nd = [num (n^3) | den (n^3)].  Block max partials, then the update.
// ---------------------------------------------------------------------------
__global__ void k_max_partials(size_t count, const float *__restrict__ x, double *__restrict__ part) {
    __shared__ float red[256];
    float m = 0.0f;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, x[t]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = (double)red[0];
}

__global__ void k_em_update(size_t count, float *__restrict__ mu, const float *__restrict__ nd,
                            const double *__restrict__ part, int nparts) {
    __shared__ float thr;
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < nparts; ++i) m = fmax(m, part[i]);
        thr = (float)(1e-12 * m);
    }
    __syncthreads();
    const float th = thr;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x) {
        float den = nd[count + t];
        if (den > th && th > 0.0f) mu[t] += nd[t] / den;
    }
}

int launch_em_update(size_t count, float *mu, const float *nd, double *part, cudaStream_t s) {
    int nb = grid_for(count, 256);
    if (nb > 1024) nb = 1024;
    MGCT_KERNEL(KK_REDUCE, s, k_max_partials<<<nb, 256, 0, s>>>(count, nd + count, part));
    MGCT_KERNEL(KK_UPDATE, s, k_em_update<<<grid_for(count), 256, 0, s>>>(count, mu, nd, part, nb));
    return MGCT_OK;
}

// out = alpha * d, alpha read from a device scalar
__global__ void k_scaled_copy(size_t count, const float *__restrict__ d, const double *__restrict__ alpha_p,
                              float *__restrict__ out) {
    const float alpha = (float)alpha_p[0];
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x)
        out[t] = alpha * d[t];
}

int launch_scaled_copy(size_t count, const float *d, const double *alpha, float *out, cudaStream_t s) {
    MGCT_KERNEL(KK_UPDATE, s, k_scaled_copy<<<grid_for(count), 256, 0, s>>>(count, d, alpha, out));
    return MGCT_OK;
}

// mu <- S_lambda(mu + beta d') when the learned line search found beta > 0
// (st[4] = beta, st[7] = non-finite flag), else mu <- S_lambda(mu + alpha d)
// (st[0] = alpha): the plain step is the fallback.
__global__ void k_update_choice(size_t count, float *__restrict__ mu, const float *__restrict__ d,
                                const float *__restrict__ dl, const double *__restrict__ st, float lam) {
    const bool learned = st[4] > 0.0 && st[7] == 0.0;
    const float a = learned ? (float)st[4] : (float)st[0];
    const float *__restrict__ dir = learned ? dl : d;
    if (a == 0.0f) return;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x) {
        float v = fmaf(a, dir[t], mu[t]);
        if (lam > 0.0f) v = copysignf(fmaxf(fabsf(v) - lam, 0.0f), v);
        mu[t] = v;
    }
}

int launch_update_choice(size_t count, float *mu, const float *d, const float *dl, const double *st, float lam,
                         cudaStream_t s) {
    MGCT_KERNEL(KK_UPDATE, s, k_update_choice<<<grid_for(count), 256, 0, s>>>(count, mu, d, dl, st, lam));
    return MGCT_OK;
}

__global__ void k_axpy(size_t count, float a, const float *__restrict__ x, float *__restrict__ y) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x)
        y[t] = fmaf(a, x[t], y[t]);
}

int launch_axpy(size_t count, float a, const float *x, float *y, cudaStream_t s) {
    MGCT_KERNEL(KK_UPDATE, s, k_axpy<<<grid_for(count), 256, 0, s>>>(count, a, x, y));
    return MGCT_OK;
}

__global__ void k_fill(size_t count, float *__restrict__ x, float v) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x) x[t] = v;
}

int launch_fill(size_t count, float *x, float v, cudaStream_t s) {
    MGCT_KERNEL(KK_UPDATE, s, k_fill<<<grid_for(count), 256, 0, s>>>(count, x, v));
    return MGCT_OK;
}

__global__ void k_copy(size_t count, const float4 *__restrict__ in, float4 *__restrict__ out) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x) out[t] = in[t];
}

int launch_copy(size_t count, const float *in, float *out, cudaStream_t s) {
    if (count % 4) return set_error(MGCT_ESHAPE, "copy size must be a multiple of 4");
    MGCT_KERNEL(KK_UPDATE, s, k_copy<<<grid_for(count / 4), 256, 0, s>>>(count / 4, reinterpret_cast<const float4 *>(in), reinterpret_cast<float4 *>(out)));
    return MGCT_OK;
}

}  // namespace mgct
