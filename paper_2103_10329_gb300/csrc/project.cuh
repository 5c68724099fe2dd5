// Ray-driven forward projector A (Joseph's method) with fused epilogues.
//
// The projection operator P of Eq. 1 (Sec. 2) is discretised by Joseph's
// method: each ray is sampled at its crossings with the voxel-centre planes
// normal to its major axis, by bilinear interpolation within the plane, and
// each sample carries the path length between planes.  One thread per ray,
// in two kernels:
//   k_project_col (tilt-free geometries, the solvers' and mgct_project's
//     path): a warp takes 32 rows of one detector column, whose rays share
//     their in-plane crossing, and reads z-fastest copies of the volume;
//   k_project (any geometry): a warp covers 32 adjacent detector columns of
//     one detector row, so at every plane its taps fall on one or two
//     contiguous rows of the volume copy whose fastest axis is the in-plane
//     horizontal axis.
// Either way, y-major rays sample plane y = i of vol [z][y][x] (taps along x,
// z) and x-major rays plane x = i of volT [z][x][y] (taps along y, z).
#pragma once

#include <type_traits>

#include "common.cuh"

namespace mgct {


struct ProjArgs {
    const ViewGeom *views;
    int n, nu, nv;
    float h;
    int view0, stride, nviews;
};

template <typename VT>
__device__ __forceinline__ float tap(const VT *__restrict__ p, int off, bool ok) {
    return ok ? to_f32(__ldg(p + off)) : 0.0f;
}

__device__ __forceinline__ float2 unpack2(uint32_t w, __nv_bfloat16) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
__device__ __forceinline__ float2 unpack2(uint32_t w, __half) {
    __half2 h = *reinterpret_cast<__half2 *>(&w);
    return __half22float2(h);
}

// Quad volume (the solvers' projector input): entry (jz, i, jb) holds the
// whole bilinear footprint of a sample in plane i whose in-plane voxel
// corner is (jz, jb) -- V(jz, jb), V(jz, jb + 1), V(jz + 1, jb),
// V(jz + 1, jb + 1), zero outside the volume -- so one sample is one
// unconditional 16-byte (float32) or 8-byte (16-bit) load.  Corners run over
// [-QD_PAD, n + 1] in both in-plane axes (the clip below keeps every sample
// of a ray inside (-2, n + 1)), stored at index corner + QD_PAD:
// [n + 2 QD_PAD - 1][n][n + 2 QD_PAD - 1] entries.
template <typename T>
struct Quad {};

template <typename VT>
struct VolTraits {
    using elem = VT;
    static constexpr bool quad = false;
};
template <>
struct VolTraits<Quad<float>> {
    using elem = float4;
    static constexpr bool quad = true;
};
template <typename T>
struct VolTraits<Quad<T>> {
    using elem = uint2;
    using half_t = T;
    static constexpr bool quad = true;
};

// Block-wide float64 sum of up to two values; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *red) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarp = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        double x = v[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp * NV + c] = x;
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            double s = 0.0;
            for (int w = 0; w < nwarp; ++w) s += red[w * NV + c];
            v[c] = s;
        }
    }
}

__device__ __forceinline__ int block_linear() {
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

// Range of planes i (as floats) where f(i) = ic + p + (i - ic) r lies in
// (-1, n), intersected into [lo, hi].
__device__ __forceinline__ void clip_planes(float p, float r, float ic, float fn, float &lo, float &hi) {
    if (r != 0.0f) {
        float t1 = ic + (-1.0f - ic - p) / r, t2 = ic + (fn - ic - p) / r;
        lo = fmaxf(lo, fminf(t1, t2));
        hi = fminf(hi, fmaxf(t1, t2));
    } else if (!(ic + p > -1.0f && ic + p < fn)) {
        hi = -1.0f;
    }
}

// Integer part and fraction of a double-float coordinate.
__device__ __forceinline__ void split_coord(DF f, int &i, float &phi) {
    float fl = floorf(f.hi);
    phi = __fadd_rn(__fsub_rn(f.hi, fl), f.lo);
    i = (int)fl;
    if (phi < 0.0f) {
        phi = __fadd_rn(phi, 1.0f);
        i -= 1;
    } else if (phi >= 1.0f) {
        phi = __fsub_rn(phi, 1.0f);
        i += 1;
    }
}

constexpr int PJ_CHUNK = 16;  // planes stepped in float32 from one double-float anchor
#ifndef MGCT_PJ_UNROLL
#define MGCT_PJ_UNROLL 1
#endif
#define MGCT_PRAGMA_S(x) _Pragma(#x)
#define MGCT_PRAGMA(x) MGCT_PRAGMA_S(x)

// Line integral of one ray; returns A vol for pixel (ju, jv) of view G.
// The ray's crossing with the central plane and its slopes are set up in
// double-float from the float64-derived view table; every PJ_CHUNK planes the
// crossing is re-anchored in double-float and split into integer voxel index
// and fraction, and the planes in between step the fraction in float32.  The
// sample positions are thus accurate to ~1e-6 voxel at any volume size.
struct RaySum {
    float acc;  // sum of the bilinear samples along the ray
    float dlh;  // path length per plane, h |w| / |w_a|; A vol = acc * dlh
};

template <typename VT>
__device__ __forceinline__ RaySum ray_integral(const ViewGeom &G, const ProjArgs &a, int ju, int jv,
                                               const typename VolTraits<VT>::elem *__restrict__ vol,
                                               const typename VolTraits<VT>::elem *__restrict__ volT) {
    using E = typename VolTraits<VT>::elem;
    const int n = a.n;
    const float ic = 0.5f * (float)(n - 1);
    const float up = (float)ju - 0.5f * (float)(a.nu - 1);
    const float vp = (float)jv - 0.5f * (float)(a.nv - 1);
    const RayDir d = ray_dir(G, up, vp);
    const int ia = d.ax, ib = 1 - d.ax;
    const DF wa = df_affine(G.Wc[ia], G.Wc_lo[ia], G.Eu[ia], G.Eu_lo[ia], G.Ev[ia], G.Ev_lo[ia], up, vp);
    const DF wb = df_affine(G.Wc[ib], G.Wc_lo[ib], G.Eu[ib], G.Eu_lo[ib], G.Ev[ib], G.Ev_lo[ib], up, vp);
    const DF wz = df_affine(G.Wc[2], G.Wc_lo[2], G.Eu[2], G.Eu_lo[2], G.Ev[2], G.Ev_lo[2], up, vp);
    const float *N = d.ax ? G.NY : G.NX;
    const float *Nl = d.ax ? G.NY_lo : G.NX_lo;
    const DF nb = df_affine(N[0], Nl[0], N[1], Nl[1], N[2], Nl[2], up, vp);
    const DF nz = df_affine(N[3], Nl[3], N[4], Nl[4], N[5], Nl[5], up, vp);
    const DF rb = df_div(wb, wa), rz = df_div(wz, wa);  // slopes per plane
    const DF pb = df_div(nb, wa), pz = df_div(nz, wa);  // centred crossing at the central plane
    const float dl_h = sqrtf(fmaf(rz.hi, rz.hi, fmaf(rb.hi, rb.hi, 1.0f)));
    const E *__restrict__ base = d.ax ? vol : volT;
    float lo = 0.0f, hi = (float)(n - 1);
    clip_planes(pb.hi, rb.hi, ic, (float)n, lo, hi);
    clip_planes(pz.hi, rz.hi, ic, (float)n, lo, hi);
    // Planes outside [floor(lo), ceil(hi)] lie beyond a boundary by at least
    // |r| (1 - rounding) and sample zero; within it both coordinates stay in
    // (-1 - |r|, n + |r|) with |r| <= 1 (x or y is the major axis and z never
    // is), i.e. in (-2, n + 1).
    if (!(lo <= hi)) return RaySum{0.0f, dl_h * a.h};
    const int i0 = max(0, (int)floorf(lo));
    const int i1 = min(n - 1, (int)ceilf(hi));
    const unsigned qmax = (unsigned)quad_elems(n) - 1u;
    (void)qmax;
    float acc = 0.0f;
    for (int c0 = i0; c0 <= i1; c0 += PJ_CHUNK) {
        const float d0 = __fsub_rn((float)c0, ic);  // exact
        int Ib, Iz;
        float phib, phiz;
        split_coord(df_add(df_add(pb, df_mul_f(rb, d0)), DF{ic, 0.0f}), Ib, phib);
        split_coord(df_add(df_add(pz, df_mul_f(rz, d0)), DF{ic, 0.0f}), Iz, phiz);
        const int cnt = min(PJ_CHUNK, i1 - c0 + 1);
        float part = 0.0f;
        MGCT_PRAGMA(unroll MGCT_PJ_UNROLL)
        for (int k = 0; k < cnt; ++k) {
            const int i = c0 + k;
            const float gb = fmaf((float)k, rb.hi, phib);
            const float gz = fmaf((float)k, rz.hi, phiz);
            const float fb0 = floorf(gb), fz0 = floorf(gz);
            const float tb = gb - fb0, tz = gz - fz0;
            const int jb = Ib + (int)fb0, jz = Iz + (int)fz0;
            const bool z0 = (unsigned)jz < (unsigned)n, z1 = (unsigned)(jz + 1) < (unsigned)n;
            float v00, v10, v01, v11;
            if constexpr (VolTraits<VT>::quad) {
                // the clip keeps q in range; the unsigned min only guarantees it
                const unsigned q = min((unsigned)(((jz + QD_PAD) * n + i) * quad_side(n) + jb + QD_PAD), qmax);
                if constexpr (std::is_same<E, float4>::value) {
                    const float4 Q = __ldg(base + q);
                    v00 = Q.x;
                    v10 = Q.y;
                    v01 = Q.z;
                    v11 = Q.w;
                } else {
                    const uint2 Q = __ldg(base + q);
                    const float2 p0 = unpack2(Q.x, typename VolTraits<VT>::half_t());
                    const float2 p1 = unpack2(Q.y, typename VolTraits<VT>::half_t());
                    v00 = p0.x;
                    v10 = p0.y;
                    v01 = p1.x;
                    v11 = p1.y;
                }
            } else {
                const bool b0 = (unsigned)jb < (unsigned)n, b1 = (unsigned)(jb + 1) < (unsigned)n;
                const int row0 = (jz * n + i) * n + jb;  // may be out of range; loads are predicated
                const int row1 = row0 + n * n;
                v00 = tap(base, row0, b0 && z0);
                v10 = tap(base, row0 + 1, b1 && z0);
                v01 = tap(base, row1, b0 && z1);
                v11 = tap(base, row1 + 1, b1 && z1);
            }
            const float a0 = fmaf(tb, v10 - v00, v00);
            const float a1 = fmaf(tb, v11 - v01, v01);
            part += fmaf(tz, a1 - a0, a0);
        }
        acc += part;
    }
    return RaySum{acc, dl_h * a.h};
}

// Epilogue interface: operator()(i_batch, k_view, jv, ju, active, acc, dlh)
// with A vol = acc * dlh at that ray, called by every thread of the block
// (block reductions inside).  "Weighted" sinograms carry the factor dlh of
// their ray, which the back-projector then need not recompute.
// Block order.  Consecutive views of the trajectory have nearby source
// heights, and one detector-row tile of nearby views meets only a z-band of
// the volume, so blocks are ordered (group of PJ_VG views, row tile, view in
// group, column tile): the blocks resident at any time share that band and
// its rows stay in L2.

#ifndef MGCT_PJ_MINB
#define MGCT_PJ_MINB 8  // 32 registers: 64 resident warps hide the gather latency
#endif
template <typename VT, typename Epi>
__global__ void __launch_bounds__(PJ_BX *PJ_BY, MGCT_PJ_MINB)
    k_project(ProjArgs a, const typename VolTraits<VT>::elem *__restrict__ vol,
              const typename VolTraits<VT>::elem *__restrict__ volT, Epi epi) {
    __shared__ ViewGeom G;
    const int vtiles = (a.nv + PJ_BY - 1) / PJ_BY;
    const int group = blockIdx.z / vtiles, vt = blockIdx.z % vtiles;
    const int i = group * PJ_VG + blockIdx.y;  // batch index
    const bool view_ok = i < a.nviews;
    const int k = a.view0 + (view_ok ? i : 0) * a.stride;
    const int tid = threadIdx.x + threadIdx.y * PJ_BX;
    if (tid < 64) reinterpret_cast<float *>(&G)[tid] = __ldg(reinterpret_cast<const float *>(a.views + k) + tid);
    __syncthreads();
    const int ju = blockIdx.x * PJ_BX + threadIdx.x;
    const int jv = vt * PJ_BY + threadIdx.y;
    const bool active = view_ok && ju < a.nu && jv < a.nv;
    RaySum rs{0.0f, 0.0f};
    if (active) rs = ray_integral<VT>(G, a, ju, jv, vol, volT);
    epi(i, k, jv, ju, active, rs.acc, rs.dlh);
}

// out = A vol
template <typename OT>
struct EpiStore {
    OT *out;
    int nu, nv;
    __device__ void operator()(int i, int, int jv, int ju, bool active, float acc, float dlh) const {
        if (active) out[((size_t)i * nv + jv) * nu + ju] = from_f32<OT>(acc * dlh);
    }
};

// out = b + A vol (out may alias b: each ray reads its own entry first)
struct EpiPlus {
    float *out;
    const float *b;
    int nu, nv;
    __device__ void operator()(int i, int, int jv, int ju, bool active, float acc, float dlh) const {
        if (active) {
            const size_t idx = ((size_t)i * nv + jv) * nu + ju;
            out[idx] = b[idx] + acc * dlh;
        }
    }
};

// r = b - A vol and the block's sum of r^2 (float64) into part[block].
// WEIGHTED = false: out = r.  WEIGHTED = true: out = r * dlh (the ray's path
// length per plane), which the back-projector then need not recompute.
template <typename OT, bool WEIGHTED = false>
struct EpiResidual {
    OT *out;
    const float *b;  // indexed like out
    double *part;    // NULL: no norm
    int nu, nv, nviews;
    __device__ void operator()(int i, int, int jv, int ju, bool active, float acc, float dlh) const {
        double s[1] = {0.0};
        if (active) {
            size_t idx = ((size_t)i * nv + jv) * nu + ju;
            float r = __ldg(b + idx) - acc * dlh;
            if (WEIGHTED) {
                out[idx] = from_f32<OT>(r * dlh);
                s[0] = (double)r * (double)r;
            } else {
                OT ro = from_f32<OT>(r);
                out[idx] = ro;
                float rf = to_f32(ro);
                s[0] = (double)rf * (double)rf;
            }
        }
        if (part) {
            __shared__ double red[PJ_BX * PJ_BY / 32];
            block_sum<1>(s, red);
            if (threadIdx.x == 0 && threadIdx.y == 0) part[block_linear()] = s[0];
        }
    }
};

// Line-search dot products per block, no sinogram write:
//   <r, A d> = sum r_w * acc  (r_w = r * dlh, the weighted residual)
//   |A d|^2  = sum (acc * dlh)^2
template <typename RT>
struct EpiDualDot {
    const RT *rw;
    double *part;  // [blocks][2]
    int nu, nv, nviews;
    __device__ void operator()(int i, int, int jv, int ju, bool active, float acc, float dlh) const {
        double s[2] = {0.0, 0.0};
        if (active) {
            float rv = to_f32(rw[((size_t)i * nv + jv) * nu + ju]);
            float ad = acc * dlh;
            s[0] = (double)rv * (double)acc;
            s[1] = (double)ad * (double)ad;
        }
        __shared__ double red[2 * PJ_BX * PJ_BY / 32];
        block_sum<2>(s, red);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            int bl = block_linear();
            part[2 * bl] = s[0];
            part[2 * bl + 1] = s[1];
        }
    }
};

// OS-EMTR (Eq. 3) sinogram terms for one subset, weighted by dlh:
//   t = exp(-A mu);  c0 = (t - exp(-b)) dlh  (I/I0 = exp(-b));  c1 = t PI dlh
// b and PI are full [K][nv][nu] arrays indexed by the view k; c is a batch
// two-channel sinogram [i][v][u][2].
struct EpiEMTerms {
    float2 *c;
    const float *b;
    const float *pi;
    int nu, nv, nviews;
    __device__ void operator()(int i, int k, int jv, int ju, bool active, float acc, float dlh) const {
        if (!active) return;
        size_t pix = (size_t)jv * nu + ju;
        size_t full = (size_t)k * nv * nu + pix;
        float t = expf(-acc * dlh);
        float2 o;
        o.x = (t - expf(-__ldg(b + full))) * dlh;
        o.y = t * __ldg(pi + full) * dlh;
        c[(size_t)i * nv * nu + pix] = o;
    }
};

// ---------------------------------------------------------------------------
// Column projector (tilt-free geometries).  The rays through one detector
// column of a view lie in one vertical plane: they share their major axis,
// they cross every plane i of that axis at the same in-plane coordinate
//   b(c_a) = ic + pb + c_a rb                  (c_a = i - ic),
// and their z crossings are affine in the row:
//   z(c_a) = ic + e0(v') + c_a e1(v'),  e0 = ez0 + v' e10,  e1 = ezc + v' e1c,
// with the column's quantities from the double-float column table.  A warp
// takes 32 consecutive rows of one column.  The in-plane half of a sample is
// then the same for the whole warp: the warp's lanes compute it for 32
// planes at a time (in double-float, from the plane's own offset, so nothing
// accumulates) into a small table in shared memory -- the fraction along b
// and the offset of the (plane, b) row of entries -- that every lane reads
// back with one broadcast load per sample.  Each lane steps its own z
// crossing in 32.32 fixed point: exact integer additions, a step rounded to
// 2^-32 voxel, so the position stays within ~1e-7 voxel over any number of
// planes with no re-anchoring; the integer part is the entry index and the
// fraction's top 23 bits become the float32 weight.
//
// The volume is read from z-fastest quads: entry (i, jb + QD_PAD, jz +
// QD_PAD) holds (V(jz, jb), V(jz + 1, jb), V(jz, jb + 1), V(jz + 1, jb + 1))
// at plane i, so the warp's 32 loads at one plane fall on one run of
// consecutive entries and the two b-rows of a footprint are float pairs
// along z (interpolated in b by one packed multiply-add).
//
// The warp walks the union of its rays' plane ranges.  A ray outside its own
// range lies beyond the top or bottom face there (the in-plane clip is the
// warp's), so its crossing's z index, clamped into the padded array, reads an
// all-zero entry; planes past the union (the last batch) read the zero entry
// row (plane 0, corner b = n + 1).  The clamp is exact, not a guard band.
// ---------------------------------------------------------------------------
#ifndef MGCT_PC_BATCH
#define MGCT_PC_BATCH 8
#endif
constexpr int PC_BATCH = MGCT_PC_BATCH;  // plane loads in flight per ray
constexpr int PC_TAB = 32;               // planes per table refill (one per lane)

template <typename E>
__device__ __forceinline__ float2 quad_pair(const E &Q, int which);
template <>
__device__ __forceinline__ float2 quad_pair<float4>(const float4 &Q, int which) {
    return which ? make_float2(Q.z, Q.w) : make_float2(Q.x, Q.y);
}

// d = a * b + c and d = a - b on float pairs (one packed instruction each)
__device__ __forceinline__ float2 fma_f2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 sub_f2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// Sample of one z-fastest quad: b-lerp of both z rows (packed), then z-lerp.
template <typename VT>
__device__ __forceinline__ float zquad_sample(const typename VolTraits<VT>::elem &Q, float2 tb2, float tz) {
    float2 r0, r1;
    if constexpr (std::is_same<typename VolTraits<VT>::elem, float4>::value) {
        r0 = make_float2(Q.x, Q.y);
        r1 = make_float2(Q.z, Q.w);
    } else {
        r0 = unpack2(Q.x, typename VolTraits<VT>::half_t());
        r1 = unpack2(Q.y, typename VolTraits<VT>::half_t());
    }
    const float2 a = fma_f2(tb2, sub_f2(r1, r0), r0);  // values at jz, jz + 1
    return fmaf(tz, a.y - a.x, a.x);
}

template <typename E>
// Pairs' sample arithmetic in packed f32x2 (z-lerp of both b columns in one
// FMA pair, their b weights into a pair of running sums): measured 16.2 ->
// 15.5 ms per projection at 256^3 / 720 views, unchanged at 512^3 / 1440
#ifndef MGCT_PC_F2
#define MGCT_PC_F2 1
#endif
struct ColTab {
    float tb, tb2;  // fraction along b (twice: a float pair)
    const E *row;   // entries of the sample's (plane, b) row
};

// Layouts of the column projector's z-fastest copies (entry (i, jb + QD_PAD,
// jz + QD_PAD) of plane i):
//   ZL_QUAD: the footprint as two z pairs, one 8-byte load a sample (16-bit
//            storage);
//   ZL_PAIR: (V(jz, jb), V(jz, jb + 1)) in float32, two 8-byte loads a
//            sample (rows jz and jz + 1, adjacent in memory).
// Measured at 256^3 / 720 views and 512^3 / 1440 views, float32 pairs took
// 16.3 and 313 ms per projection, float32 quads (one 16-byte load, twice the
// footprint) 18.2 and 415 ms, plain values (four 4-byte loads) 17.2 and
// 315 ms: the pairs' footprint, twice the volume's, keeps the band of
// planes that concurrently resident blocks read in L2.
constexpr int ZL_QUAD = 0, ZL_PAIR = 1;
template <typename VT, int LAYOUT>
struct ZElem {
    using type = typename VolTraits<VT>::elem;
};
template <typename VT>
struct ZElem<VT, ZL_PAIR> {
    using type = float2;
};

template <typename VT, int LAYOUT>
__device__ __forceinline__ RaySum column_rays(const ProjArgs &a, const float4 *__restrict__ ct, int jv, bool row_ok,
                                              const typename ZElem<VT, LAYOUT>::type *__restrict__ zqy,
                                              const typename ZElem<VT, LAYOUT>::type *__restrict__ zqx,
                                              ColTab<typename ZElem<VT, LAYOUT>::type> *__restrict__ tab) {
    using E = typename ZElem<VT, LAYOUT>::type;
    // {ax, rb, rb_lo, pb}, {pb_lo, ez0, ez0_lo, ezc}, {ezc_lo, e10, e10_lo, e1c}, {e1c_lo, 0, 0, 0}
    const float4 t0 = __ldg(ct), t1 = __ldg(ct + 1), t2 = __ldg(ct + 2), t3 = __ldg(ct + 3);
    const DF rb{t0.y, t0.z}, pb{t0.w, t1.x}, ez0{t1.y, t1.z}, ezc{t1.w, t2.x}, e10{t2.y, t2.z}, e1c{t2.w, t3.x};
    const E *__restrict__ base = t0.x != 0.0f ? zqy : zqx;
    const int n = a.n, lane = threadIdx.x & 31;
    const float ic = 0.5f * (float)(n - 1);
    const float vp = (float)jv - 0.5f * (float)(a.nv - 1);
    const DF e0 = df_add(ez0, df_mul_f(e10, vp));  // centred z crossing at the central plane
    const DF e1 = df_add(ezc, df_mul_f(e1c, vp));  // its change per plane
    const float rz = e1.hi;
    const float dl_h = sqrtf(fmaf(rz, rz, fmaf(rb.hi, rb.hi, 1.0f)));
    float lo = 0.0f, hi = (float)(n - 1);
    clip_planes(pb.hi, rb.hi, ic, (float)n, lo, hi);
    clip_planes(e0.hi, rz, ic, (float)n, lo, hi);
    int i0 = 0x7fffffff, i1 = -1;
    if (row_ok && lo <= hi) {
        i0 = max(0, (int)floorf(lo));
        i1 = min(n - 1, (int)ceilf(hi));
    }
    const int I0 = __reduce_min_sync(0xffffffffu, i0);
    const int I1 = __reduce_max_sync(0xffffffffu, i1);
    float acc = 0.0f;
    if (I0 > I1) return RaySum{acc, dl_h * a.h};
    const int side = quad_side(n);
    // largest z (and b) entry index a sample may start at: corner n + 1 (an
    // all-zero quad), or corner n where the sample reads index + 1 as well
    const unsigned emax = (unsigned)side - (LAYOUT == ZL_QUAD ? 1u : 2u);
    // z crossing at plane I0 as 32.32 fixed point, and its step per plane
    int Iz;
    float phiz;
    split_coord(df_add(df_add(e0, df_mul_f(e1, __fsub_rn((float)I0, ic))), DF{ic, 0.0f}), Iz, phiz);
    const unsigned zfrac = phiz < 1.0f ? (unsigned)__float2ull_rn(phiz * 4294967296.0f) : 0xffffffffu;
    long long zpos = ((long long)Iz << 32) | (long long)zfrac;
    const long long zstep = __float2ll_rn(e1.hi * 4294967296.0f) + __float2ll_rn(e1.lo * 4294967296.0f);
    for (int c0 = I0; c0 <= I1; c0 += PC_TAB) {
        // lane l: plane c0 + l of this warp's table
        const int pc = c0 + lane;
        float tbv = 0.0f;
        const E *row = base + (size_t)emax * side;  // plane 0, corner b = n + 1 (or n): zero entries
        if (pc <= I1) {
            int Ib;
            float phib;
            split_coord(df_add(df_add(pb, df_mul_f(rb, __fsub_rn((float)pc, ic))), DF{ic, 0.0f}), Ib, phib);
            const unsigned bq = min((unsigned)(Ib + QD_PAD), emax);
            row = base + ((size_t)pc * side + bq) * side;
            tbv = phib;
        }
        __syncwarp();
        // pairs: the b weights (1 - t_b, t_b) of the two z-lerped columns;
        // quads: t_b twice (a float pair for the packed b-lerp)
        tab[lane] = ColTab<E>{(MGCT_PC_F2 && LAYOUT == ZL_PAIR) ? 1.0f - tbv : tbv, tbv, row};
        __syncwarp();
        const int cnt = min(PC_TAB, I1 - c0 + 1);
        float part = 0.0f;
        float2 part2 = make_float2(0.0f, 0.0f);
        for (int kk = 0; kk < cnt; kk += PC_BATCH) {
            constexpr int NL = LAYOUT == ZL_QUAD ? 1 : 2;
            E Q[PC_BATCH][NL];
            float2 tb[PC_BATCH];
            float tz[PC_BATCH];
#pragma unroll
            for (int j = 0; j < PC_BATCH; ++j) {
                const ColTab<E> te = tab[kk + j];
                tb[j] = make_float2(te.tb, te.tb2);
                const unsigned zlo = (unsigned)zpos;
                const int zhi = (int)(zpos >> 32);
                tz[j] = __uint_as_float(0x3f800000u | (zlo >> 9)) - 1.0f;
                const unsigned zq = min((unsigned)(zhi + QD_PAD), emax);
                const E *q = te.row + zq;
                Q[j][0] = __ldg(q);
                if constexpr (NL == 2) Q[j][1] = __ldg(q + 1);
                zpos += zstep;
            }
#pragma unroll
            for (int j = 0; j < PC_BATCH; ++j) {
                if constexpr (LAYOUT == ZL_QUAD) {
                    part += zquad_sample<VT>(Q[j][0], tb[j], tz[j]);
                } else if (MGCT_PC_F2) {
                    // z-lerp of both b columns at once (packed), then their
                    // b weights into a packed pair of running sums
                    const float2 c = fma_f2(make_float2(tz[j], tz[j]), sub_f2(Q[j][1], Q[j][0]), Q[j][0]);
                    part2 = fma_f2(tb[j], c, part2);
                } else {
                    const float a0 = fmaf(tb[j].x, Q[j][0].y - Q[j][0].x, Q[j][0].x);
                    const float a1 = fmaf(tb[j].x, Q[j][1].y - Q[j][1].x, Q[j][1].x);
                    part += fmaf(tz[j], a1 - a0, a0);
                }
            }
        }
        acc += part + (part2.x + part2.y);
        // the last batch stepped past the chunk: re-align the z position
        zpos -= (long long)(((cnt + PC_BATCH - 1) / PC_BATCH) * PC_BATCH - cnt) * zstep;
    }
    return RaySum{acc, dl_h * a.h};
}

#ifndef MGCT_PC_MINB
#define MGCT_PC_MINB 4
#endif
template <typename VT, int LAYOUT, typename Epi>
__global__ void __launch_bounds__(PC_COLS *PC_ROWS, MGCT_PC_MINB)
    k_project_col(ProjArgs a, const float4 *__restrict__ cols, const typename ZElem<VT, LAYOUT>::type *__restrict__ zqy,
                  const typename ZElem<VT, LAYOUT>::type *__restrict__ zqx, Epi epi) {
    __shared__ __align__(16) ColTab<typename ZElem<VT, LAYOUT>::type> tab[PC_COLS][PC_TAB];
    const int rtiles = (a.nv + PC_ROWS - 1) / PC_ROWS;
    const int group = blockIdx.z / rtiles, rt = blockIdx.z - group * rtiles;
    const int i = group * PC_VG + blockIdx.y;  // batch index
    const bool view_ok = i < a.nviews;
    const int k = a.view0 + (view_ok ? i : 0) * a.stride;
    const int ju = blockIdx.x * PC_COLS + threadIdx.y;  // warp: one column
    const int jv = rt * PC_ROWS + threadIdx.x;          // lane: one row
    const bool active = view_ok && ju < a.nu && jv < a.nv;
    RaySum rs{0.0f, 0.0f};
    if (view_ok && ju < a.nu)  // uniform over the warp
        rs = column_rays<VT, LAYOUT>(a, cols + ((size_t)k * a.nu + ju) * 4, jv, jv < a.nv, zqy, zqx,
                                     tab[threadIdx.y]);
    epi(i, k, jv, ju, active, rs.acc, rs.dlh);
}

template <typename VT, int LAYOUT, typename Epi>
int launch_project_col(const mgct_geom *g, int level, int view0, int nviews, int stride,
                       const typename ZElem<VT, LAYOUT>::type *zqy, const typename ZElem<VT, LAYOUT>::type *zqx,
                       const Epi &epi, cudaStream_t s, int *nblocks = nullptr) {
    const LevelInfo &L = g->lev[level];
    ProjArgs a;
    a.views = L.d_views;
    a.n = L.n;
    a.nu = L.nu;
    a.nv = L.nv;
    a.h = (float)L.h;
    a.view0 = view0;
    a.stride = stride;
    a.nviews = nviews;
    const int groups = (nviews + PC_VG - 1) / PC_VG;
    const int vg = nviews < PC_VG ? nviews : PC_VG;
    dim3 grid((L.nu + PC_COLS - 1) / PC_COLS, vg, groups * ((L.nv + PC_ROWS - 1) / PC_ROWS));
    if (nblocks) *nblocks = (int)project_blocks_col(L.nu, L.nv, nviews);
    if (nviews == 0) return MGCT_OK;
    MGCT_KERNEL(KK_PROJECT, s,
                k_project_col<VT, LAYOUT, Epi><<<grid, dim3(PC_ROWS, PC_COLS), 0, s>>>(a, L.d_cols_df, zqy, zqx, epi));
    return MGCT_OK;
}

// The column projector applies where the geometry has no detector tilt (its
// column table exists at every grid).
inline bool use_column_projector(const mgct_geom *g, int level) {
    return g->separable && g->lev[level].d_cols_df != nullptr;
}

template <typename VT, typename Epi>
int launch_project(const mgct_geom *g, int level, int view0, int nviews, int stride,
                   const typename VolTraits<VT>::elem *vol, const typename VolTraits<VT>::elem *volT,
                   const Epi &epi, cudaStream_t s, int *nblocks = nullptr) {
    const LevelInfo &L = g->lev[level];
    ProjArgs a;
    a.views = L.d_views;
    a.n = L.n;
    a.nu = L.nu;
    a.nv = L.nv;
    a.h = (float)L.h;
    a.view0 = view0;
    a.stride = stride;
    a.nviews = nviews;
    const int groups = (nviews + PJ_VG - 1) / PJ_VG;
    const int vg = nviews < PJ_VG ? nviews : PJ_VG;
    dim3 grid((L.nu + PJ_BX - 1) / PJ_BX, vg, groups * ((L.nv + PJ_BY - 1) / PJ_BY));
    if (nblocks) *nblocks = (int)project_blocks(L.nu, L.nv, nviews);
    if (nviews == 0) return MGCT_OK;
    MGCT_KERNEL(KK_PROJECT, s, k_project<VT, Epi><<<grid, dim3(PJ_BX, PJ_BY), 0, s>>>(a, vol, volT, epi));
    return MGCT_OK;
}

// A over views [view0, view0 + nviews * stride) of volume v (type SRC), read
// through quad copies of storage type ST: the transpose of v into vT, the
// quads of both ray classes into `quads` (2 quad_elems(n) entries), then the
// column projector (tilt-free geometries) or k_project with epilogue `e`.
template <typename ST, typename SRC, typename Epi>
int project_volume(const mgct_geom *g, int level, int view0, int nviews, int stride, const SRC *v, SRC *vT,
                   void *quads, const Epi &e, cudaStream_t s, int *nb) {
    using QE = typename VolTraits<Quad<ST>>::elem;
    const LevelInfo &L = g->lev[level];
    QE *q1 = static_cast<QE *>(quads);
    QE *q2 = q1 + quad_elems(L.n);
    MGCT_TRY(launch_transpose_xy<SRC>(L.n, v, vT, s));
    if (use_column_projector(g, level)) {
        if constexpr (std::is_same<ST, float>::value) {
            float2 *z1 = static_cast<float2 *>(quads);
            float2 *z2 = z1 + quad_elems(L.n);
            MGCT_TRY((launch_build_zpairs<SRC>(L.n, v, z1, s)));
            MGCT_TRY((launch_build_zpairs<SRC>(L.n, vT, z2, s)));
            return launch_project_col<Quad<ST>, ZL_PAIR>(g, level, view0, nviews, stride, z1, z2, e, s, nb);
        } else {
            MGCT_TRY((launch_build_zquads<ST, SRC>(L.n, v, q1, s)));
            MGCT_TRY((launch_build_zquads<ST, SRC>(L.n, vT, q2, s)));
            return launch_project_col<Quad<ST>, ZL_QUAD>(g, level, view0, nviews, stride, q1, q2, e, s, nb);
        }
    }
    MGCT_TRY((launch_build_quads<ST, SRC>(L.n, v, q1, s)));
    MGCT_TRY((launch_build_quads<ST, SRC>(L.n, vT, q2, s)));
    return launch_project<Quad<ST>>(g, level, view0, nviews, stride, q1, q2, e, s, nb);
}

}  // namespace mgct
