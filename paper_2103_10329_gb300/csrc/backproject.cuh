// Voxel-driven back-projector A^T with the exact transpose of the projector's
// weights (the back-projection B of Sec. 2.1 is the adjoint of P).
//
// For voxel j and view k, a detector pixel contributes iff its ray crosses
// the voxel-centre plane of j along the ray's major axis a within one voxel of
// j in both in-plane axes; the weight is the projector's
//   dl * hat(f_b - j_b) * hat(f_z - j_z),   hat(t) = max(0, 1 - |t|).
// Such a ray passes through the cube [j-1, j+1]^3 (index units), so the
// candidates are the pixels inside the cube's projected bounding box.  With
// q = Q (j - S) the voxel centre projects to (u0, v0) = (q0, q1) / q2, and for
// a cube offset delta in [-1, 1]^3,
//   |u(delta) - u0| <= |Q_0 - u0 Q_2|_1 / (q2 - |Q_2|_1),
// likewise for v, which bounds the box without projecting the eight corners.
// Each candidate takes its ray direction and major axis from the projector's
// own routine (bit-identical axis choice), and its crossing from the centred
// numerator form (no cancellation of source-distance terms), in float32: the
// per-weight rounding (~1e-6 voxel at n = 64) averages out over the ~9 K
// contributions a voxel receives.  One thread per voxel, looping over the
// views; the per-view tables of a view chunk sit in shared memory.  No
// atomics.
#pragma once

#include "common.cuh"

namespace mgct {

constexpr int BP_BX = 32, BP_BY = 4, BP_BZ = 2;
constexpr int BP_CHUNK = 64;  // views staged in shared memory at a time

struct BPArgs {
    const ViewGeom *views;
    int n, nu, nv;
    float h;
    int view0, stride, nviews;
    int splits;  // slab kernel: view ranges per z-slab, each into its own partial volume (1: none)
};

template <int NCH, typename ST>
struct SinoLoad;
template <typename ST>
struct SinoLoad<1, ST> {
    static __device__ __forceinline__ void add(const ST *__restrict__ p, size_t idx, float w, float (&acc)[1]) {
        acc[0] = fmaf(w, to_f32(__ldg(p + idx)), acc[0]);
    }
};
template <>
struct SinoLoad<2, float2> {
    static __device__ __forceinline__ void add(const float2 *__restrict__ p, size_t idx, float w, float (&acc)[2]) {
        float2 y = __ldg(p + idx);
        acc[0] = fmaf(w, y.x, acc[0]);
        acc[1] = fmaf(w, y.y, acc[1]);
    }
};

__device__ __forceinline__ float2 load_f2(const float2 *p) { return __ldg(p); }
template <typename ST>
__device__ __forceinline__ float2 load_f2(const ST *) { return make_float2(0.0f, 0.0f); }

// Adds A^T (one view) at voxel (jx, jy, jz) into acc -- any geometry.
// WEIGHTED: the sinogram already carries each ray's dl (see the projector's
// weighted epilogues), so the weight is hat * hat; otherwise dl is computed
// per pixel.  Sinograms are [view][v][u].  Each candidate ray is set up as
// the projector sets it up: direction, slopes and centred crossing in
// double-float from the view table's double-float fields (G must hold them),
// and the crossing's offset from the voxel, p + c_a r - c, formed in
// double-float before it is rounded -- in float32 alone the numerators'
// cancellation leaves ~1e-6 voxel, 1e-5 of a weight near a hat's edge.
template <int NCH, typename ST, bool WEIGHTED>
__device__ __forceinline__ void bp_view(const ViewGeom &G, const BPArgs &a, int jx, int jy, int jz,
                                        const ST *__restrict__ sino_view, float (&acc)[NCH]) {
    const float X = (float)jx - G.S[0], Y = (float)jy - G.S[1], Z = (float)jz - G.S[2];
    const float q0 = fmaf(G.Q[2], Z, fmaf(G.Q[1], Y, G.Q[0] * X));
    const float q1 = fmaf(G.Q[5], Z, fmaf(G.Q[4], Y, G.Q[3] * X));
    const float q2 = fmaf(G.Q[8], Z, fmaf(G.Q[7], Y, G.Q[6] * X));
    const float inv = 1.0f / q2;
    const float u0 = q0 * inv, v0 = q1 * inv;
    const float den = 1.0f / (q2 - G.m2);
    const float hu = (fabsf(G.Q[0] - u0 * G.Q[6]) + fabsf(G.Q[1] - u0 * G.Q[7]) + fabsf(G.Q[2] - u0 * G.Q[8])) * den;
    const float hv = (fabsf(G.Q[3] - v0 * G.Q[6]) + fabsf(G.Q[4] - v0 * G.Q[7]) + fabsf(G.Q[5] - v0 * G.Q[8])) * den;
    const float cu = 0.5f * (float)(a.nu - 1), cv = 0.5f * (float)(a.nv - 1);
    // small absolute margin covers float32 rounding of the bound itself
    int ulo = max(0, (int)ceilf(u0 - hu + cu - 1e-3f));
    int uhi = min(a.nu - 1, (int)floorf(u0 + hu + cu + 1e-3f));
    int vlo = max(0, (int)ceilf(v0 - hv + cv - 1e-3f));
    int vhi = min(a.nv - 1, (int)floorf(v0 + hv + cv + 1e-3f));
    // voxel centre relative to the volume centre (exact half-integers)
    const float ic = 0.5f * (float)(a.n - 1);
    const float cx = (float)jx - ic, cy = (float)jy - ic, cz = (float)jz - ic;
    for (int jv = vlo; jv <= vhi; ++jv) {
        const float vp = (float)jv - cv;
        for (int ju = ulo; ju <= uhi; ++ju) {
            const float up = (float)ju - cu;
            const RayDir d = ray_dir(G, up, vp);
            const int ia = d.ax, ib = 1 - d.ax;
            const DF wa = df_affine(G.Wc[ia], G.Wc_lo[ia], G.Eu[ia], G.Eu_lo[ia], G.Ev[ia], G.Ev_lo[ia], up, vp);
            const DF wb = df_affine(G.Wc[ib], G.Wc_lo[ib], G.Eu[ib], G.Eu_lo[ib], G.Ev[ib], G.Ev_lo[ib], up, vp);
            const DF wz = df_affine(G.Wc[2], G.Wc_lo[2], G.Eu[2], G.Eu_lo[2], G.Ev[2], G.Ev_lo[2], up, vp);
            const float *N = d.ax ? G.NY : G.NX;
            const float *Nl = d.ax ? G.NY_lo : G.NX_lo;
            const DF nb = df_affine(N[0], Nl[0], N[1], Nl[1], N[2], Nl[2], up, vp);
            const DF nz = df_affine(N[3], Nl[3], N[4], Nl[4], N[5], Nl[5], up, vp);
            const DF rb = df_div(wb, wa), rz = df_div(wz, wa);
            // centred crossing of this ray with the voxel's plane, minus the voxel
            const float ca = d.ax ? cy : cx, cb = d.ax ? cx : cy;
            const DF xb = df_add(df_div(nb, wa), df_mul_f(rb, ca));
            const DF xz = df_add(df_div(nz, wa), df_mul_f(rz, ca));
            const float eb = __fadd_rn(__fsub_rn(xb.hi, cb), xb.lo);
            const float ez = __fadd_rn(__fsub_rn(xz.hi, cz), xz.lo);
            const float hb = 1.0f - fabsf(eb);
            const float hz = 1.0f - fabsf(ez);
            if (hb > 0.0f && hz > 0.0f) {
                float w = hb * hz;
                if (!WEIGHTED) w *= sqrtf(fmaf(rz.hi, rz.hi, fmaf(rb.hi, rb.hi, 1.0f))) * a.h;
                SinoLoad<NCH, ST>::add(sino_view, (size_t)jv * a.nu + ju, w, acc);
            }
        }
    }
}

// Separable geometries (no detector tilt: e_u horizontal, e_v vertical).
// Then w_x, w_y and the major axis depend on u' only, the in-plane crossing
// error e_b depends on u' only, and the z error is linear in v':
//   e_z(v') = E0 + v' E1,  E0 = (n0_z + u' nu_z + c_a Wc_z)/w_a - c_z,
//                          E1 = (nv_z + c_a Ev_z)/w_a,
// so each detector column is set up once for the thread's ZB voxels of one
// z-column, and each voxel walks exactly the pixels where |e_z| < 1.
// The column's quantities come from the double-float column table, and
// both cancellations are done in double-float: e_b = pb + c_a rb - c_b, and
// the z error is anchored at the detector row v_a nearest the thread's
// voxels (E0 + v_a E1 - c_z, small), so that in float32 only small terms
// remain -- the sample weights stay accurate to ~1e-7 at any N.
template <int NCH, typename ST, bool WEIGHTED, int ZB>
__device__ __forceinline__ void bp_view_sep(const ViewGeom &G, const float4 *__restrict__ cols, const BPArgs &a,
                                            int jx, int jy, int jz0, const ST *__restrict__ sino_view,
                                            float (&acc)[ZB][NCH]) {
    const float X = (float)jx - G.S[0], Y = (float)jy - G.S[1];
    // with no tilt the u coordinate and depth of a point ignore its z
    const float q0 = fmaf(G.Q[1], Y, G.Q[0] * X);
    const float q2 = fmaf(G.Q[7], Y, G.Q[6] * X);
    const float u0 = q0 / q2;
    const float hu = (fabsf(G.Q[0] - u0 * G.Q[6]) + fabsf(G.Q[1] - u0 * G.Q[7])) / (q2 - G.m2);
    const float cu = 0.5f * (float)(a.nu - 1), cv = 0.5f * (float)(a.nv - 1);
    const int ulo = max(0, (int)ceilf(u0 - hu + cu - 1e-3f));
    const int uhi = min(a.nu - 1, (int)floorf(u0 + hu + cu + 1e-3f));
    const float ic = 0.5f * (float)(a.n - 1);
    const float cx = (float)jx - ic, cy = (float)jy - ic;
    const float zm = (float)jz0 - ic + 0.5f * (float)(ZB - 1);  // centre of the thread's voxels (exact)
    for (int ju = ulo; ju <= uhi; ++ju) {
        const float4 t0 = __ldg(cols + 4 * ju), t1 = __ldg(cols + 4 * ju + 1);
        const float4 t2 = __ldg(cols + 4 * ju + 2), t3 = __ldg(cols + 4 * ju + 3);
        const bool ay = t0.x != 0.0f;
        const float ca = ay ? cy : cx, cb = ay ? cx : cy;
        const DF eb = df_add(df_mul_f(DF{t0.y, t0.z}, ca), DF{t0.w, t1.x});
        const float hb = 1.0f - fabsf(__fadd_rn(__fsub_rn(eb.hi, cb), eb.lo));
        if (hb <= 0.0f) continue;
        const DF Eb = df_add(DF{t1.y, t1.z}, df_mul_f(DF{t1.w, t2.x}, ca));  // centred height at v' = 0
        const DF E1d = df_add(DF{t2.y, t2.z}, df_mul_f(DF{t2.w, t3.x}, ca));
        const float E1 = E1d.hi;
        const float va = rintf((zm - Eb.hi) / E1);  // anchor row (centred units)
        if (!(fabsf(va) < 1.0e7f)) continue;
        const DF c = df_add(df_add(Eb, df_mul_f(E1d, va)), DF{-zm, 0.0f});
        const float cf = c.hi + c.lo;  // z error at the anchor row for the centre voxel
        const float rE1 = 1.0f / E1;
#pragma unroll
        for (int zz = 0; zz < ZB; ++zz) {
            const float E0 = cf - ((float)zz - 0.5f * (float)(ZB - 1));
            const float s1 = (-1.0f - E0) * rE1, s2 = (1.0f - E0) * rE1;
            const int vlo = max(0, (int)ceilf(fminf(s1, s2) + va + cv - 1e-3f));
            const int vhi = min(a.nv - 1, (int)floorf(fmaxf(s1, s2) + va + cv + 1e-3f));
            for (int jv = vlo; jv <= vhi; ++jv) {
                const float vp = (float)jv - cv;
                const float hz = 1.0f - fabsf(fmaf(vp - va, E1, E0));
                if (hz > 0.0f) {
                    float w = hb * hz;
                    if (!WEIGHTED) {
                        const float rz = fmaf(vp, t2.w, t1.w);  // (Wc_z + u' Eu_z + v' Ev_z) / w_a
                        w *= sqrtf(fmaf(rz, rz, fmaf(t0.y, t0.y, 1.0f))) * a.h;
                    }
                    SinoLoad<NCH, ST>::add(sino_view, (size_t)jv * a.nu + ju, w, acc[zz]);
                }
            }
        }
    }
}

// NF: floats of each table staged (VG_HI: the float32 part; 64: all of it)
template <typename ST, int NF = VG_HI>
__device__ __forceinline__ void stage_views(ViewGeom *Gs, const BPArgs &a, int c0, int cn, int tid, int nthreads) {
    for (int t = tid; t < cn * NF; t += nthreads) {
        const int vi = t / NF, e = t % NF;
        reinterpret_cast<float *>(&Gs[vi])[e] =
            __ldg(reinterpret_cast<const float *>(a.views + a.view0 + (c0 + vi) * a.stride) + e);
    }
}

template <int NCH, typename ST, bool WEIGHTED>
__global__ void __launch_bounds__(BP_BX *BP_BY *BP_BZ)
    k_backproject(BPArgs a, const ST *__restrict__ sino, float *__restrict__ out, int accumulate) {
    __shared__ ViewGeom Gs[BP_CHUNK];
    const int jx = blockIdx.x * BP_BX + threadIdx.x;
    const int jy = blockIdx.y * BP_BY + threadIdx.y;
    const int jz = blockIdx.z * BP_BZ + threadIdx.z;
    const bool active = jx < a.n && jy < a.n && jz < a.n;
    const int tid = threadIdx.x + BP_BX * (threadIdx.y + BP_BY * threadIdx.z);
    float acc[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) acc[c] = 0.0f;
    const size_t view_elems = (size_t)a.nu * a.nv;
    for (int c0 = 0; c0 < a.nviews; c0 += BP_CHUNK) {
        const int cn = min(BP_CHUNK, a.nviews - c0);
        __syncthreads();
        stage_views<ST, sizeof(ViewGeom) / 4>(Gs, a, c0, cn, tid, BP_BX * BP_BY * BP_BZ);
        __syncthreads();
        if (active) {
            for (int vi = 0; vi < cn; ++vi)
                bp_view<NCH, ST, WEIGHTED>(Gs[vi], a, jx, jy, jz, sino + (size_t)(c0 + vi) * view_elems, acc);
        }
    }
    if (!active) return;
    const size_t idx = ((size_t)jz * a.n + jy) * a.n + jx;
    const size_t nvox = (size_t)a.n * a.n * a.n;
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        float v = acc[c];
        if (accumulate) v += out[idx + c * nvox];
        out[idx + c * nvox] = v;
    }
}

constexpr int BPS_ZB = 4;  // voxels per thread along z (separable kernel)

template <int NCH, typename ST, bool WEIGHTED>
__global__ void __launch_bounds__(BP_BX *BP_BY *BP_BZ)
    k_backproject_sep(BPArgs a, const float4 *__restrict__ cols, const ST *__restrict__ sino, float *__restrict__ out,
                      int accumulate) {
    __shared__ ViewGeom Gs[BP_CHUNK];
    const int jx = blockIdx.x * BP_BX + threadIdx.x;
    const int jy = blockIdx.y * BP_BY + threadIdx.y;
    const int jz0 = (blockIdx.z * BP_BZ + threadIdx.z) * BPS_ZB;
    const bool active = jx < a.n && jy < a.n && jz0 < a.n;
    const int tid = threadIdx.x + BP_BX * (threadIdx.y + BP_BY * threadIdx.z);
    float acc[BPS_ZB][NCH];
#pragma unroll
    for (int z = 0; z < BPS_ZB; ++z)
#pragma unroll
        for (int c = 0; c < NCH; ++c) acc[z][c] = 0.0f;
    const size_t view_elems = (size_t)a.nu * a.nv;
    for (int c0 = 0; c0 < a.nviews; c0 += BP_CHUNK) {
        const int cn = min(BP_CHUNK, a.nviews - c0);
        __syncthreads();
        stage_views<ST>(Gs, a, c0, cn, tid, BP_BX * BP_BY * BP_BZ);
        __syncthreads();
        if (active) {
            for (int vi = 0; vi < cn; ++vi)
                bp_view_sep<NCH, ST, WEIGHTED, BPS_ZB>(Gs[vi], cols + (size_t)(a.view0 + (c0 + vi) * a.stride) * a.nu * 4,
                                                       a, jx, jy, jz0,
                                                       sino + (size_t)(c0 + vi) * view_elems, acc);
        }
    }
    if (!active) return;
    const size_t nvox = (size_t)a.n * a.n * a.n;
#pragma unroll
    for (int z = 0; z < BPS_ZB; ++z) {
        if (jz0 + z >= a.n) break;
        const size_t idx = ((size_t)(jz0 + z) * a.n + jy) * a.n + jx;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            float v = acc[z][c];
            if (accumulate) v += out[idx + c * nvox];
            out[idx + c * nvox] = v;
        }
    }
}

// Separable geometry, weighted sinogram: the solver's hot path.
// Each thread owns one (x, y) voxel column and a slab of Z voxels along z,
// accumulated in shared memory.  Per view and per detector column u' whose
// rays meet the voxel column (|e_b| < 1), the z crossing of the ray through
// pixel (u', v') is f_z(v') = E0' + v' E1 (E0' uncentred), so the voxels the
// ray touches are floor(f_z) and floor(f_z) + 1 with weights (1 - t, t),
// t = f_z - floor(f_z): the exact transpose of the projector's bilinear tap
// in z.  Each pixel of the slab's v range is visited once and splatted into
// the thread's own shared-memory column (no two threads share a column, so
// no atomics, and the order of additions is fixed).  Lanes are adjacent x
// columns, so the pixel reads of a warp fall on one detector row.
constexpr int BS_TX = 32, BS_TY = 4, BS_THREADS = BS_TX * BS_TY;
constexpr float BS_MAGIC = 12582912.0f;  // 1.5 * 2^23
constexpr int BS_MAGIC_BITS = 0x4B400000;

#ifndef MGCT_BS_PAIRS
#define MGCT_BS_PAIRS 1
#endif
#ifndef MGCT_BS_REG
#define MGCT_BS_REG 1
#endif
template <int NCH>
struct SlabCfg {
    // voxels per slab: 16 keeps the shared slab at 10 KB so that 16 blocks
    // (64 warps) fit per SM; measured 64 -> 32 -> 16: 74 -> 63 -> 55 ms per
    // grid-0 launch at 256^3 / 720 views
    static constexpr int Z = 16 / NCH;
    static constexpr int ROWS = Z + 5;  // guard rows: two below, three above (row pairs reach r + 2)
};

// DFA = true: the public A^T at any N.  The column comes from the double-
// float table and its z crossing is anchored, in double-float, at the detector
// row nearest the slab's centre, so the crossings are stepped in float32 from
// a small height relative to the slab (accurate to ~1e-6 voxel at any N; the
// float32 table's uncentred heights near z = 1000 carry ~6e-5).
template <int NCH, typename ST, bool DFA = false>
__global__ void __launch_bounds__(BS_THREADS)
    k_backproject_slab(BPArgs a, const float4 *__restrict__ cols, const ST *__restrict__ sino,
                       float *__restrict__ out, int accumulate) {
    constexpr int Z = SlabCfg<NCH>::Z, ROWS = SlabCfg<NCH>::ROWS;
    constexpr int CW = DFA ? 4 : 2;  // float4 per table entry
    __shared__ float acc[NCH][ROWS][BS_THREADS];
    const int tid = threadIdx.x;
    const int jx = blockIdx.x * BS_TX + (tid % BS_TX), jy = blockIdx.y * BS_TY + tid / BS_TX;
    // blockIdx.z = split * (z-slabs) + slab; split s takes views [i0, i1)
    // and writes partial volume s of `out`
    const int splits = DFA ? 1 : a.splits;  // the public form never splits
    const int zblocks = gridDim.z / splits;
    const int split = blockIdx.z / zblocks;
    const int z0 = (blockIdx.z - split * zblocks) * Z;
    const int per = (a.nviews + splits - 1) / splits;
    const int i0 = split * per, i1 = min(a.nviews, i0 + per);
#pragma unroll
    for (int q = 0; q < NCH; ++q)
        for (int r = 0; r < ROWS; ++r) acc[q][r][tid] = 0.0f;
    if (jx < a.n && jy < a.n) {
        const float ic = 0.5f * (float)(a.n - 1);
        const float cu = 0.5f * (float)(a.nu - 1), cv = 0.5f * (float)(a.nv - 1);
        const float cx = (float)jx - ic, cy = (float)jy - ic;
        const float zlo = (float)z0 - 1.0f, zhi = (float)(z0 + Z);  // crossings that touch the slab
        const size_t view_elems = (size_t)a.nu * a.nv;
        for (int i = i0; i < i1; ++i) {
            const int k = a.view0 + i * a.stride;
            const float *G = reinterpret_cast<const float *>(a.views + k);
            // projected u range of the voxel column (the cube bound; z-free without tilt)
            const float X = (float)jx - __ldg(G + 0), Y = (float)jy - __ldg(G + 1);
            const float Q0 = __ldg(G + 12), Q1 = __ldg(G + 13), Q6 = __ldg(G + 18), Q7 = __ldg(G + 19);
            const float q2 = fmaf(Q7, Y, Q6 * X);
            const float u0 = fmaf(Q1, Y, Q0 * X) * __frcp_rn(q2);
            const float hu = (fabsf(Q0 - u0 * Q6) + fabsf(Q1 - u0 * Q7)) * __frcp_rn(q2 - __ldg(G + 21));
            const int ulo = max(0, (int)ceilf(u0 - hu + cu - 1e-3f));
            const int uhi = min(a.nu - 1, (int)floorf(u0 + hu + cu + 1e-3f));
            const ST *__restrict__ sv = sino + (size_t)i * view_elems;
            const float4 *__restrict__ ct = cols + (size_t)k * a.nu * CW;
            for (int ju = ulo; ju <= uhi; ++ju) {
                const float4 t0 = __ldg(ct + CW * ju);
                const float4 t1 = __ldg(ct + CW * ju + 1);
                const bool ay = t0.x != 0.0f;
                const float ca = ay ? cy : cx, cb = ay ? cx : cy;
                // E0, E1: crossing height at row offset vf = 0 and its slope per
                // row; zb: the height E0 is counted from (uncentred z)
                float hb, E0, E1, vf;
                int vlo, vhi, zb;
                if constexpr (!DFA) {
                    hb = 1.0f - fabsf(fmaf(ca, t0.y, t0.z) - cb);
                    if (hb <= 0.0f) continue;
                    E0 = fmaf(ca, t1.x, t0.w) + ic;  // uncentred z crossing at v' = 0
                    E1 = fmaf(ca, t1.z, t1.y);
                    const float rE = __frcp_rn(E1);
                    const float ta = fmaf(zlo - E0, rE, cv), tb = fmaf(zhi - E0, rE, cv);
                    vlo = max(0, (int)ceilf(fminf(ta, tb) - 1e-3f));
                    vhi = min(a.nv - 1, (int)floorf(fmaxf(ta, tb) + 1e-3f));
                    vf = (float)vlo - cv;
                    zb = z0;
                } else {
                    const float4 t2 = __ldg(ct + CW * ju + 2), t3 = __ldg(ct + CW * ju + 3);
                    const DF eb = df_add(df_mul_f(DF{t0.y, t0.z}, ca), DF{t0.w, t1.x});
                    hb = 1.0f - fabsf(__fadd_rn(__fsub_rn(eb.hi, cb), eb.lo));
                    if (hb <= 0.0f) continue;
                    const DF Eb = df_add(DF{t1.y, t1.z}, df_mul_f(DF{t1.w, t2.x}, ca));   // centred, v' = 0
                    const DF E1d = df_add(DF{t2.y, t2.z}, df_mul_f(DF{t2.w, t3.x}, ca));
                    E1 = E1d.hi;
                    const float zc = (float)z0 - ic + 0.5f * (float)(Z - 1);  // slab centre, centred (exact)
                    const float va = rintf((zc - Eb.hi) / E1);                // anchor row, centred v'
                    if (!(fabsf(va) < 1.0e7f)) continue;
                    const DF c = df_add(df_add(Eb, df_mul_f(E1d, va)), DF{-zc, 0.0f});
                    E0 = (c.hi + c.lo) + 0.5f * (float)(Z - 1);  // height above z0 at the anchor row
                    const float rE = __frcp_rn(E1);
                    const float ta = fmaf(-1.0f - E0, rE, va + cv), tb = fmaf((float)Z - E0, rE, va + cv);
                    vlo = max(0, (int)ceilf(fminf(ta, tb) - 1e-3f));
                    vhi = min(a.nv - 1, (int)floorf(fmaxf(ta, tb) + 1e-3f));
                    vf = ((float)vlo - cv) - va;  // rows from the anchor (exact)
                    zb = 0;
                }
                const ST *__restrict__ px = sv + (size_t)vlo * a.nu + ju;
                int jv = vlo;
                if constexpr (NCH == 1) {
                  if (MGCT_BS_PAIRS && E1 > 0.0f && E1 < 0.999f) {
                    // two rows at a time: their crossings floor(fz) are equal or
                    // one apart (0 < E1 < 1), so the pair touches three slab
                    // rows r, r + 1, r + 2 -- three read-modify-writes, not four
                    // floor(fz) from one addition rounded toward minus infinity
                    // (fz + 1.5 * 2^23 holds it in its low mantissa bits); a
                    // row index outside the slab wraps, as unsigned, to the top
                    // guard rows
                    const int rbase = BS_MAGIC_BITS + zb - 2;
                    for (; jv + 1 <= vhi; jv += 2, vf += 2.0f, px += 2 * (size_t)a.nu) {
                        const float fz0 = fmaf(vf, E1, E0), fz1 = fmaf(vf + 1.0f, E1, E0);
                        const float m0 = __fadd_rd(fz0, BS_MAGIC), m1 = __fadd_rd(fz1, BS_MAGIC);
                        const float t0 = fz0 - (m0 - BS_MAGIC), t1 = fz1 - (m1 - BS_MAGIC);
                        const int r = (int)min((unsigned)(__float_as_int(m0) - rbase), (unsigned)(ROWS - 3));
                        const bool same = __float_as_int(m1) == __float_as_int(m0);
                        const float y0 = hb * to_f32(__ldg(px)), y1 = hb * to_f32(__ldg(px + a.nu));
                        const float a0 = y0 * t0, b0 = y1 * t1;
                        const float lo1 = y1 - b0;
                        acc[0][r][tid] += (y0 - a0) + (same ? lo1 : 0.0f);
                        acc[0][r + 1][tid] += a0 + (same ? b0 : lo1);
                        if (!same) acc[0][r + 2][tid] += b0;
                    }
                  }
                }
                for (; jv <= vhi; ++jv, vf += 1.0f, px += a.nu) {
                    const float fz = fmaf(vf, E1, E0);
                    const float fl = floorf(fz);
                    const float t = fz - fl;
                    // row of voxel floor(fz) in the guarded slab: in [0, Z + 2]
                    const int r = min(max((int)fl - zb + 2, 0), ROWS - 2);
                    if constexpr (NCH == 1) {
                        const float yw = hb * to_f32(__ldg(px));
                        const float w1 = yw * t;
                        acc[0][r][tid] += yw - w1;
                        acc[0][r + 1][tid] += w1;
                    } else {
                        const float2 y2 = load_f2(px);
                        const float ya = hb * y2.x, yb = hb * y2.y;
                        acc[0][r][tid] += ya - ya * t;
                        acc[0][r + 1][tid] += ya * t;
                        acc[NCH - 1][r][tid] += yb - yb * t;
                        acc[NCH - 1][r + 1][tid] += yb * t;
                    }
                }
            }
        }
        const size_t nvox = (size_t)a.n * a.n * a.n;
        float *o = out + (size_t)split * NCH * nvox;
        for (int zz = 0; zz < Z; ++zz) {
            const int z = z0 + zz;
            if (z >= a.n) break;
            const size_t idx = ((size_t)z * a.n + jy) * a.n + jx;
#pragma unroll
            for (int q = 0; q < NCH; ++q) {
                float v = acc[q][zz + 2][tid];
                if (accumulate) v += o[idx + q * nvox];
                o[idx + q * nvox] = v;
            }
        }
    }
}

// Register form of the solver's A^T (separable geometry, weighted rows, one
// channel) for grids whose detector rows are finer than the voxels along z:
// 1/3 < E1 < 1 for every view, column and plane (LevelInfo::e1_lo / e1_hi).
// As in the slab kernel a thread owns one (x, y) voxel column and ZS voxels
// z0 .. z0 + ZS - 1 of it, but the slab lives in registers.  Measured from
// z0 - 1, a detector column's row crossings rise by E1 < 1 per row, so the
// unit interval j of heights, [j, j + 1), j = 0 .. ZS, holds floor(1/E1) or
// ceil(1/E1) rows (K = ceil(1/E1) slots, the later ones predicated).  With
// S_j the interval's sum of y and T_j its sum of y t (t = the row's height
// above j), the tent weights give voxel z0 - 1 + j the share hb (S_j - T_j)
// and voxel z0 + j the share hb T_j -- the slab kernel's two taps per row,
// summed per interval, every accumulator index fixed at compile time.
#ifndef MGCT_BR_BX
#define MGCT_BR_BX 32
#endif
#ifndef MGCT_BR_WX
#define MGCT_BR_WX 8
#endif
// a block is BR_TX x BR_TY voxel columns; a warp BR_WX x (32 / BR_WX) of them.
// Measured per grid-0 launch at 256^3 / 720 views (512^3 / 1440): warps of
// 32 x 1 columns 31.2 ms (452), 16 x 2 30.2 (442), 8 x 4 29.5 (435), and
// 4 x 8 or 8 x 4 in 16 x 8 and 8 x 16 blocks 29.4-29.8 (433-439): on views
// whose rays run along a warp's long side, its lanes' detector columns and
// rows spread apart
constexpr int BR_TX = MGCT_BR_BX, BR_TY = 128 / BR_TX, BR_THREADS = BR_TX * BR_TY;
constexpr int BR_WX = MGCT_BR_WX, BR_WY = 32 / BR_WX;
static_assert(BR_TX % BR_WX == 0 && BR_TY % BR_WY == 0, "warp tiles must tile the block");
#ifndef MGCT_BR_Z
#define MGCT_BR_Z 16
#endif
// measured at 256^3 / 720 views per grid-0 launch (slab kernel 42.5 ms):
// 16 voxels, the later slots' rows loaded before their test, 40 registers
// (12 blocks per SM), the exact column range 31.1 ms; with the cube bound's
// column range 35.1 (each lane's weighted columns start at a different
// iteration, so a warp runs more of the expensive ones); with 24 voxels
// 37.9, with 8 voxels 57.1; with the loads behind the test 38.2; without the
// register cap (118 registers) 55.7 (cube bound for these five)
#ifndef MGCT_BR_UNCOND
#define MGCT_BR_UNCOND 1
#endif
#ifndef MGCT_BR_MINB
#define MGCT_BR_MINB 12
#endif
#ifndef MGCT_BR_EXACT
#define MGCT_BR_EXACT 1
#endif
constexpr int BR_Z = MGCT_BR_Z;                        // voxels per thread along z
constexpr float BR_E1_LO = 1.0f / 3.0f + 1e-3f;        // eligible grids: BR_E1_LO < E1 < BR_E1_HI
constexpr float BR_E1_HI = 1.0f - 1e-3f;
constexpr float BR_K2 = 0.5f + 1e-3f;                  // E1 above this: at most two rows per interval

// One detector column's rows into acc: off is the element offset of the
// first row (row v, height w in [0, E1) above z0 - 1) in the view's
// sinogram.  EDGE: rows outside [0, nv) read as zero (not loaded).
template <int ZS, int K, bool EDGE, typename ST>
__device__ __forceinline__ void br_column(float (&acc)[ZS], const ST *__restrict__ sv, int off, int nu, float w,
                                          float E1, float hb, int v, int nv) {
#pragma unroll
    for (int j = 0; j <= ZS; ++j) {
        float y = 0.0f;
        if (!EDGE || (unsigned)v < (unsigned)nv) y = to_f32(__ldg(sv + off));
        float S = y, T = y * w;
        float wn = w + E1;  // height of the next row above j
        int adv = 1;
#pragma unroll
        for (int s = 1; s < K; ++s) {
            if (MGCT_BR_UNCOND && !EDGE) {
                // the row after the interval's last lies within the rows the
                // launch checked, so the load need not wait for the test
                const float yl = to_f32(__ldg(sv + off + s * nu));
                const bool in = wn < 1.0f;
                const float ys = in ? yl : 0.0f;
                S += ys;
                T = fmaf(ys, wn, T);
                if (in) {
                    wn += E1;
                    adv = s + 1;
                }
            } else if (wn < 1.0f) {
                float ys = 0.0f;
                if (!EDGE || (unsigned)(v + s) < (unsigned)nv) ys = to_f32(__ldg(sv + off + s * nu));
                S += ys;
                T = fmaf(ys, wn, T);
                wn += E1;
                adv = s + 1;
            }
        }
        if (j >= 1) acc[j - 1] = fmaf(hb, S - T, acc[j - 1]);
        if (j < ZS) acc[j] = fmaf(hb, T, acc[j]);
        w = wn - 1.0f;  // the first row of interval j + 1
        off += adv * nu;
        if (EDGE) v += adv;
    }
}

// Detector column ju of the view whose sinogram is sv into acc, weighted hb:
// E0 is the uncentred z crossing of its rays at v' = 0 and E1 its step per
// row, at the voxel column's plane; the slab's intervals start at zlo.
template <int ZS, typename ST>
__device__ __forceinline__ void br_add_column(float (&acc)[ZS], const ST *__restrict__ sv, int ju, int nu, int nv,
                                              float E0, float E1, float hb, float zlo, float cv) {
    // the launch checks the grid's range of E1; this keeps every read in
    // bounds whatever the table holds
    if (!(E1 > 0.3f && E1 < 1.0f)) return;
    const float rE = __frcp_rn(E1);
    // first row at or above z0 - 1 (one correction for the rounded quotient)
    float vf = ceilf(fmaf(zlo - E0, rE, cv));
    if (!(fabsf(vf) < 1.0e7f)) return;
    float w = fmaf(vf - cv, E1, E0) - zlo;
    if (w < 0.0f) {
        vf += 1.0f;
        w += E1;
    } else if (w >= E1) {
        vf -= 1.0f;
        w -= E1;
    }
    const int vs = (int)vf;
    // rows read: those of heights [0, ZS + 1), at most (ZS + 1) / E1 + 1 (the
    // truncation below loses one), one more for the drift of the stepped
    // heights, two after the last that the unconditional slots may read, and
    // one spare
    constexpr int nrb_max = (int)((float)(ZS + 1) / BR_E1_LO) + 6;
    const int nrb = min(nrb_max, (int)((float)(ZS + 1) * rE) + 6);
    if (vs >= nv || vs + nrb <= 0) return;
    const int off = vs * nu + ju;
    if (vs >= 0 && vs + nrb <= nv) {
        if (E1 > BR_K2) br_column<ZS, 2, false>(acc, sv, off, nu, w, E1, hb, vs, nv);
        else br_column<ZS, 3, false>(acc, sv, off, nu, w, E1, hb, vs, nv);
    } else {
        if (E1 > BR_K2) br_column<ZS, 2, true>(acc, sv, off, nu, w, E1, hb, vs, nv);
        else br_column<ZS, 3, true>(acc, sv, off, nu, w, E1, hb, vs, nv);
    }
}

template <typename ST, int ZS>
__global__ void __launch_bounds__(BR_THREADS, MGCT_BR_MINB)
    k_backproject_reg(BPArgs a, const float4 *__restrict__ cols, const ST *__restrict__ sino,
                      float *__restrict__ out, int accumulate) {
    const int tid = threadIdx.x;
    const int w = tid >> 5, l = tid & 31;
    const int jx = blockIdx.x * BR_TX + (w % (BR_TX / BR_WX)) * BR_WX + l % BR_WX;
    const int jy = blockIdx.y * BR_TY + (w / (BR_TX / BR_WX)) * BR_WY + l / BR_WX;
    // blockIdx.z = split * (z-slabs) + slab, as in k_backproject_slab
    const int zblocks = gridDim.z / a.splits;
    const int split = blockIdx.z / zblocks;
    const int z0 = (blockIdx.z - split * zblocks) * ZS;
    const int per = (a.nviews + a.splits - 1) / a.splits;
    const int i0 = split * per, i1 = min(a.nviews, i0 + per);
    if (jx >= a.n || jy >= a.n) return;
    float acc[ZS];
#pragma unroll
    for (int q = 0; q < ZS; ++q) acc[q] = 0.0f;
    const float ic = 0.5f * (float)(a.n - 1);
    const float cu = 0.5f * (float)(a.nu - 1), cv = 0.5f * (float)(a.nv - 1);
    const float cx = (float)jx - ic, cy = (float)jy - ic;
    const float zlo = (float)z0 - 1.0f;  // interval 0 starts here
    const size_t view_elems = (size_t)a.nu * a.nv;
    for (int i = i0; i < i1; ++i) {
        const int k = a.view0 + i * a.stride;
        const float *G = reinterpret_cast<const float *>(a.views + k);
        const float X = (float)jx - __ldg(G + 0), Y = (float)jy - __ldg(G + 1);
        const float Q0 = __ldg(G + 12), Q1 = __ldg(G + 13), Q6 = __ldg(G + 18), Q7 = __ldg(G + 19);
        const float q0 = fmaf(Q1, Y, Q0 * X), q2 = fmaf(Q7, Y, Q6 * X);
        int ulo, uhi;
        if (MGCT_BR_EXACT) {
            // a column of x-major rays weights this voxel column iff its rays
            // cross the plane x = jx strictly between y = jy - 1 and jy + 1,
            // i.e. iff its u lies between the projections of those two
            // points; likewise (jx -+ 1, jy) for y-major rays.  Both intervals
            // hold the voxel column's own projection, so their union is the
            // interval from the least to the greatest of the four.
            const float ua = (q0 - Q1) * __frcp_rn(q2 - Q7), ub = (q0 + Q1) * __frcp_rn(q2 + Q7);
            const float uc = (q0 - Q0) * __frcp_rn(q2 - Q6), ud = (q0 + Q0) * __frcp_rn(q2 + Q6);
            const float umin = fminf(fminf(ua, ub), fminf(uc, ud)), umax = fmaxf(fmaxf(ua, ub), fmaxf(uc, ud));
            ulo = max(0, (int)ceilf(umin + cu - 1e-3f));
            uhi = min(a.nu - 1, (int)floorf(umax + cu + 1e-3f));
        } else {
            // projected u range of the voxel column (the cube bound)
            const float u0 = q0 * __frcp_rn(q2);
            const float hu = (fabsf(Q0 - u0 * Q6) + fabsf(Q1 - u0 * Q7)) * __frcp_rn(q2 - __ldg(G + 21));
            ulo = max(0, (int)ceilf(u0 - hu + cu - 1e-3f));
            uhi = min(a.nu - 1, (int)floorf(u0 + hu + cu + 1e-3f));
        }
        const ST *__restrict__ sv = sino + (size_t)i * view_elems;
        const float4 *__restrict__ ct = cols + (size_t)k * a.nu * 2;
        for (int ju = ulo; ju <= uhi; ++ju) {
            const float4 t0 = __ldg(ct + 2 * ju);
            const float4 t1 = __ldg(ct + 2 * ju + 1);
            const bool ay = t0.x != 0.0f;
            const float ca = ay ? cy : cx, cb = ay ? cx : cy;
            const float hb = 1.0f - fabsf(fmaf(ca, t0.y, t0.z) - cb);
            if (hb <= 0.0f) continue;
            br_add_column<ZS>(acc, sv, ju, a.nu, a.nv, fmaf(ca, t1.x, t0.w) + ic, fmaf(ca, t1.z, t1.y), hb, zlo, cv);
        }
    }
    const size_t nvox = (size_t)a.n * a.n * a.n;
    float *o = out + (size_t)split * nvox;
#pragma unroll
    for (int zz = 0; zz < ZS; ++zz) {
        const int z = z0 + zz;
        if (z < a.n) {
            const size_t idx = ((size_t)z * a.n + jy) * a.n + jx;
            float v = acc[zz];
            if (accumulate) v += o[idx];
            o[idx] = v;
        }
    }
}

// Column table (see LevelInfo::d_cols): one thread per (view, column); the
// axis choice is the projector's own ray_dir() at v' = 0.
__global__ void k_column_table(const ViewGeom *__restrict__ views, int K, int nu, float4 *__restrict__ cols) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K * nu) return;
    const int k = t / nu, ju = t % nu;
    const ViewGeom &G = views[k];
    const float up = (float)ju - 0.5f * (float)(nu - 1);
    const RayDir d = ray_dir(G, up, 0.0f);
    const float wa = d.ax ? d.wy : d.wx, wb = d.ax ? d.wx : d.wy;
    const float rinv = __frcp_rn(wa);
    const float *N = d.ax ? G.NY : G.NX;
    cols[2 * (size_t)t] = make_float4(d.ax ? 1.0f : 0.0f, wb * rinv, fmaf(up, N[1], N[0]) * rinv,
                                      fmaf(up, N[4], N[3]) * rinv);
    cols[2 * (size_t)t + 1] = make_float4(G.Wc[2] * rinv, N[5] * rinv, G.Ev[2] * rinv, 0.0f);
}

// Double-float column table (see LevelInfo::d_cols_df): same axis choice as
// k_column_table; the quotients by w_a are taken in double-float from the
// view table's double-float fields.
__global__ void k_column_table_df(const ViewGeom *__restrict__ views, int K, int nu, float4 *__restrict__ cols) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K * nu) return;
    const int k = t / nu, ju = t % nu;
    const ViewGeom &G = views[k];
    const float up = (float)ju - 0.5f * (float)(nu - 1);
    const RayDir d = ray_dir(G, up, 0.0f);
    const int ia = d.ax, ib = 1 - d.ax;
    const DF wa = df_affine(G.Wc[ia], G.Wc_lo[ia], G.Eu[ia], G.Eu_lo[ia], G.Ev[ia], G.Ev_lo[ia], up, 0.0f);
    const DF wb = df_affine(G.Wc[ib], G.Wc_lo[ib], G.Eu[ib], G.Eu_lo[ib], G.Ev[ib], G.Ev_lo[ib], up, 0.0f);
    const DF rinv = df_div(DF{1.0f, 0.0f}, wa);
    const float *N = d.ax ? G.NY : G.NX;
    const float *Nl = d.ax ? G.NY_lo : G.NX_lo;
    const DF rb = df_mul(wb, rinv);
    const DF pb = df_mul(df_affine(N[0], Nl[0], N[1], Nl[1], N[2], Nl[2], up, 0.0f), rinv);
    const DF ez0 = df_mul(df_affine(N[3], Nl[3], N[4], Nl[4], N[5], Nl[5], up, 0.0f), rinv);
    const DF ezc = df_mul(df_affine(G.Wc[2], G.Wc_lo[2], G.Eu[2], G.Eu_lo[2], G.Ev[2], G.Ev_lo[2], up, 0.0f), rinv);
    const DF e10 = df_mul(DF{N[5], Nl[5]}, rinv);
    const DF e1c = df_mul(DF{G.Ev[2], G.Ev_lo[2]}, rinv);
    float4 *o = cols + 4 * (size_t)t;
    o[0] = make_float4(d.ax ? 1.0f : 0.0f, rb.hi, rb.lo, pb.hi);
    o[1] = make_float4(pb.lo, ez0.hi, ez0.lo, ezc.hi);
    o[2] = make_float4(ezc.lo, e10.hi, e10.lo, e1c.hi);
    o[3] = make_float4(e1c.lo, 0.0f, 0.0f, 0.0f);
}

// out = (accumulate ? out : 0) + sum over s of part[s], in order of s.
__global__ void k_sum_splits(size_t len, int splits, const float *__restrict__ part, float *__restrict__ out,
                             int accumulate) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x) {
        float v = accumulate ? out[i] : 0.0f;
        for (int q = 0; q < splits; ++q) v += __ldg(part + (size_t)q * len + i);
        out[i] = v;
    }
}

// Number of view ranges for a slab launch of `blocks` blocks: enough for
// about four waves of resident blocks in all, as grid 0 has (coarse grids and
// OS-EMTR subsets otherwise fill a fraction of the SMs, and a launch of one
// or two waves loses its tail), at most 16 and what `cap` floats of partial
// volumes hold.
template <typename KF>
int slab_splits(KF kernel, int blocks, int nviews, size_t vol_floats, size_t cap) {
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, BS_THREADS, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int sp = (4 * sms * occ + blocks - 1) / blocks;
    if (sp > 16) sp = 16;
    if (sp > nviews) sp = nviews;
    if ((size_t)sp * vol_floats > cap) sp = (int)(cap / vol_floats);
    return sp < 1 ? 1 : sp;
}

// The register kernel's launch (see k_backproject_reg), with the slab
// kernel's view splits.
template <typename ST>
int launch_backproject_reg(const LevelInfo &L, BPArgs a, const ST *sino, float *out, int accumulate, cudaStream_t s,
                           float *split_buf, size_t cap) {
    dim3 grid((L.n + BR_TX - 1) / BR_TX, (L.n + BR_TY - 1) / BR_TY, (L.n + BR_Z - 1) / BR_Z);
    const size_t vol_floats = (size_t)L.n * L.n * L.n;
    if (split_buf && a.nviews > 1)
        a.splits = slab_splits(k_backproject_reg<ST, BR_Z>, (int)(grid.x * grid.y * grid.z), a.nviews, vol_floats,
                               cap);
    if (a.splits == 1) {
        MGCT_KERNEL(KK_BACKPROJECT, s,
                    k_backproject_reg<ST, BR_Z><<<grid, BR_THREADS, 0, s>>>(a, L.d_cols, sino, out, accumulate));
    } else {
        grid.z *= a.splits;
        MGCT_KERNEL(KK_BACKPROJECT, s,
                    k_backproject_reg<ST, BR_Z><<<grid, BR_THREADS, 0, s>>>(a, L.d_cols, sino, split_buf, 0));
        const int sb = (int)((vol_floats + 255) / 256 < 4096 ? (vol_floats + 255) / 256 : 4096);
        MGCT_KERNEL(KK_BACKPROJECT, s, k_sum_splits<<<sb, 256, 0, s>>>(vol_floats, a.splits, split_buf, out, accumulate));
    }
    return MGCT_OK;
}

// NCH = 2 writes channel c to out + c * n^3.  WEIGHTED: the sinogram carries
// each ray's dl already (internal solver path).  split_buf (cap floats, or
// NULL): scratch for partial volumes, with which an under-filled slab launch
// splits its views into ranges summed afterwards in a fixed order.
template <int NCH, typename ST, bool WEIGHTED = false>
int launch_backproject(const mgct_geom *g, int level, int view0, int nviews, int stride, const ST *sino,
                       float *out, int accumulate, cudaStream_t s, float *split_buf = nullptr, size_t cap = 0) {
    const LevelInfo &L = g->lev[level];
    BPArgs a;
    a.views = L.d_views;
    a.n = L.n;
    a.nu = L.nu;
    a.nv = L.nv;
    a.h = (float)L.h;
    a.view0 = view0;
    a.stride = stride;
    a.nviews = nviews;
    a.splits = 1;
    if (MGCT_BS_REG && NCH == 1 && g->separable && WEIGHTED && L.d_cols && L.e1_lo > BR_E1_LO &&
        L.e1_hi < BR_E1_HI && (size_t)L.nu * (L.nv + 64) < ((size_t)1 << 31)) {
        if constexpr (NCH == 1) return launch_backproject_reg<ST>(L, a, sino, out, accumulate, s, split_buf, cap);
    } else if (g->separable && WEIGHTED && L.d_cols) {
        constexpr int Z = SlabCfg<NCH>::Z;
        dim3 grid((L.n + BS_TX - 1) / BS_TX, (L.n + BS_TY - 1) / BS_TY, (L.n + Z - 1) / Z);
        const size_t vol_floats = (size_t)NCH * L.n * L.n * L.n;
        if (split_buf && nviews > 1)
            a.splits = slab_splits(k_backproject_slab<NCH, ST>, (int)(grid.x * grid.y * grid.z), nviews, vol_floats,
                                   cap);
        if (a.splits == 1) {
            MGCT_KERNEL(KK_BACKPROJECT, s,
                        k_backproject_slab<NCH, ST><<<grid, BS_THREADS, 0, s>>>(a, L.d_cols, sino, out, accumulate));
        } else {
            grid.z *= a.splits;
            MGCT_KERNEL(KK_BACKPROJECT, s,
                        k_backproject_slab<NCH, ST><<<grid, BS_THREADS, 0, s>>>(a, L.d_cols, sino, split_buf, 0));
            const int sb = (int)((vol_floats + 255) / 256 < 4096 ? (vol_floats + 255) / 256 : 4096);
            MGCT_KERNEL(KK_BACKPROJECT, s,
                        k_sum_splits<<<sb, 256, 0, s>>>(vol_floats, a.splits, split_buf, out, accumulate));
        }
    } else if (g->separable) {
        const int zper = BP_BZ * BPS_ZB;
        dim3 grid((L.n + BP_BX - 1) / BP_BX, (L.n + BP_BY - 1) / BP_BY, (L.n + zper - 1) / zper);
        MGCT_KERNEL(KK_BACKPROJECT, s,
                    k_backproject_sep<NCH, ST, WEIGHTED><<<grid, dim3(BP_BX, BP_BY, BP_BZ), 0, s>>>(a, L.d_cols_df, sino, out, accumulate));
    } else {
        dim3 grid((L.n + BP_BX - 1) / BP_BX, (L.n + BP_BY - 1) / BP_BY, (L.n + BP_BZ - 1) / BP_BZ);
        MGCT_KERNEL(KK_BACKPROJECT, s,
                    k_backproject<NCH, ST, WEIGHTED><<<grid, dim3(BP_BX, BP_BY, BP_BZ), 0, s>>>(a, sino, out, accumulate));
    }
    return MGCT_OK;
}

// The public A^T on tilt-free geometries.  Each ray's path length per plane,
// dl = h sqrt(1 + rb^2 + rz^2) (the projector's weight; rb per column, rz
// linear in v', both from the double-float column table), is applied to the
// caller's sinogram in one pass over it, written to the handle's quad scratch,
// and the weighted rows are splatted by the double-float-anchored slab
// kernel: the solver's scatter, for one extra read and write of the sinogram.
template <typename ST>
__global__ void k_weight_rays(BPArgs a, const float4 *__restrict__ cols, const ST *__restrict__ sino,
                              float *__restrict__ w) {
    const int ju = blockIdx.x * blockDim.x + threadIdx.x;
    if (ju >= a.nu) return;
    const int jv = blockIdx.y, i = blockIdx.z;
    const int k = a.view0 + i * a.stride;
    const float *c = reinterpret_cast<const float *>(cols + ((size_t)k * a.nu + ju) * 4);
    const float rb = __ldg(c + 1), ezc = __ldg(c + 7), e1c = __ldg(c + 11);  // rb, (Wc_z + u' Eu_z)/w_a, Ev_z/w_a
    const float rz = fmaf((float)jv - 0.5f * (float)(a.nv - 1), e1c, ezc);
    const float dl = sqrtf(fmaf(rz, rz, fmaf(rb, rb, 1.0f))) * a.h;
    const size_t idx = ((size_t)i * a.nv + jv) * a.nu + ju;
    w[idx] = dl * to_f32(__ldg(sino + idx));
}

// Runs the public A^T through k_weight_rays and the slab kernel, in chunks of
// views that fit the quad scratch, and sets *ran; leaves *ran = 0 (nothing
// launched) where it does not apply: tilted detectors, no views, or a
// scratch smaller than one view.
template <typename ST>
int launch_backproject_public(const mgct_geom *g, int level, int view0, int nviews, int stride, const ST *sino,
                              float *out, int accumulate, cudaStream_t s, int *ran) {
    *ran = 0;
    const LevelInfo &L = g->lev[level];
    const size_t view_elems = (size_t)L.nu * L.nv;
    const size_t cap = 2 * quad_elems(g->lev[0].n) * 4;  // floats in the quad scratch
    if (!g->separable || !L.d_cols_df || nviews < 1 || cap < view_elems || L.nv > 65535) return MGCT_OK;
    size_t chunk = cap / view_elems;
    if (chunk > (size_t)nviews) chunk = nviews;
    if (chunk > 65535) chunk = 65535;
    float *w = static_cast<float *>(g->d_scratch_quads);
    BPArgs a;
    a.views = L.d_views;
    a.n = L.n;
    a.nu = L.nu;
    a.nv = L.nv;
    a.h = (float)L.h;
    a.stride = stride;
    a.splits = 1;
    constexpr int Z = SlabCfg<1>::Z;
    const dim3 grid((L.n + BS_TX - 1) / BS_TX, (L.n + BS_TY - 1) / BS_TY, (L.n + Z - 1) / Z);
    for (int c0 = 0; c0 < nviews; c0 += (int)chunk) {
        const int cn = nviews - c0 < (int)chunk ? nviews - c0 : (int)chunk;
        a.view0 = view0 + c0 * stride;
        a.nviews = cn;
        const dim3 wgrid((L.nu + 127) / 128, L.nv, cn);
        MGCT_KERNEL(KK_BACKPROJECT, s,
                    k_weight_rays<ST><<<wgrid, 128, 0, s>>>(a, L.d_cols_df, sino + (size_t)c0 * view_elems, w));
        MGCT_KERNEL(KK_BACKPROJECT, s,
                    k_backproject_slab<1, float, true><<<grid, BS_THREADS, 0, s>>>(a, L.d_cols_df, w, out,
                                                                                    (accumulate || c0) ? 1 : 0));
    }
    *ran = 1;
    return MGCT_OK;
}

}  // namespace mgct
