// Ray-driven forward projector A (Joseph's method) with fused epilogues.
//
// The projection operator P of Eq. 1 (Sec. 2) is discretised by Joseph's
// method: each ray is sampled at its crossings with the voxel-centre planes
// normal to its major axis, by bilinear interpolation within the plane, and
// each sample carries the path length between planes.  One thread per ray;
// a warp covers 32 adjacent detector columns of one detector row of one view,
// so at every plane the warp's taps fall on one or two contiguous rows of the
// volume copy whose fastest axis is the in-plane horizontal axis:
//   y-major rays sample plane y = i of vol  [z][y][x]  (taps along x, z)
//   x-major rays sample plane x = i of volT [z][x][y]  (taps along y, z)
#pragma once

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

}  // namespace mgct
