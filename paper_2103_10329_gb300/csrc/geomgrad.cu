// Per-view geometry gradient: d/dphi_k of sum_rays y_ray (A mu)_ray for the
// drift parameters phi_k = (ds_u, ds_v, dd_u, dd_v, psi) (Sec. 1: drift of
// the source and detector, to be estimated jointly with the image).
//
// At fixed major axis a and plane i, the crossing of the ray from S to the
// pixel P (index units, w = P - S) is f = S + t w with t = (i - S_a) / w_a.
// Moving S by dS and P by dP moves the in-plane crossing by
//   df_b = (1 - t)(dS_b - r_b dS_a) + t (dP_b - r_b dP_a),  r_b = w_b / w_a,
// likewise for z, and the path length per plane dl = h sqrt(1 + r_b^2 + r_z^2)
// by h (r_b dr_b + r_z dr_z) / sqrt(...), dr_b = (dw_b - r_b dw_a) / w_a.
// With B the bilinear interpolant, d(A mu)/dphi = d(dl) sum B + dl sum
// (dB/df_b df_b + dB/df_z df_z), so the ray march accumulates sum B,
// sum dB/df and sum t dB/df for both in-plane axes, and the chain rule to the
// five parameters is applied once per ray:
//   ds_u, ds_v: dS = one fine pixel along e_u / e_v;  dd_u, dd_v: dP likewise;
//   psi: dP = u' Ev - v' Eu (the pixel offset turned about the normal).
// The plane set and axis are held fixed (the integral is piecewise smooth).
#include "common.cuh"
#include "project.cuh"

namespace mgct {

struct GradArgs {
    ProjArgs p;
    const float *y;  // cotangent batch sinogram [i][v][u]
    double *part;    // [nviews][ublocks][5]
};

template <typename VT>
__global__ void __launch_bounds__(PJ_BX *PJ_BY)
    k_geom_grad(GradArgs ga, const VT *__restrict__ vol, const VT *__restrict__ volT) {
    __shared__ ViewGeom G;
    __shared__ double red[5 * PJ_BX * PJ_BY / 32];
    const ProjArgs &a = ga.p;
    const int i = blockIdx.y;
    const int k = a.view0 + i * a.stride;
    const int tid = threadIdx.x + threadIdx.y * PJ_BX;
    if (tid < 64) reinterpret_cast<float *>(&G)[tid] = __ldg(reinterpret_cast<const float *>(a.views + k) + tid);
    __syncthreads();
    const int n = a.n;
    const float ic = 0.5f * (float)(n - 1);
    const int ju = blockIdx.x * PJ_BX + threadIdx.x;
    double gsum[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int v0 = 0; v0 < a.nv; v0 += PJ_BY) {
        const int jv = v0 + threadIdx.y;
        if (ju >= a.nu || jv >= a.nv) continue;
        const float yv = __ldg(ga.y + ((size_t)i * a.nv + jv) * a.nu + ju);
        if (yv == 0.0f) continue;
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
        const DF rb = df_div(wb, wa), rz = df_div(wz, wa);
        const DF pb = df_div(nb, wa), pz = df_div(nz, wa);
        const float dl_h = sqrtf(fmaf(rz.hi, rz.hi, fmaf(rb.hi, rb.hi, 1.0f)));
        const VT *__restrict__ base = d.ax ? vol : volT;
        float lo = 0.0f, hi = (float)(n - 1);
        clip_planes(pb.hi, rb.hi, ic, (float)n, lo, hi);
        clip_planes(pz.hi, rz.hi, ic, (float)n, lo, hi);
        const int i0 = max(0, (int)floorf(lo) - 1);
        const int i1 = min(n - 1, (int)ceilf(hi) + 1);
        // t(i) = (i - S_a) / w_a
        const float rwa = 1.0f / wa.hi;
        const float Sa = G.S[ia];
        float acc = 0.0f, gb = 0.0f, gbt = 0.0f, gz = 0.0f, gzt = 0.0f;
        for (int c0 = i0; c0 <= i1; c0 += PJ_CHUNK) {
            const float d0 = __fsub_rn((float)c0, ic);
            int Ib, Iz;
            float phib, phiz;
            split_coord(df_add(df_add(pb, df_mul_f(rb, d0)), DF{ic, 0.0f}), Ib, phib);
            split_coord(df_add(df_add(pz, df_mul_f(rz, d0)), DF{ic, 0.0f}), Iz, phiz);
            const int cnt = min(PJ_CHUNK, i1 - c0 + 1);
            for (int kk = 0; kk < cnt; ++kk) {
                const int pl = c0 + kk;
                const float gbk = fmaf((float)kk, rb.hi, phib);
                const float gzk = fmaf((float)kk, rz.hi, phiz);
                const float fb0 = floorf(gbk), fz0 = floorf(gzk);
                const float tb = gbk - fb0, tz = gzk - fz0;
                const int jb = Ib + (int)fb0, jz = Iz + (int)fz0;
                const bool b0 = (unsigned)jb < (unsigned)n, b1 = (unsigned)(jb + 1) < (unsigned)n;
                const bool z0 = (unsigned)jz < (unsigned)n, z1 = (unsigned)(jz + 1) < (unsigned)n;
                const int row0 = (jz * n + pl) * n + jb;
                const int row1 = row0 + n * n;
                const float v00 = tap(base, row0, b0 && z0);
                const float v10 = tap(base, row0 + 1, b1 && z0);
                const float v01 = tap(base, row1, b0 && z1);
                const float v11 = tap(base, row1 + 1, b1 && z1);
                const float e0 = v10 - v00, e1 = v11 - v01;
                const float a0 = fmaf(tb, e0, v00), a1 = fmaf(tb, e1, v01);
                const float t = ((float)pl - Sa) * rwa;
                const float dbz = a1 - a0;             // dB / df_z
                const float dbb = fmaf(tz, e1 - e0, e0);  // dB / df_b
                acc += fmaf(tz, dbz, a0);
                gb += dbb;
                gbt = fmaf(t, dbb, gbt);
                gz += dbz;
                gzt = fmaf(t, dbz, gzt);
            }
        }
        // chain rule to the five parameters
        const float rbv = rb.hi, rzv = rz.hi, h = a.h;
        const float gb0 = gb - gbt, gz0 = gz - gzt;  // sums weighted by (1 - t)
        float dS[3], dP[3];
#pragma unroll
        for (int p = 0; p < 5; ++p) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                dS[q] = p == 0 ? G.Du[q] : (p == 1 ? G.Dv[q] : 0.0f);
                dP[q] = p == 2 ? G.Du[q] : (p == 3 ? G.Dv[q] : (p == 4 ? up * G.Ev[q] - vp * G.Eu[q] : 0.0f));
            }
            const float sa = dS[ia], sb = dS[ib], sz = dS[2];
            const float pa = dP[ia], pbv = dP[ib], pzv = dP[2];
            const float cbS = sb - rbv * sa, cbP = pbv - rbv * pa;
            const float czS = sz - rzv * sa, czP = pzv - rzv * pa;
            const float dwa = pa - sa, dwb = pbv - sb, dwz = pzv - sz;
            const float drb = (dwb - rbv * dwa) * rwa, drz = (dwz - rzv * dwa) * rwa;
            const float ddl = (rbv * drb + rzv * drz) / dl_h;
            const float dI = h * (ddl * acc + dl_h * (gb0 * cbS + gbt * cbP + gz0 * czS + gzt * czP));
            gsum[p] += (double)yv * (double)dI;
        }
    }
    block_sum<5>(gsum, red);
    if (tid == 0) {
        double *o = ga.part + ((size_t)i * gridDim.x + blockIdx.x) * 5;
#pragma unroll
        for (int p = 0; p < 5; ++p) o[p] = gsum[p];
    }
}

// out[i][5] = sum over the u-blocks of view i, in order.
__global__ void k_view_sums(const double *__restrict__ part, int nub, int nviews, double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nviews) return;
    double s[5] = {0, 0, 0, 0, 0};
    for (int b = 0; b < nub; ++b)
        for (int p = 0; p < 5; ++p) s[p] += part[((size_t)i * nub + b) * 5 + p];
    for (int p = 0; p < 5; ++p) out[(size_t)i * 5 + p] = s[p];
}

}  // namespace mgct

using namespace mgct;

extern "C" int mgct_geometry_grad(const mgct_geom *g, int level, int view0, int nviews, int stride, const float *vol,
                                  const float *y, double *dphi, mgct_stream stream) {
    MGCT_TRY(validate_level(g, level));
    MGCT_TRY(validate_views(g, view0, nviews, stride));
    MGCT_TRY(check_ptr(vol, "vol"));
    MGCT_TRY(check_ptr(y, "y", nviews == 0));
    MGCT_TRY(check_ptr(dphi, "dphi", nviews == 0));
    if (nviews == 0) return MGCT_OK;
    const LevelInfo &L = g->lev[level];
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int nub = (L.nu + PJ_BX - 1) / PJ_BX;
    if ((size_t)nviews * nub * 5 > g->scratch_part_count)
        return set_error(MGCT_ESHAPE, "geometry_grad: too many views for the handle's scratch");
    float *volT = static_cast<float *>(g->d_scratch_vol);
    MGCT_TRY(launch_transpose_xy<float>(L.n, vol, volT, s));
    GradArgs ga;
    ga.p.views = L.d_views;
    ga.p.n = L.n;
    ga.p.nu = L.nu;
    ga.p.nv = L.nv;
    ga.p.h = (float)L.h;
    ga.p.view0 = view0;
    ga.p.stride = stride;
    ga.p.nviews = nviews;
    ga.y = y;
    ga.part = g->d_scratch_part;
    dim3 grid(nub, nviews);
    MGCT_KERNEL(KK_GEOMGRAD, s, k_geom_grad<float><<<grid, dim3(PJ_BX, PJ_BY), 0, s>>>(ga, vol, volT));
    MGCT_KERNEL(KK_REDUCE, s, k_view_sums<<<(nviews + 127) / 128, 128, 0, s>>>(g->d_scratch_part, nub, nviews, dphi));
    return MGCT_OK;
}
