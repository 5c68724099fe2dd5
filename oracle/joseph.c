/*
 * FP64 CPU oracle for the cone-beam projection operator P (= A) and its
 * adjoint back-projection B (= A^T).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; it exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can compare the CUDA library against a
 * plain, slow, obviously correct implementation.  It shares no code with the
 * CUDA library.
 *
 * What it computes.  The paper's data model (Sec. 2, Eq. 1) needs line
 * integrals of the attenuation mu along the rays from the source to each
 * detector pixel; P is the discrete operator, and B is its adjoint (Sec. 2.1,
 * the text under Eq. 2).  The paper does not say how P is discretised.  The
 * reading used here is Joseph's method:
 *   - a ray with direction w = pixel - source has major axis a, the axis of
 *     largest |w_i| (ties go to the lowest index: x before y before z);
 *   - for every voxel-centre plane i_a = 0..N-1 of that axis, the ray's
 *     crossing point gives continuous indices (f_b, f_c) of the two other
 *     axes, and mu is sampled there by bilinear interpolation, with zero
 *     outside [0, N-1];
 *   - each sample is weighted by the path length between planes,
 *     dl = h * |w| / |w_a|.
 * B is the exact transpose of that matrix, computed here by scattering each
 * ray's samples back (a different loop from the GPU's voxel-driven gather).
 *
 * Geometry is passed in per view: source position src[k][3], the centre of
 * detector pixel (0,0) det[k][3], and the pixel steps pu[k][3] (one pixel
 * along u) and pv[k][3] (one pixel along v), all in world units; the volume
 * is the cube [-1/2, 1/2]^3 with voxel size h = 1/N, voxel i centred at
 * (i - (N-1)/2) h, stored [z][y][x] with x fastest.  Sinograms are
 * [view][v][u] with u fastest.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double s[3];   /* source */
    double w[3];   /* direction source -> pixel centre (unnormalised) */
    int a, b, c;   /* major axis and the two others, b < c */
    double dl;     /* path length per plane step: h |w| / |w_a| */
} ray_t;

/* Returns 0, or -1 if the major axis would be z (the geometry never allows it). */
static int make_ray(const double *src, const double *det, const double *pu, const double *pv,
                    int ju, int jv, double h, ray_t *r)
{
    double aw[3];
    for (int i = 0; i < 3; ++i) {
        double p = det[i] + ju * pu[i] + jv * pv[i];
        r->s[i] = src[i];
        r->w[i] = p - src[i];
        aw[i] = fabs(r->w[i]);
    }
    int a = 0;
    if (aw[1] > aw[a]) a = 1;
    if (aw[2] > aw[a]) a = 2;
    if (a == 2) return -1;
    r->a = a;
    r->b = (a == 0) ? 1 : 0;
    r->c = 2;
    double nw = sqrt(r->w[0] * r->w[0] + r->w[1] * r->w[1] + r->w[2] * r->w[2]);
    r->dl = h * nw / aw[a];
    return 0;
}

/* Crossing of the ray with the plane of axis a at voxel-centre index ia:
 * continuous indices of the b and c axes. */
static void crossing(const ray_t *r, int n, double h, int ia, double *fb, double *fc)
{
    double half = 0.5 * (n - 1);
    double cpos = (ia - half) * h;
    double t = (cpos - r->s[r->a]) / r->w[r->a];
    double xb = r->s[r->b] + t * r->w[r->b];
    double xc = r->s[r->c] + t * r->w[r->c];
    *fb = xb / h + half;
    *fc = xc / h + half;
}

static size_t vox_index(int n, int a, int b, int c, int ia, int ib, int ic)
{
    int idx[3];
    idx[a] = ia;
    idx[b] = ib;
    idx[c] = ic;
    return ((size_t)idx[2] * n + idx[1]) * n + idx[0];
}

/* Line integral of vol along one ray (Joseph). */
static double ray_integral(const ray_t *r, int n, double h, const double *vol)
{
    double sum = 0.0;
    for (int ia = 0; ia < n; ++ia) {
        double fb, fc;
        crossing(r, n, h, ia, &fb, &fc);
        double fb0 = floor(fb), fc0 = floor(fc);
        double tb = fb - fb0, tc = fc - fc0;
        int ib = (int)fb0, ic = (int)fc0;
        for (int db = 0; db < 2; ++db) {
            int jb = ib + db;
            if (jb < 0 || jb >= n) continue;
            double wb = db ? tb : 1.0 - tb;
            for (int dc = 0; dc < 2; ++dc) {
                int jc = ic + dc;
                if (jc < 0 || jc >= n) continue;
                double wc = dc ? tc : 1.0 - tc;
                sum += wb * wc * vol[vox_index(n, r->a, r->b, r->c, ia, jb, jc)];
            }
        }
    }
    return sum * r->dl;
}

/* Scatter y * (row of A for this ray) into acc. */
static void ray_scatter(const ray_t *r, int n, double h, double y, double *acc)
{
    double yw = y * r->dl;
    if (yw == 0.0) return;
    for (int ia = 0; ia < n; ++ia) {
        double fb, fc;
        crossing(r, n, h, ia, &fb, &fc);
        double fb0 = floor(fb), fc0 = floor(fc);
        double tb = fb - fb0, tc = fc - fc0;
        int ib = (int)fb0, ic = (int)fc0;
        for (int db = 0; db < 2; ++db) {
            int jb = ib + db;
            if (jb < 0 || jb >= n) continue;
            double wb = db ? tb : 1.0 - tb;
            for (int dc = 0; dc < 2; ++dc) {
                int jc = ic + dc;
                if (jc < 0 || jc >= n) continue;
                double wc = dc ? tc : 1.0 - tc;
                acc[vox_index(n, r->a, r->b, r->c, ia, jb, jc)] += yw * wb * wc;
            }
        }
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* sino[k][v][u] = (A vol) for views 0..nviews-1.  Returns 0 or -1 (z-major ray). */
int orc_project(int n, int nu, int nv, int nviews,
                const double *src, const double *det, const double *pu, const double *pv,
                const double *vol, double *sino)
{
    double h = 1.0 / n;
    int bad = 0;
#pragma omp parallel for collapse(2) schedule(dynamic, 4) reduction(| : bad)
    for (int k = 0; k < nviews; ++k) {
        for (int jv = 0; jv < nv; ++jv) {
            for (int ju = 0; ju < nu; ++ju) {
                ray_t r;
                if (make_ray(src + 3 * k, det + 3 * k, pu + 3 * k, pv + 3 * k, ju, jv, h, &r)) {
                    bad = 1;
                    continue;
                }
                sino[((size_t)k * nv + jv) * nu + ju] = ray_integral(&r, n, h, vol);
            }
        }
    }
    return bad ? -1 : 0;
}

/* vol = A^T sino, by scattering every ray (thread-private accumulators,
 * summed in thread order). */
int orc_backproject(int n, int nu, int nv, int nviews,
                    const double *src, const double *det, const double *pu, const double *pv,
                    const double *sino, double *vol)
{
    double h = 1.0 / n;
    size_t nvox = (size_t)n * n * n;
    int nthr = orc_num_threads();
    /* bound the private accumulators to about 8 GB */
    size_t cap = (size_t)8 << 30;
    if ((size_t)nthr * nvox * sizeof(double) > cap) {
        nthr = (int)(cap / (nvox * sizeof(double)));
        if (nthr < 1) nthr = 1;
    }
    double *acc = (double *)calloc((size_t)nthr * nvox, sizeof(double));
    if (!acc) return -2;
    int bad = 0;
#pragma omp parallel num_threads(nthr) reduction(| : bad)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *my = acc + (size_t)t * nvox;
        /* static schedule: the same views always land in the same accumulator,
         * so repeated calls sum in the same order */
#pragma omp for schedule(static, 1)
        for (int k = 0; k < nviews; ++k) {
            for (int jv = 0; jv < nv; ++jv) {
                for (int ju = 0; ju < nu; ++ju) {
                    ray_t r;
                    if (make_ray(src + 3 * k, det + 3 * k, pu + 3 * k, pv + 3 * k, ju, jv, h, &r)) {
                        bad = 1;
                        continue;
                    }
                    ray_scatter(&r, n, h, sino[((size_t)k * nv + jv) * nu + ju], my);
                }
            }
        }
    }
    memset(vol, 0, nvox * sizeof(double));
    for (int t = 0; t < nthr; ++t) {
        const double *my = acc + (size_t)t * nvox;
        for (size_t i = 0; i < nvox; ++i) vol[i] += my[i];
    }
    free(acc);
    return bad ? -1 : 0;
}

/* Line integrals for a list of rays rays[i] = (view, v, u). */
int orc_project_rays(int n, const double *src, const double *det, const double *pu,
                     const double *pv, const double *vol, int count, const int32_t *rays,
                     double *out)
{
    double h = 1.0 / n;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (int i = 0; i < count; ++i) {
        int k = rays[3 * i], jv = rays[3 * i + 1], ju = rays[3 * i + 2];
        ray_t r;
        if (make_ray(src + 3 * k, det + 3 * k, pu + 3 * k, pv + 3 * k, ju, jv, h, &r)) {
            bad = 1;
            out[i] = 0.0;
            continue;
        }
        out[i] = ray_integral(&r, n, h, vol);
    }
    return bad ? -1 : 0;
}

static double hat(double t)
{
    double v = 1.0 - fabs(t);
    return v > 0.0 ? v : 0.0;
}

/* One matrix entry A[(view, v, u), (x, y, z)], written directly from the
 * definition: the ray's crossing of the voxel's own plane along the ray's
 * major axis, weighted by the two in-plane hat functions and dl.  Independent
 * of the plane loop above.  Returns NaN for a z-major ray. */
double orc_weight(int n, const double *src, const double *det, const double *pu,
                  const double *pv, int ju, int jv, int ix, int iy, int iz)
{
    double h = 1.0 / n;
    ray_t r;
    if (make_ray(src, det, pu, pv, ju, jv, h, &r)) return NAN;
    int idx[3] = {ix, iy, iz};
    double fb, fc;
    crossing(&r, n, h, idx[r.a], &fb, &fc);
    return r.dl * hat(fb - idx[r.b]) * hat(fc - idx[r.c]);
}

/* (A^T y) at a list of voxels vox[i] = (x, y, z): per view, the voxel centre is
 * projected onto the detector (line source -> voxel centre cut with the
 * detector plane), and the weight function is summed over a (2 radius + 1)^2
 * pixel window around that point.  edge[i] is set to 1 when any weight on the
 * window's border is non-zero, i.e. when the window may have been too small. */
int orc_backproject_voxels(int n, int nu, int nv, int nviews,
                           const double *src, const double *det, const double *pu,
                           const double *pv, const double *sino, int count,
                           const int32_t *vox, int radius, double *out, int32_t *edge)
{
    double h = 1.0 / n;
    double half = 0.5 * (n - 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < count; ++i) {
        int ix = vox[3 * i], iy = vox[3 * i + 1], iz = vox[3 * i + 2];
        double x[3] = {(ix - half) * h, (iy - half) * h, (iz - half) * h};
        double acc = 0.0;
        int hit_edge = 0;
        for (int k = 0; k < nviews; ++k) {
            const double *s = src + 3 * k, *d0 = det + 3 * k, *eu = pu + 3 * k, *ev = pv + 3 * k;
            /* solve s + t (x - s) = d0 + a eu + b ev  for (t, a, b) by Cramer's rule */
            double m[3][3], rhs[3];
            for (int q = 0; q < 3; ++q) {
                m[q][0] = x[q] - s[q];
                m[q][1] = -eu[q];
                m[q][2] = -ev[q];
                rhs[q] = d0[q] - s[q];
            }
            double det3 = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
                        - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
                        + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
            double da = m[0][0] * (rhs[1] * m[2][2] - m[1][2] * rhs[2])
                      - rhs[0] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
                      + m[0][2] * (m[1][0] * rhs[2] - rhs[1] * m[2][0]);
            double db = m[0][0] * (m[1][1] * rhs[2] - rhs[1] * m[2][1])
                      - m[0][1] * (m[1][0] * rhs[2] - rhs[1] * m[2][0])
                      + rhs[0] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
            double uc = da / det3, vc = db / det3;
            int u0 = (int)floor(uc) - radius, v0 = (int)floor(vc) - radius;
            for (int jv = v0; jv <= v0 + 2 * radius + 1; ++jv) {
                for (int ju = u0; ju <= u0 + 2 * radius + 1; ++ju) {
                    if (ju < 0 || ju >= nu || jv < 0 || jv >= nv) continue;
                    double w = orc_weight(n, s, d0, eu, ev, ju, jv, ix, iy, iz);
                    if (w == 0.0) continue;
                    if (ju == u0 || jv == v0 || ju == u0 + 2 * radius + 1 || jv == v0 + 2 * radius + 1)
                        hit_edge = 1;
                    acc += w * sino[((size_t)k * nv + jv) * nu + ju];
                }
            }
        }
        out[i] = acc;
        edge[i] = hit_edge;
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Derivative of the line integrals with respect to the ray end points, for
 * the per-view geometry gradient (joint estimation of drift, Sec. 1).
 *
 * For a ray from s to the pixel centre p (w = p - s), Joseph's integral is
 * I = dl * sum_i B(f_b(i), f_c(i)), dl = h |w| / |w_a|, with the crossing of
 * plane c_i: t_i = (c_i - s_a) / w_a, x = s + t_i w, f = x / h + (N-1)/2.
 * Differentiating at fixed major axis a and fixed plane set:
 *   dt/ds_a = (c - p_a) / w_a^2,   dt/dp_a = -t / w_a,
 *   dx_q/ds_q = 1 - t, dx_q/dp_q = t (q != a), dx_q/d(s_a, p_a) = w_q dt/d(.),
 *   d dl / dw_j = h (w_j / (|w| |w_a|) - [j = a] |w| sign(w_a) / w_a^2),
 * and B's gradient is that of the bilinear interpolant (zero padding).
 * Per view it returns sums weighted by the cotangent y:
 *   gs[k][3]  = sum y dI/ds,          gp[k][3]  = sum y dI/dp,
 *   gpu[k][3] = sum y dI/dp * ju',    gpv[k][3] = sum y dI/dp * jv',
 * with ju' = ju - (nu-1)/2, jv' = jv - (nv-1)/2 (centred pixel indices).
 * ------------------------------------------------------------------------ */
static void ray_grad(const ray_t *r, int n, double h, const double *vol, double *dI_ds, double *dI_dp)
{
    const double half = 0.5 * (n - 1);
    const int a = r->a, b = r->b, c = r->c;
    const double wa = r->w[a];
    double nw = sqrt(r->w[0] * r->w[0] + r->w[1] * r->w[1] + r->w[2] * r->w[2]);
    double sum = 0.0;
    double g_s[3] = {0, 0, 0}, g_p[3] = {0, 0, 0};
    for (int ia = 0; ia < n; ++ia) {
        double cpos = (ia - half) * h;
        double t = (cpos - r->s[a]) / wa;
        double xb = r->s[b] + t * r->w[b], xc = r->s[c] + t * r->w[c];
        double fb = xb / h + half, fc = xc / h + half;
        double fb0 = floor(fb), fc0 = floor(fc);
        double tb = fb - fb0, tc = fc - fc0;
        int ib = (int)fb0, ic = (int)fc0;
        double v[2][2];
        for (int db = 0; db < 2; ++db)
            for (int dc = 0; dc < 2; ++dc) {
                int jb = ib + db, jc = ic + dc;
                v[db][dc] = (jb >= 0 && jb < n && jc >= 0 && jc < n)
                                ? vol[vox_index(n, a, b, c, ia, jb, jc)] : 0.0;
            }
        double val = (1 - tb) * (1 - tc) * v[0][0] + tb * (1 - tc) * v[1][0]
                   + (1 - tb) * tc * v[0][1] + tb * tc * v[1][1];
        double dB_dfb = (1 - tc) * (v[1][0] - v[0][0]) + tc * (v[1][1] - v[0][1]);
        double dB_dfc = (1 - tb) * (v[0][1] - v[0][0]) + tb * (v[1][1] - v[1][0]);
        sum += val;
        double dt_dsa = (cpos - (r->s[a] + wa)) / (wa * wa);  /* (c - p_a) / w_a^2 */
        double dt_dpa = -t / wa;
        /* dx_b, dx_c with respect to s and p */
        g_s[b] += dB_dfb / h * (1 - t);
        g_p[b] += dB_dfb / h * t;
        g_s[c] += dB_dfc / h * (1 - t);
        g_p[c] += dB_dfc / h * t;
        g_s[a] += (dB_dfb * r->w[b] + dB_dfc * r->w[c]) / h * dt_dsa;
        g_p[a] += (dB_dfb * r->w[b] + dB_dfc * r->w[c]) / h * dt_dpa;
    }
    double dl = h * nw / fabs(wa);
    for (int j = 0; j < 3; ++j) {
        double ddl_dw = h * (r->w[j] / (nw * fabs(wa)));
        if (j == a) ddl_dw -= h * nw * (wa > 0 ? 1.0 : -1.0) / (wa * wa);
        /* w = p - s */
        dI_dp[j] = ddl_dw * sum + dl * g_p[j];
        dI_ds[j] = -ddl_dw * sum + dl * g_s[j];
    }
}

int orc_project_grad(int n, int nu, int nv, int nviews, const double *src, const double *det,
                     const double *pu, const double *pv, const double *vol, const double *y,
                     double *gs, double *gp, double *gpu, double *gpv)
{
    double h = 1.0 / n;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int k = 0; k < nviews; ++k) {
        double as[3] = {0, 0, 0}, ap[3] = {0, 0, 0}, apu[3] = {0, 0, 0}, apv[3] = {0, 0, 0};
        for (int jv = 0; jv < nv; ++jv) {
            for (int ju = 0; ju < nu; ++ju) {
                double yy = y[((size_t)k * nv + jv) * nu + ju];
                if (yy == 0.0) continue;
                ray_t r;
                if (make_ray(src + 3 * k, det + 3 * k, pu + 3 * k, pv + 3 * k, ju, jv, h, &r)) {
                    bad = 1;
                    continue;
                }
                double ds[3], dp[3];
                ray_grad(&r, n, h, vol, ds, dp);
                double uc = ju - 0.5 * (nu - 1), vc = jv - 0.5 * (nv - 1);
                for (int j = 0; j < 3; ++j) {
                    as[j] += yy * ds[j];
                    ap[j] += yy * dp[j];
                    apu[j] += yy * dp[j] * uc;
                    apv[j] += yy * dp[j] * vc;
                }
            }
        }
        for (int j = 0; j < 3; ++j) {
            gs[3 * k + j] = as[j];
            gp[3 * k + j] = ap[j];
            gpu[3 * k + j] = apu[j];
            gpv[3 * k + j] = apv[j];
        }
    }
    return bad ? -1 : 0;
}
