// Geometry set-up (host, float64 -> float32 tables), status strings, error
// and launch bookkeeping.
//
// The acquisition geometry follows Sec. 2 / Eq. 1: a point source and a flat
// detector placed along the scanning trajectory Theta, with the source-to-axis
// and source-to-detector distances measured from the source point.  Per-view
// drift (Sec. 1: thermal drift of the components) shifts source and detector
// and tilts the detector.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "common.cuh"

namespace mgct {

static thread_local std::string g_last_error;
static thread_local uint64_t g_launches = 0;

int set_error(int status, const std::string &msg) {
    g_last_error = msg;
    return status;
}

int check_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return MGCT_OK;
    return set_error(e == cudaErrorMemoryAllocation ? MGCT_ENOMEM : MGCT_ECUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}

void count_launch(int n) { g_launches += (uint64_t)n; }

int check_ptr(const void *p, const char *name, bool may_be_null) {
    if (!p) {
        if (may_be_null) return MGCT_OK;
        return set_error(MGCT_EINVAL, std::string(name) + " is NULL");
    }
    if (reinterpret_cast<uintptr_t>(p) % 16 != 0)
        return set_error(MGCT_EALIGN, std::string(name) + " is not 16-byte aligned");
    return MGCT_OK;
}

int validate_level(const mgct_geom *g, int level) {
    if (!g) return set_error(MGCT_EINVAL, "geometry handle is NULL");
    if (level < 0 || level >= g->levels)
        return set_error(MGCT_EINVAL, "level " + std::to_string(level) + " outside [0, " +
                                          std::to_string(g->levels) + ")");
    return MGCT_OK;
}

int validate_views(const mgct_geom *g, int view0, int nviews, int stride) {
    int K = g->desc.n_views;
    if (nviews < 0 || stride < 1 || view0 < 0)
        return set_error(MGCT_EINVAL, "bad view selection");
    if (nviews > 65535) return set_error(MGCT_EINVAL, "at most 65535 views per call");
    if (nviews > 0 && (int64_t)view0 + (int64_t)(nviews - 1) * stride >= K)
        return set_error(MGCT_EINVAL, "view selection runs past the last view");
    return MGCT_OK;
}

// ---------------------------------------------------------------------------
// Float64 construction of one view's table on one grid.
// ---------------------------------------------------------------------------
struct V3 {
    double x, y, z;
};
static inline V3 add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
static inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
static inline V3 mul(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
static inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline V3 cross(V3 a, V3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

static int build_view(const mgct_geom *g, int level, int k, ViewGeom *out, std::string *why) {
    const mgct_geom_desc &d = g->desc;
    int f = 1 << level;
    int n = d.n / f, nu = d.nu / f, nv = d.nv / f;
    double h = 1.0 / n;
    double pitch = d.pixel_pitch * f;
    double th = g->theta[k];
    double c = std::cos(th), s = std::sin(th);
    V3 eu = {-s, c, 0.0}, ev = {0.0, 0.0, 1.0}, nrm = {-c, -s, 0.0};
    const V3 eu_nom = eu, ev_nom = ev;
    V3 base = {d.src_axis_dist * c, d.src_axis_dist * s, g->z[k]};
    V3 src = base;
    V3 dcen = add(base, mul(d.src_det_dist, nrm));
    if (g->has_drift) {
        const double *ph = &g->drift[5 * (size_t)k];
        src = add(src, add(mul(ph[0] * d.pixel_pitch, eu), mul(ph[1] * d.pixel_pitch, ev)));
        dcen = add(dcen, add(mul(ph[2] * d.pixel_pitch, eu), mul(ph[3] * d.pixel_pitch, ev)));
        double cp = std::cos(ph[4]), sp = std::sin(ph[4]);
        V3 eu2 = add(mul(cp, eu), mul(sp, ev));
        V3 ev2 = add(mul(-sp, eu), mul(cp, ev));
        eu = eu2;
        ev = ev2;
    }
    double half = 0.5 * (n - 1);
    V3 S = add(mul(1.0 / h, src), {half, half, half});
    V3 Wc = mul(1.0 / h, sub(dcen, src));
    V3 Eu = mul(pitch / h, eu);
    V3 Ev = mul(pitch / h, ev);
    // Q = inverse of the matrix with columns Eu, Ev, Wc: rows are the cross
    // products of the other two columns divided by the determinant.
    double det = dot(Eu, cross(Ev, Wc));
    if (!(std::fabs(det) > 0)) {
        *why = "degenerate detector frame";
        return MGCT_ESHAPE;
    }
    V3 r0 = mul(1.0 / det, cross(Ev, Wc));
    V3 r1 = mul(1.0 / det, cross(Wc, Eu));
    V3 r2 = mul(1.0 / det, cross(Eu, Ev));
    // (1) z never the major axis: every ray direction w satisfies w.n = const
    // over the flat detector (n its unit normal); with n horizontal,
    // max(|w_x|,|w_y|) >= |w.n| / sqrt(2), while |w_z| is largest at a corner.
    V3 nh = cross(Eu, Ev);
    nh = mul(1.0 / std::sqrt(dot(nh, nh)), nh);
    if (std::fabs(nh.z) > 1e-12) {
        *why = "detector normal is not horizontal";
        return MGCT_ESHAPE;
    }
    double wn = std::fabs(dot(Wc, nh));
    double uh = 0.5 * (nu - 1), vh = 0.5 * (nv - 1);
    double wzmax = 0.0;
    for (int cu = -1; cu <= 1; cu += 2)
        for (int cv = -1; cv <= 1; cv += 2) {
            V3 w = add(Wc, add(mul(cu * uh, Eu), mul(cv * vh, Ev)));
            wzmax = std::fmax(wzmax, std::fabs(w.z));
        }
    if (!(wzmax < wn / std::sqrt(2.0) * (1.0 - 1e-9))) {
        *why = "a ray could have z as its major axis (detector too tall for the distances)";
        return MGCT_ESHAPE;
    }
    // (2) every voxel cube [j-1, j+1]^3 lies in front of the source
    double m2 = std::fabs(r2.x) + std::fabs(r2.y) + std::fabs(r2.z);
    double qmin = 1e300;
    for (int cx = 0; cx < 2; ++cx)
        for (int cy = 0; cy < 2; ++cy)
            for (int cz = 0; cz < 2; ++cz) {
                V3 X = {cx ? (double)n : -1.0, cy ? (double)n : -1.0, cz ? (double)n : -1.0};
                qmin = std::fmin(qmin, dot(r2, sub(X, S)));
            }
    if (!(qmin - m2 > 1e-9)) {
        *why = "part of the volume lies behind or too near the source";
        return MGCT_ESHAPE;
    }
    auto split = [](double v, float *hi, float *lo) {
        *hi = (float)v;
        *lo = (float)(v - (double)*hi);
    };
    std::memset(out, 0, sizeof(ViewGeom));
    const double sv[3] = {S.x, S.y, S.z}, wc[3] = {Wc.x, Wc.y, Wc.z}, eu3[3] = {Eu.x, Eu.y, Eu.z},
                 ev3[3] = {Ev.x, Ev.y, Ev.z};
    const double q[9] = {r0.x, r0.y, r0.z, r1.x, r1.y, r1.z, r2.x, r2.y, r2.z};
    for (int i = 0; i < 3; ++i) {
        out->S[i] = (float)sv[i];
        split(wc[i], &out->Wc[i], &out->Wc_lo[i]);
        split(eu3[i], &out->Eu[i], &out->Eu_lo[i]);
        split(ev3[i], &out->Ev[i], &out->Ev_lo[i]);
    }
    for (int i = 0; i < 9; ++i) out->Q[i] = (float)q[i];
    out->m2 = (float)m2;
    const V3 du = mul(d.pixel_pitch / h, eu_nom), dv = mul(d.pixel_pitch / h, ev_nom);
    out->Du[0] = (float)du.x;
    out->Du[1] = (float)du.y;
    out->Du[2] = (float)du.z;
    out->Dv[0] = (float)dv.x;
    out->Dv[1] = (float)dv.y;
    out->Dv[2] = (float)dv.z;
    // crossing numerators with the central plane of the major axis a:
    // P_b = (s'_b w_a - s'_a w_b) / w_a with s' = S - ic, expanded in (u', v')
    const double sc[3] = {S.x - half, S.y - half, S.z - half};
    auto numer = [&](int a, int b, double *o3) {
        o3[0] = sc[b] * wc[a] - sc[a] * wc[b];
        o3[1] = sc[b] * eu3[a] - sc[a] * eu3[b];
        o3[2] = sc[b] * ev3[a] - sc[a] * ev3[b];
    };
    double t[3];
    numer(0, 1, t);
    for (int i = 0; i < 3; ++i) split(t[i], &out->NX[i], &out->NX_lo[i]);
    numer(0, 2, t);
    for (int i = 0; i < 3; ++i) split(t[i], &out->NX[3 + i], &out->NX_lo[3 + i]);
    numer(1, 0, t);
    for (int i = 0; i < 3; ++i) split(t[i], &out->NY[i], &out->NY_lo[i]);
    numer(1, 2, t);
    for (int i = 0; i < 3; ++i) split(t[i], &out->NY[3 + i], &out->NY_lo[3 + i]);
    return MGCT_OK;
}

// Range of E1 = (nv_z + c_a Ev_z) / w_a over every view, column and plane
// c_a in [-ic, ic] where the column's rays cross the volume (|e_b| <= ic + 1,
// e_b = c_a rb + pb, the planes at which a voxel column can take them), from
// the float32 view tables in float64 -- the column table's own quantities.
// Where |w_x| and |w_y| are within a part in 1e5 of each other both axis
// choices are counted.
static void e1_range(LevelInfo &L, const std::vector<ViewGeom> &hv) {
    double lo = 1e300, hi = -1e300;
    const double ic = 0.5 * (L.n - 1), cu = 0.5 * (L.nu - 1);
    for (const ViewGeom &G : hv) {
        for (int ju = 0; ju < L.nu; ++ju) {
            const double up = ju - cu;
            const double wx = (double)G.Wc[0] + up * G.Eu[0], wy = (double)G.Wc[1] + up * G.Eu[1];
            for (int ax = 0; ax < 2; ++ax) {
                const double wa = ax ? wy : wx, wb = ax ? wx : wy;
                if (std::fabs(wa) < std::fabs(wb) * (1.0 - 1e-5)) continue;
                const float *N = ax ? G.NY : G.NX;
                const double rb = wb / wa, pb = ((double)N[0] + up * N[1]) / wa;
                double c0 = -ic, c1 = ic;  // planes where |c_a rb + pb| <= ic + 1
                if (std::fabs(rb) > 1e-12) {
                    double e0 = (-ic - 1.0 - pb) / rb, e1 = (ic + 1.0 - pb) / rb;
                    if (e0 > e1) std::swap(e0, e1);
                    c0 = std::max(c0, e0);
                    c1 = std::min(c1, e1);
                } else if (std::fabs(pb) > ic + 1.0) {
                    continue;
                }
                if (c0 > c1) continue;
                const double e10 = (double)N[5] / wa, e1c = (double)G.Ev[2] / wa;
                const double a = e10 + c0 * e1c, b = e10 + c1 * e1c;
                lo = std::min(lo, std::min(a, b));
                hi = std::max(hi, std::max(a, b));
            }
        }
    }
    L.e1_lo = (float)lo;
    L.e1_hi = (float)hi;
}

static int upload_tables(mgct_geom *g) {
    int K = g->desc.n_views;
    g->separable = 1;
    for (int l = 0; l < g->levels; ++l) {
        auto &hv = g->h_views[l];
        hv.resize(K);
        for (int k = 0; k < K; ++k) {
            std::string why;
            int st = build_view(g, l, k, &hv[k], &why);
            if (st) return set_error(st, "view " + std::to_string(k) + ", grid " + std::to_string(l) + ": " + why);
            const ViewGeom &v = hv[k];
            if (v.Ev[0] != 0.0f || v.Ev[1] != 0.0f || v.Eu[2] != 0.0f || v.Ev_lo[0] != 0.0f ||
                v.Ev_lo[1] != 0.0f || v.Eu_lo[2] != 0.0f || v.Q[2] != 0.0f || v.Q[8] != 0.0f)
                g->separable = 0;
        }
        MGCT_TRY(check_cuda(cudaMemcpy(g->lev[l].d_views, hv.data(), K * sizeof(ViewGeom),
                                       cudaMemcpyHostToDevice),
                            "upload view tables"));
    }
    for (int l = 0; l < g->levels; ++l) {
        LevelInfo &L = g->lev[l];
        if (!g->separable) continue;
        e1_range(L, g->h_views[l]);
        if (!L.d_cols)
            MGCT_TRY(check_cuda(cudaMalloc(&L.d_cols, (size_t)K * L.nu * 2 * sizeof(float4)), "allocate column table"));
        if (!L.d_cols_df)
            MGCT_TRY(check_cuda(cudaMalloc(&L.d_cols_df, (size_t)K * L.nu * 4 * sizeof(float4)),
                                "allocate column table"));
        MGCT_TRY(launch_column_table(g, l, 0));
        MGCT_TRY(launch_column_table_df(g, l, 0));
    }
    return check_cuda(cudaDeviceSynchronize(), "column tables");
}

}  // namespace mgct

using namespace mgct;

extern "C" {

const char *mgct_status_string(int st) {
    switch (st) {
        case MGCT_OK: return "ok";
        case MGCT_EINVAL: return "invalid argument";
        case MGCT_ESHAPE: return "inconsistent or unsupported sizes";
        case MGCT_EDTYPE: return "unsupported dtype";
        case MGCT_EALIGN: return "misaligned pointer";
        case MGCT_ECUDA: return "CUDA error";
        case MGCT_ENOMEM: return "out of memory or workspace too small";
        case MGCT_ENONFINITE: return "non-finite value";
        case MGCT_EDEVICE: return "device-side check failed";
        case MGCT_ETIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

const char *mgct_last_error(void) { return g_last_error.c_str(); }

uint64_t mgct_launch_count(int reset) {
    uint64_t v = g_launches;
    if (reset) g_launches = 0;
    return v;
}

void mgct_geometry_destroy(mgct_geom *g) {
    if (!g) return;
    for (int l = 0; l < 8; ++l) {
        if (g->lev[l].d_views) cudaFree(g->lev[l].d_views);
        if (g->lev[l].d_cols) cudaFree(g->lev[l].d_cols);
        if (g->lev[l].d_cols_df) cudaFree(g->lev[l].d_cols_df);
    }
    if (g->d_scratch_vol) cudaFree(g->d_scratch_vol);
    if (g->d_scratch_quads) cudaFree(g->d_scratch_quads);
    if (g->d_scratch_part) cudaFree(g->d_scratch_part);
    delete g;
}

int mgct_geometry_create(const mgct_geom_desc *d, mgct_geom **out) {
    if (!d || !out) return set_error(MGCT_EINVAL, "desc and out must not be NULL");
    *out = nullptr;
    if (!d->theta || !d->z) return set_error(MGCT_EINVAL, "theta and z must be host arrays");
    if (d->levels < 1 || d->levels > 8) return set_error(MGCT_EINVAL, "levels must be 1..8");
    if (d->n_views < 1) return set_error(MGCT_EINVAL, "n_views must be >= 1");
    int f = 1 << (d->levels - 1);
    if (d->n < 4 || d->nu < 1 || d->nv < 1 || d->n % f || d->nu % f || d->nv % f || d->n / f < 2)
        return set_error(MGCT_ESHAPE, "n, nu, nv must be divisible by 2^(levels-1) (and n/2^(levels-1) >= 2)");
    if (d->n > 1024)
        return set_error(MGCT_ESHAPE, "volume too large (n <= 1024)");
    if ((int64_t)d->nu * d->nv > ((int64_t)1 << 31))
        return set_error(MGCT_ESHAPE, "detector too large");
    if (!(d->src_axis_dist > 0.8660254037844387) || !(d->src_det_dist > d->src_axis_dist) ||
        !(d->pixel_pitch > 0))
        return set_error(MGCT_EINVAL, "need src_axis_dist > sqrt(3)/2, src_det_dist > src_axis_dist, pitch > 0");
    if (d->p_slice_axis < 0 || d->p_slice_axis > 2) return set_error(MGCT_EINVAL, "p_slice_axis must be 0, 1 or 2");
    mgct_geom *g = new mgct_geom();
    std::memset(g->lev, 0, sizeof(g->lev));
    g->d_scratch_vol = nullptr;
    g->d_scratch_quads = nullptr;
    g->d_scratch_part = nullptr;
    g->desc = *d;
    g->desc.theta = g->desc.z = g->desc.drift = nullptr;
    g->levels = d->levels;
    int K = d->n_views;
    g->theta.assign(d->theta, d->theta + K);
    g->z.assign(d->z, d->z + K);
    g->has_drift = d->drift != nullptr;
    if (g->has_drift) g->drift.assign(d->drift, d->drift + 5 * (size_t)K);
    cudaGetDevice(&g->device);
    for (int l = 0; l < g->levels; ++l) {
        int fl = 1 << l;
        LevelInfo &L = g->lev[l];
        L.n = d->n / fl;
        L.nu = d->nu / fl;
        L.nv = d->nv / fl;
        L.h = 1.0 / L.n;
        L.pitch = d->pixel_pitch * fl;
        int st = check_cuda(cudaMalloc(&L.d_views, K * sizeof(ViewGeom)), "allocate view tables");
        if (st) {
            mgct_geometry_destroy(g);
            return st;
        }
    }
    int st = upload_tables(g);
    if (st) {
        mgct_geometry_destroy(g);
        return st;
    }
    size_t nvox = (size_t)d->n * d->n * d->n;
    // partials: one per projector block (either projector's tiling), two values each
    size_t blocks = project_blocks_any(d->nu, d->nv, K);
    size_t vblocks = (nvox + 255) / 256;
    size_t gblocks = 5 * (size_t)K * ((d->nu + PJ_BX - 1) / PJ_BX);  // geometry-gradient partials
    g->scratch_part_count = 2 * (blocks > vblocks ? blocks : vblocks) + 64;
    if (gblocks > g->scratch_part_count) g->scratch_part_count = gblocks;
    st = check_cuda(cudaMalloc(&g->d_scratch_vol, nvox * 4), "allocate scratch volume");
    if (!st)
        st = check_cuda(cudaMalloc(&g->d_scratch_quads, 2 * quad_elems(g->lev[0].n) * sizeof(float4)),
                        "allocate scratch quads");
    if (!st) st = check_cuda(cudaMalloc(&g->d_scratch_part, g->scratch_part_count * sizeof(double)),
                             "allocate scratch partials");
    if (!st) st = check_cuda(cudaDeviceSynchronize(), "geometry_create");
    if (st) {
        mgct_geometry_destroy(g);
        return st;
    }
    *out = g;
    return MGCT_OK;
}

int mgct_geometry_set_preconditioner(mgct_geom *g, const double *kernel) {
    if (!g) return set_error(MGCT_EINVAL, "geometry handle is NULL");
    if (!kernel) {
        g->has_pkernel = 0;
        return MGCT_OK;
    }
    for (int i = 0; i < 27; ++i)
        if (!std::isfinite(kernel[i])) return set_error(MGCT_EINVAL, "kernel coefficients must be finite");
    for (int i = 0; i < 27; ++i) g->pkernel[i] = (float)kernel[i];
    g->has_pkernel = 1;
    return MGCT_OK;
}

int mgct_geometry_set_drift(mgct_geom *g, const double *drift) {
    if (!g) return set_error(MGCT_EINVAL, "geometry handle is NULL");
    int K = g->desc.n_views;
    g->has_drift = drift != nullptr;
    if (drift) g->drift.assign(drift, drift + 5 * (size_t)K);
    else g->drift.clear();
    MGCT_TRY(upload_tables(g));
    return check_cuda(cudaDeviceSynchronize(), "geometry_set_drift");
}

int mgct_geometry_level(const mgct_geom *g, int level, int32_t *n, int32_t *nu, int32_t *nv,
                        double *h, double *pitch) {
    MGCT_TRY(validate_level(g, level));
    const LevelInfo &L = g->lev[level];
    if (n) *n = L.n;
    if (nu) *nu = L.nu;
    if (nv) *nv = L.nv;
    if (h) *h = L.h;
    if (pitch) *pitch = L.pitch;
    return MGCT_OK;
}

}  // extern "C"
