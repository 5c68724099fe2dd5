// C-ABI entry points: projector, back-projector, filters, grid transfer, and
// the solvers built from them -- the preconditioned Landweber step (Eq. 4,
// Eq. 2 without the filter), the OS-EMTR pass (Eq. 3) and the recursive
// multigrid iteration (Alg. 1).  The solvers run entirely on the stream: the
// step size is computed on the device and read there by the update kernel,
// so an iteration issues no host synchronisation.
#include <cstring>
#include <type_traits>

#include "backproject.cuh"
#include "common.cuh"
#include "project.cuh"

namespace mgct {

int launch_precondition(int n, int slice_axis, const float *in, float *out, cudaStream_t s, const float *custom);
int launch_restrict_volume(int n_fine, const float *in, float *out, cudaStream_t s);
int launch_restrict_sino(int k, int nv, int nu, const float *in, float *out, cudaStream_t s);
int launch_prolong_add(int nc, const float *cn, const float *co, float *fine, cudaStream_t s);
int launch_step_size(const double *sums, const double *r2, double fixed_alpha, double *stats, cudaStream_t s);
int launch_update(size_t count, float *mu, const float *d, const double *alpha, float lam, cudaStream_t s);
int launch_em_update(size_t count, float *mu, const float *nd, double *part, cudaStream_t s);
int launch_fill(size_t count, float *x, float v, cudaStream_t s);
int launch_copy(size_t count, const float *in, float *out, cudaStream_t s);
int launch_scaled_copy(size_t count, const float *d, const double *alpha, float *out, cudaStream_t s);
int launch_update_choice(size_t count, float *mu, const float *d, const float *dl, const double *st, float lam,
                         cudaStream_t s);
int launch_axpy(size_t count, float a, const float *x, float *y, cudaStream_t s);
int launch_bilateral(int n, const float *in, float *out, double sigma_s, double sigma_r, int radius, cudaStream_t s);

int launch_column_table_df(const mgct_geom *g, int level, cudaStream_t s) {
    const LevelInfo &L = g->lev[level];
    const int K = g->desc.n_views;
    const int total = K * L.nu;
    MGCT_KERNEL(KK_OTHER, s, k_column_table_df<<<(total + 255) / 256, 256, 0, s>>>(L.d_views, K, L.nu, L.d_cols_df));
    return MGCT_OK;
}

int launch_column_table(const mgct_geom *g, int level, cudaStream_t s) {
    const LevelInfo &L = g->lev[level];
    const int K = g->desc.n_views;
    const int total = K * L.nu;
    MGCT_KERNEL(KK_OTHER, s, k_column_table<<<(total + 255) / 256, 256, 0, s>>>(L.d_views, K, L.nu, L.d_cols));
    return MGCT_OK;
}

// ---------------------------------------------------------------------------
// Workspace carving
// ---------------------------------------------------------------------------
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

static size_t vox(const LevelInfo &L) { return (size_t)L.n * L.n * L.n; }
static size_t sino_elems(const mgct_geom *g, const LevelInfo &L) {
    return (size_t)g->desc.n_views * L.nv * L.nu;
}
static size_t proj_blocks(const mgct_geom *g, const LevelInfo &L) {
    return project_blocks_any(L.nu, L.nv, g->desc.n_views);
}

struct LWSpace {
    float *r, *grad, *d, *muT;
    float4 *quads;                // projector input: quad copies for y-major then x-major rays
    double *part, *sums, *stats;  // sums: [0] r2, [1] <r,Ad>, [2] |Ad|^2 ; stats: 4
};

static LWSpace carve_lw(const mgct_geom *g, int level, Carver &c) {
    const LevelInfo &L = g->lev[level];
    LWSpace w;
    w.r = c.take<float>(sino_elems(g, L));
    w.grad = c.take<float>(vox(L));
    w.d = c.take<float>(vox(L));
    w.muT = c.take<float>(vox(L));
    w.quads = c.take<float4>(2 * quad_elems(L.n));  // sized for float32 quads (16-bit ones use half)
    w.part = c.take<double>(2 * proj_blocks(g, L) + 64);
    w.sums = c.take<double>(8);
    w.stats = c.take<double>(8);
    return w;
}

struct EMSpace {
    float2 *c2;
    float *nd, *muT;
    double *part;
};

static EMSpace carve_em(const mgct_geom *g, int level, Carver &c) {
    const LevelInfo &L = g->lev[level];
    EMSpace w;
    w.c2 = c.take<float2>(sino_elems(g, L));  // worst case: one subset holding every view
    w.nd = c.take<float>(2 * vox(L));
    w.muT = c.take<float>(vox(L));
    w.part = c.take<double>(1024);
    return w;
}

struct MGSpace {
    float *b[8], *mu[8], *old[8];
    float *bf[8];  // FAS coarse data per grid (grids 1 .. L-1)
    float *pi;
    int prepared_flag;
    void *lw_base, *em_base;
    size_t lw_bytes, em_bytes;
};

static MGSpace carve_mg(const mgct_geom *g, Carver &c) {
    MGSpace m;
    std::memset(&m, 0, sizeof(m));
    for (int l = 1; l < g->levels; ++l) {
        m.b[l] = c.take<float>(sino_elems(g, g->lev[l]));
        m.bf[l] = c.take<float>(sino_elems(g, g->lev[l]));
        m.mu[l] = c.take<float>(vox(g->lev[l]));
        m.old[l] = c.take<float>(vox(g->lev[l]));
    }
    int lc = g->levels - 1;
    m.pi = g->levels > 1 ? c.take<float>(sino_elems(g, g->lev[lc])) : nullptr;
    // sub-workspaces: Landweber sized for grid 0 (the largest), OS-EMTR for the coarsest
    Carver probe(nullptr);
    carve_lw(g, 0, probe);
    m.lw_bytes = probe.off;
    m.lw_base = c.take<char>(m.lw_bytes);
    Carver probe2(nullptr);
    carve_em(g, lc, probe2);
    m.em_bytes = probe2.off;
    m.em_base = c.take<char>(m.em_bytes);
    return m;
}

static size_t ws_bytes(const mgct_geom *g, int op, int level) {
    Carver c(nullptr);
    if (op == MGCT_WS_LANDWEBER) carve_lw(g, level, c);
    else if (op == MGCT_WS_OSEMTR) carve_em(g, level, c);
    else carve_mg(g, c);
    return c.off + 256;
}

static int check_ws(const mgct_geom *g, int op, int level, const void *ws, size_t bytes) {
    MGCT_TRY(check_ptr(ws, "workspace"));
    if (reinterpret_cast<uintptr_t>(ws) % 256)
        return set_error(MGCT_EALIGN, "workspace must be 256-byte aligned");
    size_t need = ws_bytes(g, op, level);
    if (bytes < need)
        return set_error(MGCT_ENOMEM, "workspace too small: need " + std::to_string(need) + " bytes");
    return MGCT_OK;
}

// ---------------------------------------------------------------------------
// Solver steps
// ---------------------------------------------------------------------------
// A v over every view through quad copies of v in storage type ST (see
// project_volume): vT is a float32 scratch volume, `quads` holds both ray
// classes' copies.
template <typename ST, typename Epi>
static int project_quads(const mgct_geom *g, int level, const float *v, float *vT, float4 *quads, const Epi &e,
                         cudaStream_t s, int *nb) {
    return project_volume<ST, float>(g, level, 0, g->desc.n_views, 1, v, vT, quads, e, s, nb);
}

// ST: storage type of the copies the projector and back-projector read (the
// shadow of mu, the residual sinogram, the shadow of the search direction).
//
// Phase 1 (direction): r = b - A mu (stored weighted, |r|^2 into sums[0]),
// grad = A^T r, d = p * grad (or grad).  Returns d.
template <typename ST>
static int lw_direction(const mgct_geom *g, int level, const float *mu, const float *b, const LWSpace &w,
                        const mgct_lw_opts &o, float **d_out, cudaStream_t s) {
    const LevelInfo &L = g->lev[level];
    const int K = g->desc.n_views;
    const size_t nv3 = vox(L);
    constexpr bool F32 = std::is_same<ST, float>::value;
    MGCT_TRY(check_cuda(cudaMemsetAsync(w.sums, 0, 8 * sizeof(double), s), "memset"));
    ST *r = reinterpret_cast<ST *>(w.r);
    int nb = 0;
    EpiResidual<ST, true> er{r, b, w.part, L.nu, L.nv, K};
    (void)F32;
    MGCT_TRY(project_quads<ST>(g, level, mu, w.muT, w.quads, er, s, &nb));
    (void)nv3;
    MGCT_TRY(launch_sum_partials(w.part, nb, 1, w.sums + 0, s));
    // the quads are free until the line search: room for partial volumes
    MGCT_TRY(launch_backproject<1, ST, true>(g, level, 0, K, 1, r, w.grad, 0, s, reinterpret_cast<float *>(w.quads),
                                             2 * quad_elems(L.n) * 4));
    *d_out = w.grad;
    if (o.precondition) {
        MGCT_TRY(launch_precondition(L.n, g->desc.p_slice_axis, w.grad, w.d, s, g->has_pkernel ? g->pkernel : nullptr));
        *d_out = w.d;
    }
    return MGCT_OK;
}

// Phase 2 (line search along dir): <r, A dir>, |A dir|^2 into sums[slot],
// sums[slot+1]; `spare` (one float32 volume) holds the projector's copies.
template <typename ST>
static int lw_line_search(const mgct_geom *g, int level, const float *dir, float *spare, const LWSpace &w, int slot,
                          cudaStream_t s) {
    const LevelInfo &L = g->lev[level];
    const int K = g->desc.n_views;
    const size_t nv3 = vox(L);
    int nb = 0;
    EpiDualDot<ST> ed{reinterpret_cast<ST *>(w.r), w.part, L.nu, L.nv, K};
    MGCT_TRY(project_quads<ST>(g, level, dir, spare, w.quads, ed, s, &nb));
    (void)nv3;
    return launch_sum_partials(w.part, nb, 2, w.sums + slot, s);
}

template <typename ST>
static int landweber_t(const mgct_geom *g, int level, float *mu, const float *b, void *ws, const mgct_lw_opts &o,
                       mgct_lw_stats *stats_out, cudaStream_t s) {
    const LevelInfo &L = g->lev[level];
    Carver c(ws);
    LWSpace w = carve_lw(g, level, c);
    double *stats = stats_out ? reinterpret_cast<double *>(stats_out) : w.stats;
    float *d = nullptr;
    MGCT_TRY(lw_direction<ST>(g, level, mu, b, w, o, &d, s));
    float *spare = d == w.d ? w.grad : w.d;  // the gradient is no longer needed
    if (!(o.alpha > 0.0)) MGCT_TRY(lw_line_search<ST>(g, level, d, spare, w, 1, s));
    MGCT_TRY(launch_step_size(w.sums + 1, w.sums + 0, o.alpha > 0.0 ? o.alpha : 0.0, stats, s));
    return launch_update(vox(L), mu, d, stats, (float)o.lambda, s);
}

// The step alpha d of one Landweber step (no update), into out.
template <typename ST>
static int direction_t(const mgct_geom *g, int level, const float *mu, const float *b, void *ws, const mgct_lw_opts &o,
                       float *out, mgct_lw_stats *stats_out, cudaStream_t s) {
    trace_tag(level);
    const LevelInfo &L = g->lev[level];
    Carver c(ws);
    LWSpace w = carve_lw(g, level, c);
    double *stats = stats_out ? reinterpret_cast<double *>(stats_out) : w.stats;
    float *d = nullptr;
    MGCT_TRY(lw_direction<ST>(g, level, mu, b, w, o, &d, s));
    float *spare = d == w.d ? w.grad : w.d;
    if (!(o.alpha > 0.0)) MGCT_TRY(lw_line_search<ST>(g, level, d, spare, w, 1, s));
    MGCT_TRY(launch_step_size(w.sums + 1, w.sums + 0, o.alpha > 0.0 ? o.alpha : 0.0, stats, s));
    return launch_scaled_copy(vox(L), d, stats, out, s);
}

// Learned Landweber step: step = alpha d as usual, corrected step d' =
// net(alpha d), a second exact line search beta along d', and the update
// mu += beta d' (or alpha d when beta <= 0).  stats: 8 doubles, the plain
// {alpha, r2, r2_pred, nonfinite} then the learned {beta, r2, r2_pred, nonfinite}.
template <typename ST>
static int learned_t(const mgct_geom *g, int level, float *mu, const float *b, void *ws, const mgct_lw_opts &o,
                     const mgct_net *net, void *net_ws, size_t net_bytes, double *stats, cudaStream_t s) {
    trace_tag(level);
    const LevelInfo &L = g->lev[level];
    Carver c(ws);
    LWSpace w = carve_lw(g, level, c);
    const size_t nv3 = vox(L);
    float *d = nullptr;
    MGCT_TRY(lw_direction<ST>(g, level, mu, b, w, o, &d, s));
    float *spare = d == w.d ? w.grad : w.d;
    MGCT_TRY(lw_line_search<ST>(g, level, d, spare, w, 1, s));
    MGCT_TRY(launch_step_size(w.sums + 1, w.sums + 0, 0.0, stats, s));
    float *step = spare;       // alpha d
    float *dl = w.muT;         // net(alpha d); muT is free after the residual
    MGCT_TRY(launch_scaled_copy(nv3, d, stats, step, s));
    MGCT_TRY(mgct_net_apply(net, 1, L.n, L.n, L.n, step, dl, net_ws, net_bytes, reinterpret_cast<mgct_stream>(s)));
    MGCT_TRY(lw_line_search<ST>(g, level, dl, spare, w, 3, s));
    MGCT_TRY(launch_step_size(w.sums + 3, w.sums + 0, 0.0, stats + 4, s));
    return launch_update_choice(nv3, mu, d, dl, stats, (float)o.lambda, s);
}

static int landweber(const mgct_geom *g, int level, float *mu, const float *b, void *ws, const mgct_lw_opts &o,
                     mgct_lw_stats *stats_out, cudaStream_t s) {
    trace_tag(level);
    switch (o.storage) {
        case MGCT_BF16: return landweber_t<__nv_bfloat16>(g, level, mu, b, ws, o, stats_out, s);
        case MGCT_F16: return landweber_t<__half>(g, level, mu, b, ws, o, stats_out, s);
        default: return landweber_t<float>(g, level, mu, b, ws, o, stats_out, s);
    }
}

static int osemtr(const mgct_geom *g, int level, int M, float *mu, const float *b, const float *pi, void *ws,
                  cudaStream_t s) {
    trace_tag(level);
    const LevelInfo &L = g->lev[level];
    Carver c(ws);
    EMSpace w = carve_em(g, level, c);
    const int K = g->desc.n_views;
    const size_t nv3 = vox(L);
    for (int m = 0; m < M; ++m) {
        int cnt = (K - m + M - 1) / M;
        if (cnt <= 0) continue;
        MGCT_TRY(launch_transpose_xy<float>(L.n, mu, w.muT, s));
        EpiEMTerms e{w.c2, b, pi, L.nu, L.nv, cnt};
        MGCT_TRY(launch_project<float>(g, level, m, cnt, M, mu, w.muT, e, s));
        // c2 holds room for every view; past this subset's views it is free
        const size_t used = (size_t)cnt * L.nu * L.nv;
        MGCT_TRY(launch_backproject<2, float2, true>(g, level, m, cnt, M, w.c2, w.nd, 0, s,
                                                     reinterpret_cast<float *>(w.c2 + used),
                                                     2 * (sino_elems(g, L) - used)));
        MGCT_TRY(launch_em_update(nv3, mu, w.nd, w.part, s));
    }
    return MGCT_OK;
}

// Alg. 1 on grid `level` with this grid's data `b`: restrict mu, recurse (or
// one OS-EMTR pass on the coarsest grid), add the prolongated coarse change,
// then one Landweber step (unless skip_landweber).  The coarse data is R b,
// prepared once (m.b), or with o.coarse_fas the full-approximation-scheme
// data R (b - A mu) + A_c (R mu), built here every call (m.bf): a variant
// outside the paper under which the fine solution is a fixed point.
static int multigrid_level(const mgct_geom *g, int level, float *mu, const MGSpace &m, const float *b,
                           const mgct_lw_opts &o, mgct_lw_stats *stats, cudaStream_t s, bool skip_landweber = false) {
    const int Lc = g->levels;
    trace_tag(level);
    if (level + 1 < Lc) {
        const LevelInfo &F = g->lev[level], &C = g->lev[level + 1];
        const int K = g->desc.n_views;
        float *mc = m.mu[level + 1], *oc = m.old[level + 1];
        MGCT_TRY(launch_restrict_volume(F.n, mu, mc, s));
        MGCT_TRY(launch_copy(vox(C), mc, oc, s));
        const float *bc = m.b[level + 1];
        if (o.coarse_fas) {
            // the Landweber workspace's residual, transpose and quads serve as scratch
            Carver cw(m.lw_base);
            LWSpace w = carve_lw(g, 0, cw);
            int nb = 0;
            EpiResidual<float, false> er{w.r, b, nullptr, F.nu, F.nv, K};
            MGCT_TRY(project_quads<float>(g, level, mu, w.muT, w.quads, er, s, &nb));
            MGCT_TRY(launch_restrict_sino(K, F.nv, F.nu, w.r, m.bf[level + 1], s));
            trace_tag(level + 1);
            EpiPlus ep{m.bf[level + 1], m.bf[level + 1], C.nu, C.nv};
            MGCT_TRY(project_quads<float>(g, level + 1, mc, w.muT, w.quads, ep, s, &nb));
            trace_tag(level);
            bc = m.bf[level + 1];
        }
        if (level + 1 < Lc - 1) {
            MGCT_TRY(multigrid_level(g, level + 1, mc, m, bc, o, stats, s));
        } else {
            int M = o.n_subsets > 0 ? o.n_subsets : 8;
            MGCT_TRY(osemtr(g, level + 1, M, mc, bc, m.pi, m.em_base, s));
        }
        trace_tag(level);
        MGCT_TRY(launch_prolong_add(C.n, mc, oc, mu, s));
    }
    if (skip_landweber) return MGCT_OK;
    MGCT_TRY(landweber(g, level, mu, b, m.lw_base, o, stats ? stats + level : nullptr, s));
    if (o.bilateral_radius > 0) {
        // Alg. 1 BilateralFilter; the Landweber workspace's gradient volume is free now
        Carver cw(m.lw_base);
        LWSpace w = carve_lw(g, 0, cw);
        const int n = g->lev[level].n;
        MGCT_TRY(launch_bilateral(n, mu, w.grad, o.bilateral_sigma_s, o.bilateral_sigma_r, o.bilateral_radius, s));
        MGCT_TRY(check_cuda(cudaMemcpyAsync(mu, w.grad, vox(g->lev[level]) * sizeof(float), cudaMemcpyDeviceToDevice, s),
                            "copy filtered volume"));
    }
    return MGCT_OK;
}

static int check_opts(const mgct_lw_opts *o) {
    if (!o) return set_error(MGCT_EINVAL, "opts is NULL");
    if (o->learned_corr) return set_error(MGCT_EINVAL, "learned_corr is reserved and must be NULL");
    if (!(o->lambda >= 0.0)) return set_error(MGCT_EINVAL, "lambda must be >= 0");
    if (o->n_subsets < 0) return set_error(MGCT_EINVAL, "n_subsets must be >= 0");
    if (o->storage < MGCT_F32 || o->storage > MGCT_F16)
        return set_error(MGCT_EINVAL, "storage must be MGCT_F32, MGCT_BF16 or MGCT_F16");
    if (o->coarse_fas != 0 && o->coarse_fas != 1) return set_error(MGCT_EINVAL, "coarse_fas must be 0 or 1");
    if (o->reserved1 != 0) return set_error(MGCT_EINVAL, "reserved1 must be 0");
    if (o->bilateral_radius < 0 || o->bilateral_radius > 4) return set_error(MGCT_EINVAL, "bilateral_radius must be 0..4");
    if (o->bilateral_radius > 0 && !(o->bilateral_sigma_s > 0.0 && o->bilateral_sigma_r > 0.0))
        return set_error(MGCT_EINVAL, "bilateral sigmas must be > 0");
    return MGCT_OK;
}

}  // namespace mgct

using namespace mgct;

extern "C" {

int mgct_project(const mgct_geom *g, int level, int view0, int nviews, int stride, const void *vol, mgct_dtype vt,
                 void *out, mgct_dtype ot, const float *b, double *sumsq, mgct_stream stream) {
    trace_tag(level);
    MGCT_TRY(validate_level(g, level));
    MGCT_TRY(validate_views(g, view0, nviews, stride));
    MGCT_TRY(check_ptr(vol, "vol"));
    MGCT_TRY(check_ptr(out, "out", nviews == 0));
    MGCT_TRY(check_ptr(b, "b", true));
    if (sumsq && reinterpret_cast<uintptr_t>(sumsq) % 8) return set_error(MGCT_EALIGN, "sumsq must be 8-byte aligned");
    if (vt < MGCT_F32 || vt > MGCT_F16 || ot < MGCT_F32 || ot > MGCT_F16)
        return set_error(MGCT_EDTYPE, "dtype must be MGCT_F32, MGCT_BF16 or MGCT_F16");
    if (sumsq && !b) return set_error(MGCT_EINVAL, "sumsq needs b (it is the residual norm)");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const LevelInfo &L = g->lev[level];
    if (nviews == 0) {
        if (sumsq) MGCT_TRY(check_cuda(cudaMemsetAsync(sumsq, 0, sizeof(double), s), "memset"));
        return MGCT_OK;
    }
    int nb = 0;
    double *part = sumsq ? g->d_scratch_part : nullptr;
    // the volume's quads (in its own precision) for both ray classes
    auto run = [&](auto vtag, auto otag) -> int {
        using VT = decltype(vtag);
        using OT = decltype(otag);
        const VT *v = static_cast<const VT *>(vol);
        VT *vT = static_cast<VT *>(g->d_scratch_vol);
        if (b) {
            EpiResidual<OT> e{static_cast<OT *>(out), b, part, L.nu, L.nv, nviews};
            return project_volume<VT, VT>(g, level, view0, nviews, stride, v, vT, g->d_scratch_quads, e, s, &nb);
        }
        EpiStore<OT> e{static_cast<OT *>(out), L.nu, L.nv};
        return project_volume<VT, VT>(g, level, view0, nviews, stride, v, vT, g->d_scratch_quads, e, s, &nb);
    };
    auto run_v = [&](auto vtag) -> int {
        switch (ot) {
            case MGCT_F32: return run(vtag, float());
            case MGCT_BF16: return run(vtag, __nv_bfloat16());
            default: return run(vtag, __half());
        }
    };
    int st;
    switch (vt) {
        case MGCT_F32: st = run_v(float()); break;
        case MGCT_BF16: st = run_v(__nv_bfloat16()); break;
        default: st = run_v(__half()); break;
    }
    MGCT_TRY(st);
    if (sumsq) MGCT_TRY(launch_sum_partials(part, nb, 1, sumsq, s));
    return MGCT_OK;
}

int mgct_backproject(const mgct_geom *g, int level, int view0, int nviews, int stride, const void *sino,
                     mgct_dtype st, float *vol_out, int accumulate, mgct_stream stream) {
    trace_tag(level);
    MGCT_TRY(validate_level(g, level));
    MGCT_TRY(validate_views(g, view0, nviews, stride));
    MGCT_TRY(check_ptr(sino, "sino", nviews == 0));
    MGCT_TRY(check_ptr(vol_out, "vol_out"));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int ran = 0;
    switch (st) {
        case MGCT_F32:
            MGCT_TRY(launch_backproject_public<float>(g, level, view0, nviews, stride,
                                                      static_cast<const float *>(sino), vol_out, accumulate, s, &ran));
            break;
        case MGCT_BF16:
            MGCT_TRY(launch_backproject_public<__nv_bfloat16>(g, level, view0, nviews, stride,
                                                              static_cast<const __nv_bfloat16 *>(sino), vol_out,
                                                              accumulate, s, &ran));
            break;
        case MGCT_F16:
            MGCT_TRY(launch_backproject_public<__half>(g, level, view0, nviews, stride,
                                                       static_cast<const __half *>(sino), vol_out, accumulate, s,
                                                       &ran));
            break;
        default: break;
    }
    if (ran) return MGCT_OK;
    switch (st) {
        case MGCT_F32:
            return launch_backproject<1, float>(g, level, view0, nviews, stride, static_cast<const float *>(sino),
                                                vol_out, accumulate, s);
        case MGCT_BF16:
            return launch_backproject<1, __nv_bfloat16>(g, level, view0, nviews, stride,
                                                        static_cast<const __nv_bfloat16 *>(sino), vol_out,
                                                        accumulate, s);
        case MGCT_F16:
            return launch_backproject<1, __half>(g, level, view0, nviews, stride, static_cast<const __half *>(sino),
                                                 vol_out, accumulate, s);
        default: return set_error(MGCT_EDTYPE, "dtype must be MGCT_F32, MGCT_BF16 or MGCT_F16");
    }
}

int mgct_precondition(const mgct_geom *g, int level, const float *in, float *out, mgct_stream stream) {
    MGCT_TRY(validate_level(g, level));
    MGCT_TRY(check_ptr(in, "in"));
    MGCT_TRY(check_ptr(out, "out"));
    if (in == out) return set_error(MGCT_EINVAL, "in and out must not overlap");
    return launch_precondition(g->lev[level].n, g->desc.p_slice_axis, in, out, reinterpret_cast<cudaStream_t>(stream),
                               g->has_pkernel ? g->pkernel : nullptr);
}

int mgct_restrict_volume(int n_fine, const float *in, float *out, mgct_stream stream) {
    if (n_fine < 2 || n_fine % 2 || n_fine > 2048) return set_error(MGCT_ESHAPE, "n_fine must be even, 2..2048");
    MGCT_TRY(check_ptr(in, "in"));
    MGCT_TRY(check_ptr(out, "out"));
    return launch_restrict_volume(n_fine, in, out, reinterpret_cast<cudaStream_t>(stream));
}

int mgct_restrict_sino(int k, int nv, int nu, const float *in, float *out, mgct_stream stream) {
    if (k < 1 || nv < 2 || nu < 2 || nv % 2 || nu % 2) return set_error(MGCT_ESHAPE, "k >= 1, nv and nu even");
    MGCT_TRY(check_ptr(in, "in"));
    MGCT_TRY(check_ptr(out, "out"));
    return launch_restrict_sino(k, nv, nu, in, out, reinterpret_cast<cudaStream_t>(stream));
}

int mgct_prolong_add(int n_coarse, const float *cn, const float *co, float *fine, mgct_stream stream) {
    if (n_coarse < 1 || n_coarse > 1024) return set_error(MGCT_ESHAPE, "n_coarse must be 1..1024");
    MGCT_TRY(check_ptr(cn, "coarse_new"));
    MGCT_TRY(check_ptr(co, "coarse_old"));
    MGCT_TRY(check_ptr(fine, "fine"));
    return launch_prolong_add(n_coarse, cn, co, fine, reinterpret_cast<cudaStream_t>(stream));
}

size_t mgct_workspace_bytes(const mgct_geom *g, int op, int level) {
    if (!g || op < 0 || op > 2) return 0;
    if (op != MGCT_WS_MULTIGRID && (level < 0 || level >= g->levels)) return 0;
    return ws_bytes(g, op, level);
}

int mgct_landweber_step(const mgct_geom *g, int level, float *vol, const float *b, void *ws, size_t bytes,
                        const mgct_lw_opts *o, mgct_lw_stats *stats, mgct_stream stream) {
    MGCT_TRY(validate_level(g, level));
    MGCT_TRY(check_opts(o));
    MGCT_TRY(check_ptr(vol, "vol"));
    MGCT_TRY(check_ptr(b, "b"));
    MGCT_TRY(check_ptr(stats, "stats", true));
    MGCT_TRY(check_ws(g, MGCT_WS_LANDWEBER, level, ws, bytes));
    return landweber(g, level, vol, b, ws, *o, stats, reinterpret_cast<cudaStream_t>(stream));
}

int mgct_osemtr_pass(const mgct_geom *g, int level, int n_subsets, float *vol, const float *b, const float *pi,
                     void *ws, size_t bytes, mgct_stream stream) {
    MGCT_TRY(validate_level(g, level));
    if (n_subsets < 1 || n_subsets > g->desc.n_views) return set_error(MGCT_EINVAL, "n_subsets must be 1..n_views");
    MGCT_TRY(check_ptr(vol, "vol"));
    MGCT_TRY(check_ptr(b, "b"));
    MGCT_TRY(check_ptr(pi, "pi"));
    MGCT_TRY(check_ws(g, MGCT_WS_OSEMTR, level, ws, bytes));
    return osemtr(g, level, n_subsets, vol, b, pi, ws, reinterpret_cast<cudaStream_t>(stream));
}

int mgct_bilateral(int n, const float *in, float *out, double sigma_s, double sigma_r, int radius, mgct_stream stream) {
    if (n < 1) return set_error(MGCT_ESHAPE, "n must be >= 1");
    MGCT_TRY(check_ptr(in, "in"));
    MGCT_TRY(check_ptr(out, "out"));
    if (in == out) return set_error(MGCT_EINVAL, "in and out must differ");
    if (radius < 1 || radius > 4) return set_error(MGCT_EINVAL, "radius must be 1..4");
    if (!(sigma_s > 0.0 && sigma_r > 0.0)) return set_error(MGCT_EINVAL, "sigmas must be > 0");
    return launch_bilateral(n, in, out, sigma_s, sigma_r, radius, reinterpret_cast<cudaStream_t>(stream));
}

int mgct_multigrid_prepare(const mgct_geom *g, const float *b, void *ws, size_t bytes, mgct_stream stream) {
    if (!g) return set_error(MGCT_EINVAL, "geometry handle is NULL");
    MGCT_TRY(check_ptr(b, "b"));
    MGCT_TRY(check_ws(g, MGCT_WS_MULTIGRID, 0, ws, bytes));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Carver c(ws);
    MGSpace m = carve_mg(g, c);
    const int K = g->desc.n_views;
    const float *prev = b;
    for (int l = 1; l < g->levels; ++l) {
        const LevelInfo &F = g->lev[l - 1];
        MGCT_TRY(launch_restrict_sino(K, F.nv, F.nu, prev, m.b[l], s));
        prev = m.b[l];
    }
    if (g->levels > 1) {
        // PI = A 1 on the coarsest grid (Eq. 3: projected support length)
        int lc = g->levels - 1;
        const LevelInfo &C = g->lev[lc];
        float *ones = m.mu[lc];
        MGCT_TRY(launch_fill(vox(C), ones, 1.0f, s));
        // the projector mgct_project runs, with the Landweber workspace's
        // transpose and quads as scratch
        Carver cw(m.lw_base);
        LWSpace w = carve_lw(g, 0, cw);
        EpiStore<float> e{m.pi, C.nu, C.nv};
        int nb = 0;
        MGCT_TRY((project_volume<float, float>(g, lc, 0, K, 1, ones, w.muT, w.quads, e, s, &nb)));
    }
    return MGCT_OK;
}

int mgct_multigrid_iteration(const mgct_geom *g, float *vol, const float *b, void *ws, size_t bytes,
                             const mgct_lw_opts *o, mgct_lw_stats *stats, mgct_stream stream) {
    if (!g) return set_error(MGCT_EINVAL, "geometry handle is NULL");
    MGCT_TRY(check_opts(o));
    MGCT_TRY(check_ptr(vol, "vol"));
    MGCT_TRY(check_ptr(b, "b"));
    MGCT_TRY(check_ptr(stats, "stats", true));
    MGCT_TRY(check_ws(g, MGCT_WS_MULTIGRID, 0, ws, bytes));
    Carver c(ws);
    MGSpace m = carve_mg(g, c);
    return multigrid_level(g, 0, vol, m, b, *o, stats, reinterpret_cast<cudaStream_t>(stream));
}

int mgct_multigrid_coarse(const mgct_geom *g, float *vol, const float *b, void *ws, size_t bytes,
                          const mgct_lw_opts *o, mgct_lw_stats *stats, mgct_stream stream) {
    if (!g) return set_error(MGCT_EINVAL, "geometry handle is NULL");
    MGCT_TRY(check_opts(o));
    MGCT_TRY(check_ptr(vol, "vol"));
    MGCT_TRY(check_ptr(b, "b", !o->coarse_fas));
    MGCT_TRY(check_ptr(stats, "stats", true));
    MGCT_TRY(check_ws(g, MGCT_WS_MULTIGRID, 0, ws, bytes));
    Carver c(ws);
    MGSpace m = carve_mg(g, c);
    return multigrid_level(g, 0, vol, m, b, *o, stats, reinterpret_cast<cudaStream_t>(stream), true);
}

int mgct_landweber_direction(const mgct_geom *g, int level, const float *vol, const float *b, void *ws, size_t bytes,
                             const mgct_lw_opts *o, float *step, mgct_lw_stats *stats, mgct_stream stream) {
    MGCT_TRY(validate_level(g, level));
    MGCT_TRY(check_opts(o));
    MGCT_TRY(check_ptr(vol, "vol"));
    MGCT_TRY(check_ptr(b, "b"));
    MGCT_TRY(check_ptr(step, "step"));
    MGCT_TRY(check_ptr(stats, "stats", true));
    MGCT_TRY(check_ws(g, MGCT_WS_LANDWEBER, level, ws, bytes));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (o->storage) {
        case MGCT_BF16: return direction_t<__nv_bfloat16>(g, level, vol, b, ws, *o, step, stats, s);
        case MGCT_F16: return direction_t<__half>(g, level, vol, b, ws, *o, step, stats, s);
        default: return direction_t<float>(g, level, vol, b, ws, *o, step, stats, s);
    }
}

int mgct_landweber_learned(const mgct_geom *g, int level, float *vol, const float *b, void *ws, size_t bytes,
                           const mgct_lw_opts *o, const mgct_net *net, void *net_ws, size_t net_bytes,
                           double *stats, mgct_stream stream) {
    MGCT_TRY(validate_level(g, level));
    MGCT_TRY(check_opts(o));
    if (!net) return set_error(MGCT_EINVAL, "net is NULL");
    if (o->alpha > 0.0) return set_error(MGCT_EINVAL, "the learned step always line-searches (opts->alpha must be <= 0)");
    MGCT_TRY(check_ptr(vol, "vol"));
    MGCT_TRY(check_ptr(b, "b"));
    MGCT_TRY(check_ptr(stats, "stats"));
    MGCT_TRY(check_ws(g, MGCT_WS_LANDWEBER, level, ws, bytes));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (o->storage) {
        case MGCT_BF16: return learned_t<__nv_bfloat16>(g, level, vol, b, ws, *o, net, net_ws, net_bytes, stats, s);
        case MGCT_F16: return learned_t<__half>(g, level, vol, b, ws, *o, net, net_ws, net_bytes, stats, s);
        default: return learned_t<float>(g, level, vol, b, ws, *o, net, net_ws, net_bytes, stats, s);
    }
}

int mgct_axpy(size_t count, float a, const float *x, float *y, mgct_stream stream) {
    MGCT_TRY(check_ptr(x, "x"));
    MGCT_TRY(check_ptr(y, "y"));
    return launch_axpy(count, a, x, y, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
