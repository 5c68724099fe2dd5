/*
 * mgct — cone-beam CT preconditioned multigrid Landweber reconstruction on one
 * NVIDIA GB300 (sm_103a).  C ABI of the CUDA library libmgct.so.
 *
 * Method: G. R. Myers et al., "Rapidly-converging multigrid reconstruction of
 * cone-beam tomographic data" (arXiv 2103.10329).  Each entry point cites the
 * passage of the paper that defines the operation.
 *
 * Conventions shared by every call
 * --------------------------------
 * World units: the reconstruction volume is the cube [-1/2, 1/2]^3.  On grid
 * g (g = 0 finest) the volume has n_g = n / 2^g voxels per side, voxel size
 * h_g = 1 / n_g, voxel i centred at (i - (n_g - 1)/2) h_g; the detector has
 * nu_g = nu / 2^g by nv_g = nv / 2^g pixels at pitch 2^g * pixel_pitch.
 * All views are present on every grid (Alg. 1 passes Theta unchanged).
 *
 * Layouts: volumes are [z][y][x], x fastest, C-contiguous; sinograms are
 * [view][v][u], u fastest.  A "batch" sinogram holds the selected views
 * contiguously in selection order.  Two-channel sinograms (OS-EMTR) are
 * [view][v][u][2].
 *
 * Pointers: unless stated otherwise every array argument is DEVICE memory of
 * the current CUDA device, allocated and owned by the caller, with 16-byte
 * aligned base address (MGCT_EALIGN otherwise).  Descriptor structs and
 * arrays documented as host arrays are read during the call only.
 *
 * Streams: every call that launches work is ordered on `stream` (a
 * cudaStream_t; NULL is the legacy default stream) and returns without
 * synchronising, unless its comment says it synchronises.
 *
 * Errors: every call returns an int status: MGCT_OK (0) or a negative
 * MGCT_E* code.  Argument errors are detected on the host before anything is
 * launched; nothing aborts the process.  mgct_last_error() returns a
 * thread-local message describing the most recent failure.  Conditions only
 * the device can see (a non-finite step size) are reported in the device-side
 * stats structs documented below.
 *
 * Thread safety: a geometry handle may be used by one stream at a time (it
 * owns the scratch buffers of mgct_project/mgct_backproject); different
 * handles are independent.
 */
#ifndef MGCT_H
#define MGCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *mgct_stream; /* == cudaStream_t */

enum {
    MGCT_OK = 0,
    MGCT_EINVAL = -1,     /* bad argument (NULL pointer, out-of-range value) */
    MGCT_ESHAPE = -2,     /* sizes inconsistent or unsupported */
    MGCT_EDTYPE = -3,     /* unsupported dtype combination */
    MGCT_EALIGN = -4,     /* pointer not 16-byte aligned */
    MGCT_ECUDA = -5,      /* a CUDA runtime call failed */
    MGCT_ENOMEM = -6,     /* device allocation failed or workspace too small */
    MGCT_ENONFINITE = -7, /* non-finite value where a finite one is required */
    MGCT_EDEVICE = -8,    /* device-side check failed */
    MGCT_ETIMEOUT = -9    /* bounded device wait expired */
};

typedef enum { MGCT_F32 = 0, MGCT_BF16 = 1, MGCT_F16 = 2 } mgct_dtype;

/* ---------------------------------------------------------------------------
 * Geometry (Sec. 2, Eq. 1: the source and detector positions Theta along the
 * scanning trajectory; Sec. 1 motivates per-view drift parameters)
 *
 * View k: source s_k = (D cos th_k, D sin th_k, z_k) with D = src_axis_dist;
 * flat detector centred at s_k + L (-cos th_k, -sin th_k, 0), L =
 * src_det_dist (both distances measured from the source point as in Sec. 2);
 * detector axes e_u = (-sin th_k, cos th_k, 0), e_v = (0, 0, 1); pixel
 * (ju, jv) centred at offset ((ju - (nu-1)/2) pitch, (jv - (nv-1)/2) pitch).
 * Optional drift[k] = (ds_u, ds_v, dd_u, dd_v, psi): the source moves by
 * (ds_u e_u + ds_v e_v) * pixel_pitch, the detector centre by
 * (dd_u e_u + dd_v e_v) * pixel_pitch, and the detector axes turn by psi
 * radians about the detector normal.
 * ------------------------------------------------------------------------- */
typedef struct mgct_geom mgct_geom; /* opaque, library-owned */

typedef struct {
    int32_t n;          /* finest volume side, 4..1024; divisible by 2^(levels-1) */
    int32_t nu, nv;     /* finest detector size; divisible by 2^(levels-1) */
    int32_t n_views;    /* K >= 1 */
    int32_t levels;     /* number of grids L, 1..8 */
    double src_axis_dist;  /* D > sqrt(3)/2 (source outside the volume) */
    double src_det_dist;   /* L > D */
    double pixel_pitch;    /* finest pitch, world units, > 0 */
    const double *theta;   /* host [K] radians */
    const double *z;       /* host [K] source height */
    const double *drift;   /* host [K*5] or NULL (no drift) */
    int32_t p_slice_axis;  /* Eq. 5 outer index axis: 2 = z (default), 0 = x, 1 = y */
} mgct_geom_desc;

/* Builds the per-grid, per-view float32 tables from float64 host arithmetic
 * and uploads them; allocates the handle's scratch (one finest volume plus
 * reduction partials).  Rejects geometries in which a ray could have z as its
 * major axis or a voxel could lie behind the source (MGCT_ESHAPE).
 * Synchronises the current device.  *out receives the handle. */
int mgct_geometry_create(const mgct_geom_desc *desc, mgct_geom **out);

/* Replaces the drift of every view (host [K*5], or NULL for none) and
 * re-uploads the tables.  Synchronises the current device. */
/* Preconditioner in place of Eq. 5 for mgct_precondition and the Landweber
 * steps on every grid (the paper asks for better kernels than Eq. 5, Sec. 3):
 * kernel = 27 doubles [dz][dy][dx], dz, dy, dx in {-1, 0, 1}, applied as the
 * correlation out(p) = sum_d kernel[d] in(p + d) with zero padding (the
 * slice-axis option does not apply to it).  NULL restores Eq. 5.  Not
 * concurrent with calls that use the handle. */
int mgct_geometry_set_preconditioner(mgct_geom *geom, const double *kernel);
int mgct_geometry_set_drift(mgct_geom *geom, const double *drift);

/* Frees the handle and its device memory.  NULL is ignored. */
void mgct_geometry_destroy(mgct_geom *geom);

/* Sizes of grid `level`: n_g, nu_g, nv_g, voxel size h_g, pitch. */
int mgct_geometry_level(const mgct_geom *geom, int level, int32_t *n, int32_t *nu, int32_t *nv,
                        double *h, double *pitch);

/* ---------------------------------------------------------------------------
 * Projection P = A (Sec. 2, Eq. 1; one projection per iteration, Sec. 1).
 *
 * Joseph's method: each ray (source -> pixel centre, direction w) has major
 * axis a = argmax |w_i| over x, y (z never, see geometry_create; ties to x);
 * it is sampled where it crosses each voxel-centre plane of axis a, by
 * bilinear interpolation in that plane (zero outside the volume), each sample
 * weighted by h_g |w| / |w_a|.  Accumulation is float32.
 *
 * Views: view0 + i * view_stride for i = 0..nviews-1 (must lie in [0, K)).
 * vol: [n_g]^3 of dtype vt.  out: batch sinogram [nviews][nv_g][nu_g] of
 * dtype ot.  b: NULL (out = A vol) or a float32 batch sinogram (out = b - A
 * vol).  sumsq: NULL or device double[1] receiving sum(out^2) in float64.
 * Uses the handle's scratch.
 * ------------------------------------------------------------------------- */
int mgct_project(const mgct_geom *geom, int level, int view0, int nviews, int view_stride,
                 const void *vol, mgct_dtype vt, void *out, mgct_dtype ot, const float *b,
                 double *sumsq, mgct_stream stream);

/* ---------------------------------------------------------------------------
 * Back-projection B = A^T (Sec. 2.1: B is the adjoint of the projection).
 *
 * The exact transpose of mgct_project's weights: for each voxel and view,
 * every detector pixel whose ray crosses the voxel's plane (along that ray's
 * major axis) within one voxel of it contributes
 * y * h_g|w|/|w_a| * hat(db) * hat(dc).  On tilt-free geometries each ray's
 * y * h_g|w|/|w_a| is formed in the handle's quad scratch (in chunks of
 * views) and splatted by z-slab into shared memory; with detector tilt, or a
 * scratch smaller than one view, a per-voxel gather computes the same sums.
 * No atomics: the result is deterministic.  sino: batch sinogram of dtype
 * st; vol_out: float32 [n_g]^3, overwritten (accumulate = 0) or added to
 * (accumulate = 1).  Uses the handle's scratch.
 * ------------------------------------------------------------------------- */
int mgct_backproject(const mgct_geom *geom, int level, int view0, int nviews, int view_stride,
                     const void *sino, mgct_dtype st, float *vol_out, int accumulate,
                     mgct_stream stream);

/* ---------------------------------------------------------------------------
 * Preconditioner p (Eq. 4 and Eq. 5): out = p * in, the 3x3x3 kernel of
 * Eq. 5 with its outer index along the handle's p_slice_axis, zero outside
 * the volume.  float32 [n_g]^3; in and out must not overlap.
 * ------------------------------------------------------------------------- */
int mgct_precondition(const mgct_geom *geom, int level, const float *in, float *out,
                      mgct_stream stream);

/* ---------------------------------------------------------------------------
 * Grid transfer (Alg. 1 Restrict and Prolongate).
 * restrict_volume: out[n/2]^3 = 2x2x2 mean of in[n]^3 (n even).
 * restrict_sino:   out[k][nv/2][nu/2] = 2x2 mean of each view's log data.
 * prolong_add:     fine[2n]^3 += Prolongate(coarse_new - coarse_old), cell-
 *                  centred trilinear (3/4, 1/4 per axis, edges clamped).
 * All float32.
 * ------------------------------------------------------------------------- */
int mgct_restrict_volume(int n_fine, const float *in, float *out, mgct_stream stream);
int mgct_restrict_sino(int k, int nv, int nu, const float *in, float *out, mgct_stream stream);
int mgct_prolong_add(int n_coarse, const float *coarse_new, const float *coarse_old, float *fine,
                     mgct_stream stream);

/* ---------------------------------------------------------------------------
 * Solvers.  Workspaces are caller-allocated device memory of at least
 * mgct_workspace_bytes(geom, op, level) bytes, 256-byte aligned.
 * ------------------------------------------------------------------------- */
enum { MGCT_WS_LANDWEBER = 0, MGCT_WS_OSEMTR = 1, MGCT_WS_MULTIGRID = 2 };

size_t mgct_workspace_bytes(const mgct_geom *geom, int op, int level);

typedef struct {
    double alpha;         /* > 0: fixed step; <= 0: exact line search <r,Ad>/|Ad|^2 */
    double lambda;        /* soft-threshold level (Alg. 1 SoftThreshold); 0 = none */
    int32_t precondition; /* 1: d = p * B r (Eq. 4); 0: d = B r (SIRT, Eq. 2) */
    int32_t n_subsets;    /* OS-EMTR subsets M on the coarsest grid (multigrid only) */
    int32_t storage;      /* mgct_dtype of the copies the projector and back-projector read:
                             MGCT_F32, or MGCT_BF16 / MGCT_F16 for a 16-bit shadow of mu and
                             of the search direction and a 16-bit residual sinogram; mu itself
                             (the master copy), b, the filter and the update stay float32,
                             accumulation is float32, alpha and the norms float64 */
    int32_t coarse_fas;   /* multigrid only.  0: the coarse problem's data is the restricted
                             radiographs R b (Alg. 1).  1: the full-approximation-scheme data
                             R (b_g - A_g mu) + A_c (R mu), rebuilt each iteration (one extra A
                             on every grid but the coarsest; not in the paper): the fine
                             solution becomes a fixed point, removing the plateau of the
                             plain recursion on consistent data */
    const float *learned_corr; /* reserved, must be NULL */
    /* Alg. 1 BilateralFilter after each grid's Landweber step and soft threshold
     * in the multigrid recursion (mgct_multigrid_iteration / _coarse; see
     * mgct_bilateral).  The paper gives no parameters: radius 0 = off. */
    double bilateral_sigma_s;  /* spatial sigma, voxels of the grid (> 0 when on) */
    double bilateral_sigma_r;  /* range sigma, attenuation units (> 0 when on) */
    int32_t bilateral_radius;  /* window half-width, 0 (off) .. 4 */
    int32_t reserved1;         /* must be 0 */
} mgct_lw_opts;

/* Device-side record of one Landweber step (float64). */
typedef struct {
    double alpha;       /* step used (0 if |A d| = 0 or a non-finite value was met) */
    double r2;          /* |b - A mu|^2 before the step */
    double r2_pred;     /* |b - A (mu + alpha d)|^2 predicted by the line search */
    double nonfinite;   /* 1 if a non-finite alpha was replaced by 0, else 0; with alpha = 0 the
                           volume is left untouched */
} mgct_lw_stats;

/* One preconditioned Landweber step on grid `level` (Eq. 4; Eq. 2 when
 * opts->precondition = 0), followed by soft thresholding (Alg. 1):
 *   r = b - A mu;  d = p * (A^T r);  alpha = <r, A d> / |A d|^2 (or fixed);
 *   mu <- S_lambda(mu + alpha d).
 * vol: float32 [n_g]^3 in place; b: float32 [K][nv_g][nu_g], all views.
 * stats: NULL or a device mgct_lw_stats.  No host synchronisation. */
int mgct_landweber_step(const mgct_geom *geom, int level, float *vol, const float *b,
                        void *workspace, size_t ws_bytes, const mgct_lw_opts *opts,
                        mgct_lw_stats *stats, mgct_stream stream);

/* One OS-EMTR pass on grid `level` (Eq. 3) over n_subsets ordered subsets,
 * subset m = views k with k mod M = m, in order m = 0..M-1:
 *   mu <- mu + B{exp(-A mu) - exp(-b)} / B{exp(-A mu) * PI}
 * where voxels whose denominator is not above 1e-12 of its maximum keep
 * their value.  pi: float32 [K][nv_g][nu_g] = A 1 (mgct_project of ones). */
int mgct_osemtr_pass(const mgct_geom *geom, int level, int n_subsets, float *vol,
                     const float *b, const float *pi, void *workspace, size_t ws_bytes,
                     mgct_stream stream);

/* Alg. 1 BilateralFilter (its parameters are not given in the paper):
 *   out(p) = sum_q w(p,q) in(q) / sum_q w(p,q),
 *   w(p,q) = exp(-|p-q|^2 / (2 sigma_s^2)) exp(-(in(p)-in(q))^2 / (2 sigma_r^2)),
 * q over the (2 radius + 1)^3 window around p inside the volume, distances in
 * voxels.  in, out: float32 [n]^3, distinct (out-of-place).  sigma_s > 0,
 * sigma_r > 0, 1 <= radius <= 4. */
int mgct_bilateral(int n, const float *in, float *out, double sigma_s, double sigma_r, int radius,
                   mgct_stream stream);

/* Alg. 1.  mgct_multigrid_prepare stores b on every grid (2x2 restriction)
 * and PI = A 1 on the coarsest grid in the workspace; then each
 * mgct_multigrid_iteration runs one recursive multigrid call at grid 0:
 * restrict mu, recurse (or one OS-EMTR pass on the coarsest grid), add the
 * prolongated coarse change, one preconditioned Landweber step, soft
 * threshold.  stats: NULL or device mgct_lw_stats[levels] (one per grid,
 * grid 0 first; the coarsest entry stays untouched when levels > 1).
 * b: float32 [K][nv][nu] grid-0 data, the same array given to prepare. */
int mgct_multigrid_prepare(const mgct_geom *geom, const float *b, void *workspace,
                           size_t ws_bytes, mgct_stream stream);
int mgct_multigrid_iteration(const mgct_geom *geom, float *vol, const float *b, void *workspace,
                             size_t ws_bytes, const mgct_lw_opts *opts, mgct_lw_stats *stats,
                             mgct_stream stream);

/* Alg. 1 without the grid-0 Landweber step: restrict mu, recurse (or one
 * OS-EMTR pass on the coarsest grid) and add the prolongated coarse change.
 * mgct_multigrid_iteration = mgct_multigrid_coarse + mgct_landweber_step at
 * grid 0.  Same arguments as mgct_multigrid_iteration; b (the grid-0 data)
 * may be NULL unless opts->coarse_fas. */
int mgct_multigrid_coarse(const mgct_geom *geom, float *vol, const float *b, void *workspace,
                          size_t ws_bytes, const mgct_lw_opts *opts, mgct_lw_stats *stats,
                          mgct_stream stream);

/* The step alpha d of one Landweber step (Eq. 4: d = p * A^T (b - A mu),
 * alpha from the line search or fixed) into step (float32 [n_g]^3), without
 * changing vol.  Used to collect training pairs for the learned correction. */
int mgct_landweber_direction(const mgct_geom *geom, int level, const float *vol, const float *b,
                             void *workspace, size_t ws_bytes, const mgct_lw_opts *opts,
                             float *step, mgct_lw_stats *stats, mgct_stream stream);

/* y += a x, float32 (count elements). */
int mgct_axpy(size_t count, float a, const float *x, float *y, mgct_stream stream);

/* ---------------------------------------------------------------------------
 * Geometry gradient (Sec. 1: drift of the source and detector, estimated
 * jointly with the image).  dphi[i][5] = d/dphi of sum_rays y * (A vol) over
 * the rays of view view0 + i * view_stride, for phi = (ds_u, ds_v, dd_u,
 * dd_v [fine pixels], psi [rad]) of that view (the drift of
 * mgct_geometry_desc), at fixed major axis and plane set (A is piecewise
 * smooth in phi).  vol: float32 [n_g]^3; y: float32 batch sinogram; dphi:
 * device double [nviews * 5], overwritten.  Uses the handle's scratch.
 * ------------------------------------------------------------------------- */
int mgct_geometry_grad(const mgct_geom *geom, int level, int view0, int nviews, int view_stride,
                       const float *vol, const float *y, double *dphi, mgct_stream stream);

/* ---------------------------------------------------------------------------
 * Learned preconditioner correction (Sec. 3 discussion: a more effective
 * preconditioning kernel than Eq. 5 is wanted; this network learns a
 * correction on top of it).
 *
 * Network f: four 3x3x3 convolutions at full resolution (zero padding),
 * 1 -> 16 -> 32 -> 64 -> 1 channels, ReLU after the first three, on the BF16
 * tensor cores (tcgen05, accumulators in tensor memory) with float32
 * accumulation and BF16 activations; float32
 * master weights trained by Adam.  Volumes are [B][D][H][W] float32, B
 * volumes of D x H x W voxels, B*D*H*W < 2^31.
 *
 * mgct_net_apply: out = s (x + f(x)) with x = dir / s, s = RMS(dir): the
 *   corrected step for the step dir (alpha d of a Landweber step).
 * mgct_net_forward_backward: for scaled input x and target t, loss =
 *   mean((x + f(x) - t)^2) into *loss (device double) and the gradients of
 *   every parameter into the net (mgct_net_get_grads reads them).
 * mgct_net_adam_step: one Adam step (beta 0.9 / 0.999, eps 1e-8) with the
 *   last gradients.
 * Parameters are exchanged as float32, layer by layer: weights
 * [27][cout][cin] (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)) then biases [cout];
 * mgct_net_param_count() values in all.  mgct_net_create initialises with
 * He-normal weights from `seed`, zero biases and a zero output layer.
 * Workspaces: mgct_net_workspace_bytes(B*D*H*W, training) bytes, 256-byte
 * aligned.  mgct_net_apply (and so mgct_landweber_learned) also accepts a
 * smaller workspace and then runs the volume in z-slabs: S planes at a time,
 * S the largest depth with mgct_net_workspace_bytes((S + 8) H W, 0) <= the
 * workspace, each slab computed with 4 extra planes on either side (the
 * receptive field of the four 3x3x3 layers), so the result is the same;
 * the RMS s is that of the whole volume.
 * ------------------------------------------------------------------------- */
typedef struct mgct_net mgct_net;
int mgct_net_create(uint64_t seed, mgct_net **out);
void mgct_net_destroy(mgct_net *net);
size_t mgct_net_param_count(void);
int mgct_net_set_params(mgct_net *net, const float *host, size_t count);
int mgct_net_get_params(const mgct_net *net, float *host, size_t count);
int mgct_net_get_grads(const mgct_net *net, float *host, size_t count);
size_t mgct_net_workspace_bytes(int64_t nvox, int training);
int mgct_net_apply(const mgct_net *net, int B, int D, int H, int W, const float *dir, float *out,
                   void *workspace, size_t ws_bytes, mgct_stream stream);
int mgct_net_forward_backward(mgct_net *net, int B, int D, int H, int W, const float *x,
                              const float *t, void *workspace, size_t ws_bytes, double *loss,
                              mgct_stream stream);
int mgct_net_adam_step(mgct_net *net, double lr, mgct_stream stream);
/* The convolutions run on the tcgen05 tensor cores and wait on their MMAs
 * with bounded waits; when a wait expires the kernel records it in a device
 * word of the net, skips its stores and returns.  The pass's results are
 * then NaN (mgct_net_apply's output, mgct_net_forward_backward's loss).
 * mgct_net_check synchronises `stream`, clears the word and returns
 * MGCT_ETIMEOUT if it was set, MGCT_OK otherwise. */
int mgct_net_check(const mgct_net *net, mgct_stream stream);

/* Learned Landweber step on grid `level`: the plain step alpha d (Eq. 4 with
 * the exact line search), the corrected step d' = mgct_net_apply(alpha d),
 * a second exact line search beta = <r, A d'> / |A d'|^2, and the update
 * mu <- S_lambda(mu + beta d'), or mu <- S_lambda(mu + alpha d) when beta is
 * not positive and finite (the plain filter is the fallback).  opts->alpha
 * must be <= 0.  net_ws: mgct_net_workspace_bytes(n_g^3, 0) bytes.  stats:
 * device double[8] = {alpha, r2, r2_pred, nonfinite, beta, r2, r2_pred
 * (learned), nonfinite}. */
int mgct_landweber_learned(const mgct_geom *geom, int level, float *vol, const float *b,
                           void *workspace, size_t ws_bytes, const mgct_lw_opts *opts,
                           const mgct_net *net, void *net_ws, size_t net_ws_bytes, double *stats,
                           mgct_stream stream);

/* ---------------------------------------------------------------------------
 * Residual projection without any device allocation.  The paper has no
 * counterpart: this is a library service.
 *
 * Same result as mgct_project(geom, level, view0, nviews, view_stride, vol,
 * MGCT_F32, out, MGCT_F32, b, sumsq, stream): out = b - A vol and
 * *sumsq = |out|^2 in float64 (sumsq required).  It is meant for callers
 * that may not allocate device memory themselves -- a plug-in whose host
 * pipeline owns every device buffer through its own pool or caching
 * allocator, or a process with a device-memory budget fixed at start-up.
 * Instead of the handle's scratch it uses one static device array inside the
 * library, mgct_project_residual_static_bytes() bytes (about 10 MiB), which
 * every GPU that loads the library's device code holds until the process
 * exits.  With lazy module loading (the CUDA default) that memory is taken
 * when the device code is first used on a device, at the latest by the first
 * call of this entry point there: a caller whose device-memory budget is
 * fixed later should make one warm-up call at start-up.  Limits:
 * at most 128^3 voxels on the chosen grid and at most 262144 projector
 * blocks (ceil(nu_g/32) * ceil(nv_g/8) * nviews, with nviews rounded up to a
 * multiple of 32 above 32 views); larger requests fail with
 * MGCT_ESHAPE and a message naming the limit.  It calls no cudaMalloc,
 * cudaFree or other allocating routine.  The first call in a device's
 * context looks up the array's device address (cudaGetSymbolAddress) with
 * that device current and keeps it for that context (a context created anew,
 * e.g. after cudaDeviceReset, gets its own lookup); make that first call
 * before any stream capture.  All calls share
 * the one array, so calls that overlap on the GPU (different streams, or
 * different host threads, without ordering between them) race on it and give
 * wrong results; the array keeps the last call's contents, and every word a
 * call reads is written by that call first.
 * ------------------------------------------------------------------------- */
int mgct_project_residual_static(const mgct_geom *geom, int level, int view0, int nviews,
                                 int view_stride, const float *vol, float *out, const float *b,
                                 double *sumsq, mgct_stream stream);
size_t mgct_project_residual_static_bytes(void);

/* ---------------------------------------------------------------------------
 * Diagnostics
 * ------------------------------------------------------------------------- */
const char *mgct_status_string(int status);
const char *mgct_last_error(void);
/* Kernel launches issued by this thread since the last reset (host counter). */
uint64_t mgct_launch_count(int reset);

/* Self-check of the failure path of the library's device waits (the paper
 * has no counterpart).  Every wait in the library's kernels on another
 * agent's progress (the tensor-core convolutions' waits for their MMAs) is
 * bounded by the SM clock, about a second, after which the kernel reports
 * the expiry (see mgct_net_check) instead of hanging.  This runs that same
 * bounded wait for `seconds` (0 < seconds <= 10) on a barrier nothing ever
 * completes, synchronises `stream`, and sets *expired = 1 when the wait gave
 * up as designed.  Returns MGCT_OK (the device context stays usable). */
int mgct_check_bounded_wait(double seconds, int *expired, mgct_stream stream);

/* Measures the two on-chip peaks the projector and back-projector are held
 * against (the paper has no counterpart): *fp32_tflops, the FP32 rate of
 * independent FMA chains (2 flop each) on every SM, and *lds_gbs, the rate
 * of conflict-free 16-byte shared-memory loads (the L1 data path), each the
 * median of five CUDA-event-timed launches on `stream` after one untimed
 * launch.  Allocates nothing; synchronises `stream`.  A few milliseconds. */
int mgct_measure_onchip_peaks(double *fp32_tflops, double *lds_gbs, mgct_stream stream);

/* Kernel trace (tracing subsystem; the paper has none).  mgct_trace_enable(1)
 * clears the record and starts recording a CUDA event pair on the launching
 * stream around every kernel the library issues; 0 stops and clears.
 * mgct_trace_read waits for the recorded events and writes, per kernel kind
 * (0 project, 1 backproject, 2 precondition, 3 transpose, 4 restrict/prolong,
 * 5 updates/fills/copies, 6 reductions, 7 geometry gradient, 8 convolution,
 * 9 other), the summed milliseconds and launch counts into host arrays of
 * nkinds entries. */
#define MGCT_TRACE_KINDS 10
int mgct_trace_enable(int on);
int mgct_trace_read(double *ms, uint64_t *launches, int nkinds);
/* The same, restricted to launches made for grid `level` (solver steps and
 * mgct_project / mgct_backproject tag their launches with their grid). */
int mgct_trace_read_level(int level, double *ms, uint64_t *launches, int nkinds);

#ifdef __cplusplus
}
#endif
#endif /* MGCT_H */
