// Internal definitions shared by the translation units of libmgct.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mgct.h"

namespace mgct {

// ---------------------------------------------------------------------------
// Per-view geometry on one grid, float32, index units of that grid (voxel i
// centred at index i; the volume centre is at ic = (n-1)/2 on each axis).
//   S   : source position in continuous voxel indices
//   Wc  : direction from the source to the detector centre
//   Eu  : one pixel step along u;  Ev: one pixel step along v
//   Q   : inverse of the 3x3 matrix [Eu Ev Wc] (row-major), so that a point X
//         projects to centred pixel coordinates (q0/q2, q1/q2), q = Q (X - S)
//   m2  : |Q row 2|_1 (bounds the change of q2 over a +-1 voxel cube)
//   NX  : for x-major rays, the numerators (n0, nu, nv) of the y and z
//         coordinates of the crossing with the central plane x = ic:
//         P_y = (n0_y + u' nu_y + v' nv_y) / w_x, likewise P_z (centred);
//   NY  : the same for y-major rays (x and z coordinates over w_y).
// The numerators are s'_b w_a - s'_a w_b with s' = S - ic, expanded in
// (u', v') on the host in float64: no large terms cancel on the device.
// Pixel (ju, jv) has centred coordinates u' = ju - (nu-1)/2, v' = jv - (nv-1)/2
// and ray direction w = Wc + u' Eu + v' Ev.  The *_lo fields hold the float64
// rounding residue of the matching fields (double-float, used by the
// projector's per-ray set-up).
// ---------------------------------------------------------------------------
constexpr int VG_HI = 36;  // floats of the float32 part (the back-projector stages only these)
struct ViewGeom {
    float S[3];
    float Wc[3];
    float Eu[3];
    float Ev[3];
    float Q[9];
    float m2;
    float NX[6];  // n0_y, nu_y, nv_y, n0_z, nu_z, nv_z
    float NY[6];  // n0_x, nu_x, nv_x, n0_z, nu_z, nv_z
    float pad0[2];
    float Wc_lo[3];
    float Eu_lo[3];
    float Ev_lo[3];
    float NX_lo[6];
    float NY_lo[6];
    float Du[3];  // drift directions (index units of this grid): one fine pixel
    float Dv[3];  // along the untilted detector axes e_u, e_v
    float pad1;
};
static_assert(sizeof(ViewGeom) == 256, "ViewGeom layout");

struct LevelInfo {
    int n, nu, nv;
    double h, pitch;
    ViewGeom *d_views;  // device [K]
    float4 *d_cols;     // device [K][nu][2] detector-column table (separable geometries), or NULL
    float4 *d_cols_df;  // device [K][nu][4] the same quantities in double-float, or NULL
    // range of the column table's z step per detector row, E1 = e10 + c_a e1c,
    // over every view, column and voxel-centre plane c_a (separable geometries)
    float e1_lo, e1_hi;
};

// Detector-column table of a separable geometry (no detector tilt): for view
// k and column u' every ray of the column has the same major axis and
// horizontal slope, and its z crossing is linear in v'.  With (c_a, c_b) the
// centred voxel coordinates along the column's major axis and the other
// horizontal axis, the back-projector needs
//   e_b = c_a rb + pb - c_b,   E0 + c_z = ez0 + c_a ezc,   E1 = e10 + c_a e1c.
// Entry: {ax, rb, pb, ez0}, {ezc, e10, e1c, 0}.
int launch_column_table(const mgct_geom *g, int level, cudaStream_t s);
// The same column quantities as double-float pairs (hi, lo), for the public
// back-projector's accuracy at large N: entry {ax, rb, rb_lo, pb},
// {pb_lo, ez0, ez0_lo, ezc}, {ezc_lo, e10, e10_lo, e1c}, {e1c_lo, 0, 0, 0}
// (centred: E0 + c_z = ez0 + c_a ezc).
int launch_column_table_df(const mgct_geom *g, int level, cudaStream_t s);

}  // namespace mgct

struct mgct_geom {
    mgct_geom_desc desc;        // pointers inside are not kept
    std::vector<double> theta, z, drift;
    int has_drift;
    int separable;  // 1 if no view has a tilted detector (e_u horizontal, e_v vertical)
    int levels;
    mgct::LevelInfo lev[8];
    std::vector<mgct::ViewGeom> h_views[8];
    // scratch owned by the handle (mgct_project / mgct_backproject)
    void *d_scratch_vol;        // one finest volume, 4 bytes per voxel
    void *d_scratch_quads;      // projector quads of the finest grid, both ray classes (16 bytes per entry)
    double *d_scratch_part;     // reduction partials
    size_t scratch_part_count;
    int device;
    // preconditioner replacing Eq. 5 (mgct_geometry_set_preconditioner), [dz][dy][dx]
    float pkernel[27];
    int has_pkernel;
};

namespace mgct {

// ---------------------------------------------------------------------------
// Errors and launch accounting
// ---------------------------------------------------------------------------
int set_error(int status, const std::string &msg);
int check_cuda(cudaError_t e, const char *what);
void count_launch(int n = 1);

// Kernel kinds for the optional event trace (mgct_trace_enable / _read).
enum KernelKind {
    KK_PROJECT = 0,
    KK_BACKPROJECT = 1,
    KK_PRECONDITION = 2,
    KK_TRANSPOSE = 3,
    KK_GRID = 4,     // restrict / prolong
    KK_UPDATE = 5,   // Landweber update, OS-EMTR update, fills, copies
    KK_REDUCE = 6,
    KK_GEOMGRAD = 7,
    KK_CONV = 8,
    KK_OTHER = 9,
    KK_COUNT = 10
};
void trace_begin(int kind, cudaStream_t s);
void trace_end(int kind, cudaStream_t s);
void trace_tag(int tag);  // grid level of the launches that follow (this thread)
int check_ptr(const void *p, const char *name, bool may_be_null = false);

#define MGCT_TRY(...)                   \
    do {                                \
        int _st = (__VA_ARGS__);        \
        if (_st != MGCT_OK) return _st; \
    } while (0)

#define MGCT_LAUNCH_CHECK(what) MGCT_TRY(::mgct::check_cuda(cudaGetLastError(), what))

// Launch a kernel with launch accounting, optional event tracing and an
// error check: MGCT_KERNEL(kind, stream, kernel<<<...>>>(...));
#define MGCT_KERNEL(kind, stream, ...)                 \
    do {                                               \
        ::mgct::trace_begin(kind, stream);             \
        __VA_ARGS__;                                   \
        ::mgct::count_launch();                        \
        ::mgct::trace_end(kind, stream);               \
        MGCT_LAUNCH_CHECK("kernel launch");            \
    } while (0)

int validate_level(const mgct_geom *g, int level);
int validate_views(const mgct_geom *g, int view0, int nviews, int stride);

// ---------------------------------------------------------------------------
// dtype helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float to_f32(__half x) { return __half2float(x); }

template <typename T> __device__ __forceinline__ T from_f32(float x);
template <> __device__ __forceinline__ float from_f32<float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float x) {
    return __float2bfloat16_rn(x);
}
template <> __device__ __forceinline__ __half from_f32<__half>(float x) { return __float2half_rn(x); }

inline size_t dtype_size(mgct_dtype t) { return t == MGCT_F32 ? 4 : 2; }

// ---------------------------------------------------------------------------
// Ray direction and major axis, shared by the projector and the
// back-projector and written with explicit round-to-nearest intrinsics, so
// both kernels assign every ray to the same axis bit for bit.
// ---------------------------------------------------------------------------
struct RayDir {
    float wx, wy, wz;
    int ax;  // major axis: 0 = x, 1 = y (z never: checked at geometry creation)
};

__device__ __forceinline__ RayDir ray_dir(const ViewGeom &G, float up, float vp) {
    RayDir r;
    r.wx = __fmaf_rn(vp, G.Ev[0], __fmaf_rn(up, G.Eu[0], G.Wc[0]));
    r.wy = __fmaf_rn(vp, G.Ev[1], __fmaf_rn(up, G.Eu[1], G.Wc[1]));
    r.wz = __fmaf_rn(vp, G.Ev[2], __fmaf_rn(up, G.Eu[2], G.Wc[2]));
    r.ax = fabsf(r.wy) > fabsf(r.wx) ? 1 : 0;
    return r;
}

// ---------------------------------------------------------------------------
// Double-float arithmetic (value = hi + lo), error-free transformations with
// non-contracted intrinsics.
// ---------------------------------------------------------------------------
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF quick_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
    float s = __fadd_rn(x.hi, y.hi);
    float bb = __fsub_rn(s, x.hi);
    float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y.hi, bb));
    e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
    return quick_two_sum(s, e);
}
__device__ __forceinline__ DF df_mul_f(DF x, float f) {
    float p = __fmul_rn(x.hi, f);
    float e = __fmaf_rn(x.hi, f, -p);
    e = __fmaf_rn(x.lo, f, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ DF df_mul(DF x, DF y) {
    float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ DF df_div(DF x, DF y) {
    float q1 = __fdiv_rn(x.hi, y.hi);
    DF qy = df_mul_f(y, q1);
    DF r = df_add(x, DF{-qy.hi, -qy.lo});
    float q2 = __fdiv_rn(r.hi, y.hi);
    return quick_two_sum(q1, q2);
}
// c + up * a + vp * b, all coefficients double-float, up/vp exact floats
__device__ __forceinline__ DF df_affine(float c, float c_lo, float a, float a_lo, float b, float b_lo,
                                        float up, float vp) {
    return df_add(df_add(DF{c, c_lo}, df_mul_f(DF{a, a_lo}, up)), df_mul_f(DF{b, b_lo}, vp));
}

// ---------------------------------------------------------------------------
// Projector launch shape (shared with the buffers sized for its per-block
// partial sums): 32 x 8 pixel tiles, views in groups of PJ_VG.
// ---------------------------------------------------------------------------
constexpr int PJ_BX = 32;  // detector columns per block
constexpr int PJ_BY = 8;   // detector rows per block
#ifndef MGCT_PJ_VG
#define MGCT_PJ_VG 32
#endif
constexpr int PJ_VG = MGCT_PJ_VG;  // views per block group

inline size_t project_blocks(int nu, int nv, int nviews) {
    if (nviews <= 0) return 0;
    const size_t groups = (size_t)(nviews + PJ_VG - 1) / PJ_VG;
    const size_t vg = nviews < PJ_VG ? nviews : PJ_VG;
    return (size_t)((nu + PJ_BX - 1) / PJ_BX) * vg * groups * ((nv + PJ_BY - 1) / PJ_BY);
}
// Column projector (tilt-free geometries): a block is PC_COLS detector
// columns (one warp each) by PC_ROWS rows (one lane each).
constexpr int PC_COLS = 8;
constexpr int PC_ROWS = 32;
#ifndef MGCT_PC_VG
#define MGCT_PC_VG 32
#endif
constexpr int PC_VG = MGCT_PC_VG;  // views per block group (column projector)
inline size_t project_blocks_col(int nu, int nv, int nviews) {
    if (nviews <= 0) return 0;
    const size_t groups = (size_t)(nviews + PC_VG - 1) / PC_VG;
    const size_t vg = nviews < PC_VG ? nviews : PC_VG;
    return (size_t)((nu + PC_COLS - 1) / PC_COLS) * vg * groups * ((nv + PC_ROWS - 1) / PC_ROWS);
}
// Blocks of either projector: the size of per-block partial-sum buffers.
inline size_t project_blocks_any(int nu, int nv, int nviews) {
    const size_t a = project_blocks(nu, nv, nviews), b = project_blocks_col(nu, nv, nviews);
    return a > b ? a : b;
}

// ---------------------------------------------------------------------------
// Internal kernels used across translation units (host launchers)
// ---------------------------------------------------------------------------
// Quad copies of a volume for the projector (see Quad in project.cuh):
// corners (jz, jb) over [-QD_PAD, n + 1] stored at corner + QD_PAD.
constexpr int QD_PAD = 3;
__host__ __device__ constexpr int quad_side(int n) { return n + 2 * QD_PAD - 1; }
__host__ __device__ inline size_t quad_elems(int n) { return (size_t)quad_side(n) * n * quad_side(n); }
// src [z][i][b] (float32, bf16 or fp16) -> quads of T (float4 for float, two
// packed 16-bit pairs for bf16 / fp16) [z + QD_PAD][i][b + QD_PAD]
template <typename T, typename SRC = float>
int launch_build_quads(int n, const SRC *src, void *dst, cudaStream_t s);
// z-fastest quad copies for the column projector: src [z][i][b] ->
// dst[i][b + QD_PAD][z + QD_PAD], each entry the footprint as two z pairs
// (V(jz, jb), V(jz + 1, jb)), (V(jz, jb + 1), V(jz + 1, jb + 1))
template <typename T, typename SRC = float>
int launch_build_zquads(int n, const SRC *src, void *dst, cudaStream_t s);
// float32 z-fastest pairs for the column projector: (V(jz, jb), V(jz, jb + 1))
// at dst[i][jb + QD_PAD][jz + QD_PAD], zero outside the volume
template <typename SRC = float>
int launch_build_zpairs(int n, const SRC *src, void *dst, cudaStream_t s);
template <typename T>
int launch_transpose_xy(int n, const T *in, T *out, cudaStream_t s);

int launch_sum_partials(const double *part, int count, int nvals, double *out, cudaStream_t s);

}  // namespace mgct
