/*
 * CPU oracle for the SG-Splatting rasterizer -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg
 * may load this library.  It shares no code, header or constant table with the CUDA
 * path under paper_2501_00342_b300/; both sides are written separately from the
 * paper (Eq. 2-9) and from the 3D Gaussian splatting rasterizer conventions it builds
 * on (3-sigma support, alpha clamp 0.99, alpha cutoff 1/255, early stop below
 * transmittance 1e-4, EWA dilation 0.3 px).
 *
 * Three parts:
 *   mirror32.cpp   FP32 "binning mirror": the integer decisions of the method taken in
 *                  single precision with a fixed, written-out operation order (depth
 *                  bits, screen mean, radius, tile rectangle, conic, tile|depth keys,
 *                  stable sort, per-tile ranges, per-pixel support membership).
 *   forward64.cpp  FP64 brute-force renderer: per pixel, every Gaussian whose support
 *                  holds the pixel centre, ordered by (FP32 depth bits, index), blended
 *                  front to back.  No tiles.
 *   adjoint64.cpp  Hand-written FP64 reverse mode of forward64.
 *
 * Scene planes are the float32 SoA arrays described in paper_2501_00342_b300/inputs.py.
 * Cameras are float32 rows of 22: viewmat[12] (row-major world->camera 3x4),
 * campos[3], fx, fy, cx, cy, width, height, near.
 */
#ifndef SGS_ORACLE_H
#define SGS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int64_t n, stride;
    int32_t sh_degree, num_lobes, axis_mode; /* axis_mode: 0 free axes, 1 world axes */
    const float *mean, *scale, *rot, *opacity, *sh, *sg_amp, *sg_axis, *sg_sharp;
    /* Adaptive SH degree (Sec. "Mixing Spherical Harmonics and Spherical Gaussians"): when
     * sh_adaptive is 1, a record sums the SH bands l <= D, D = 0 below radius threshold
     * sh_radius[0], 1 below sh_radius[1], else 2, capped at sh_degree; the radius is the
     * mirror's integer pixel radius ceil(3 sqrt(lambda_max)). */
    int32_t sh_adaptive;
    float sh_radius[2];
} orc_scene;

typedef struct { /* double planes with the same [..][stride] layout as the scene */
    double *mean, *scale, *rot, *opacity, *sh, *sg_amp, *sg_axis, *sg_sharp;
} orc_grads;

/* ---- FP32 binning mirror ---- */
/* Per record r = v*n + i: visible flag, depth bits, mean2d, conic, radius, rect
 * (x0,y0,x1,y1 inclusive tile coords), tiles touched. */
void orc_mirror_preprocess(const orc_scene* s, const float* cams, int32_t B, int32_t tile_w,
                           int32_t tile_h, uint8_t* visible, uint32_t* depth_bits,
                           float* mean2d, float* conic, float* radius, int32_t* rect,
                           uint32_t* tiles_touched);
/* Total number of tiles over all views. */
int64_t orc_num_tiles(const float* cams, int32_t B, int32_t tile_w, int32_t tile_h);
/* Number of (record, tile) instances. */
int64_t orc_mirror_count(const orc_scene* s, const float* cams, int32_t B, int32_t tile_w,
                         int32_t tile_h);
/* Keys/values before and after a stable sort by key, and per-tile [start,end). */
void orc_mirror_bin(const orc_scene* s, const float* cams, int32_t B, int32_t tile_w,
                    int32_t tile_h, uint64_t* keys_in, uint32_t* vals_in, uint64_t* keys_out,
                    uint32_t* vals_out, uint32_t* ranges);
/* Stable sort of (key, value) pairs by key (std::stable_sort). */
void orc_stable_sort_pairs(int64_t m, uint64_t* keys, uint32_t* vals);

/* ---- FP64 forward ---- */
/* Per record: visible (from the mirror), mean2d, conic, rgb (clamped), opacity, view
 * depth; all FP64. */
void orc_preprocess64(const orc_scene* s, const float* cams, int32_t B, uint8_t* visible,
                      double* mean2d, double* conic, double* rgb, double* depth);
/* Render the listed pixels (rows of view, x, y).  margin = smallest relative distance of
 * any discrete FP64 decision (alpha < 1/255, 0.99 clamp, T < 1e-4 stop) from its
 * threshold; sig = hash of the contributor set and clamp states. */
void orc_render_pixels(const orc_scene* s, const float* cams, int32_t B, const double* bg,
                       const int32_t* pix, int64_t P, double* out_rgb, double* out_T,
                       double* out_margin, int32_t* out_ncontrib, uint64_t* out_sig,
                       int32_t threads);

/* ---- FP64 adjoint ---- */
/* Gradients of L = sum_p dL_drgb[p] . rgb[p] over the listed pixels, w.r.t. every scene
 * parameter (overwritten). */
void orc_adjoint_pixels(const orc_scene* s, const float* cams, int32_t B, const double* bg,
                        const int32_t* pix, int64_t P, const double* dL_drgb, orc_grads* g,
                        int32_t threads);

/* Real SH basis value Y_lm(d) for unit d, index l*l + l + m (exposed for pins). */
double orc_sh_basis(int32_t l, int32_t m, const double* d);

#ifdef __cplusplus
}
#endif
#endif
