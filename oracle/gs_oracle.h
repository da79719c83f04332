/*
 * gs_oracle.h -- FP64 CPU oracle of the Turbo-GS dilated 3DGS rasterizer hot path.
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline leg (and its --impl reference arm) may load this library. The
 * product path (paper_2412_13547_b300) never imports, links or calls it, and it
 * shares no code, header, table or constant with the CUDA kernels.
 *
 * Every quantity is computed in double precision, one Gaussian or one pixel at
 * a time, in the order the method defines it:
 *   - 3D Gaussian and covariance R S S^T R^T                 (Sec. 3, Eq. 1)
 *   - EWA projection with the original focal length plus a
 *     low-pass term, 3-sigma radius                          (Sec. 3.1)
 *   - centre and radius in the downsampled tile grid         (Sec. 3.1, Eq. 3-4)
 *   - tile/depth keys, sort, per-tile ranges                 (Sec. 3, Sec. 3.1)
 *   - front-to-back alpha blending of the strided hr pixels  (Sec. 3 Eq. 2, Sec. 3.1 Eq. 5)
 *   - analytic backward, densification statistics           (Sec. 3.3)
 *   - Adam update                                            (Sec. 4.1)
 * Readings of points the paper leaves open are stated beside the code.
 */
#ifndef GS_ORACLE_H
#define GS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Pinhole camera. World point m goes to camera space as t = R m + T (R row-major),
 * x right, y down, z forward. Pixel centres sit at integer coordinates:
 * p = (fx t_x / t_z + cx, fy t_y / t_z + cy) on the width x height hr image. */
typedef struct {
    double R[9];
    double T[3];
    double fx, fy, cx, cy;
    int32_t width, height;
    double z_near;
} OrcCamera;

/* Dilation (Sec. 3.1): stride d, offsets 0 <= ox, oy < d. center_mode 0 bins the
 * Gaussian at (p - o)/d (lattice-aligned), 1 at (p - (d-1)/2)/d (Eq. 3 with
 * Eq. 5 read literally). tile is the tile edge in downsampled pixels (16). */
typedef struct {
    int32_t d, ox, oy, center_mode, tile;
} OrcDilation;

/* Ambiguity flags: an integer or branch decision of this Gaussian lies so close
 * to its threshold that FP32 arithmetic may take the other side. */
enum {
    ORC_FLAG_RADIUS = 1u << 0,   /* 3 sqrt(lambda_max) near an integer          */
    ORC_FLAG_RECT   = 1u << 1,   /* a tile-rect bound near a tile boundary       */
    ORC_FLAG_NEAR   = 1u << 2,   /* depth near the near plane                    */
    ORC_FLAG_CLAMP  = 1u << 3,   /* t_x/t_z or t_y/t_z near the Jacobian clamp   */
    ORC_FLAG_RGB    = 1u << 4,   /* a colour channel near the max(0, .) clamp    */
    ORC_FLAG_CULLED = 1u << 5    /* not a flag of ambiguity: Gaussian is culled  */
};

/* Sizes of the downsampled image and its tile grid. */
void orc_grid(const OrcCamera* cam, const OrcDilation* dil,
              int32_t* w_ds, int32_t* h_ds, int32_t* tiles_x, int32_t* tiles_y);

/* Real spherical harmonics basis (Condon-Shortley phase, index l*l+l+m) of
 * degree <= deg at the unit direction dir; out gets (deg+1)^2 values. */
void orc_sh_basis(int32_t deg, const double dir[3], double* out);

/* Projection. sh is n x (deg+1)^2 x 3. Outputs (all n-sized rows):
 * xy (2), conic (3: A, B, C of A dx^2 + 2B dx dy + C dy^2), opacity, rgb (3),
 * depth, cov2d (3: a, b, c of Sigma' incl. low-pass), radius (0 = culled),
 * rect (4: x0, y0, x1, y1 inclusive ds tile indices), tiles_touched,
 * flags (ORC_FLAG_*). Returns the number of visible Gaussians. */
int64_t orc_project(int32_t n, int32_t sh_degree,
                    const double* means, const double* log_scales, const double* quats,
                    const double* opacity_logits, const double* sh,
                    const OrcCamera* cam, const OrcDilation* dil,
                    double* xy, double* conic, double* opacity, double* rgb, double* depth,
                    double* cov2d, int32_t* radius, int32_t* rect, int64_t* tiles_touched,
                    uint32_t* flags);

/* Binning over the whole tile grid. depth_bits are the IEEE float32 bit
 * patterns of the depths (the sort key). Emits, for every touched tile of every
 * Gaussian, key = (tile_id << 32) | depth_bits and value = Gaussian index,
 * sorts ascending by (key, index), and writes per-tile [start, end) ranges
 * (tiles_x * tiles_y pairs). keys/vals must hold sum(tiles_touched) entries.
 * Returns the number of pairs. */
int64_t orc_bin(int32_t n, const int32_t* rect, const int64_t* tiles_touched,
                const uint32_t* depth_bits, int32_t tiles_x, int32_t tiles_y,
                uint64_t* keys, uint32_t* vals, uint32_t* ranges);

/* Binning of a subset of tiles: for each of the n_tiles tile ids, the depth
 * ordered list of Gaussians whose rect contains the tile. With vals == NULL
 * only counts[k] are written; otherwise vals holds the lists back to back and
 * ranges[2k], ranges[2k+1] bound list k. Returns the total length. */
int64_t orc_bin_tiles(int32_t n, const int32_t* rect, const uint32_t* depth_bits,
                      int32_t tiles_x, int32_t n_tiles, const int32_t* tile_ids,
                      uint32_t* vals, uint32_t* ranges);

/* Forward blend. With tile_ids == NULL every tile of the grid is rendered and
 * ranges are indexed by tile id; otherwise only the n_tiles listed tiles are
 * rendered and ranges[2k..2k+1] belongs to tile_ids[k]. img is the
 * w_ds x h_ds x 3 image (HWC), t_final and last are per ds pixel; last is the
 * list position (relative to the range start) + 1 of the last blended entry.
 * ambiguous (nullable) gets 1 where a gate value lies within the stated margin
 * of its threshold. counts (nullable) accumulates [entries evaluated, entries
 * blended]. */
void orc_render_fwd(const double* xy, const double* conic, const double* opacity,
                    const double* rgb, const double* depth,
                    const uint32_t* vals, const uint32_t* ranges,
                    int32_t n_tiles, const int32_t* tile_ids,
                    const OrcCamera* cam, const OrcDilation* dil, const double bg[3],
                    double* img, double* t_final, uint32_t* last, uint8_t* ambiguous,
                    uint64_t* counts);

/* Backward blend: accumulates (+=) dL/dxy, dL/dconic, dL/dopacity, dL/drgb
 * per Gaussian for the pixels of the listed tiles given dL/dimg (HWC). */
void orc_render_bwd(const double* xy, const double* conic, const double* opacity,
                    const double* rgb,
                    const uint32_t* vals, const uint32_t* ranges,
                    int32_t n_tiles, const int32_t* tile_ids,
                    const OrcCamera* cam, const OrcDilation* dil, const double bg[3],
                    const double* dl_dimg,
                    double* dxy, double* dconic, double* dopacity, double* drgb);

/* L1 loss over the rendered pixels against the hr target (height x width x 3)
 * sampled at the lattice pixels; writes dL/dimg and returns L. */
double orc_loss_l1(const OrcCamera* cam, const OrcDilation* dil, const double* img,
                   const double* target, double* dl_dimg);

/* Projection backward: from the per-Gaussian 2D gradients to the parameter
 * gradients (overwritten). Culled Gaussians get zero gradients. */
void orc_project_bwd(int32_t n, int32_t sh_degree,
                     const double* means, const double* log_scales, const double* quats,
                     const double* opacity_logits, const double* sh,
                     const OrcCamera* cam, const OrcDilation* dil,
                     const double* dxy, const double* dconic, const double* dopacity,
                     const double* drgb,
                     double* d_means, double* d_log_scales, double* d_quats,
                     double* d_opacity_logits, double* d_sh);

/* Densification statistics (Sec. 3.3): for every Gaussian with tiles_touched > 0,
 * pos_acc += |dL/dxy|_2 (hr pixel units), col_acc += |dL/drgb|_2, count += 1. */
void orc_densify_stats(int32_t n, const int64_t* tiles_touched, const double* dxy,
                       const double* drgb, double* pos_acc, double* col_acc,
                       int32_t* count);

/* Adam (Kingma & Ba) on one flat tensor of rows of row_width elements; step is
 * 1-based. With row_mask != NULL rows whose mask is 0 are left untouched. */
void orc_adam(int64_t numel, int32_t row_width, double* param, const double* grad,
              double* m, double* v, double lr, double beta1, double beta2, double eps,
              int32_t step, const uint8_t* row_mask);

#ifdef __cplusplus
}
#endif
#endif
