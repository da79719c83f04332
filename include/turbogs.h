/*
 * turbogs.h -- C ABI of the B300 (sm_103a) hot path of Turbo-GS fitting:
 * a differentiable tile-based 3D Gaussian splatting rasterizer with dilated
 * rendering (arXiv 2412.13547, Sec. 3.1), the per-Gaussian densification
 * statistics it feeds (Sec. 3.3) and a fused Adam step (Sec. 4.1).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Pointers named d_* or documented as "device" are CUDA device pointers; the
 *   caller owns all of them. The library never allocates device memory (scratch
 *   is passed in, sized by the *_workspace_size queries). GsCamera, GsDilation,
 *   bg[3] and GsAdamTensor arrays are read on the host at call time.
 * - Every call is asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *   default stream) and returns a status: GS_OK, GS_ERR_ARG for a bad argument
 *   (nothing is launched), GS_ERR_CUDA when a launch failed (gs_last_error()
 *   gives the CUDA error string of the calling thread).
 * - Arrays are contiguous, row-major, FP32 unless stated. Per-Gaussian arrays
 *   have n rows; images are height x width x 3 (HWC).
 * - Image geometry: an hr image of width x height pixels with pixel centres at
 *   integer coordinates. A dilation (d, ox, oy) renders the lattice of hr pixels
 *   (d*u + ox, d*v + oy) as a w_ds x h_ds image, w_ds = ceil((width - ox)/d),
 *   h_ds = ceil((height - oy)/d), tiled by tile x tile downsampled pixels
 *   (tiles_x = ceil(w_ds/tile), tiles_y = ceil(h_ds/tile)); tile ids are
 *   row-major, ty * tiles_x + tx.
 */
#ifndef TURBOGS_H
#define TURBOGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void* gs_stream_t; /* cudaStream_t */

enum {
    GS_OK = 0,
    GS_ERR_ARG = 1,
    GS_ERR_CAPACITY = 2,
    GS_ERR_CUDA = 3,
    GS_ERR_TIMEOUT = 4
};

/* Storage type of the SH coefficients (and of Adam's optional shadow copy). */
enum { GS_DTYPE_F32 = 0, GS_DTYPE_BF16 = 1, GS_DTYPE_F16 = 2 };

/* Pinhole camera (Sec. 3.1 projects with the original, hr focal length).
 * A world point m maps to camera space t = R m + T (R row-major; x right,
 * y down, z forward) and to the hr pixel (fx t_x/t_z + cx, fy t_y/t_z + cy).
 * Gaussians with t_z <= z_near are culled. */
typedef struct {
    float R[9];
    float T[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float z_near;
} GsCamera;

/* Dilated rendering (Sec. 3.1): stride d >= 1, offsets 0 <= ox, oy < d.
 * center_mode 0 bins a Gaussian around the downsampled centre (p - o)/d, the
 * lattice the offset renders; 1 uses (p - (d-1)/2)/d, Eq. 3 combined with the
 * pixel map of Eq. 5. Eq. 4: the downsampled radius is r/d. tile is the tile
 * edge in downsampled pixels (Sec. 3.1 fixes 16; 8 and 32 are accepted): the
 * unit of the tile-Gaussian lists the blend walks.
 * bin_shift (0, 1 or 2) coarsens only the binning: pairs are formed with tiles
 * of tile << bin_shift pixels (fewer pairs to bin), and each blend tile keeps
 * from its binning tile's list exactly the entries of its own list, in order.
 * Images, transmittances and gradients do not depend on it; only the list
 * positions stored in `last` do. */
typedef struct {
    int32_t d, ox, oy, center_mode, tile, bin_shift;
} GsDilation;

/* Width of the per-Gaussian records below, in floats. */
#define GS_SPLAT_FLOATS 16
#define GS_GRAD2D_FLOATS 12

/* Splat record written by gs_project (64 bytes per Gaussian):
 *   [0] x_hi  [1] y_hi  [2] conic A  [3] conic B
 *   [4] conic C  [5] opacity  [6] r  [7] g
 *   [8] b  [9] depth t_z  [10] x_lo  [11] y_lo
 *   [12..15] int32 x0, y0, x1, y1: inclusive rectangle of blend tiles touched
 * The hr image-plane centre is (x_hi + x_lo, y_hi + y_lo), kept as an unevaluated
 * float-float sum so that pixel offsets at 4K stay accurate. The conic is the
 * inverse 2D covariance: G = exp(-(A dx^2 + C dy^2)/2 - B dx dy) (Sec. 3, Eq. 1).
 *
 * 2D gradient record accumulated by gs_render_bwd (48 bytes per Gaussian):
 *   [0] dL/dx  [1] dL/dy  [2] dL/dA  [3] dL/dB
 *   [4] dL/dC  [5] dL/dopacity  [6] dL/dr  [7] dL/dg
 *   [8] dL/db  [9..11] zero padding                                       */

/* Library version (major*10000 + minor*100 + patch) and the per-thread error. */
int32_t gs_version(void);
const char* gs_last_error(void);

/* Size of the downsampled image and of its blend tile grid (host arithmetic
 * only; the grid of the blend launches and of the tile orders). */
int32_t gs_grid(const GsCamera* cam, const GsDilation* dil,
                int32_t* w_ds, int32_t* h_ds, int32_t* tiles_x, int32_t* tiles_y);

/* The binning tile grid: ceil(tiles_x / 2^bin_shift) x ceil(tiles_y /
 * 2^bin_shift) (the grid of rects, gs_bin_sort and ranges). */
int32_t gs_bin_grid(const GsCamera* cam, const GsDilation* dil, int32_t* bin_tiles_x, int32_t* bin_tiles_y);

/* ---------------------------------------------------------------------------
 * gs_project -- Sec. 3 (Sigma = R S S^T R^T, opacity, SH colour) and Sec. 3.1
 * (EWA projection Sigma' = J W Sigma W^T J^T with the hr focal length plus a
 * 0.3 px^2 low-pass term, 3-sigma radius r = ceil(3 sqrt(lambda_max)) in hr
 * pixels, downsampled centre and radius r/d of Eq. 3-4, and the rectangle of
 * downsampled tiles it touches).
 *   means (n x 3), log_scales (n x 3, scale = exp), quats (n x 4, (w,x,y,z),
 *   any norm > 0), opacity_logits (n, opacity = sigmoid), sh (n x K x 3 with
 *   K = (sh_degree+1)^2, sh_degree <= 3, of type sh_dtype): device inputs.
 *   Colour = max(0, sum_k Y_k(dir) sh_k + 0.5), dir = unit(mean - camera centre),
 *   real SH with Condon-Shortley phase, index l*l + l + m.
 * Outputs (device): splats (n x 16, layout above), radii (n, 0 = culled),
 *   rects (n x 4: x0, y0, x1, y1 inclusive binning tile indices, the blend
 *   tile rectangle shifted right by bin_shift; culled: 0, 0, -1, -1),
 *   tiles_touched (n: binning tiles in the rect; > 0 = visible),
 *   depth_keys (nullable, n uint32: the depth sort key of gs_bin_sort, the
 *   float32 bits of the depth t_z of a visible Gaussian, at most 0xfffffffe,
 *   and 0xffffffff for a culled one; given to gs_bin_sort, it saves its
 *   pass over the splat records).
 *   A Gaussian is culled (radius 0, empty rect) when its blend tile rectangle
 *   is empty, whatever bin_shift.
 * Errors: GS_ERR_ARG for n < 0, a null pointer with n > 0, sh_degree outside
 *   0..3, a bad dtype, d < 1 or d > 64, offsets outside [0, d), tile not in
 *   {8, 16, 32}, or a non-positive image size or focal length. */
int32_t gs_project(int32_t n, int32_t sh_degree, int32_t sh_dtype,
                   const float* means, const float* log_scales, const float* quats,
                   const float* opacity_logits, const void* sh,
                   const GsCamera* cam, const GsDilation* dil,
                   float* splats, int32_t* radii, int32_t* rects, int32_t* tiles_touched,
                   uint32_t* depth_keys, gs_stream_t stream);

/* ---------------------------------------------------------------------------
 * gs_bin_sort -- the tile-Gaussian pairs of the tile-based rasterizer (Sec. 3,
 * and the "duplicateWithKeys"/"sortPairs" stages profiled in Sec. 3.1): for
 * every tile of every Gaussian's rect, the pair (key = tile_id << 32 |
 * float32 bits of the depth, value = Gaussian index), sorted ascending by
 * (key, value), and per-tile [start, end) ranges into the sorted values.
 * Inputs (device): rects, tiles_touched (from gs_project for the same
 *   dilation), splats (depth = [9]); depth_keys (nullable: gs_project's keys
 *   for the same call, used instead of reading the depths from splats);
 *   tiles_x, tiles_y: the binning grid (gs_bin_grid). Rects outside the grid
 *   are ignored.
 * Outputs (device): sorted_ids (capacity entries; the first num_pairs hold the
 *   Gaussian ids tile by tile, front to back), ranges (tiles_x*tiles_y x 2,
 *   uint32 start/end; (0, 0) for a tile no Gaussian touches), num_pairs (one
 *   int64: the pair count K), num_pairs_max (nullable, one int64: raised to K
 *   when K is larger and never lowered by the library, so that a caller can
 *   check once, after many calls, that none overflowed its capacity).
 * No host synchronisation: K is computed and consumed on the device. When
 *   K > capacity, *num_pairs still receives K, no pair is written beyond
 *   capacity, every range is set empty (the render then sees no Gaussian) and
 *   the caller must grow the buffers and call again; K <= 2^31 - 1.
 * workspace: device scratch of gs_bin_sort_workspace_size(n, capacity,
 *   tiles_x, tiles_y) bytes, 256-byte aligned; its contents need no init. The
 *   size also covers every smaller grid (tx <= tiles_x, ty <= tiles_y), so one
 *   workspace serves all dilations of an image.
 * Method: the pairs are never materialised with keys nor sorted. The
 *   Gaussians are radix-sorted by (depth bits, id); a two-level counting
 *   scatter then writes every id straight into its slot: first into per-row
 *   lists (one entry per tile row of the rect), then each row list into its
 *   tiles, both levels stable. tiles_x, tiles_y <= 4096.
 * Output form: the 64-bit (tile << 32 | depth bits) keys are implied, not
 *   written. The sorted key of entry j of tile t's range is t << 32 | the
 *   float32 bits of splats[sorted_ids[j]][9], so (sorted_ids, ranges) is the
 *   whole result of sorting the (key, value) pairs: the same list, position
 *   for position, as the key sort of the tile-based rasterizer (Sec. 3) on
 *   the downsampled tile grid (Sec. 3.1).
 * Errors: GS_ERR_ARG for bad sizes, null pointers or a short workspace. */
size_t gs_bin_sort_workspace_size(int32_t n, int64_t capacity, int32_t tiles_x, int32_t tiles_y);
int32_t gs_bin_sort(int32_t n, const int32_t* rects, const int32_t* tiles_touched,
                    const float* splats, const uint32_t* depth_keys, int32_t tiles_x, int32_t tiles_y,
                    void* workspace, size_t workspace_bytes, int64_t capacity,
                    uint32_t* sorted_ids, uint32_t* ranges, int64_t* num_pairs,
                    int64_t* num_pairs_max, gs_stream_t stream);

/* ---------------------------------------------------------------------------
 * gs_bin_sort_static -- gs_bin_sort for callers that cannot allocate device
 * memory: a renderer plugin or embedded host that only hands over its own input
 * and output buffers, or a serving process whose device memory budget is fixed
 * once at start-up and forbids cudaMalloc afterwards. The paper has no
 * counterpart; it exists for those callers only.
 * Same arguments, results and errors as gs_bin_sort, minus the workspace: the
 * scratch lives in one array of GS_BIN_SORT_STATIC_SCRATCH_BYTES (32 MiB)
 * compiled into the library, which every GPU that loads the library holds
 * until the process exits. Calls whose gs_bin_sort_workspace_size(n, capacity,
 * tiles_x, tiles_y) exceeds that size return GS_ERR_ARG (nothing launched) with
 * the required size in gs_last_error(); for example n = 256K Gaussians with
 * 1.5M pairs on a 1920x1080 grid fits. The call allocates nothing and calls no
 * allocating routine.
 * Every call looks up the array's device address in the calling thread's
 * current CUDA context, so the call is valid in any context (a plugin's own
 * context, or a new one after cudaDeviceReset). With lazy module loading (the
 * CUDA default since 12.2) the array is reserved when the library's module is
 * first used on a device, which can fail with out-of-memory in a process
 * whose device memory is already spoken for: make one call at start-up (it
 * also loads the module, so make it before any stream capture), or set
 * CUDA_MODULE_LOADING=EAGER to reserve the array when the library loads.
 * All calls share the one array and it keeps the last call's contents: calls
 * that may overlap on the GPU (different streams, or different host threads
 * on one device) race on it, so serialise them. */
#define GS_BIN_SORT_STATIC_SCRATCH_BYTES (32u << 20)
int32_t gs_bin_sort_static(int32_t n, const int32_t* rects, const int32_t* tiles_touched,
                           const float* splats, const uint32_t* depth_keys, int32_t tiles_x,
                           int32_t tiles_y, int64_t capacity,
                           uint32_t* sorted_ids, uint32_t* ranges, int64_t* num_pairs,
                           int64_t* num_pairs_max, gs_stream_t stream);

/* ---------------------------------------------------------------------------
 * gs_tile_order -- a launch order for the blend kernels: the tile ids sorted
 * by descending list length (end - start of ranges), bucketed 8 buckets per
 * power of two. Started longest-first, the tiles of uneven load finish close
 * together instead of leaving a tail. Inputs (device): ranges (num_tiles x 2).
 * Output (device): order (num_tiles). For a dilation with bin_shift > 0 (blend
 * tiles differ from binning tiles) use gs_tile_order_batch. */
int32_t gs_tile_order(const uint32_t* ranges, int32_t num_tiles, uint32_t* order, gs_stream_t stream);

/* ---------------------------------------------------------------------------
 * gs_render_fwd -- front-to-back alpha blending (Sec. 3, Eq. 2) of the lattice
 * pixels of the dilated image (Sec. 3.1: tile lists from the downsampled grid,
 * Gaussian evaluated at the hr pixel (d*u + ox, d*v + oy), Eq. 5).
 * Per pixel, walking its tile's list: alpha = min(0.99, opacity * G); entries
 * with alpha < 1/255 (or a positive exponent) are skipped; the walk stops
 * before an entry that would take the transmittance below 1e-4; finally
 * C += T * bg. Both gates are decided in FP32 on log2(opacity * G), in the
 * same arithmetic as gs_render_bwd's replay.
 * Inputs (device): splats, sorted_ids, ranges (from gs_bin_sort). bg: host
 *   float[3].
 * Each blend tile walks its binning tile's list (the same list when
 *   bin_shift is 0) and keeps the entries whose splat record rectangle
 *   ([12..15]) contains it: its own list, in depth order.
 * Outputs (device): img (h_ds x w_ds x 3), t_final (h_ds x w_ds), last
 *   (h_ds x w_ds: position + 1, in the binning tile's list, of the last
 *   blended entry, 0 if none),
 *   counts (nullable, 3 x uint64 accumulated with +=: list entries evaluated,
 *   entries blended, and entries the backward replays, i.e. the sum over
 *   pixels of the own-list position of their last blended entry; the caller
 *   zeroes it).
 * pixels_per_thread: launch shape, not semantics -- each thread of the
 *   tile's CTA handles this many pixels: 0 = the library default (1 for tile
 *   8, else 2; gs_render_bwd: 4 for tile 16 when the launch has at least 4096
 *   tiles), else 1 or 2 for tile 8, 1, 2 or 4 for tile 16, 2 or 4 for tile 32
 *   (whole warps, at most 512 threads; others give GS_ERR_ARG). Results are
 *   identical for every value.
 * tile_order (nullable, device, tiles_x*tiles_y entries): the blend tiles in
 *   the order their CTAs should start, e.g. from gs_tile_order_batch.
 *   Scheduling only: the results do not depend on it. */
int32_t gs_render_fwd(int32_t n, const float* splats, const uint32_t* sorted_ids,
                      const uint32_t* ranges, const GsCamera* cam, const GsDilation* dil,
                      const float* bg, float* img, float* t_final, uint32_t* last,
                      unsigned long long* counts, int32_t pixels_per_thread,
                      const uint32_t* tile_order, gs_stream_t stream);

/* ---------------------------------------------------------------------------
 * Targets. A target image (height x width x 3, row-major) is FP32 values in
 * [0, 1] (GS_TARGET_F32), or 8-bit values t as photographs are stored
 * (GS_TARGET_U8), which every kernel reads as the FP32 product t * (1/255),
 * 1/255 rounded to FP32 (0x3B808081): a quarter of the bytes to copy to the
 * device and to read per step. */
#define GS_TARGET_F32 0
#define GS_TARGET_U8 1

/* ---------------------------------------------------------------------------
 * gs_loss_l1 -- L1 photometric loss of the rendered lattice pixels against the
 * hr target sampled at the same pixels (supervision with "corresponding
 * high-resolution pixels", Sec. 3.1): L = mean |img - target| over h_ds*w_ds*3
 * values, dL/dimg = sign(img - target) / (3 * h_ds * w_ds) (sign(0) = 0).
 * Inputs (device): img (h_ds x w_ds x 3), target (height x width x 3, of
 *   target_dtype, GS_TARGET_F32 or GS_TARGET_U8).
 * Outputs (device): dl_dimg (h_ds x w_ds x 3), loss (one float, overwritten). */
int32_t gs_loss_l1(const GsCamera* cam, const GsDilation* dil, const float* img,
                   const void* target, int32_t target_dtype, float* dl_dimg, float* loss, gs_stream_t stream);

/* ---------------------------------------------------------------------------
 * gs_render_fwd_l1 -- gs_render_fwd and gs_loss_l1 in one launch (plus a
 * one-thread kernel that zeroes *loss first): each pixel's L1 term and
 * dL/dimg come from the colour the blend holds in registers, with
 * gs_loss_l1's arithmetic (dl_dimg bit-identical; *loss equal up to the order
 * of the float additions). grad2d_zero (nullable, n x 12, 16-byte aligned):
 * zeroed by the same launch, for a gs_render_bwd with zero_grad2d = 0. The
 * forward is bound by its arithmetic and leaves DRAM idle, so the loss and the
 * zeroing cost it little, where as separate passes they would be paid in full.
 * Other arguments, outputs and errors as gs_render_fwd and gs_loss_l1. */
#define GS_FWD_L1 1
#define GS_FWD_ZERO_GRAD2D 2
int32_t gs_render_fwd_l1(int32_t n, const float* splats, const uint32_t* sorted_ids,
                         const uint32_t* ranges, const GsCamera* cam, const GsDilation* dil,
                         const float* bg, float* img, float* t_final, uint32_t* last,
                         const void* target, int32_t target_dtype, float* dl_dimg, float* loss,
                         float* grad2d_zero, unsigned long long* counts, int32_t pixels_per_thread,
                         const uint32_t* tile_order, gs_stream_t stream);

/* ---------------------------------------------------------------------------
 * gs_ssim -- SSIM, the structural-similarity index (Wang et al. 2004) the
 * paper reports beside PSNR (Sec. 4, metrics), of the rendered lattice image
 * against the hr target sampled at the same pixels (as gs_loss_l1 samples it).
 * Per channel and lattice pixel p, with the 11 x 11 Gaussian window (sigma
 * 1.5, weights summing to 1) sums m_x, m_y, E_xx, E_yy, E_xy around p:
 *   SSIM_p = (2 m_x m_y + C1)(2 (E_xy - m_x m_y) + C2)
 *            / ((m_x^2 + m_y^2 + C1)(E_xx - m_x^2 + E_yy - m_y^2 + C2)),
 * C1 = 0.01^2, C2 = 0.03^2 (values in [0, 1]). mode 0 ("valid"): the mean over
 * the pixels whose window lies inside the lattice image (at least 11 x 11);
 * mode 1 ("same"): the mean over all pixels, zeros outside the image (the
 * form 3DGS fitting trains with). Channels are averaged.
 * Inputs (device): img (h_ds x w_ds x 3), target (height x width x 3, of
 *   target_dtype as for gs_loss_l1).
 * Outputs (device): *ssim_out (one float, overwritten); d_img (nullable,
 *   h_ds x w_ds x 3): d (mean SSIM) / d img, overwritten.
 * workspace: gs_ssim_workspace_size(cam, dil) bytes, 256-byte aligned (9
 *   floats per lattice pixel and two accumulators; no init needed).
 * Errors: GS_ERR_ARG for a bad camera/dilation/mode, null pointers, a short or
 *   misaligned workspace, or a lattice under 11 x 11 in mode 0. */
size_t gs_ssim_workspace_size(const GsCamera* cam, const GsDilation* dil);
int32_t gs_ssim(const GsCamera* cam, const GsDilation* dil, const float* img, const void* target,
                int32_t target_dtype, int32_t mode, float* ssim_out, float* d_img, void* workspace,
                size_t workspace_bytes, gs_stream_t stream);

/* gs_loss_l1_dssim -- the photometric loss of 3DGS fitting, which the paper's
 * method builds on (the paper's own loss is the L1 of gs_loss_l1):
 *   L = (1 - lambda) L1 + lambda (1 - SSIM),  0 <= lambda <= 1,
 * L1 as in gs_loss_l1 and SSIM as in gs_ssim (mode as there), over the lattice
 * pixels. Outputs (device): dl_dimg (h_ds x w_ds x 3, overwritten) = dL/dimg,
 * *loss (overwritten). workspace as gs_ssim. */
int32_t gs_loss_l1_dssim(const GsCamera* cam, const GsDilation* dil, const float* img, const void* target,
                         int32_t target_dtype, float lambda, int32_t mode, float* dl_dimg, float* loss, void* workspace,
                         size_t workspace_bytes, gs_stream_t stream);

/* ---------------------------------------------------------------------------
 * gs_render_bwd -- backward of gs_render_fwd. The per-pixel blend state is not
 * stored: each pixel replays its list back to front from t_final and last,
 * recovering T_i = T_{i+1} / (1 - alpha_i), and the per-Gaussian gradients of
 * the pixels of a tile are reduced in registers/shared memory before one set
 * of atomics per (tile, Gaussian).
 * Inputs (device): as gs_render_fwd plus t_final, last and dl_dimg.
 * Output (device): grad2d (n x 12, layout above), accumulated with +=; with
 *   zero_grad2d != 0 the library first zeroes it on the stream.
 * pixels_per_thread, tile_order: as for gs_render_fwd (results equal up to
 *   the order of the floating-point atomic additions). */
int32_t gs_render_bwd(int32_t n, const float* splats, const uint32_t* sorted_ids,
                      const uint32_t* ranges, const GsCamera* cam, const GsDilation* dil,
                      const float* bg, const float* t_final, const uint32_t* last,
                      const float* dl_dimg, float* grad2d, int32_t zero_grad2d,
                      int32_t pixels_per_thread, const uint32_t* tile_order,
                      gs_stream_t stream);

/* ---------------------------------------------------------------------------
 * gs_project_bwd -- chain rule of gs_project: from grad2d to the parameter
 * gradients (overwritten, FP32, same shapes as the parameters; d_sh is
 * n x K x 3 FP32 whatever sh_dtype is). Culled Gaussians get zero gradients.
 * With pos_acc, col_acc and count non-null it also performs gs_densify_stats.
 * Inputs (device): the gs_project inputs, tiles_touched, grad2d. */
int32_t gs_project_bwd(int32_t n, int32_t sh_degree, int32_t sh_dtype,
                       const float* means, const float* log_scales, const float* quats,
                       const float* opacity_logits, const void* sh,
                       const GsCamera* cam, const GsDilation* dil,
                       const int32_t* tiles_touched, const float* grad2d,
                       float* d_means, float* d_log_scales, float* d_quats,
                       float* d_opacity_logits, float* d_sh,
                       float* pos_acc, float* col_acc, int32_t* count,
                       gs_stream_t stream);

/* ---------------------------------------------------------------------------
 * gs_project_bwd_adam -- gs_project_bwd, gs_densify_stats and gs_adam fused
 * into one pass over the Gaussians (the gradient of each Gaussian goes from
 * its 2D record straight into its Adam update, never through HBM). Results
 * equal gs_project_bwd followed by gs_adam with the same settings up to FP32
 * rounding (the two kernels may contract the shared gradient arithmetic into
 * FMAs differently); the Adam update itself is the same pinned arithmetic.
 * adam->param[0..4] are the FP32 parameters (means, log_scales, quats,
 * opacity_logits, sh), updated in place; m, v their moments (FP32, also for
 * the SH); lr per tensor. sh_store (device) is the SH storage the forward
 * projection read. Three forms of SH storage:
 *   - FP32: sh_store is adam->param[4] (or param[4] is NULL: the same array).
 *   - low precision only (the precision form: SH and colours stored in
 *     BF16/FP16, blend and accumulation in FP32): adam->param[4] = NULL and
 *     sh_dtype BF16 or FP16. sh_store is the parameter itself, updated in place:
 *     the update is computed in FP32 from the stored value and rounded
 *     stochastically to sh_dtype (the neighbour away from zero with probability
 *     equal to the value's position between the two neighbours, from 16 bits
 *     of the PCG hash of Jarzynski & Olano 2020: elements 2k and 2k + 1 take
 *     the low and high halves of hash(base + k), e = g * 3 (sh_degree+1)^2 + j
 *     the element index, base = hash(hash(sr_seed) xor t), t the Adam step:
 *     *adam->step_dev when given, else adam->step). No FP32
 *     copy of the SH exists, so the pass moves 2 instead of 4 bytes per SH
 *     value in each direction. adam->sh_shadow must be NULL.
 *   - FP32 master with a low-precision copy: adam->param[4] FP32 and sh_store
 *     its BF16/FP16 copy, refreshed (round to nearest) from the updated FP32
 *     values when adam->sh_shadow points at it.
 * With adam->sparse != 0 Gaussians with tiles_touched == 0 are left untouched
 * (no moment decay).
 * grads_out (nullable host array of 5 device pointers, each nullable) receives
 * the gradients as gs_project_bwd would write them. pos_acc/col_acc/count:
 * as in gs_project_bwd. bias_dev (nullable device pointer to two floats
 * (1/(1-beta1^t), 1/(1-beta2^t)), as gs_adam_advance writes them) replaces the
 * bias correction computed on the host from step, so that a CUDA graph
 * holding this call stays valid while the step advances; step is then
 * ignored. */
typedef struct {
    float* param[5];
    float* m[5];
    float* v[5];
    float lr[5];
    float beta1, beta2, eps;
    int32_t step;
    int32_t sparse;
    void* sh_shadow;
    int32_t sh_shadow_dtype;
    const float* bias_dev;
    const int32_t* step_dev;   /* nullable device int32: t of the rounding stream */
    uint32_t sr_seed;          /* seed of the stochastic rounding (low-precision SH) */
} GsAdamParams;
int32_t gs_project_bwd_adam(int32_t n, int32_t sh_degree, int32_t sh_dtype, const void* sh_store,
                            const GsCamera* cam, const GsDilation* dil,
                            const int32_t* tiles_touched, const float* grad2d,
                            const GsAdamParams* adam, float* pos_acc, float* col_acc,
                            int32_t* count, float* const* grads_out, gs_stream_t stream);

/* gs_adam_advance -- one device thread adds 1 to *step_dev (device int32, the
 * Adam step t, 0 before the first step) and writes the bias corrections of the
 * new t to bias_dev[0..1] = (1/(1-beta1^t), 1/(1-beta2^t)), evaluated in
 * double and rounded to float like the host path of gs_project_bwd_adam. One
 * call per optimizer step, before the fused step that reads bias_dev. */
int32_t gs_adam_advance(int32_t* step_dev, float beta1, float beta2, float* bias_dev,
                        gs_stream_t stream);

/* ---------------------------------------------------------------------------
 * gs_densify_stats -- position-appearance densification scores (Sec. 3.3): for
 * every Gaussian with tiles_touched > 0, pos_acc += |(dL/dx, dL/dy)|_2 (hr
 * pixel units), col_acc += |(dL/dr, dL/dg, dL/db)|_2, count += 1 (device). */
int32_t gs_densify_stats(int32_t n, const int32_t* tiles_touched, const float* grad2d,
                         float* pos_acc, float* col_acc, int32_t* count, gs_stream_t stream);

/* ---------------------------------------------------------------------------
 * gs_adam -- one fused Adam step (Kingma & Ba, bias-corrected; Sec. 4.1 trains
 * with Adam) over up to GS_ADAM_MAX_TENSORS tensors in a single launch:
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * Each tensor has numel elements in rows of row_width (one row per Gaussian);
 * with row_mask (device, one byte per row, shared by all tensors) non-null,
 * rows whose byte is 0 are left untouched ("sparse" Adam over visible
 * Gaussians). shadow (nullable) receives the updated parameter converted to
 * shadow_dtype (e.g. the BF16 SH storage the projection reads). With param
 * NULL and shadow non-null of BF16/FP16 type, shadow is the parameter itself
 * (no FP32 copy): the update is computed in FP32 from the stored value and
 * rounded stochastically, element e of the tensor drawing its 16 random bits
 * as gs_project_bwd_adam does (seed sr_seed, t = step).
 * The GsAdamTensor array is read on the host; all its pointers are device. */
#define GS_ADAM_MAX_TENSORS 8
typedef struct {
    float* param;
    const float* grad;
    float* m;
    float* v;
    void* shadow;
    int64_t numel;
    int32_t row_width;
    int32_t shadow_dtype;
    float lr;
    uint32_t sr_seed;
} GsAdamTensor;
int32_t gs_adam(const GsAdamTensor* tensors, int32_t count, float beta1, float beta2,
                float eps, int32_t step, const uint8_t* row_mask, gs_stream_t stream);

/* ===========================================================================
 * Batched views: several views (cameras, resolutions, dilations) of one set of
 * Gaussians in one launch per stage. The view table is read on the host and
 * passed to the kernels by value; every pointer in it is a device buffer owned
 * by the caller, sized for that view as in the single-view calls. All views of
 * a batch use the same tile size.
 * =========================================================================== */
#define GS_MAX_VIEWS 16
typedef struct {
    GsCamera cam;
    GsDilation dil;
    float* splats;             /* n x 16 (gs_project)                         */
    int32_t* radii;            /* n                                            */
    int32_t* rects;            /* n x 4                                        */
    int32_t* tiles_touched;    /* n                                            */
    uint32_t* sorted_ids;      /* from gs_bin_sort of this view                */
    uint32_t* ranges;          /* binning tiles x 2                            */
    float* img;                /* h_ds x w_ds x 3                              */
    float* t_final;            /* h_ds x w_ds                                  */
    uint32_t* last;            /* h_ds x w_ds                                  */
    const void* target;        /* height x width x 3 (hr), of target_dtype     */
    float* dl_dimg;            /* h_ds x w_ds x 3                              */
    float* grad2d;             /* n x 12                                       */
    float* loss;               /* one float                                    */
    uint32_t* depth_keys;      /* n, nullable (gs_project's depth_keys)         */
    int32_t target_dtype;      /* GS_TARGET_F32 or GS_TARGET_U8                */
} GsView;

/* gs_project for every view of the table (one launch). */
int32_t gs_project_batch(int32_t n, int32_t sh_degree, int32_t sh_dtype,
                         const float* means, const float* log_scales, const float* quats,
                         const float* opacity_logits, const void* sh,
                         const GsView* views, int32_t nviews, gs_stream_t stream);

/* gs_tile_order over the blend tiles of all views, numbered view by view
 * (view v's tiles follow those of views 0..v-1): order gets sum_v tiles_v ids,
 * longest (binning tile) list first. This is the work queue of the batched
 * blend launches. */
int32_t gs_tile_order_batch(const GsView* views, int32_t nviews, uint32_t* order, gs_stream_t stream);

/* gs_tile_order_by_last_batch -- the launch order for the backward blend
 * (gs_render_bwd_batch, or gs_render_bwd with a one-view table), after the
 * forward: the blend tiles of all views, numbered as in gs_tile_order_batch,
 * longest-first by the largest `last` over each tile's pixels (the list
 * positions its backward replays), 8 buckets per power of two. With coarse
 * binning this ranks the blend tiles of one binning tile by their own work,
 * which the list length cannot. Input (device): each view's last
 * (h_ds x w_ds). Output (device): order (sum_v tiles_v). Above
 * 49152 tiles in all, the keys do not fit the sort's shared memory and the
 * list-length order of gs_tile_order_batch is written instead. Scheduling
 * only: the backward's results do not depend on it. */
int32_t gs_tile_order_by_last_batch(const GsView* views, int32_t nviews, uint32_t* order, gs_stream_t stream);

/* gs_render_fwd / gs_loss_l1 / gs_render_bwd for every view in one launch each;
 * the blend launches take the tiles of all views from one work queue
 * (tile_order, nullable = view by view). counts as in gs_render_fwd, summed
 * over views. gs_render_bwd_batch zeroes each view's grad2d first when
 * zero_grad2d != 0. gs_render_fwd_batch's flags (0, or GS_FWD_L1 and/or
 * GS_FWD_ZERO_GRAD2D, as gs_render_fwd_l1 does for one view): GS_FWD_L1 also
 * computes every view's L1 loss into its loss and dl_dimg from its target;
 * GS_FWD_ZERO_GRAD2D zeroes every view's grad2d. */
int32_t gs_render_fwd_batch(int32_t n, const GsView* views, int32_t nviews, const float* bg,
                            const uint32_t* tile_order, unsigned long long* counts,
                            int32_t pixels_per_thread, int32_t flags, gs_stream_t stream);
int32_t gs_loss_l1_batch(const GsView* views, int32_t nviews, gs_stream_t stream);
int32_t gs_render_bwd_batch(int32_t n, const GsView* views, int32_t nviews, const float* bg,
                            const uint32_t* tile_order, int32_t zero_grad2d,
                            int32_t pixels_per_thread, gs_stream_t stream);

/* gs_project_bwd_adam over a batch: for each Gaussian the gradient is summed
 * over the views (each view's projection backward from its own grad2d), the
 * densification statistics accumulate once per view the Gaussian is visible
 * in, and Adam is applied once with the summed gradient. Parameters, moments
 * and the SH storage cross HBM once per batch. */
int32_t gs_project_bwd_adam_batch(int32_t n, int32_t sh_degree, int32_t sh_dtype, const void* sh_store,
                                  const GsView* views, int32_t nviews, const GsAdamParams* adam,
                                  float* pos_acc, float* col_acc, int32_t* count,
                                  float* const* grads_out, gs_stream_t stream);

/* gs_project_bwd_adam_next -- gs_project_bwd_adam (one view, dense Adam:
 * adam->sparse must be 0) followed, in the same launch, by gs_project of the
 * updated parameters into the next training step's view: next->cam and
 * next->dil, outputs into next->splats (16-byte aligned), radii, rects
 * (16-byte aligned), tiles_touched and depth_keys (nullable), exactly as
 * gs_project(..., next->cam, next->dil, ...) would write them after this
 * call: the same formulas on the same stored values, so radii, rects, tile
 * counts, depth keys, centres, opacities and colours are equal, and the conic
 * equal up to FP32 rounding (the two kernels may contract its products into
 * FMAs differently); the parameters equal gs_project_bwd_adam's up to the
 * same rounding of the gradient arithmetic. The
 * next step then skips its projection: the parameters cross HBM once per step
 * instead of twice. next's output buffers may be the ones this call's
 * tiles_touched lives in (each Gaussian's count is read before it is
 * rewritten). Errors: as gs_project_bwd_adam, plus GS_ERR_ARG for sparse Adam
 * or a null or misaligned next buffer. */
int32_t gs_project_bwd_adam_next(int32_t n, int32_t sh_degree, int32_t sh_dtype, const void* sh_store,
                                 const GsCamera* cam, const GsDilation* dil, const int32_t* tiles_touched,
                                 const float* grad2d, const GsAdamParams* adam, float* pos_acc,
                                 float* col_acc, int32_t* count, float* const* grads_out,
                                 const GsView* next, gs_stream_t stream);

/* ===========================================================================
 * Densification and pruning under a Gaussian budget (Sec. 3.2, Sec. 3.3).
 * Run once per densification interval. The host reads the device counts the
 * selection calls write (num_selected, num_keep) to size the next arrays.
 * =========================================================================== */

/* Bytes of the workspace gs_densify_select and gs_prune_select need for n
 * Gaussians (device memory, caller-owned, any alignment). */
size_t gs_densify_workspace_size(int32_t n);

/* gs_densify_select -- position-appearance densification (Sec. 3.3) with the
 * budget cut. For every i < n with count[i] > 0, in FP32 with IEEE division:
 *   sp = pos_acc[i] / count[i];  sc = col_acc[i] / count[i]
 *   candidate  <=>  sp > tau_pos  or  (color_branch != 0 and sc > tau_color)
 *   score = max(sp / tau_pos, color_branch ? sc / tau_color : 0)
 * (the paper takes tau_color = 0.01 tau_pos and activates the colour branch
 * with probability 0.2; the caller draws it). When there are more than
 * max_new candidates, the max_new with the highest score are kept, equal
 * scores in index order. selected (device, >= min(n, max_new) entries)
 * receives the kept indices in ascending order, *num_selected (device) their
 * count. pos_acc, col_acc, count: device, n entries (gs_densify_stats). */
int32_t gs_densify_select(int32_t n, const float* pos_acc, const float* col_acc, const int32_t* count,
                          float tau_pos, float tau_color, int32_t color_branch, int32_t max_new,
                          void* workspace, size_t workspace_bytes, int32_t* selected,
                          int32_t* num_selected, gs_stream_t stream);

/* gs_prune_select -- indices (ascending, device, n entries) of the Gaussians
 * kept: opacity_logits[i] >= logit_min (the opacity sigmoid(logit) is at
 * least sigmoid(logit_min)) and, when log_scales (n x 3, nullable) is given,
 * max_k log_scales[i][k] <= log_scale_max. *num_keep (device): their count. */
int32_t gs_prune_select(int32_t n, const float* opacity_logits, float logit_min,
                        const float* log_scales, float log_scale_max, void* workspace,
                        size_t workspace_bytes, int32_t* keep, int32_t* num_keep,
                        gs_stream_t stream);

/* A row tensor: one row of row_bytes (a multiple of 4) per Gaussian, from
 * src to dst (distinct device buffers). role tells the growth what to do with
 * it; the gather copies every role but GS_ROW_ZERO. */
#define GS_MAX_ROW_TENSORS 24
#define GS_ROW_COPY 0        /* copied (opacity, SH, their BF16/FP16 copy, ...)   */
#define GS_ROW_MEANS 1       /* 3 floats: moved for split children                */
#define GS_ROW_LOG_SCALES 2  /* 3 floats: reduced by log(1.6) for split children  */
#define GS_ROW_QUATS 3       /* 4 floats (w,x,y,z), 16-byte aligned: copied       */
#define GS_ROW_STATE 4       /* optimizer moments: zero for new rows and split parents */
#define GS_ROW_ZERO 5        /* zeroed in every row (densification statistics)    */
typedef struct {
    const void* src;
    void* dst;
    int32_t row_bytes;
    int32_t role;
} GsRowTensor;

/* gs_gather_rows -- dst row i = src row index[i] for i < n_out (index: device
 * int32, e.g. gs_prune_select's keep list); GS_ROW_ZERO tensors are zeroed.
 * The tensor table is read on the host. */
int32_t gs_gather_rows(int32_t n_out, const int32_t* index, const GsRowTensor* tensors,
                       int32_t count, gs_stream_t stream);

/* gs_densify_grow -- clone / split of the m selected Gaussians (the 3DGS
 * baseline Sec. 3.3 follows), from n_old rows in src to n_old + m rows in dst:
 * rows < n_old are copied, row n_old + j is a copy of row selected[j]. A
 * selected Gaussian whose largest log-scale exceeds log_split_scale is split:
 * its two children sit at mean + R(q) diag(exp(log_scales)) z_k with the
 * standard normals z_k = noise[6 j + 3 k .. +3] (device, m x 2 x 3, drawn by
 * the caller), their log-scales reduced by log(1.6); child 0 replaces the
 * parent, child 1 is row n_old + j. GS_ROW_STATE rows of new rows and of split
 * parents are zero; GS_ROW_ZERO tensors are zero. Needs exactly one MEANS, one
 * LOG_SCALES and one QUATS tensor. selected: device, ascending or not. */
int32_t gs_densify_grow(int32_t n_old, int32_t m, const int32_t* selected, const float* noise,
                        float log_split_scale, const GsRowTensor* tensors, int32_t count,
                        gs_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* TURBOGS_H */
