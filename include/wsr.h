/*
 * wsr.h — C ABI of the GB300 (sm_103a) Weighted Sum Rendering library.
 *
 * Weighted Sum Rendering (WSR) renders a 3D Gaussian scene without sorting:
 * every pixel is the order-independent weighted sum of Eq. 7 of "Sort-free
 * Gaussian Splatting via Weighted Sum Rendering" (arXiv 2410.18931),
 *
 *     C = (c_B w_B + sum_i c_i a_i) / (w_B + sum_i a_i),
 *     a_i = u_i w(d_i) exp(-q_i / 2),      q_i <= 9 (3-sigma footprint),
 *
 * with the depth weights w(d) of Eqs. 8-10 and the view-dependent opacity
 * u_i of Eq. 11.  The hot path is four calls:
 *
 *     wsr_project     per-Gaussian projection (Sec. 3 Eqs. 3-5, Eq. 4, Eq. 11,
 *                     Eqs. 8-10) into a 48-byte render record per view
 *     wsr_bin         sort-free tile binning: per-tile count, prefix scan and
 *                     unordered scatter (Sec. 4.1, Fig. 2 without the sort)
 *     wsr_render_fwd  per-pixel accumulation of Eq. 7
 *     wsr_render_bwd  gradient of Eq. 7 and of the projection chain with
 *                     respect to every stored parameter
 *
 * Conventions for every call:
 *   - All data pointers are DEVICE pointers owned by the caller.  The library
 *     allocates no memory; scratch comes from a caller-provided workspace
 *     whose size wsr_workspace_size() returns (256-byte aligned).
 *   - Alignment: render records and gradient records (read and updated as
 *     16-byte vectors), the workspace and the parameter arrays 16-byte
 *     aligned; every other array to its element size.  A misaligned
 *     pointer is WSR_ERR_INVALID_ARG.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy stream).  All
 *     work is enqueued asynchronously on it; no call synchronises the stream
 *     except wsr_check() and wsr_bin_total().
 *   - Every call returns a wsr_status.  Argument errors are found on the host
 *     before anything is enqueued (WSR_ERR_INVALID_ARG / WSR_ERR_UNSUPPORTED).
 *     Errors found on the device (tile-list overflow) are recorded in the
 *     workspace and reported by wsr_check().  Launch failures return
 *     WSR_ERR_CUDA.  No call aborts, throws or exits.
 *   - Camera convention: world-to-camera rotation R (row-major) and
 *     translation T, camera axes x right, y down, z forward; pixel (x, y) has
 *     its centre at (x + 0.5, y + 0.5).
 */
#ifndef WSR_H
#define WSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WSR_OK = 0,
    WSR_ERR_INVALID_ARG = 1,  /* null pointer, bad size, bad enum, too-small workspace */
    WSR_ERR_CAPACITY = 2,     /* the tile list did not fit in list_capacity */
    WSR_ERR_CUDA = 3,         /* a CUDA launch or runtime call failed */
    WSR_ERR_TIMEOUT = 4,      /* reserved: no kernel of this library waits on another */
    WSR_ERR_UNSUPPORTED = 5   /* valid but unsupported combination (e.g. tile shape) */
} wsr_status;

/* Storage types of Gaussian parameter arrays. */
enum { WSR_F32 = 0, WSR_F16 = 1, WSR_BF16 = 2 };
/* Depth-weight functions: Eq. 8 (DIR), Eq. 9 (EXP), Eq. 10 (LC). */
enum { WSR_WEIGHT_DIR = 0, WSR_WEIGHT_EXP = 1, WSR_WEIGHT_LC = 2 };
/* Opacity: sigmoid of a logit (Eq. 3's t_i) or view-dependent SH (Eq. 11). */
enum { WSR_OPACITY_LOGIT = 0, WSR_OPACITY_SH = 1 };

#define WSR_MAX_VIEWS 32
#define WSR_RECORD_FLOATS 12      /* one render record: 48 bytes */
#define WSR_GRAD_RECORD_FLOATS 12 /* one 2D gradient record: 48 bytes (9 used) */
#define WSR_GRAD_RECORD_FLOATS_DET 32 /* one record in deterministic mode: 128 bytes */
#define WSR_DET_MAX_SEGMENT 8192  /* deterministic mode: most instances one tile may hold */
#define WSR_SCAN_ONE_BLOCK_TILES 32768  /* wsr_bin scans (and orders) up to this many tiles in one kernel */

/* Pinhole camera (passed by value through host memory). */
typedef struct {
    float R[9];          /* world -> camera rotation, row-major */
    float T[3];          /* world -> camera translation */
    float fx, fy;        /* focal lengths, pixels */
    float cx, cy;        /* principal point, pixels */
    int32_t width, height;
    float znear;         /* Gaussians with camera z <= znear are culled (App. C) */
} wsr_camera;

/*
 * Gaussian scene 𝒢 = {(p_i, t_i or H^alpha_i, q_i, s_i, H_i)} (Sec. 3).
 * K = (sh_degree + 1)^2.  All arrays are dense, row-major, device memory.
 *   means       [n, 3]  float32                    centres p_i
 *   log_scales  [n, 3]  dtype_scales_quats          log s_i  (s = exp(.))
 *   quats       [n, 4]  dtype_scales_quats          q_i = (w, x, y, z), any norm
 *   sh          [n, K, 3] dtype_sh                  colour SH H_i (Eq. 4)
 *   opacity     [n] logit (WSR_OPACITY_LOGIT) or [n, K] SH (WSR_OPACITY_SH),
 *               dtype_sh
 *   lc_v        [n] float32, the per-Gaussian v_i of Eq. 10 (required for LC,
 *               ignored otherwise, may then be NULL)
 * Reduced-precision storage: dtype_scales_quats in {WSR_F32, WSR_BF16},
 * dtype_sh in {WSR_F32, WSR_F16}.  Every array must be 16-byte aligned.
 */
typedef struct {
    int64_t n;
    int32_t sh_degree;           /* 0..3 */
    int32_t opacity_mode;        /* WSR_OPACITY_LOGIT or WSR_OPACITY_SH */
    int32_t dtype_scales_quats;
    int32_t dtype_sh;
    const float* means;
    const void* log_scales;
    const void* quats;
    const void* sh;
    const void* opacity;
    const float* lc_v;
} wsr_gaussians;

/*
 * Depth weight w(d) and background.  `params` points to 6 device floats:
 * [sigma, beta, w_B, c_B.r, c_B.g, c_B.b].  EXP (Eq. 9) uses sigma and beta,
 * LC (Eq. 10) uses sigma (and the per-Gaussian v_i), DIR (Eq. 8) neither.
 * Keeping them on the device lets them change between graph replays.
 */
typedef struct {
    int32_t kind;                /* WSR_WEIGHT_* */
    const float* params;         /* device [6] */
} wsr_weight;

/* Work schedule of the render kernels. */
enum {
    WSR_SCHEDULE_TILE_BLOCKS = 0,  /* one thread block per tile */
    WSR_SCHEDULE_PERSISTENT = 1    /* one block per SM slot, tiles taken heaviest first */
};

/*
 * Tile shape for binning and rendering (supported: 16x16, 8x8, 32x8, 16x8),
 * the render schedule and the backward's Gaussians per block.  With
 * WSR_SCHEDULE_PERSISTENT, wsr_bin also orders the tiles by decreasing
 * instance count (a bucketed longest-first order kept in the workspace) and
 * the render calls launch one block per resident slot (wsr_render_fwd: at
 * most 16 warps per SM, the forward's fastest grid) that takes tiles from
 * that order through a counter in the workspace; the same workspace and tiles
 * must then be passed to wsr_bin and the renderers.  `chunk` is how many of a
 * tile's Gaussians one block of wsr_render_bwd takes at a time: 0 for the
 * default 128 (blocks of 256 threads), 64 (blocks of 128 threads, twice as
 * many resident), 256 or 512 (blocks of 256 threads, fewer barriers per
 * Gaussian); other values return WSR_ERR_UNSUPPORTED.  It changes the schedule only, not the result
 * beyond rounding order.
 *
 * `deterministic` = 1 makes every result bitwise reproducible from run to run
 * for the same inputs and tiles (0, the default, lets the order of atomics
 * decide the last bits):
 *   - wsr_bin sorts each tile's list by record index after the scatter (a tile
 *     with more than WSR_DET_MAX_SEGMENT instances leaves WSR_ERR_UNSUPPORTED
 *     in the workspace for wsr_check);
 *   - wsr_render_bwd_tiles first takes the largest pixel term of the image
 *     (G/D and (G.C)/D), then walks the tiles once, adding each record term
 *     as 64-bit fixed point (exact integer sums) in units that a bound of the
 *     Gaussian's own fixes (the sum of its absolute pixel terms over the
 *     whole footprint: footprint pixels x that largest term x the record's
 *     factors); grad_records then holds WSR_GRAD_RECORD_FLOATS_DET floats per
 *     record (9 int64 sums, the 9 bounds as float bits), and the background
 *     terms are reduced in tile order;
 *   - wsr_project_bwd, given the same tiles, reads those records and reduces
 *     its sigma/beta terms in a fixed order.
 * The backward then takes about 1.4 times as long.
 */
typedef struct {
    int32_t tile_w, tile_h;
    int32_t schedule;            /* WSR_SCHEDULE_* */
    int32_t chunk;               /* Gaussians per backward block: 0 (128), 64, 256, 512 */
    int32_t deterministic;       /* 0, or 1: bitwise-reproducible results */
} wsr_tiles;

/*
 * Gradient outputs (device float32, OVERWRITTEN by wsr_render_bwd), shaped
 * like the parameters: means [n,3], log_scales [n,3], quats [n,4],
 * sh [n,K,3], opacity [n] or [n,K], lc_v [n], weight_params [6] (sigma, beta,
 * w_B, c_B).  Gradients over several views are summed.  A NULL member skips
 * writing that output (the others are still computed).
 */
typedef struct {
    float* means;
    float* log_scales;
    float* quats;
    float* sh;
    float* opacity;
    float* lc_v;
    float* weight_params;
} wsr_grads;

/* Human-readable message of a status code (static string). */
const char* wsr_status_string(wsr_status s);

/* Library version, as major * 10000 + minor * 100 + patch. */
int32_t wsr_version(void);

/* Total tiles over all views for the tile shape (0 on invalid arguments). */
int64_t wsr_num_tiles(const wsr_camera* cams, int32_t n_cams, const wsr_tiles* tiles);

/* Total pixels over all views (the rows of out_rgb / out_den). */
int64_t wsr_num_pixels(const wsr_camera* cams, int32_t n_cams);

/*
 * Workspace bytes needed by wsr_bin / wsr_render_fwd / wsr_render_bwd for
 * these views and tile shape (the same workspace serves all of them; it may
 * be reused across calls on the same stream).  0 on invalid arguments.
 */
size_t wsr_workspace_size(const wsr_camera* cams, int32_t n_cams, const wsr_tiles* tiles);

/*
 * wsr_project — projection of every Gaussian into every view.
 * Sec. 3 Eq. 3 (Sigma = R S S^t R^t), Eq. 5 (Sigma_2D = J W Sigma W^t J^t,
 * plus the 3DGS 0.3-pixel dilation and Jacobian clamp), Eq. 4 (SH colour,
 * RGB = max(0, Y.H + 0.5)), Eq. 11 / Eq. 3 (opacity), Eqs. 8-10 (weight),
 * App. C (near-plane culling).
 *   records  [n_cams, n, 12] float32 output.  Per Gaussian and view:
 *            {mu_x, mu_y, qs, qw, qd, u w, c_r u w, c_g u w, c_b u w,
 *             rx, ry, depth}, where the Mahalanobis distance of a pixel
 *            offset (dx, dy) is written as a sum of squares,
 *              q log2(e)/2 = (qs dy + qw dx)^2 + qd dx^2,
 *            i.e. with Sigma_2D = [[a, b], [b, c]] and det its determinant:
 *            qs = sqrt(k a / det), qw = -(b / a) qs, qd = k / a, k = log2(e)/2
 *            (no cancellation for needle-like footprints), and rx, ry are the
 *            3-sigma half extents in pixels.  rx < 0 marks a culled Gaussian.
 */
wsr_status wsr_project(const wsr_gaussians* g, const wsr_camera* cams, int32_t n_cams,
                       const wsr_weight* w, float* records, void* stream);

/*
 * wsr_bin — sort-free tile binning (Sec. 4.1: tiles and per-tile replication
 * as in 3DGS, with the depth sort removed because Eq. 7 is order-independent).
 *   records        [n_cams, n, 12] from wsr_project
 *   tile_offsets   [num_tiles + 1] uint32 output: exclusive prefix sum of the
 *                  per-tile counts; tile t owns tile_list[offsets[t], offsets[t+1])
 *   tile_list      [list_capacity] uint32 output: record indices (view * n + i),
 *                  in no particular order within a tile
 *   list_capacity  entries available in tile_list
 * The total instance count is tile_offsets[num_tiles].  If it exceeds
 * list_capacity, nothing is written past the end, every offset is clamped to
 * list_capacity (so the render calls stay in bounds, with incomplete tiles),
 * the workspace records WSR_ERR_CAPACITY (see wsr_check) and the true total
 * (wsr_bin_total); the caller grows the list and runs the frame again.
 *   total_dev      [1] uint64 device output, may be NULL: the true instance
 *                  count of this call, written on `stream` after the scan (a
 *                  captured graph learns from it how far to grow the list
 *                  without a host read inside the graph)
 */
wsr_status wsr_bin(const float* records, int64_t n, const wsr_camera* cams, int32_t n_cams,
                   const wsr_tiles* tiles, uint32_t* tile_offsets, uint32_t* tile_list,
                   uint64_t list_capacity, uint64_t* total_dev, void* workspace, size_t workspace_bytes,
                   void* stream);

/*
 * wsr_bin_count — first half of wsr_bin (count + scan only), for callers that
 * size tile_list exactly: read the total with wsr_bin_total afterwards.
 * tile_offsets is written unclamped.
 */
wsr_status wsr_bin_count(const float* records, int64_t n, const wsr_camera* cams, int32_t n_cams,
                         const wsr_tiles* tiles, uint32_t* tile_offsets, void* workspace,
                         size_t workspace_bytes, void* stream);

/*
 * Synchronises `stream` and returns in *total the number of tile instances
 * (Gaussian-tile pairs) counted by the last wsr_bin / wsr_bin_count that used
 * this workspace, before any clamping to the list capacity.
 */
wsr_status wsr_bin_total(const void* workspace, size_t workspace_bytes, uint64_t* total, void* stream);

/*
 * wsr_render_fwd — Eq. 7 per pixel, one thread block per tile.
 *   out_rgb  [num_pixels, 3] float32 output, views concatenated in order, each
 *            view row-major (y * width + x)
 *   out_den  [num_pixels] float32 output: the full denominator w_B + sum a_i
 *            (kept for the backward pass)
 */
wsr_status wsr_render_fwd(const float* records, int64_t n, const uint32_t* tile_offsets,
                          const uint32_t* tile_list, const wsr_camera* cams, int32_t n_cams,
                          const wsr_tiles* tiles, const wsr_weight* w, float* out_rgb,
                          float* out_den, void* workspace, size_t workspace_bytes, void* stream);

/*
 * wsr_render_bwd — gradient of a scalar loss L through Eq. 7 and the
 * projection, given grad_rgb = dL/dC.  Two stages:
 *   (1) per tile, recompute every (pixel, Gaussian) term from the records and
 *       reduce into grad_records [n_cams, n, 12] float32 (overwritten):
 *       {Sr, Sx, Srr, Srx, Sxx, dL/d(uw) at fixed c uw, dL/d(c uw) (3),
 *        0, 0, 0}, where, over the Gaussian's pixels with q <= 9 and with
 *       gq = dL/dq' (q' = q log2(e)/2 = r^2 + qd dx^2, r = qs dy + qw dx,
 *       dx, dy = pixel centre - mu, qs, qw, qd as in the render record):
 *       Sr = sum gq r, Sx = sum gq dx, Srr = sum gq r^2, Srx = sum gq r dx,
 *       Sxx = sum gq dx^2.  Then dL/dmu_x = -2 (qw Sr + qd Sx),
 *       dL/dmu_y = -2 qs Sr and, with w = (qw, qs), e1 = (1, 0),
 *       dL/dSigma_2D = -(Srr w w^t + qd Srx (w e1^t + e1 w^t)
 *                        + qd^2 Sxx e1 e1^t) / (log2(e)/2);
 *       plus the background terms dL/dw_B, dL/dc_B;
 *   (2) per Gaussian, chain grad_records back to the stored parameters.
 * `g` must be the scene given to wsr_project; out_rgb / out_den come from
 * wsr_render_fwd on the same records.
 */
wsr_status wsr_render_bwd(const wsr_gaussians* g, const float* records, const uint32_t* tile_offsets,
                          const uint32_t* tile_list, const wsr_camera* cams, int32_t n_cams,
                          const wsr_tiles* tiles, const wsr_weight* w, const float* out_rgb,
                          const float* out_den, const float* grad_rgb, float* grad_records,
                          const wsr_grads* grads, void* workspace, size_t workspace_bytes,
                          void* stream);

/*
 * The two stages of wsr_render_bwd as separate calls (same arguments and
 * semantics; wsr_render_bwd is exactly wsr_render_bwd_tiles followed by
 * wsr_project_bwd).  wsr_render_bwd_tiles overwrites grad_records and
 * accumulates the background terms in the workspace; wsr_project_bwd adds the
 * sigma/beta terms there and writes grads (weight_params included).  `tiles`
 * of wsr_project_bwd may be NULL; only its `deterministic` field is read, and
 * it must match the wsr_render_bwd_tiles call that wrote grad_records.
 */
wsr_status wsr_render_bwd_tiles(const float* records, int64_t n, const uint32_t* tile_offsets,
                                const uint32_t* tile_list, const wsr_camera* cams, int32_t n_cams,
                                const wsr_tiles* tiles, const wsr_weight* w, const float* out_rgb,
                                const float* out_den, const float* grad_rgb, float* grad_records,
                                void* workspace, size_t workspace_bytes, void* stream);
wsr_status wsr_project_bwd(const wsr_gaussians* g, const wsr_camera* cams, int32_t n_cams,
                           const wsr_tiles* tiles, const wsr_weight* w, const float* grad_records,
                           const wsr_grads* grads, void* workspace, size_t workspace_bytes, void* stream);

/*
 * wsr_loss_l1 — mean absolute error against a target and its gradient
 * (the L1 part of the 3DGS loss of Sec. 4.4, used to drive the backward).
 *   loss_out [1] float32 (overwritten), grad_rgb [num_pixels * 3] (overwritten);
 *   rgb, target and grad_rgb 16-byte aligned (WSR_ERR_INVALID_ARG otherwise)
 */
wsr_status wsr_loss_l1(const float* rgb, const float* target, int64_t count, float* loss_out,
                       float* grad_rgb, void* stream);

/*
 * wsr_loss_3dgs — the rendering loss the paper trains with (Sec. 4.4:
 * the 3DGS loss, L1 plus D-SSIM weighted 0.2) and its
 * gradient with respect to the rendered pixels:
 *     L = (1 - lambda) * L1 + lambda * (1 - SSIM)
 *   L1    mean |rgb - target| over every pixel and channel of every view;
 *   SSIM  mean of the SSIM map (Wang et al. 2004) over the same elements,
 *         each view and channel filtered on its own with the 11 x 11 Gaussian
 *         window of standard deviation 1.5 (normalised to sum 1), pixels
 *         outside the image taken as zero, C1 = 0.01^2, C2 = 0.03^2.
 *   rgb, target  [num_pixels * 3] float32 device, the views concatenated as
 *                wsr_render_fwd writes them (row-major per view, RGB
 *                interleaved); 4-byte aligned
 *   cams, n_cams the views (only width and height are used)
 *   lambda       weight of the D-SSIM term, in [0, 1] (the paper: 0.2)
 *   loss_out     [3] float32 device, overwritten: {L, L1, SSIM}
 *   grad_rgb     [num_pixels * 3] float32 device, overwritten: dL/drgb, with
 *                d|d|/dd taken as 0 at d = 0
 * Summation order across tiles is not fixed (float atomics), so L varies in
 * the last bits between runs; grad_rgb does not.
 * Errors: WSR_ERR_INVALID_ARG (null pointer, bad cameras, lambda outside
 * [0, 1]) before anything is enqueued; WSR_ERR_CUDA on a launch failure.
 */
wsr_status wsr_loss_3dgs(const float* rgb, const float* target, const wsr_camera* cams, int32_t n_cams,
                         float lambda, float* loss_out, float* grad_rgb, void* stream);

/*
 * wsr_adam_step — one Adam update (Kingma & Ba 2015) of a flat float32
 * parameter buffer, the optimiser the paper's PyTorch training uses (Sec.
 * 4.4, as 3DGS does):
 *     m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
 *     p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
 * with t the step number kept in the device state (advanced by this call).
 *   params, grads, exp_avg, exp_avg_sq  flat float32 device buffers, 16-byte
 *       aligned; exp_avg and exp_avg_sq start at zero (caller-owned)
 *   groups[n_groups] (host, n_groups <= WSR_ADAM_MAX_GROUPS): element ranges
 *       updated, each with its learning rate; offset a multiple of 4, count
 *       below 2^32; ranges must not overlap.  Elements outside every group are
 *       not touched.  Element e of a group (0-based) uses lr, or lr_tail when
 *       period > 0 and e % period >= head (e.g. the higher SH bands of
 *       [n, K, 3] coefficients: period 3K, head 3).
 *   hp (host): beta1, beta2 in [0, 1), eps >= 0
 *   state  device wsr_adam_state (16 bytes, 4-byte aligned), zeroed by the
 *       caller before the first step; step counts the updates made, skipped
 *       the calls that made none
 *   guard_workspace, guard_bytes  optional (NULL, 0): a wsr_bin / render
 *       workspace; when it holds a device-side error (e.g. WSR_ERR_CAPACITY
 *       from a wsr_bin earlier on the stream) the call changes nothing but
 *       state->skipped.  Everything is read on the device, so a captured
 *       graph replays correct steps.
 * Errors: WSR_ERR_INVALID_ARG before anything is enqueued; WSR_ERR_CUDA.
 */
#define WSR_ADAM_MAX_GROUPS 16
typedef struct {
    int64_t offset;
    int64_t count;
    float lr;
    float lr_tail;
    int32_t period;
    int32_t head;
} wsr_adam_group;

typedef struct {
    double beta1;
    double beta2;
    double eps;
} wsr_adam_hparams;

typedef struct {
    int32_t step;     /* updates made so far */
    float c1;         /* 1 / (1 - beta1^step) */
    float c2;         /* 1 / sqrt(1 - beta2^step) */
    int32_t skipped;  /* calls that updated nothing (guard error) */
} wsr_adam_state;

wsr_status wsr_adam_step(float* params, const float* grads, float* exp_avg, float* exp_avg_sq,
                         const wsr_adam_group* groups, int32_t n_groups, const wsr_adam_hparams* hp,
                         wsr_adam_state* state, const void* guard_workspace, size_t guard_bytes,
                         void* stream);

/*
 * wsr_bin_static — wsr_bin for callers that cannot allocate device memory.
 *
 * Some callers cannot call cudaMalloc at all once they are running: a frame
 * loop inside a host application that owns the GPU's memory budget and
 * forbids device allocations after start-up (an allocation can synchronise
 * the whole device and stall the frame), or a plug-in that is handed only its
 * input and output buffers by its host.  This entry point needs no workspace:
 * its scratch (per-tile counters, scan partial sums, a small header) lives in
 * one fixed device array inside this library, WSR_BIN_STATIC_BYTES =
 * 270,848 bytes (264.5 KiB), which every GPU that loads the library holds
 * until the process exits.  The paper has no counterpart; this is an
 * integration entry point, not part of the method.
 *
 * Arguments and results are those of wsr_bin, except:
 *   - there is no workspace: at most WSR_BIN_STATIC_MAX_TILES tiles over all
 *     views, and only the per-tile schedule (WSR_SCHEDULE_TILE_BLOCKS); other
 *     calls return WSR_ERR_UNSUPPORTED before anything is enqueued;
 *   - total_dev [1] uint64 device output (may be NULL): the true number of tile
 *     instances.  When it exceeds list_capacity the list is incomplete and the
 *     offsets are clamped to list_capacity, as in wsr_bin;
 *   - status_dev [1] int32 device output (may be NULL): the device-side status
 *     of this call, written on `stream` after its last kernel: WSR_OK,
 *     WSR_ERR_CAPACITY (the list was too small: see total_dev), or, in the
 *     deterministic mode, WSR_ERR_UNSUPPORTED (a tile holds more than
 *     WSR_DET_MAX_SEGMENT instances and its list was left unsorted).  It is
 *     the only place such errors surface, since wsr_check reads a workspace.
 * The array's device address is looked up (cudaGetSymbolAddress, which
 * allocates nothing) on every call made outside stream capture, with the
 * calling thread's current device; a call inside a capture reuses the address
 * the last call outside capture found on that device, so make one call on a
 * device before capturing it (and again after a cudaDeviceReset); a first
 * call inside a capture returns WSR_ERR_UNSUPPORTED.  Every call shares the
 * one array, and the array keeps the last call's contents (each call clears
 * what it needs cleared): calls that overlap on the GPU (on different
 * streams, or from different threads) race on it.  The call allocates
 * nothing: no cudaMalloc, no cudaFree, no allocating library routine.
 */
#define WSR_BIN_STATIC_MAX_TILES 65536
#define WSR_BIN_STATIC_BYTES 270848
wsr_status wsr_bin_static(const float* records, int64_t n, const wsr_camera* cams, int32_t n_cams,
                          const wsr_tiles* tiles, uint32_t* tile_offsets, uint32_t* tile_list,
                          uint64_t list_capacity, uint64_t* total_dev, int32_t* status_dev, void* stream);

/*
 * wsr_count_pairs — diagnostic: the work of the render kernels over all views,
 * written to count_dev [3] (device uint64, overwritten, 8-byte aligned):
 *   [0] (pixel, Gaussian) pairs with q <= 9, i.e. the terms of the sums of
 *       Eq. 7 (the algorithmic work of both render kernels);
 *   [1] (pixel, Gaussian) slots wsr_render_fwd evaluates: for each Gaussian of
 *       a tile, the pixels of every warp whose region of the tile its footprint
 *       reaches (the forward tests q at each of them);
 *   [2] (pixel, Gaussian) slots wsr_render_bwd evaluates: for each Gaussian
 *       of a tile, the rows from its first span to its last, each of tile
 *       width columns, or of half the tile width when none of its row spans
 *       is longer than that.
 * Arguments as for wsr_render_fwd.  Not part of a timed step.
 */
wsr_status wsr_count_pairs(const float* records, int64_t n, const uint32_t* tile_offsets,
                           const uint32_t* tile_list, const wsr_camera* cams, int32_t n_cams,
                           const wsr_tiles* tiles, uint64_t* count_dev, void* stream);

/*
 * wsr_check — synchronises `stream` and returns the first device-side error
 * recorded in the workspace (WSR_OK if none), then clears it.
 */
wsr_status wsr_check(void* workspace, size_t workspace_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* WSR_H */
