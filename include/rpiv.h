/*
 * rpiv.h - C ABI of librpiv, a GB300 (sm_103a) implementation of the
 * correction hot path of RapidPIV (Bollt, Foxman, Gharib, arXiv 2504.17987).
 *
 * What the library computes (paper Sec. 2, "RapidPIV"): for an image pair
 * (A, B) and a displacement predictor, frame B is warped by the predictor
 * (bilinear image deformation), each interrogation window of A is correlated
 * against the warped B with the zero-normalised correlation coefficient over
 * a +-r integer search, the integer peak is refined by a three-point Gaussian
 * fit per axis, the universal outlier detector (normalised median test,
 * threshold 2, regulariser 0.1 px in Sec. 3.1/3.2) flags outliers and replaces
 * them by the median of their non-outlier neighbours, and vorticity is derived
 * from the final field.  The paper obtains the predictor from a fixed-function
 * optical-flow engine; here a coarse-to-fine correlation pyramid (2x2 box
 * levels) computed by the same kernels stands in for it, or the caller
 * supplies one (e.g. the previous field of a camera stream).  r = 0 is the
 * paper's fixed 5-point stencil centred on the predicted displacement.
 *
 * Conventions for every entry point
 *   - Image and field pointers are DEVICE pointers owned by the caller unless
 *     stated; they must stay valid until the work enqueued on `cuda_stream`
 *     has completed.  The handle owns only its workspace, streams, events and
 *     captured CUDA graphs.
 *   - Images are single-channel, row-major, `pitch_bytes` between rows
 *     (pitch_bytes >= width * bytes per pixel); uint8 or uint16 (12-bit data
 *     is stored LSB-aligned, 0..4095).  x = column, y = row (downwards).
 *   - Vector grids of window w and step s = w (1 - overlap) have
 *     nx = floor((W - w)/s) + 1 columns and ny rows; node (i, j) sits at the
 *     window centre (i s + (w-1)/2, j s + (w-1)/2); arrays are ny x nx
 *     row-major float32 (u, v in px/frame, vorticity in 1/frame), the mask is
 *     uint8 (1 = passed the outlier test, 0 = flagged/replaced or invalid).
 *   - Work is enqueued asynchronously on `cuda_stream` (a cudaStream_t; NULL
 *     = the legacy default stream).  Nothing synchronises except
 *     rpiv_destroy.  Calls on one handle must not run concurrently from
 *     several host threads; the handle orders its own launches so that calls
 *     on different streams do not overlap on the device.
 *   - Nothing throws across the ABI.  Every call returns an rpiv_status;
 *     rpiv_last_error() gives a human-readable message for the calling thread.
 */
#ifndef RPIV_H
#define RPIV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RPIV_MAX_PASSES 4
#define RPIV_MAX_BATCH 64
#define RPIV_MAX_RADIUS 16
#define RPIV_MAX_LEVELS 4

typedef enum {
    RPIV_OK = 0,
    RPIV_ERR_INVALID_ARG = 1, /* a null pointer, a size or parameter out of range */
    RPIV_ERR_UNSUPPORTED = 2, /* valid request this build does not implement     */
    RPIV_ERR_OOM = 3,         /* device or pinned host allocation failed         */
    RPIV_ERR_CUDA = 4,        /* a CUDA runtime call failed (message has detail) */
    RPIV_ERR_TIMEOUT = 5,     /* rpiv_wait gave up before the work completed      */
    RPIV_ERR_BUSY = 6,        /* reserved                                        */
    RPIV_ERR_NO_DEVICE = 7    /* no usable CUDA device                           */
} rpiv_status;

typedef enum { RPIV_U8 = 1, RPIV_U16 = 2, RPIV_F32 = 3 } rpiv_pixfmt;

/* Arithmetic of the correlation plane.  The argmax is taken on this plane;
 * the 5-point stencil for the Gaussian fit is always recomputed in FP32.  */
typedef enum { RPIV_FP32 = 0, RPIV_BF16 = 1, RPIV_FP16 = 2 } rpiv_precision;

/* Image deformation: frame B only (B'(x) = B(x + d(x)), default) or central
 * (A'(x) = A(x - d/2), B'(x) = B(x + d/2), the paper's "central difference"). */
typedef enum { RPIV_DEFORM_B = 0, RPIV_DEFORM_CENTRAL = 1 } rpiv_deform;

typedef struct {
    int width, height;          /* image size, px                                  */
    rpiv_pixfmt fmt;            /* RPIV_U8, RPIV_U16, or RPIV_F32 (pre-processed)  */
    int bit_depth;              /* 8, 12 or 16 (informational; no rescaling)        */
    int n_passes;               /* full-resolution passes, 1..RPIV_MAX_PASSES       */
    int window[RPIV_MAX_PASSES];     /* even, 8..128, in pass order                 */
    float overlap[RPIV_MAX_PASSES];  /* [0, 1); w (1 - overlap) must be an integer  */
    int search_radius[RPIV_MAX_PASSES]; /* 0..RPIV_MAX_RADIUS                       */
    int predictor_levels;       /* coarse-to-fine pyramid levels (0 = zero or caller
                                   predictor); each level runs a pass with
                                   window[0], overlap[0], search_radius[0]          */
    float uod_threshold;        /* normalised-median threshold (paper: 2)          */
    float uod_eps;              /* regulariser, px (paper: 0.1)                     */
    int replace_outliers;       /* 1: replace by neighbour median; 0: flag only    */
    rpiv_precision precision;   /* correlation-plane arithmetic                    */
    rpiv_deform deform_mode;    /* RPIV_DEFORM_B (default) or RPIV_DEFORM_CENTRAL   */
    int max_batch;              /* 1..RPIV_MAX_BATCH pairs per rpiv_process_batch   */
    int host_frames;            /* 0: img_a / img_b of rpiv_process_batch and
                                   rpiv_process_pair are device memory; 1: they are
                                   page-locked host memory (cudaHostAlloc,
                                   cudaMallocHost), which every launch sequence
                                   reads once into the handle's workspace with one
                                   upload kernel (part of the captured graph), so
                                   that no copy call is made per image           */
} rpiv_config;

typedef struct rpiv_handle rpiv_handle;

/* Fills *cfg with the paper's settings for a 1 MP 8-bit pair: 16 px windows,
 * 50 % overlap (Sec. 3.1, 4.1), UOD threshold 2 / 0.1 px, r = 1, FP32,
 * frame-B deformation, no pyramid, max_batch 1.                              */
rpiv_status rpiv_config_default(rpiv_config *cfg);

/* Host-only validation of a configuration (no device access).  On success
 * writes the final-pass grid size.  Rejects: null pointers, image smaller than
 * window + 2 (radius + 1) at any level, odd or out-of-range windows, overlap
 * outside [0, 1) or a non-integer step, radius outside [0, 16], more than
 * 4 passes or levels, batch outside [1, 64], unknown enums.                  */
rpiv_status rpiv_validate_config(const rpiv_config *cfg, int *nx, int *ny);

/* Creates a handle on CUDA device `device`: validates cfg, allocates the
 * workspace for cfg->max_batch pairs (pyramid levels and per-stage fields)
 * and a pinned host ring for per-call pointer tables.  *out is set only on
 * RPIV_OK.  Errors: INVALID_ARG, NO_DEVICE, OOM, CUDA.                       */
rpiv_status rpiv_create(const rpiv_config *cfg, int device, rpiv_handle **out);

/* Final-pass grid size of a handle.                                          */
rpiv_status rpiv_grid_shape(const rpiv_handle *h, int *nx, int *ny);

/* Device bytes the handle holds (workspace), for admission control.         */
rpiv_status rpiv_workspace_bytes(const rpiv_handle *h, size_t *bytes);

/* One image pair through the whole schedule (pyramid or caller predictor,
 * every pass with deformation, correlation, peak, Gaussian fit and outlier
 * test, vorticity).
 *   img_a, img_b   device images, fmt of the config, pitch_bytes apart rows.
 *   pred_u, pred_v nullable device arrays on the FINAL-pass grid: when given
 *                  they replace the pyramid as the predictor of pass 1
 *                  (interpolated onto its grid).  Both or neither.
 *   u, v, vort     device float arrays, ny x nx of the final pass.
 *   mask           device uint8 array, ny x nx.  vort and mask may be NULL.
 * Errors: INVALID_ARG (nulls, pitch too small), CUDA.                        */
rpiv_status rpiv_process_pair(rpiv_handle *h, const void *img_a, const void *img_b, size_t pitch_bytes,
                              const float *pred_u, const float *pred_v, float *u, float *v, float *vort,
                              uint8_t *mask, void *cuda_stream);

/* n pairs of the handle's size and format in one launch sequence (pairs are
 * independent; the batch index only selects data).  Every pointer argument
 * is a HOST array of n device pointers; pred_u/pred_v may be NULL (no pair
 * has a predictor) or hold NULL entries (that pair uses the pyramid), vort
 * and mask may be NULL or hold NULL entries.  Launch sequences are captured
 * once per (n, predictor pattern) as a CUDA graph and replayed.
 * With cfg.host_frames = 1 the image pointers are page-locked host memory,
 * read by the device (checked per call: RPIV_ERR_INVALID_ARG otherwise).
 * Errors: INVALID_ARG (n outside [1, max_batch], nulls), CUDA.               */
rpiv_status rpiv_process_batch(rpiv_handle *h, int n, const void *const *img_a, const void *const *img_b,
                               size_t pitch_bytes, const float *const *pred_u, const float *const *pred_v,
                               float *const *u, float *const *v, float *const *vort, uint8_t *const *mask,
                               void *cuda_stream);

/* Score S = sum over the windows of pass 1's grid (window[0], overlap[0]) of
 * the zero-shift correlation coefficient between A and B warped by the field
 * (u, v) on that grid (frame-B deformation), and its adjoint
 *     grad_u = grad_score * dS/du,  grad_v = grad_score * dS/dv,
 * through the bilinear image interpolation and the bilinear field-to-pixel
 * weights (deformed windows are recomputed, not stored).  grad_u/grad_v may
 * both be NULL (score only); score_out (device float) may be NULL.  The
 * gradient is accumulated deterministically (no floating-point atomics).
 * Errors: INVALID_ARG, CUDA.                                                 */
rpiv_status rpiv_backward(rpiv_handle *h, const void *img_a, const void *img_b, size_t pitch_bytes,
                          const float *u, const float *v, float grad_score, float *grad_u, float *grad_v,
                          float *score_out, void *cuda_stream);

/* Gradient-ascent refinement of the field by the score of rpiv_backward (the
 * differentiation pattern applied to the paper's correction, Sec. 2: the
 * correlation coefficient of the warped pair is raised directly).  The step
 * rule: g0 = dS/d(u, v) at the start; step k moves along the current
 * gradient by eta_k = eta0 * 0.5^k / max|g0|; a step is kept only if S
 * increases, otherwise eta is halved and the step retried, at most
 * `halvings` times (the field stays where it was if every try fails).
 *   u, v     device float arrays on pass 1's grid (window[0], overlap[0]),
 *            read as the start and overwritten with the result.
 *   hist     HOST float array of steps + 1 scores (the start, then after each
 *            step), or NULL.
 * Every score is read back to decide the step, so the call synchronises
 * cuda_stream once per evaluation; it returns when the result is in u, v.
 * Work buffers are owned by the handle (allocated on first use).
 * Errors: INVALID_ARG (nulls, steps < 0, halvings < 0, eta0 <= 0), OOM, CUDA. */
rpiv_status rpiv_refine(rpiv_handle *h, const void *img_a, const void *img_b, size_t pitch_bytes, float *u, float *v,
                        int steps, float eta0, int halvings, float *hist, void *cuda_stream);

/* Blocks until the handle's enqueued work has finished, polling for at most
 * timeout_ms milliseconds (host watchdog).  RPIV_ERR_TIMEOUT if it has not.  */
rpiv_status rpiv_wait(rpiv_handle *h, int timeout_ms);

/* Stage tracing.  While enabled, rpiv_process_batch/rpiv_process_pair run
 * their launch sequence eagerly (no graph replay) and bracket every kernel
 * launch with CUDA events on the caller's stream.  rpiv_trace_read
 * synchronises the handle's work and returns one record per traced stage
 * (aggregated over calls since the last read, then cleared): name (e.g.
 * "pass/p2" for full-resolution pass 2, "pass/L1" for pyramid level 1,
 * "uod/p2", "interp/p2", "down/L1", "vort"), launches, total milliseconds,
 * and the stage geometry (image size, window, step, radius, grid, pairs per
 * launch) from which throughput is derived.  cap = capacity of out; *n = number
 * of records (may exceed cap; only cap are written).                         */
typedef struct {
    char name[24];
    int launches;
    float total_ms;
    int width, height, window, step, radius, nx, ny, pairs;
} rpiv_trace_record;

rpiv_status rpiv_trace_enable(rpiv_handle *h, int enable);
rpiv_status rpiv_trace_read(rpiv_handle *h, rpiv_trace_record *out, int cap, int *n);

/* Synchronises and frees everything the handle owns.  NULL is a no-op.      */
rpiv_status rpiv_destroy(rpiv_handle *h);

/* Message describing the last failing call on this thread ("" if none).
 * Valid until the next rpiv_* call on the same thread.                      */
const char *rpiv_last_error(void);

/* ------------------------------------------------------------------------
 * Stage entry points.  Each runs one step of the method on caller buffers
 * (device pointers, one pair, enqueued on cuda_stream) with the same kernels
 * the handle uses; they exist for stage-by-stage verification and for
 * callers composing their own schedules.  No handle and no allocation.
 * ---------------------------------------------------------------------- */

/* One correlation pass (paper Sec. 2: warp, correlation coefficient around
 * the peak, Gaussian sub-pixel fit) on the grid (w, step) of a W x H image.
 *   fmt        RPIV_U8, RPIV_U16, or 0 for float32 images (pyramid levels).
 *   pred_u/v   predictor on this grid's nodes (device, ny x nx float), or
 *              both NULL for a zero predictor.
 *   u, v       raw (pre-validation) result, ny x nx float.
 *   info       ny x nx int32: bit 0 valid window, bits 8..15 the integer peak
 *              ky and bits 16..23 kx as int8.
 *   scratch    caller-owned device buffer of at least the size returned by
 *              rpiv_stage_correlate_scratch_bytes (frame A as float, or
 *              the warped A' for the central warp, and the warped B'),
 *              256-byte aligned; it must not be in use by other work on the
 *              device.
 * Errors: INVALID_ARG (sizes, nulls, radius, small or unaligned scratch), UNSUPPORTED
 * (precision not built for this radius or step), CUDA.                      */
rpiv_status rpiv_stage_correlate(const void *img_a, const void *img_b, size_t pitch_bytes, int fmt, int width,
                                 int height, int window, int step, int radius, rpiv_precision precision,
                                 rpiv_deform deform_mode, const float *pred_u, const float *pred_v, float *u,
                                 float *v, int32_t *info, void *scratch, size_t scratch_bytes, void *cuda_stream);

/* Scratch bytes rpiv_stage_correlate needs for a W x H image and radius r:
 * two float images grown by M = r + 1 rounded up to a multiple of 4 pixels
 * per side, rows padded to a multiple of 32 floats (either warp mode).      */
rpiv_status rpiv_stage_correlate_scratch_bytes(int width, int height, int radius, rpiv_deform deform_mode,
                                               size_t *bytes);

/* Status of the stage calls (rpiv_stage_correlate and its allocation-free
 * form) queued on cuda_stream: waits for the stream with a host watchdog (at
 * most timeout_ms), then reads and clears the device's stage error word.  Its
 * kernels never wait without a limit: a copy or MMA completion that does not
 * arrive in time makes the tile report its windows invalid (info 0, the
 * predictor passed through) and sets the word.  The word is one per device,
 * shared by every stage call on it, so a status covers all of them since the
 * last read.  The correction step is the paper's (Sec. 2); the bounded waits
 * and this status are this library's.
 * Errors: TIMEOUT (the stream did not finish in time, or a bounded wait gave
 * up), CUDA.                                                                 */
rpiv_status rpiv_stage_status(void *cuda_stream, int timeout_ms);

/* The same pass as rpiv_stage_correlate for callers that cannot allocate
 * device memory when they run it (no cudaMalloc/cudaFree or allocating
 * library call happens inside).  This entry point has no counterpart in the
 * paper: it exists for callers such as a real-time acquisition loop that must
 * not enter the device allocator, or a host application that owns all device
 * memory through its own pool.  Its scratch is a 32 MiB array compiled into
 * the library, held by every GPU that loads the library until the process
 * exits; images needing more (rpiv_stage_correlate_scratch_bytes > 32 MiB,
 * about 2000 x 2000 pixels) are rejected with
 * RPIV_ERR_INVALID_ARG.  Every call looks up the array's device address
 * (cudaGetSymbolAddress, which allocates nothing once the library's module is
 * loaded on the device); the first call on a device loads it, and that is
 * when the array's memory is taken.  All calls
 * share the one array, so calls whose work overlaps on the GPU (different
 * streams, or other devices' calls are fine) race and must be serialised by
 * the caller; a later call on the same stream is ordered after the earlier.
 * Arguments, outputs and other errors as rpiv_stage_correlate.              */
rpiv_status rpiv_stage_correlate_noalloc(const void *img_a, const void *img_b, size_t pitch_bytes, int fmt,
                                         int width, int height, int window, int step, int radius,
                                         rpiv_precision precision, rpiv_deform deform_mode, const float *pred_u,
                                         const float *pred_v, float *u, float *v, int32_t *info,
                                         void *cuda_stream);

/* Normalised median test + median replacement (paper Sec. 2, Westerweel &
 * Scarano 2005) on an nx x ny field; info (nullable) marks invalid windows
 * (bit 0 clear) which are always treated as outliers.  Writes u_out, v_out
 * and mask (1 passed, 0 flagged).  Input and output arrays must not alias.  */
rpiv_status rpiv_stage_validate(const float *u, const float *v, const int32_t *info, int nx, int ny,
                                float threshold, float eps, int replace, float *u_out, float *v_out,
                                uint8_t *mask, void *cuda_stream);

/* Bilinear interpolation of a source grid field (snx x sny, window sw, step
 * ss) onto the nodes of a destination grid (dnx x dny, window dw, step ds)
 * whose image is `levels_up` pyramid levels finer (position map
 * x_src = (x_dst + 0.5)/2^L - 0.5, values times 2^L).  Outside the source node
 * hull the border value is extended.                                         */
rpiv_status rpiv_stage_interp(const float *su, const float *sv, int snx, int sny, int sw, int ss, float *du,
                              float *dv, int dnx, int dny, int dw, int ds, int levels_up, void *cuda_stream);

/* omega = dv/dx - du/dy on an nx x ny grid of step s: central differences
 * inside, one-sided on the border, zero along an axis with one node.        */
rpiv_status rpiv_stage_vorticity(const float *u, const float *v, int nx, int ny, int step, float *vort,
                                 void *cuda_stream);

/* 2x2 box average of a W x H image (fmt RPIV_U8, RPIV_U16 or 0 = float32,
 * pitch in bytes) into a floor(W/2) x floor(H/2) float32 image, row-major
 * without padding.                                                          */
rpiv_status rpiv_stage_downsample(const void *img, size_t pitch_bytes, int fmt, int width, int height,
                                  float *out, void *cuda_stream);

/* Pre-processing before the flow estimate (paper Sec. 2): a high-pass filter
 * against the static background, then contrast-limited adaptive histogram
 * equalisation (Zuiderveld 1994).  The paper gives no parameters; this build
 * reads them as:
 *   high-pass  d = max(0, n I - S), S the clamp-to-edge sum of I over the
 *              (2 hp_radius + 1)^2 box, n its pixel count (hp_radius = 0:
 *              d = I, n = 1); the filtered value is d / n
 *   CLAHE      256 bins over [0, vmax + 1): bin = floor(256 d / (n (vmax+1)));
 *              tiles_x x tiles_y tiles of ceil(W/tiles_x) x ceil(H/tiles_y)
 *              pixels; per tile of N pixels the histogram is clipped at
 *              max(1, floor(clip_percent N / 25600)), the excess E spread as
 *              E / 256 to every bin plus one to the first E mod 256 bins;
 *              map = cumulative count * vmax / N; each pixel blends the maps
 *              of the four tiles whose centres surround it, bilinearly;
 *              clip_percent = 0 skips the equalisation.
 *   img        device, fmt RPIV_U8 or RPIV_U16, rows pitch_bytes apart.
 *   out        device float32, width x height, rows `width` floats apart.
 *   scratch    device, at least rpiv_stage_preprocess_scratch_bytes.
 * The result, in [0, vmax], can be handed to an engine created with
 * fmt RPIV_F32.  Errors: INVALID_ARG (nulls, sizes, hp_radius > 64, tiles
 * outside [1, 64] or larger than the image, vmax outside [1, 65535], small
 * scratch), CUDA.                                                           */
rpiv_status rpiv_stage_preprocess_scratch_bytes(int width, int height, int tiles_x, int tiles_y, size_t *bytes);
rpiv_status rpiv_stage_preprocess(const void *img, size_t pitch_bytes, int fmt, int width, int height, int vmax,
                                  int hp_radius, int tiles_x, int tiles_y, int clip_percent, float *out,
                                  void *scratch, size_t scratch_bytes, void *cuda_stream);

/* Exponential smoothing in time (paper Sec. 2: the optical-flow estimate is
 * smoothed with a constant alpha_1 before it predicts, and the sub-pixel
 * field with alpha_2 before it is output):
 *     state[i] = init ? x[i] : alpha * x[i] + (1 - alpha) * state[i]
 * over n floats of device memory, in FP32.  x and state may not overlap
 * unless they are the same array.  Errors: INVALID_ARG (null pointers with
 * n > 0, alpha outside [0, 1]), CUDA.                                       */
rpiv_status rpiv_stage_ema(const float *x, float *state, size_t n, float alpha, int init, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* RPIV_H */
