/*
 * C ABI of the GB300 (sm_103a) implementation of the local stereo method of
 * Chang & Maruyama, "Real-Time High-Quality Stereo Matching System on a GPU"
 * (arXiv 2212.00488).
 *
 * Pipeline (Sec. III, steps 1-8): grey -> 2x mean-pool downscale (Eq. 2) ->
 * mini-census + cross arms -> matching cost AD + mini-census (Eqs. 3-6) ->
 * cross-based aggregation along x then y (Eqs. 7-8) -> winner-take-all for
 * the left and right base images (Eq. 9) -> GCP cross-check (Eq. 10) ->
 * median filter -> bilateral estimation fill (Eq. 11) -> upscale (Step 8).
 *
 * Conventions shared by every entry point:
 *  - Every function returns STEREO_OK (0) or a negative STEREO_E* code and
 *    never throws; stereo_last_error() then holds a one-line reason.
 *  - Images are RGB, uint8, HWC interleaved, row pitch 3*W bytes, no padding.
 *  - Buffers named "device" are CUDA device (or managed) memory that the
 *    caller owns and keeps alive until the work on the stream has finished.
 *    The context owns only its workspace.
 *  - Work is asynchronous on the given stream (NULL = the context's own
 *    stream; cudaStreamLegacy and cudaStreamPerThread are accepted);
 *    synchronise that stream, or call stereo_sync(), before reading.
 *  - Dmax counts disparities: d in [0, Dmax-1] (Sec. II). With downscaling,
 *    the processed image is (W/2) x (H/2) and D = ceil(Dmax/2) (Sec. I);
 *    processed-size maps (dl, dr, gcp) hold processed-resolution disparities,
 *    and the final float map holds full-resolution disparities.
 *  - A context is not thread-safe: calls on one context must not overlap.
 */
#ifndef STEREO_H
#define STEREO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STEREO_API __attribute__((visibility("default")))

enum {
    STEREO_OK = 0,
    STEREO_EINVAL = -1,   /* bad argument: size, pointer, parameter or stage */
    STEREO_ENOMEM = -2,   /* the workspace would exceed the context's memory cap, or allocation failed */
    STEREO_ECUDA = -3,    /* a CUDA runtime call or kernel launch failed */
    STEREO_ETIMEOUT = -4  /* a bounded device-side wait gave up */
};

/* Pipeline stages, in order, as reported by stereo_stage_ms() (the columns of
 * Table II, with W+- and W*+- merged into one support stage). */
enum {
    STEREO_STAGE_SCALEDOWN = 0, /* grey + mean-pool downscale (SD) */
    STEREO_STAGE_SUPPORT = 1,   /* mini-census codes and the four cross arms (W+-, W*+-) */
    STEREO_STAGE_COSTAGG = 2,   /* fused cost + x/y aggregation + WTA, both bases (C+CA_x, CA) */
    STEREO_STAGE_REFINE = 3,    /* cross-check + median + bilateral fill (CC, Post), and with
                                   downscaling the scale-up (SU) in the same kernel */
    STEREO_STAGE_UPSCALE = 4,   /* scale-up (SU): part of stage 3; launches nothing, reports 0 */
    STEREO_NUM_STAGES = 5
};

/* Method parameters. Defaults (stereo_default_params) are the paper's values
 * (Sec. V: lambda_AD = 0.3, lambda_MC = 2.3, T = 3; Table II footnote:
 * W_x = 21, W_y = 31 per side, TC = 13) plus values for what the paper
 * leaves open (cost scale, fill mode, downscaling). */
typedef struct {
    double lambda_ad; /* Eq. 4, on intensities scaled to [0, 1]; 0.3 */
    double lambda_mc; /* Eq. 5; 2.3 */
    int tc;           /* arm brightness threshold delta (strict <), Sec. III-C; 13 */
    int wx;           /* horizontal arm cap per side, 0..141 (Table I); 21 */
    int wy;           /* vertical arm cap per side, 1..31; 31 */
    int t_fill;       /* T of the bilateral estimation (Sec. III-E); 3 */
    int downscale;    /* 1: K = 2, m = 1 mean-pool with Dmax halved (Sec. III-A); 0: none */
    int cost_scale;   /* integer cost mode: each term is round(cost_scale * value); 512.
                         (2*wx+1)*(2*wy+1)*(AD(255)+MC(6)) must stay below 2^24. */
    int fill_mode;    /* non-GCP fill between the nearest GCPs a (left, distance i) and b
                         (right, distance j), Sec. III-E: 0 = the paper's bilateral
                         estimation (default); 1 = the closer GCP (Fig. 5a prior art; the
                         left one when i < j, else the right one); 2 = the smaller
                         disparity (Fig. 5b prior art). One-sided and empty rows are
                         filled alike in every mode. */
} stereo_params;

typedef struct stereo_ctx stereo_ctx;

/* Fills *out with the defaults listed above. */
STEREO_API void stereo_default_params(stereo_params *out);

/* Creates a context bound to CUDA device `device` with its own non-blocking
 * stream. p = NULL takes the defaults; a copy of *p is kept. mem_cap_bytes
 * bounds the device workspace the context may allocate (0 = no cap).
 * Returns EINVAL for a NULL out, bad parameters or a device that is not
 * sm_103; ECUDA when the device cannot be initialised. On failure *out is NULL. */
STEREO_API int stereo_create(stereo_ctx **out, int device, const stereo_params *p,
                             size_t mem_cap_bytes);

/* Releases the workspace, stream and context. NULL is a no-op. Waits for the
 * context's own stream first. */
STEREO_API void stereo_destroy(stereo_ctx *ctx);

/* One-line description of the last failure on this context ("" if none). The
 * string belongs to the context and stays valid until its next call. */
STEREO_API const char *stereo_last_error(const stereo_ctx *ctx);

/* The whole method on one pair (Sec. III steps 1-8).
 *  left_rgb, right_rgb: device, H*W*3 bytes each.
 *  W, H: input size, 1..8192 each; with downscaling both must be >= 2.
 *  Dmax: 1..256 without downscaling, 1..511 with it (D <= 256 after halving).
 *  disp_out: device float, required. With downscaling: H*W full-resolution
 *    disparities (Step 8 output); without: H*W filled map D+ (Step 7 output).
 *  dl_out, dr_out: optional (NULL to skip) device uint8 [Y][X] winner-take-all
 *    maps D^L, D^R of the processed image (Eq. 9), X*Y bytes each.
 *  gcp_out: optional device uint8 [Y][X], 1 where Eq. 10 holds, else 0.
 *  stream: cudaStream_t or NULL for the context's stream.
 * The workspace grows on demand (ENOMEM past the cap). Asynchronous. */
STEREO_API int stereo_compute(stereo_ctx *ctx, const uint8_t *left_rgb, const uint8_t *right_rgb,
                              int W, int H, int Dmax, float *disp_out, uint8_t *dl_out,
                              uint8_t *dr_out, uint8_t *gcp_out, void *stream);

/* stereo_compute on HOST buffers: copies the two images in, runs the
 * pipeline, copies the float map (and the optional uint8 maps) back and waits
 * for the stream. Sizes and layouts as for stereo_compute; every pointer is
 * host memory (pinned memory makes the copies asynchronous-capable and faster).
 * Uses a device staging area inside the workspace. Synchronous. */
STEREO_API int stereo_compute_host(stereo_ctx *ctx, const uint8_t *left_rgb, const uint8_t *right_rgb,
                                   int W, int H, int Dmax, float *disp_out, uint8_t *dl_out,
                                   uint8_t *dr_out, uint8_t *gcp_out);

/* stereo_compute_host without the final wait: the copies in, the pipeline and
 * the copies out are queued on the context's stream and the call returns.
 * The host buffers must stay valid and untouched until the work is done
 * (stereo_sync); with pinned host memory the copies run on the copy engines
 * while the SMs work, so two contexts fed alternately overlap one frame's
 * copies with the other's compute. Calls on one context run in order on its
 * stream and reuse one staging area. A bounded-wait timeout is reported by
 * the next stereo_sync. */
STEREO_API int stereo_compute_host_async(stereo_ctx *ctx, const uint8_t *left_rgb, const uint8_t *right_rgb,
                                         int W, int H, int Dmax, float *disp_out, uint8_t *dl_out,
                                         uint8_t *dr_out, uint8_t *gcp_out);

/* Blocks until all work on the context's own stream has finished, then
 * reports STEREO_ETIMEOUT if a bounded wait inside the fused kernel gave up
 * during the last compute (the kernel then returned early and its maps are
 * not valid). Work enqueued on a caller's stream must be synchronised by the
 * caller first. */
STEREO_API int stereo_sync(stereo_ctx *ctx);

/* Polls each bounded wait of the fused kernel makes before it gives up, sets
 * the error word and returns. The waiting warp sleeps at most 256 ns between
 * polls, so the default of 2^20 polls bounds a wait by about 0.3 s, far above
 * any legitimate wait (the waits are between warps of one CTA and last one
 * image row at most). 0 makes every wait give up at its first poll, which
 * exercises the error path. */
STEREO_API int stereo_set_wait_limit(stereo_ctx *ctx, uint32_t polls);

/* Copies intermediates of the last stereo_compute on this context into device
 * buffers (any may be NULL), enqueued on `stream` after that compute:
 *  grey_l, grey_r: uint8 [Y][X] processed grey images (after Eq. 2);
 *  census_l, census_r: uint8 [Y][X] six-bit mini-census codes, bit k for the
 *    neighbour (dx,dy) = (-1,-1),(+1,-1),(-2,0),(+2,0),(-1,+1),(+1,+1) darker;
 *  arms_l, arms_r: uint32 [Y][X], bytes (low to high) = left, right, up, down
 *    arm lengths (m, n, M, N of Eqs. 7-8);
 *  dm: uint8 [Y][X] median-filtered D^L; dplus: float [Y][X] filled map D+.
 * Returns EINVAL when no compute has run. */
STEREO_API int stereo_debug_planes(stereo_ctx *ctx, uint8_t *grey_l, uint8_t *grey_r,
                                   uint8_t *census_l, uint8_t *census_r, uint32_t *arms_l,
                                   uint32_t *arms_r, uint8_t *dm, float *dplus, void *stream);

/* Re-launches one stage (STEREO_STAGE_*) of the last stereo_compute on this
 * context, with the same inputs, outputs and workspace, on `stream`. Used to
 * time a single kernel. The caller keeps the last compute's buffers alive.
 * Returns EINVAL when no compute has run or the stage is out of range. */
STEREO_API int stereo_launch_stage(stereo_ctx *ctx, int stage, void *stream);

/* Turns per-stage timing on or off and clears the accumulated times.
 *  on: 0 = off; n >= 1 = every n-th stereo_compute from now on (the first
 *    one included) records CUDA events between its stages on its stream.
 *    The events sit between the kernels, so a profiled frame runs a few us
 *    slower; n > 1 keeps that cost off most frames.
 * The events of a frame are read back only when their slot in a ring of 64 is
 * reused, so profiling adds no synchronisation between frames. Returns
 * EINVAL for on < 0. */
STEREO_API int stereo_set_profiling(stereo_ctx *ctx, int on);

/* Mean per-stage device times (ms) over every compute profiled since
 * profiling was turned on, waiting for the outstanding events. ms must hold n
 * entries, n <= STEREO_NUM_STAGES; a stage that did not run reports 0.
 * Returns the number of frames averaged (>= 1), or EINVAL when none was
 * profiled. */
STEREO_API int stereo_stage_ms(stereo_ctx *ctx, float *ms, int n);

/* Number of kernels (memsets excluded) the last stereo_compute launched. */
STEREO_API int stereo_last_launch_count(const stereo_ctx *ctx);

/* Tile shapes of the fused cost + aggregation + WTA kernel (columns per base
 * x disparities per CTA, row-prefix width); every consumer thread holds one
 * column and 4 disparities of its tile:
 * 0: 104x4 16-bit for wx up to 26, 1: 104x4 16-bit for wx up to 58,
 * 2: 104x4 32-bit for wx up to 26, 3: 104x4 32-bit for wx up to 58,
 * 4: 64x4 16-bit, 5: 100x4 16-bit with 12 row-prefix producer warps
 * instead of 8, 6: 48x8 32-bit (slabs of 8 disparities, two threads per
 * column), 7: 64x4 32-bit for wx up to 174 with 8 producer warps (the wide
 * windows of Table I, up to the library's limit of 141), 8: 88x4 32-bit for
 * wx up to 66 with 8 producer warps.
 * 16-bit row prefixes need max(2*wx+1, 7) times the largest matching cost
 * below 2^16. Every shape gives the same result; they differ only in speed.
 * A compute with a shape that does not fit the parameters fails with EINVAL. */
#define STEREO_NUM_TILES 9

/* Fixes the tile shape used by later computes on this context (-1 = pick
 * automatically from the frame shape and the SM count, the default).
 * Returns EINVAL for an id outside [-1, STEREO_NUM_TILES-1]. */
STEREO_API int stereo_set_tile(stereo_ctx *ctx, int tile);

/* The tile shape a compute of this frame shape would use (>= 0), or EINVAL. */
STEREO_API int stereo_get_tile(stereo_ctx *ctx, int W, int H, int Dmax);

/* One frame of a batch (stereo_compute_batch): the arguments of
 * stereo_compute for one pair. Frames of a batch may differ in W, H and Dmax. */
typedef struct {
    const uint8_t *left_rgb;   /* device, H*W*3 bytes */
    const uint8_t *right_rgb;  /* device, H*W*3 bytes */
    int W, H, Dmax;
    float *disp_out;           /* device, required */
    uint8_t *dl_out, *dr_out, *gcp_out;   /* device, optional (NULL) */
} stereo_job;

/* Up to 32 pairs in one call (the batched form of the method; the paper
 * processes one pair at a time). Preparation and post-processing run per
 * frame, the fused cost + aggregation + WTA of all frames runs as one
 * persistent kernel taking (frame, strip, slab) tiles largest frame first;
 * the whole batch is one CUDA graph, re-captured and updated in place on each
 * call. Each frame's maps equal stereo_compute's for that frame exactly.
 * With the automatic tile (stereo_set_tile(-1)) the first batch of a given
 * signature (frame shapes, parameters, GPU) times every tile shape that fits
 * and remembers the fastest; stereo_tune_save / stereo_tune_load keep those
 * choices across processes. Asynchronous on `stream` (NULL: the context's
 * stream). The batch uses a workspace of its own next to the single-frame
 * one; both count against the memory cap. */
STEREO_API int stereo_compute_batch(stereo_ctx *ctx, int n, const stereo_job *jobs, void *stream);

/* Device bytes one frame of W x H with Dmax disparities takes in the batch
 * workspace of stereo_compute_batch under parameters p (NULL = the defaults):
 * its grey planes, support words, WTA keys, median and filled maps, plus a
 * 256-byte share of the batch's tile counter. A batch's workspace is at most
 * the sum of its frames' figures; a context created with mem_cap_bytes at
 * least that sum runs the batch without STEREO_ENOMEM (if it holds no
 * single-frame workspace). The caller's input and output buffers are not
 * included. Host arithmetic only: needs no device and no context. Returns 0
 * for parameters or a frame size the entry points reject. */
STEREO_API size_t stereo_job_bytes(const stereo_params *p, int W, int H, int Dmax);

/* Tile shape used by the last batch (-1 if none); when tune_ms is not NULL
 * it receives, for up to n tile ids, the autotuner's time of that shape in
 * ms (-1 where it did not fit or no tuning ran in that call). */
STEREO_API int stereo_batch_tile(const stereo_ctx *ctx, float *tune_ms, int n);

/* Writes the autotuner's choices (one "signature<TAB>tile" line each) to a
 * text file; returns the number written or EINVAL. */
STEREO_API int stereo_tune_save(stereo_ctx *ctx, const char *path);

/* Adds the choices of a file written by stereo_tune_save; returns how many
 * were read or EINVAL. */
STEREO_API int stereo_tune_load(stereo_ctx *ctx, const char *path);

/* Differentiable form (a training form of the method; the paper has only the
 * forward WTA). Left base, processed resolution W x H (no downscaling),
 * D disparities, B pairs. Per pair, in FP32:
 *   g        = (77 R + 150 G + 29 B) / 256 of the float RGB on [0, 1]
 *   C        = w_AD (1 - exp(-|gL(x,y) - gR(x-d,y)| / l_AD))
 *            + w_MC (1 - exp(-MC(x,y,d) / l_MC))  (Eqs. 3-5), the constant
 *              w_AD (1 - exp(-1/l_AD)) + w_MC (1 - exp(-6/l_MC)) when x < d
 *   CA       = the cross aggregation of Eqs. 7-8 divided by the support size
 *   dhat     = sum_d d softmax_d(-CA(x,y,d) / tau)
 * The census codes MC and the arms are frozen: they come from the uint8
 * images left_u8 / right_u8 through the integer path (grey, census, arms with
 * the context's tc, wx, wy) and are not differentiated.
 *  left, right: device float [B][H][W][3]; left_u8, right_u8: device uint8
 *    [B][H][W][3]; theta: device float [4] = (w_AD, w_MC, l_AD, l_MC).
 *  dhat: device float [B][H][W] out; stats: device float [B][H][W][2] out
 *    (softmax maximum and sum per pixel, needed by the backward).
 * H up to 8192, W up to 4096, D up to 256, B up to 64. Asynchronous.
 * The context's workspace for this form holds planes of every pair (all
 * pairs of a batch run in each launch): about 200 bytes per pixel and pair,
 * 70 MB for one 718x496 pair; STEREO_ENOMEM past the context's cap. */
STEREO_API int stereo_diff_forward(stereo_ctx *ctx, int B, int W, int H, int D, const float *left,
                                   const float *right, const uint8_t *left_u8, const uint8_t *right_u8,
                                   const float *theta, float tau, float *dhat, float *stats, void *stream);

/* Backward of stereo_diff_forward for the incoming gradient grad_dhat
 * (device float [B][H][W]): writes the gradients of sum(grad_dhat * dhat)
 * for left and right (device float [B][H][W][3], overwritten) and theta
 * (device float [4], overwritten). The aggregated cost is recomputed a slab
 * of disparities at a time, never stored; the adjoint of the aggregation is
 * the same arm sums transposed over the frozen supports. dhat and stats must
 * be the forward's outputs for the same inputs. Deterministic. */
STEREO_API int stereo_diff_backward(stereo_ctx *ctx, int B, int W, int H, int D, const float *left,
                                    const float *right, const uint8_t *left_u8, const uint8_t *right_u8,
                                    const float *theta, float tau, const float *dhat, const float *stats,
                                    const float *grad_dhat, float *grad_left, float *grad_right,
                                    float *grad_theta, void *stream);

/* stereo_compute without any allocation at call time. The paper has no
 * counterpart: this entry point exists for callers that must not allocate
 * device memory while they run, such as a real-time frame loop that may not
 * stall on, or fail in, an allocation, or a program whose memory pool owns the
 * device and forbids other allocations. It needs no context.
 *
 * All intermediates live in one fixed 32 MiB device array inside the library,
 * which every GPU that loads the library holds until the process exits. A
 * frame fits when its workspace does: with the default parameters that is
 * about 11.8 bytes per input pixel with downscaling (1436x992 needs 17 MB; up
 * to about 2.8 Mpixel) and about 43 bytes per pixel without it (up to about
 * 0.78 Mpixel). A larger frame is rejected with STEREO_ENOMEM and a message in
 * err. Nothing is allocated: no cudaMalloc, cudaFree or allocating library
 * call.
 *
 *  params: NULL for stereo_default_params().
 *  left_rgb, right_rgb, W, H, Dmax, disp_out, dl_out, dr_out, gcp_out,
 *    stream: as for stereo_compute, on the current CUDA device; stream NULL
 *    is the legacy default stream.
 *  err, err_len: optional buffer for a one-line message on failure.
 * The first call on a device looks up the array's device address and sets the
 * kernels' attributes; make that first call before any stream capture. The
 * cost tables are copied from host memory, so a call may wait for work
 * already queued on its stream. Every call shares the one array and its
 * contents stay from the last call: calls whose work overlaps on the GPU (on
 * different streams or host threads) race and give wrong maps. A bounded wait
 * that gives up inside the fused kernel is not reported by this entry point. */
STEREO_API int stereo_compute_noalloc(const stereo_params *params, const uint8_t *left_rgb,
                                      const uint8_t *right_rgb, int W, int H, int Dmax, float *disp_out,
                                      uint8_t *dl_out, uint8_t *dr_out, uint8_t *gcp_out, void *stream,
                                      char *err, size_t err_len);

/* Throughput microbenchmarks for the roofline of the fused kernel (no
 * counterpart in the paper): 32-bit integer add/xor/min, population count and
 * 16-byte shared-memory loads, each as independent chains with every SM of
 * the device full of warps, timed with CUDA events (about 10 ms in all).
 *  device: CUDA device index.
 *  int_ops_per_s, popc_per_s, lds_bytes_per_s: results (operations or bytes
 *    per second, whole device).
 * Allocates a few KB of device memory for the duration of the call. Returns
 * STEREO_OK, STEREO_EINVAL for a null pointer, STEREO_ECUDA on a CUDA error. */
STEREO_API int stereo_measure_peaks(int device, double *int_ops_per_s, double *popc_per_s,
                                    double *lds_bytes_per_s);

#ifdef __cplusplus
}
#endif

#endif /* STEREO_H */
