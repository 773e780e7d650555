/*
 * rs.h -- C ABI of the B300 (sm_103a) reconstruction-filter resampler.
 *
 * What the library computes.  For an image of in_h x in_w pixels with
 * `channels` interleaved samples per pixel (HWC), each output sample is a
 * normalised weighted sum of input samples under a separable reconstruction
 * kernel:
 *
 *     out[y][x][c] = sum_j sum_i  wy(y, j) wx(x, i) in[B_h(j)][B_w(i)][c]
 *
 * with, per axis (n_in input samples, n_out output samples):
 *   - half-pixel centres: output i sits at c_i = (i + 1/2) n_in / n_out;
 *   - antialiasing: the kernel is widened by sc = max(1, n_in / n_out), so
 *     its argument is x = ((2j+1) n_out - (2i+1) n_in) / D with the exact
 *     integer denominator D = 2 max(n_in, n_out) (D = 2 n_out with
 *     RS_NO_ANTIALIAS);
 *   - taps: the integers j with |x| < R (R the kernel's support radius); the
 *     first tap is j_lo = floor(((2i+1) n_in - R D - n_out) / (2 n_out)) + 1,
 *     computed in 64-bit integers, so tap indices are exact;
 *   - weights: w = K(x) evaluated in FP64, divided by their FP64 sum, then
 *     rounded to the working precision; the rounding residual 1 - sum(w) is
 *     added to the largest-magnitude weight and that weight re-rounded;
 *   - kernels (standard published definitions):
 *       RS_K_LINEAR    tent 1 - |x|, R = 1
 *       RS_K_CUBIC     Keys cubic convolution with parameter a = `param`
 *                      (R. Keys, IEEE Trans. ASSP 29(6), 1981), R = 2
 *       RS_K_LANCZOS   sinc(x) sinc(x / R), R = `param` (integer 1..16)
 *                      (C. Duchon, J. Appl. Meteor. 18, 1979)
 *       RS_K_BSPLINE3  cubic B-spline (M. Unser, IEEE SP Mag. 16(6), 1999),
 *                      used directly as an approximating kernel, R = 2
 *       RS_K_MITCHELL  Mitchell-Netravali cubic (D. Mitchell, A. Netravali,
 *                      SIGGRAPH 1988) with B = `param` and C = (1 - B) / 2
 *                      (the B + 2C = 1 line; B = 1/3 the authors' choice,
 *                      B = 0 is Keys a = -1/2, B = 1 the cubic B-spline), R = 2
 *       RS_K_GAUSSIAN  exp(-x^2 / (2 s^2)), s = `param` in (0, 4], truncated
 *                      at R = ceil(3 s)
 *   - boundary maps B for an axis of n samples:
 *       RS_B_CLAMP       min(max(j, 0), n - 1)
 *       RS_B_MIRROR      half-sample symmetric (edge sample repeated),
 *                        period 2n, folds any number of times
 *       RS_B_REFLECT101  whole-sample symmetric, period 2n - 2
 *       RS_B_TRUNCATE    out-of-range taps dropped, the rest renormalised
 *   - no clamping of the result (cubic and Lanczos overshoot is kept).
 *
 * The paper this library accompanies (arXiv:1110.5450) states no resampling
 * formula of its own; every definition above is the standard one cited beside
 * it.
 *
 * Conventions for every entry point.
 *   - Pointers named d_* are CUDA device pointers on the current device;
 *     pointers named h_* are host pointers.  `stream` is a cudaStream_t cast
 *     to void* (NULL = the legacy default stream).
 *   - The caller owns every image buffer.  A plan owns its weight tables and
 *     any intermediate buffer; rs_destroy frees them (NULL is accepted).
 *   - Work is enqueued asynchronously on the stream; argument errors are
 *     returned synchronously before anything is enqueued.  Errors raised on
 *     the device (RS_CHECK bounds words, bounded waits that ran out) are
 *     reported by rs_plan_check / rs_batch_poll after the stream has drained.
 *   - No C++ exception crosses this interface.  rs_last_error() returns a
 *     thread-local message describing the most recent failure on the calling
 *     thread.
 *   - A plan may be used from one host thread at a time.
 */
#ifndef RS_H
#define RS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RS_API __attribute__((visibility("default")))
#else
#define RS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RS_OK = 0,
    RS_ERR_INVALID_ARG = 1, /* malformed descriptor, NULL pointer, bad size   */
    RS_ERR_UNSUPPORTED = 2, /* valid request this build does not implement    */
    RS_ERR_OOM = 3,         /* a device allocation failed                     */
    RS_ERR_BUDGET = 4,      /* a server's memory budget cannot hold a request */
    RS_ERR_CUDA = 5,        /* a CUDA runtime call failed                     */
    RS_ERR_TIMEOUT = 6,     /* a bounded device or host wait ran out          */
    RS_ERR_BUSY = 7,        /* queue full or work still in flight             */
    RS_ERR_DEVICE = 8       /* a device-side check (RS_CHECK) failed          */
} rs_status;

typedef enum { RS_F64 = 0, RS_F32 = 1, RS_F16 = 2, RS_BF16 = 3 } rs_dtype;

typedef enum {
    RS_K_LINEAR = 0,
    RS_K_CUBIC = 1,   /* param = a, e.g. -0.5 */
    RS_K_LANCZOS = 2, /* param = R, e.g. 3    */
    RS_K_BSPLINE3 = 3,
    RS_K_MITCHELL = 4, /* param = B (C = (1 - B) / 2), e.g. 1/3 */
    RS_K_GAUSSIAN = 5  /* param = sigma, e.g. 0.5              */
} rs_kernel;

typedef enum {
    RS_B_CLAMP = 0,
    RS_B_MIRROR = 1,
    RS_B_REFLECT101 = 2,
    RS_B_TRUNCATE = 3
} rs_boundary;

/* Plan flags. */
#define RS_NO_ANTIALIAS 0x01u /* do not widen the kernel when downscaling        */
#define RS_FORCE_SIMT 0x02u   /* never pick the tensor-core (tcgen05) path        */
#define RS_FORCE_TC 0x04u     /* pick the tcgen05 banded-GEMM path (F16/BF16)     */
/* The tcgen05 path runs the vertical (first) pass of the fused kernel as a
 * banded GEMM on the tensor cores.  It needs F16/BF16 storage, a row pitch of
 * whole 16 bytes, in_w * channels a multiple of 8, and at rs_resample an input
 * pointer aligned to 16 bytes (RS_ERR_INVALID_ARG otherwise).  Without a flag
 * it is chosen for such plans when the vertical axis has 16 or more taps
 * (wide antialiasing); with RS_FORCE_TC a plan that cannot take it fails with
 * RS_ERR_UNSUPPORTED.  Batches and the server always run the SIMT kernel. */
#define RS_TWO_PASS 0x08u     /* separate H-then-V kernels through an HBM buffer  */
#define RS_CHECK 0x10u        /* device table checks before every resample (below) */
#define RS_NO_STREAM 0x20u    /* never pick the row-streaming kernel              */
#define RS_FORCE_STREAM 0x40u /* pick the row-streaming kernel (FP32/FP16/BF16, 1 or 3
                                 channels; bands of 4 outputs of at most 40 / 32
                                 inputs across / down); RS_ERR_UNSUPPORTED where
                                 it cannot apply.  A 16-bit downscale of 12 or
                                 more taps across runs its tensor-core form
                                 (stream form 3, plan path 5) where that applies */
#define RS_PREFILTER 0x100u   /* interpolating cubic B-spline: with RS_K_BSPLINE3, the
                                 input is first replaced by its B-spline coefficients
                                 (per axis (c[k-1] + 4 c[k] + c[k+1]) / 6 = s[k], c
                                 extended by the boundary rule), so the result passes
                                 through the samples (M. Unser, IEEE SP Mag. 16(6),
                                 1999).  FP32 or FP64 storage; clamp, mirror or
                                 reflect101; not in batches or the server.  The plan
                                 holds the coefficients (in_h x in_row_stride FP32/FP64). */
#define RS_FORCE_VFIRST 0x80u /* pick the vertical-first two-pass kernels (FP32/FP16/
                                 BF16, 1 or 3 channels, out_h <= in_h, bands of at
                                 most 256); RS_ERR_UNSUPPORTED where they cannot apply */
/* The vertical-first path runs the vertical pass from the input into an FP32
 * intermediate of out_h x in_w pixels (plan-owned), then the horizontal pass
 * into the output: no staged halo, so it suits strong downscales with wide
 * bands (x0.125: 48 taps).  rs_plan_autotune times it against the other
 * kernels; it runs untuned only when forced. */
/* The row-streaming kernel runs the horizontal pass first on staged input rows
 * and the vertical pass on a ring of filtered rows (FP32 whatever the storage
 * type), with deep TMA prefetch and coalesced output rows.  It is chosen for
 * FP32, FP16 and BF16 plans of 1 or 3 channels whose bands of 4 outputs need
 * at most 40 input pixels across and 32 input rows down, with a 16-byte row
 * pitch -- except 16-bit plans that take the tensor-core tiles (wide
 * antialiasing), which keep them unless this kernel is forced or the
 * autotuner measures it faster; an input pointer that is not 16-byte aligned
 * at rs_resample falls back to the tile kernel of the same plan. */

/* Debugging knobs: the environment variable RS_PLAN_FLAGS (read once per
 * process) adds kernel-choice flags to every plan created, e.g.
 * RS_PLAN_FLAGS=FORCE_SIMT,CHECK; accepted names: FORCE_SIMT, FORCE_TC,
 * TWO_PASS, CHECK, NO_STREAM, FORCE_STREAM, FORCE_VFIRST (an unknown name
 * makes rs_plan_create return RS_ERR_INVALID_ARG).  Every API call that
 * launches work opens an NVTX range named after it (no cost without a
 * profiler). */

/* Plan descriptor.  Sizes are in samples/elements, not bytes. */
typedef struct {
    int32_t in_h, in_w, channels; /* source grid, HWC interleaved, 1 <= channels <= 64 */
    int32_t out_h, out_w;         /* target grid; 0 => derive from scale_h / scale_w   */
    double scale_h, scale_w;      /* used iff out_* == 0: out = max(1, floor(n s + 1/2)) */
    int32_t kernel;               /* rs_kernel                                          */
    double param;                 /* a for RS_K_CUBIC, R for RS_K_LANCZOS, else ignored */
    int32_t boundary;             /* rs_boundary                                        */
    int32_t in_dtype, out_dtype;  /* rs_dtype; must be equal.  Accumulation is FP64 for
                                     RS_F64 and FP32 otherwise                          */
    uint32_t flags;               /* RS_* flags above                                   */
    int64_t in_row_stride;        /* elements between input rows; 0 => in_w * channels  */
    int64_t out_row_stride;       /* elements between output rows; 0 => out_w*channels  */
} rs_plan_desc;

typedef struct rs_plan rs_plan;

/* The output size a descriptor derives (out_h / out_w as given, or
 * max(1, floor(n s + 1/2)) from scale_h / scale_w where they are 0), after the
 * same checks as rs_plan_create.  Host only: no device work, no allocation. */
RS_API rs_status rs_desc_out_size(const rs_plan_desc *desc, int32_t *out_h, int32_t *out_w);

/* Create a plan: validates the descriptor, derives the output size, allocates
 * the weight tables on the current device and enqueues the FP64 weight-table
 * kernel on `stream`, then synchronises that stream once to read back the
 * tap-span statistics that choose the pass kernel.  On success *out receives
 * the plan; on failure *out is set to NULL and nothing stays allocated.
 * Limits: sides 1 .. 2^22, taps per output (before boundary folding) <= 256. */
RS_API rs_status rs_plan_create(const rs_plan_desc *desc, void *stream, rs_plan **out);

/* Resample one image: d_in holds in_h rows of in_row_stride elements of
 * in_dtype, d_out receives out_h rows of out_row_stride elements of
 * out_dtype.  Buffers must not overlap.  Asynchronous on `stream`. */
RS_API rs_status rs_resample(rs_plan *plan, const void *d_in, void *d_out, void *stream);

/* Re-run the weight-table kernels of a plan on `stream` into the plan's
 * existing tables (no allocation, no synchronisation).  The tables are a
 * deterministic function of the descriptor, so this reproduces them bit for
 * bit; it exists so that a timed step can include the table computation. */
RS_API rs_status rs_plan_recompute(rs_plan *plan, void *stream);

/* Measured autotuning of the fused path (the kernel tile shape, outputs per
 * thread group, staged-buffer count and the split of warps between the two
 * pipelined passes): times candidate configurations on the caller's buffers
 * (d_in / d_out as for rs_resample; d_out is overwritten) and keeps the
 * fastest for this plan.  Synchronises `stream`; allocates and frees band
 * tables while it runs.  cache_path (may be NULL) names a JSON-lines file of
 * earlier results keyed by device, dtype, channels, kernel, boundary and
 * geometry; a hit applies the cached choice without timing, a miss appends
 * the new result.  Unless RS_FORCE_TC or RS_FORCE_STREAM is set, the
 * winner is also timed against the two-pass path (H then V through an HBM
 * intermediate of in_h x out_w x channels accumulation samples, allocated
 * for the trial and kept only if that path wins: small problems such as
 * FP64 256x256 -> 512x512); the chosen path is in rs_plan_info.path.  Plans
 * created on the two-pass path return RS_OK unchanged. */
RS_API rs_status rs_plan_autotune(rs_plan *plan, const void *d_in, void *d_out, void *stream,
                                  const char *cache_path);

/* Forms of the row-streaming kernel (plan path 3).  kind 0: the band kernel
 * with phases that alternate between block barriers; 1: the band kernel with
 * warps specialised on the two passes; 2: the pipelined kernel (upscales and
 * scale 1 with 4 or 6 taps per output on both axes: groups of 4 outputs on
 * bands of taps + 3 inputs built on chip from the plan's weight tables, a
 * producer warp and horizontal / vertical warps handing staged blocks over
 * through mbarriers); 3: the tensor-core downscale (plan path 5; FP16 /
 * BF16 plans that downscale both axes, in_w * channels a multiple of 8, at
 * most 128 vertical taps): the horizontal pass as a tcgen05 GEMM per strip
 * of 48 output samples against the strip's weight matrix (hi + lo 16-bit
 * parts, held in shared memory), 128 input rows per MMA block with TMA-staged
 * chunks and two tensor-memory accumulators, and the vertical pass in FP32 on
 * the filtered rows read back from tensor memory.  Zeros choose a field's
 * default.  Forms 0-2 compute the same sums (each output's taps in increasing
 * order, FP32 accumulation; band zeros add exact zeros); form 3 sums each
 * horizontal window in the tensor cores' order (FP32 accumulation), so its
 * results may differ from the others in the last bits. */
typedef struct {
    int32_t kind;          /* 0, 1, 2 or 3 as above                                   */
    int32_t h_warps;       /* warps on the horizontal pass (kind 1: 2..6; kind 2: 1..8) */
    int32_t staged_blocks; /* staged 32-row input blocks, 2..4 (kind 3: staged chunks of
                              128 rows x 64 samples, 2..6)                            */
    int32_t strip_width;   /* output pixels per strip (a multiple of 4; kind 3: 0 to set,
                              48 / channels reported)                                 */
    int32_t prefetch;      /* kind 2: 1 = prefetch the block after the staging ring
                              into L2; kind 3: 1 = prefetch the chunk 2 rings ahead  */
    int32_t v_warps;       /* kind 2: warps on the vertical pass (a CTA has one producer
                              warp plus h_warps + v_warps <= 15; above 11 the CTA
                              takes a whole SM); kind 3: 1..8                         */
    int32_t row_ranges;    /* kind 2: output row ranges, one CTA per (strip, range);
                              1..255                                                  */
} rs_stream_form;

/* Makes the plan run the row-streaming kernel in the given form (configuring
 * it on `stream`, which it does not synchronise).  RS_ERR_UNSUPPORTED when the
 * plan cannot take that form (then the plan keeps its previous kernel);
 * RS_ERR_INVALID_ARG for a malformed form.  rs_plan_autotune chooses among the
 * same forms by timing them. */
RS_API rs_status rs_plan_set_stream_form(rs_plan *plan, const rs_stream_form *form, void *stream);

/* The form the plan's streaming kernel is configured in (RS_ERR_UNSUPPORTED
 * if the plan has no streaming configuration); whether rs_resample runs it is
 * rs_plan_info.path == 3 (kinds 0-2) or 5 (kind 3). */
RS_API rs_status rs_plan_get_stream_form(const rs_plan *plan, rs_stream_form *form);

/* Free a plan after waiting for its work to finish.  NULL is accepted. */
RS_API rs_status rs_destroy(rs_plan *plan);

/* Facts about a created plan. */
typedef struct {
    int32_t out_h, out_w;     /* derived output size                              */
    int32_t taps_h, taps_w;   /* raw taps per output (max over outputs), per axis */
    int32_t table_h, table_w; /* stored (boundary-folded) taps per output         */
    int32_t path;             /* 0 = fused tiles (SIMT), 1 = two-pass SIMT, 2 = fused
                                 tiles with the tcgen05 vertical pass, 3 = row-streaming,
                                 4 = vertical-first two-pass, 5 = tensor-core
                                 streaming downscale (stream form kind 3)           */
    int32_t tile_h, tile_w;   /* output tile of the chosen pass kernel            */
    int32_t group_h, group_w; /* outputs per thread group along each axis         */
    int32_t span_h, span_w;   /* band width (inputs per group)                    */
    int32_t warps_pass1;      /* fused path: warps on staging + vertical pass      */
    int32_t stages;           /* fused path: staged input buffers (TMA)           */
    int32_t smem_bytes;       /* fused path: dynamic shared memory per CTA        */
    int32_t ctas_per_sm;      /* fused path: resident CTAs per SM                 */
    int64_t scratch_bytes;    /* device bytes owned by the plan                   */
} rs_plan_info;

RS_API rs_status rs_plan_get_info(const rs_plan *plan, rs_plan_info *info);

/* Copy one axis' tables to the host (synchronises the device).  axis 0 = rows
 * (height), 1 = columns (width).  Each h_* may be NULL to skip it; arrays are
 * sized for n_out entries (h_w64: n_out * table entries, row-major).
 *   h_jlo    first raw tap j_lo (may be negative or >= n_in)
 *   h_count  number of raw taps with |x| < R
 *   h_start  first input index of the stored, boundary-folded window
 *   h_w64    folded, normalised FP64 weights (window position k <-> index
 *            h_start + k)
 *   h_wwork  weights rounded to the working precision and residual-corrected,
 *            widened to double for the copy */
RS_API rs_status rs_plan_get_tables(const rs_plan *plan, int axis, int32_t *h_jlo, int32_t *h_count,
                             int32_t *h_start, double *h_w64, double *h_wwork);

/* Allocation-free resample.  For callers that cannot call cudaMalloc -- a
 * plug-in inside an application whose own allocator owns the device memory, or
 * a real-time loop that may not pay for cudaMalloc/cudaFree (cudaFree
 * synchronises the whole device).  The paper has no counterpart of this entry
 * point; it is a deployment convenience.
 *
 * Same descriptor (checked exactly as rs_plan_create checks it) and buffers as
 * rs_plan_create + rs_resample, but no plan: each call computes the weight
 * tables and runs the separate H-then-V pass kernels with the tables and the
 * intermediate placed in one library-owned static device array of
 * RS_STATIC_SCRATCH_BYTES (32 MiB).  No cudaMalloc, cudaFree or other
 * allocating call is made on the caller's behalf.  The only flag it takes is
 * RS_NO_ANTIALIAS (any other: RS_ERR_UNSUPPORTED).  A request whose tables
 * plus intermediate (in_h * out_w * channels * 4 bytes, 8 for RS_F64) exceed
 * the array returns RS_ERR_BUDGET with the sizes in rs_last_error().
 *
 * The array comes into existence when the CUDA runtime loads the library's
 * device code that holds it: with lazy module loading (the CUDA default) at
 * the first call of this entry point on a device, with eager loading
 * (CUDA_MODULE_LOADING=EAGER) when the device's context is created; the
 * device keeps it until the process exits.  Make the first call on each
 * device at start-up, before the application's allocator takes the device
 * memory (if the device has no room left then, it returns RS_ERR_OOM) and
 * outside any stream capture.  Every call looks the array's device address up
 * again (cudaGetSymbolAddress: no allocation once it exists), so a call after
 * a device reset uses the re-created array.  All calls share the array and it
 * keeps the previous call's contents; calls whose GPU work overlaps (different
 * streams or host threads) race on it, so issue them on one stream.
 * Asynchronous on `stream`; device errors of the table kernel are not reported
 * by this entry point. */
#define RS_STATIC_SCRATCH_BYTES (32u << 20)
RS_API rs_status rs_resample_noalloc(const rs_plan_desc *desc, const void *d_in, void *d_out, void *stream);

/* ------------------------------------------------------------------------
 * Batches: uneven images resampled by one persistent kernel launch.
 *
 * Every image keeps its own descriptor (size, scale, kernel, boundary and
 * flags may differ); channels (1 or 3) and dtype must be equal across the
 * batch.  Work items are (image, output tile) pairs of the concatenated tile
 * list, dealt round-robin to the persistent CTAs, so every image's tiles
 * spread over the whole GPU.  The launch (parameter upload, kernel) is a CUDA
 * graph built at creation and replayed by rs_batch_run.  In a batch planned
 * for TMA, images of at least 2^18 output pixels that the row-streaming
 * kernels take leave the tile list and run on them instead
 * (rs_batch_info.n_streamed): the images of one streaming kernel share one
 * multi-image launch (where it takes several images, each is first
 * re-planned for its share of the SMs within that launch, strip width and
 * row ranges chosen anew for that share; a band kernel with
 * one image keeps a launch of its own), spread
 * over four side streams that are forked from and joined back into the
 * caller's stream around the graph.
 * ---------------------------------------------------------------------- */
typedef struct rs_batch rs_batch;

/* Plans n images (n >= 1) and builds the batch's CUDA graphs.  Synchronises
 * `stream`.  Returns RS_ERR_UNSUPPORTED when an image cannot use the fused
 * kernel (more than 4 channels, or bands too wide). */
RS_API rs_status rs_batch_create(const rs_plan_desc *descs, int32_t n, void *stream, rs_batch **out);

/* Resamples image i from d_in[i] into d_out[i] (device pointers laid
 * out as for rs_resample of descriptor i) by replaying the batch graph on
 * `stream`; asynchronous.  The host arrays are read during the call.  When the
 * batch was planned for TMA (all row pitches 16-byte multiples), every d_in[i]
 * must be 16-byte aligned (RS_ERR_INVALID_ARG otherwise). */
RS_API rs_status rs_batch_run(rs_batch *batch, const void *const *d_in, void *const *d_out, void *stream);

/* Measured autotuning of the batch launch (group size, per-image tile
 * budget, warp split) on the given buffers (outputs are overwritten).
 * Synchronises `stream`.  cache_path as for rs_plan_autotune (may be NULL). */
RS_API rs_status rs_batch_autotune(rs_batch *batch, const void *const *d_in, void *const *d_out, void *stream,
                                   const char *cache_path);

typedef struct {
    int32_t n_images, total_tiles;
    int32_t group, warps_pass1, stages, use_tma;
    int32_t smem_bytes, ctas_per_sm, grid;
    int64_t out_pixels;          /* sum of out_h * out_w                      */
    int64_t in_bytes, out_bytes; /* algorithmic bytes: every input and output once */
    int32_t n_streamed;          /* images on the row-streaming kernel        */
} rs_batch_info;

RS_API rs_status rs_batch_get_info(const rs_batch *batch, rs_batch_info *info);

/* The kernel path image `index` runs on in this batch: 0 the persistent tile
 * kernel, 3 a row-streaming kernel (the band kernels one launch per image, the
 * pipelined kernel in a multi-image launch), 5 the tensor-core streaming
 * downscale; the streamed images run their plan's untuned streaming form.
 * RS_ERR_INVALID_ARG for a bad index. */
RS_API rs_status rs_batch_image_path(const rs_batch *batch, int32_t index, int32_t *path);

/* Frees the batch after waiting for its work.  NULL is accepted. */
RS_API rs_status rs_batch_destroy(rs_batch *batch);

/* ------------------------------------------------------------------------
 * Serving: a continuous-batching request loop on one device.
 *
 * Requests (one image each; size, scale, kernel and boundary free) are
 * submitted from any host thread.  A scheduler thread admits them in arrival
 * order while their device state (weight and band tables, and the output
 * when the request passes d_out = NULL) fits the server's memory budget -- a
 * device arena allocated once -- plans each one without any host
 * synchronisation, and launches everything admitted since the previous launch
 * as one persistent fused launch per (channels, dtype, group size, TMA)
 * class, on up to max_inflight streams at once.  A request of at least 2^20
 * output pixels (16-byte row pitches, not RS_F64, not RS_NO_STREAM) runs
 * alone on the row-streaming kernels in their untuned form, its window
 * starts computed on the host in closed form; when no streaming form takes
 * it, it runs on the tile kernel like the rest.  Requests arriving while
 * others run are admitted as memory frees and run concurrently with them.
 * Completion is timestamped (host steady clock) by a host callback queued
 * behind each launch.  Every request's result is bit-identical to the same
 * resample run alone: on the tile kernel (RS_FORCE_SIMT | RS_NO_STREAM), or
 * for a large request on the plan's untuned streaming form.
 * ---------------------------------------------------------------------- */
typedef struct rs_server rs_server;

typedef struct {
    uint64_t budget_bytes; /* device bytes for in-flight requests (>= 1 MiB)      */
    int32_t max_inflight;  /* launches in flight (1..8), one stream each         */
    int32_t max_batch;     /* requests per launch (1..4096)                      */
    int32_t warps_pass1;   /* fused-kernel warp split (0 => 4)                   */
    int32_t reserved;
} rs_server_desc;

typedef struct {
    rs_plan_desc desc; /* one image; channels 1 or 3; in_dtype == out_dtype            */
    const void *d_in;  /* device input laid out as for rs_resample (client-owned)      */
    void *d_out;       /* device output, or NULL: the server allocates it in its budget
                          and keeps it until rs_server_release                        */
} rs_request;

typedef struct {
    int32_t status;         /* RS_ERR_BUSY while pending, RS_OK when done, else the error */
    int32_t launch_id;      /* launch that ran the request                              */
    int32_t batch_size;     /* requests in that launch                                  */
    int32_t out_h, out_w;
    int64_t out_row_stride; /* elements                                                 */
    void *d_out;            /* the result (device), valid once status == RS_OK          */
    uint64_t t_submit_ns, t_admit_ns, t_launch_ns, t_done_ns; /* host steady clock */
    /* GPU clock (%globaltimer, ns) when the launch that ran the request started
     * and finished its work on the device (one-thread stamp kernels on its
     * stream around it): launches whose intervals intersect ran concurrently */
    uint64_t t_gpu_start_ns, t_gpu_end_ns;
} rs_request_state;

typedef struct {
    uint64_t completed, rejected, launches, out_pixels, pending;
    uint64_t bytes_in_use, max_bytes_in_use, max_batch;
    uint64_t streamed; /* launches of one large request on the row-streaming kernels */
    uint64_t launch_host_ns; /* scheduler time spent issuing launches (host work + API calls) */
    uint64_t stream_host_ns; /* of which issuing the large requests' launches              */
} rs_server_stats;

RS_API rs_status rs_server_create(const rs_server_desc *desc, rs_server **out);
/* Enqueues n requests; tickets first_ticket .. first_ticket + n - 1.  Requests
 * that can never fit the budget complete with RS_ERR_BUDGET; malformed ones
 * with RS_ERR_INVALID_ARG / RS_ERR_UNSUPPORTED. */
RS_API rs_status rs_batch_submit(rs_server *server, const rs_request *reqs, int32_t n, uint64_t *first_ticket);
RS_API rs_status rs_batch_poll(rs_server *server, uint64_t ticket, rs_request_state *state);
/* Forgets a finished request and returns its server-allocated output to the budget. */
RS_API rs_status rs_server_release(rs_server *server, uint64_t ticket);
/* Waits (host, bounded by timeout_ms) until nothing is pending or in flight,
 * then reports any device-side error word (RS_ERR_DEVICE). */
RS_API rs_status rs_server_drain(rs_server *server, int64_t timeout_ms);
RS_API rs_status rs_server_get_stats(rs_server *server, rs_server_stats *stats);
/* Drains (up to 60 s), stops the scheduler and frees the server.  NULL is accepted. */
RS_API rs_status rs_server_destroy(rs_server *server);

/* Tensor-core self-test.  The paper has no counterpart: this checks the
 * fifth-generation tensor-core building blocks the banded-GEMM passes use.
 * One CTA computes D = A * B^T with tcgen05 MMAs (16-bit operands, FP32
 * accumulators in tensor memory): A is m x k, B is n x k, both row-major
 * 16-bit patterns on the host (bf16 != 0: BF16, else FP16), D is m x n
 * floats on the host.  a_mn / b_mn store A / B MN-major in shared memory
 * (else K-major); variant 0 encodes the core-matrix stride along K as the
 * descriptor's leading offset and the stride along M (N) as its stride
 * offset, variant 1 the other way round.  m = 128, n and k multiples of
 * 16 up to 256 with n * k <= 49152.  Synchronous; allocates and frees its own
 * device buffers. */
RS_API rs_status rs_tc_selftest(int32_t m, int32_t n, int32_t k, int32_t a_mn, int32_t b_mn, int32_t variant,
                                int32_t bf16, const uint16_t *h_a, const uint16_t *h_b, float *h_d);

/* RS_CHECK.  A plan created with RS_CHECK runs a table check on the device
 * before every resample (on the same stream): per output of both axes, the
 * stored window lies in the input (0 <= h_start <= n_in - table entries) and
 * its working-precision weights are finite and sum to one within 1e-5 (FP32,
 * FP16, BF16 storage) or 1e-12 (FP64).  These are what every pass kernel
 * relies on when it reads a window; a failure sets the plan's error word
 * (rs_plan_check then returns RS_ERR_DEVICE) and the resample still runs. */

/* Synchronise the device and report any device-side error word the plan's
 * kernels set; clears the word.  RS_ERR_TIMEOUT: a bounded device wait ran
 * out (every wait of every kernel gives up after 2 s); RS_ERR_DEVICE: any
 * other device-side check (the weight-table kernel's tap and sum checks, a
 * band that does not fit its staged tile, RS_CHECK). */
RS_API rs_status rs_plan_check(rs_plan *plan);

/* Replace one axis' working-precision weights (axis 0 = rows, 1 = columns)
 * with the caller's: h_wwork holds n_out x (table entries) values, row-major,
 * laid out as rs_plan_get_tables returns h_wwork; they are rounded to the
 * working precision.  The windows (h_start) stay the plan's, so every read
 * stays inside the input whatever the weights are; they are used as given
 * (RS_CHECK checks them before each resample).  The band tables of the
 * kernels that have them are rebuilt on `stream`; rs_plan_recompute restores
 * the computed weights.  RS_ERR_UNSUPPORTED when both axes share one table
 * (identical geometry).  Synchronises `stream` for FP32 / FP16 / BF16 plans. */
RS_API rs_status rs_plan_set_weights(rs_plan *plan, int32_t axis, const double *h_wwork, void *stream);

/* Bounded-wait self-test: enqueues on `stream` a one-warp kernel that runs the
 * same bounded mbarrier wait as every kernel of the library on a barrier
 * nobody arrives on, with a limit of limit_us microseconds (1 .. 2,000,000).
 * The wait gives up, sets the plan's error word to the timeout code and the
 * kernel returns, so the next rs_plan_check reports RS_ERR_TIMEOUT and the
 * context stays usable.  The paper has no counterpart: this checks the
 * library's failure path without stopping a GPU. */
RS_API rs_status rs_plan_wait_selftest(rs_plan *plan, int32_t limit_us, void *stream);

/* ------------------------------------------------------------------------
 * Affine warps with elliptical weighted average filtering (non-separable):
 * P. Heckbert, "Fundamentals of Texture Mapping and Image Warping", 1989;
 * N. Greene and P. Heckbert, IEEE CG&A 6(6), 1986.
 *
 * Output pixel (x, y) maps to the input point
 *   u = a[0] (x + 1/2) + a[1] (y + 1/2) + a[2],  v = a[3] (x + 1/2) + a[4] (y + 1/2) + a[5]
 * (input sample (i, j) sits at (i + 1/2, j + 1/2)).  With J = [[a0, a1],
 * [a3, a4]] the filter covariance is V = sigma^2 (J J^T + I) (a Gaussian
 * reconstruction filter of width sigma convolved with the prefilter of the
 * same width in output pixels); input sample s weighs
 * exp(-Q / 2) - exp(-cutoff^2 / 2) for Q = (s - c)^T V^-1 (s - c) < cutoff^2,
 * else 0; the result is the weighted mean (0 where no weight is left, e.g.
 * far outside with RS_B_TRUNCATE).  Boundary maps as for resampling.  FP32
 * weights and accumulation; storage FP32, FP16 or BF16; 1-4 channels, HWC.
 * Stateless: one call, one kernel launch on `stream`.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t in_h, in_w, channels;     /* source grid, HWC interleaved, 1..4 channels */
    int32_t out_h, out_w;             /* target grid                                 */
    double a[6];                      /* output centre -> input point (see above)    */
    double sigma;                     /* filter width in pixels, (0, 64]; e.g. 0.5   */
    double cutoff;                    /* ellipse radius in filter widths, (0, 8]     */
    int32_t boundary;                 /* rs_boundary                                 */
    int32_t dtype;                    /* rs_dtype: RS_F32, RS_F16 or RS_BF16         */
    int64_t in_row_stride, out_row_stride; /* elements; 0 => packed                  */
} rs_warp_desc;

/* Warps d_in into d_out (device pointers, layouts per the descriptor). */
RS_API rs_status rs_warp(const rs_warp_desc *desc, const void *d_in, void *d_out, void *stream);

/* ------------------------------------------------------------------------
 * Clustering: the paper's parallel merging of ToF frames (arXiv:1110.5450,
 * Sec. "Parallel Merging Algorithm" and "Merging Criterion").
 *
 * Every pixel of a frame starts as a region whose ID is its linear index
 * (y * width + x), with descriptor w = (z, phi), phi = arctan(d sqrt(I))
 * (z: distance along the optical axis, d: radial distance, I: intensity).
 * In synchronous rounds every region picks, among its 4-neighbourhood
 * neighbour regions S with |z - z_S| <= t_z and |phi - phi_S| <= t_phi
 * (Eq. 1), the one minimising f = alpha_z |dz| + alpha_phi |dphi| (Eq. 2),
 * ties to the larger ID; mutual choices merge into the larger ID, whose
 * descriptor becomes the mean over the merged pixels.  Rounds repeat until no
 * region has a qualifying neighbour (or max_rounds; 0 = no limit but the pixel
 * count).  Decisions are taken in FP32, each operation rounded on its own.
 * Table 1 of the paper: t_z = 0.04 m, t_phi = 0.009 rad, alpha_z = 8 / pi,
 * alpha_phi = 4 / 3.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t n_frames, height, width; /* frames per run, 1 <= height * width <= 2^24 */
    float t_z, t_phi;                /* merge thresholds (Eq. 1), >= 0                 */
    float alpha_z, alpha_phi;        /* weights of f (Eq. 2), >= 0                     */
    int32_t max_rounds;              /* 0: until no region has a partner               */
} rs_cluster_desc;

typedef struct rs_cluster rs_cluster;

/* Allocates the per-frame region state (72 bytes per pixel per frame). */
RS_API rs_status rs_cluster_create(const rs_cluster_desc *desc, rs_cluster **out);

/* Clusters n_frames frames, one thread block each, asynchronously on
 * `stream`.  Device pointers, frames back to back, row-major:
 * z, d, intensity [n_frames][height][width] (FP32, read only);
 * labels [n_frames][height][width] (int32, written: each pixel's region ID);
 * rounds [n_frames] (int32, written: merge rounds run);
 * region_z, region_phi [n_frames][height * width] (FP32) and region_size
 * (int32), indexed by region ID: the final descriptor and pixel count of
 * every region (size 0 for IDs merged away); each may be NULL. */
RS_API rs_status rs_cluster_run(rs_cluster *c, const float *z, const float *d, const float *intensity,
                                int32_t *labels, int32_t *rounds, float *region_z, float *region_phi,
                                int32_t *region_size, void *stream);

/* Waits for the device and frees.  NULL is accepted. */
RS_API rs_status rs_cluster_destroy(rs_cluster *c);

RS_API const char *rs_status_string(rs_status status);
RS_API const char *rs_last_error(void);

/* Library version, for the Python binding's sanity check. */
RS_API int32_t rs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RS_H */
