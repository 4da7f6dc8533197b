/*
 * sobel4.h — C ABI of the GB300 (sm_103a) four-directional 5x5 Sobel library.
 *
 * The operator (Section 3.1 of "Multi-directional Sobel operator kernel on
 * GPUs"): for every pixel of an 8-bit grayscale image, the four 5x5 integer
 * masks G_x, G_y, G_d, G_dt of Eq. (3) are applied in correlation order
 * (mask row 0 meets input row y-2, mask column 0 meets input column x-2, the
 * orientation of Eq. (6) and Eq. (13)), giving the responses
 *     R_k(y,x) = sum_{i,j} K_k[i][j] * I(y+i-2, x+j-2),  k in {x, y, d, dt},
 * and the magnitude of Eq. (4),
 *     G = sqrt(R_x^2 + R_y^2 + R_d^2 + R_dt^2).
 * All integer work is exact (|R_k| <= 12240, S = sum R_k^2 <= 599,270,400).
 * The F32 output is sqrtf((float)S): int -> fp32 round-to-nearest-even, then
 * the IEEE-754 correctly rounded single-precision square root.  It matches a
 * plain CPU evaluation of that definition bit for bit.
 *
 * Conventions for every entry point below:
 *  - Image pointers passed to sobel4_run / sobel4_run_batched are DEVICE
 *    pointers owned by the caller.  A handle owns only its own scratch.
 *  - Calls that take a cudaStream_t are asynchronous: they validate their
 *    arguments on the host, enqueue work on `stream` (0 = legacy default
 *    stream) and return.  A call that returns an error enqueued nothing.
 *  - Device faults surface on the caller's next synchronisation, as with any
 *    CUDA library.
 *  - One handle per host thread, or serialise calls on a handle externally.
 */
#ifndef SOBEL4_H_
#define SOBEL4_H_

#include <stddef.h>
#include <stdint.h>

#ifndef __DRIVER_TYPES_H__
struct CUstream_st;
typedef struct CUstream_st *cudaStream_t;
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque handle; created by sobel4_create, released by sobel4_destroy. */
typedef struct sobel4_ctx *sobel4_handle;

typedef enum {
  SOBEL4_OK = 0,
  SOBEL4_ERR_INVALID_ARG = 1, /* an argument broke a rule stated below */
  SOBEL4_ERR_UNSUPPORTED = 2, /* valid request this build cannot serve */
  SOBEL4_ERR_OOM = 3,         /* device or pinned host allocation failed */
  SOBEL4_ERR_CUDA = 4,        /* a CUDA call failed; see sobel4_last_cuda_error */
  SOBEL4_ERR_TIMEOUT = 5      /* a bounded wait ran out */
} sobel4_status;

/*
 * Border rules.  VALID is the paper's: the kernel output is 2r = 4 rows and
 * columns smaller than its input (Section 4.3.2); here the 2-pixel frame is
 * written as 0 so input and output have the same shape.  The three padded
 * rules evaluate every pixel with the missing neighbours supplied by:
 *   REPLICATE  : the nearest edge pixel (indices clamped),
 *   REFLECT101 : reflection about the edge pixel (-1 -> 1, -2 -> 2,
 *                n -> n-2, n+1 -> n-3); needs height, width >= 3,
 *   CONSTANT0  : zeros.
 */
typedef enum {
  SOBEL4_BORDER_VALID = 0,
  SOBEL4_BORDER_REPLICATE = 1,
  SOBEL4_BORDER_REFLECT101 = 2,
  SOBEL4_BORDER_CONSTANT0 = 3
} sobel4_border;

/*
 * Output formats (dst element type and layout; rows are dst_pitch bytes apart):
 *   F32   : float G = sqrtf((float)S), 4 bytes per pixel.
 *   U8    : uint8 min(255, round(sqrt(S))), 1 byte per pixel.
 *   S16X4 : the four responses R_x, R_y, R_d, R_dt as int16, in four planes;
 *           plane k starts at dst + k * height * dst_pitch.
 *   U16   : uint16 round(sqrt(S)) by the exact integer rule, unsaturated (the
 *           largest value of Eq. 3 is 24480), 2 bytes per pixel.  Runs on the
 *           TMA-family and DIRECT kernels (the lane-copy variant and the
 *           allocation-free entry point return UNSUPPORTED).
 *   EDGE8 : uint8 edge map, 255 where sqrt(S) >= T (exactly: S >= ceil(T^2))
 *           and 0 elsewhere (the VALID frame is 0); T is the handle's
 *           threshold (sobel4_set_threshold, 128 by default); 1 byte per
 *           pixel.  Same kernels as U16.
 */
typedef enum {
  SOBEL4_OUT_F32 = 0,
  SOBEL4_OUT_U8 = 1,
  SOBEL4_OUT_S16X4 = 2,
  SOBEL4_OUT_U16 = 3,
  SOBEL4_OUT_EDGE8 = 4
} sobel4_format;

/*
 * Kernel variants.  AUTO picks the fastest for the request (autotuned when
 * enabled).  DIRECT evaluates the 25-tap sums of Eq. (3) per output pixel from
 * global memory (the paper's "GM" kernel, Section 5.2).  RG is the
 * register-window kernel (Section 4.3): threads across columns, rows walked
 * sequentially, the x/y masks factored into 1x5 passes (Eq. 6-7), the
 * diagonals through K_d+ / K_d- (Eq. 10-19), next rows prefetched.  RG
 * stages rows with asynchronous copies into a per-warp shared-memory ring:
 * 2-D tensor copies (TMA) when the source address and pitch are multiples of
 * 16 bytes, else 1-D bulk copies of each row's 16-byte granules; destinations
 * that are not vector-aligned take lane-shifted aligned stores.
 * RG_LANECOPY selects the older staging in which each lane copies granules
 * itself (cp.async).  TC runs the tensor-core kernel (the masks of Eq. 3 as
 * banded f16 matrix products with fp32 accumulators in tensor memory) on the
 * images it covers (VALID, F32, source and destination rows on 16-byte
 * boundaries, width a multiple of 4) and RG on the others; AUTO uses it for
 * a shape only where sobel4_tune measured it fastest.  The LADDER_* variants
 * are the paper's kernel ladder (Section 5.2, Table 1), kept to re-measure its
 * ablation: LADDER_SM stages a 32 x 8 tile and its halo in shared memory and
 * sums the 25 taps per mask there; LADDER_SM_P adds prefetching (the next
 * tile's loads issued before the current tile is summed, double-buffered);
 * LADDER_RG is the plain register window (one column per lane, 28 output
 * columns per warp, neighbours by warp shuffles, K_x and K_y factored, the
 * diagonals summed over a 5x5 register window); LADDER_RG_V1 computes the
 * diagonals through K_d+ (factored) and K_d- (Eq. 10-15); LADDER_RG_V2 also
 * factors K_d- (Eq. 16-19).  They serve every border rule and format, take
 * rows_per_strip as the RG strip height (default: up to 64 rows, fewer where
 * an image would leave under 16 warps per SM), run one launch per
 * image of a batch, and ignore runtime weights (a handle with weights set
 * runs those as any other handle does).  All variants give identical results.
 */
typedef enum {
  SOBEL4_VARIANT_AUTO = 0,
  SOBEL4_VARIANT_DIRECT = 1,
  SOBEL4_VARIANT_RG = 2,
  SOBEL4_VARIANT_RG_LANECOPY = 3,
  SOBEL4_VARIANT_TC = 4,
  SOBEL4_VARIANT_LADDER_SM = 5,
  SOBEL4_VARIANT_LADDER_SM_P = 6,
  SOBEL4_VARIANT_LADDER_RG = 7,
  SOBEL4_VARIANT_LADDER_RG_V1 = 8,
  SOBEL4_VARIANT_LADDER_RG_V2 = 9
} sobel4_variant;

/*
 * Creation options; pass NULL for defaults (all fields 0 / NULL).
 * autotune = 1: the first sobel4_run of a shape bucket (ceil log2 height,
 * ceil log2 width, format) that has no tuned entry first runs sobel4_tune
 * for that shape (synchronous: scratch buffers, ~30 timed launches per
 * candidate; the call returns after the tune and its own launch are
 * enqueued); skipped while the call's stream is capturing, and each bucket
 * is tried once.  Batches are tuned only by sobel4_tune_batched.
 * cache_path: a tuning cache file (the sobel4_tune_save format), loaded at
 * creation when present (before SOBEL4_TUNE_CACHE, which it replaces) and
 * rewritten (atomically) after every automatic tune.  The string is copied.
 */
typedef struct {
  int32_t variant;               /* sobel4_variant; 0 = AUTO */
  int32_t rows_per_strip;        /* RG strip height R (rows per thread per strip); 0 = auto */
  int32_t persistent_ctas_per_sm;/* batched kernel CTAs per SM; 0 = auto */
  int32_t columns_per_lane;      /* RG columns per thread: 2 or 4; 0 = default */
  int32_t autotune;              /* 1 = tune each new single-image shape bucket on first use */
  const char *cache_path;        /* tuning cache file, or NULL */
} sobel4_options;

/* One image of a batch (all pointers are device pointers). */
typedef struct {
  const uint8_t *src; /* height rows of width bytes, src_pitch bytes apart */
  size_t src_pitch;
  void *dst;          /* output in the batch's format, dst_pitch bytes apart */
  size_t dst_pitch;
  int32_t height;
  int32_t width;
} sobel4_image;

/*
 * Create a handle bound to CUDA device `device` (made current for the call).
 * `opt` may be NULL.  Allocates the handle's scratch (a small device buffer
 * for batch descriptors and the work-queue counter, and pinned host staging).
 * Errors: INVALID_ARG (out == NULL, bad option values, bad device),
 * OOM, CUDA.  On error *out is set to NULL.
 */
sobel4_status sobel4_create(sobel4_handle *out, int32_t device, const sobel4_options *opt);

/*
 * Gradient output of one image (Eq. 3 and Eq. 4 for every pixel).
 *   d_src     : device pointer to height rows of width uint8 pixels.
 *   src_pitch : bytes between rows; >= width.  Any alignment is accepted.
 *   d_dst     : device pointer to the output (layout per `fmt`).
 *   dst_pitch : bytes between output rows; >= width * element size; for F32 a
 *               multiple of 4 and d_dst 4-byte aligned; for S16X4 a multiple of
 *               2 and d_dst 2-byte aligned.
 *   height, width >= 1 (REFLECT101: >= 3).
 *   The source and destination ranges must not overlap.
 * Asynchronous on `stream`.  Errors: INVALID_ARG (nothing enqueued), CUDA.
 */
sobel4_status sobel4_run(sobel4_handle h, const uint8_t *d_src, size_t src_pitch, void *d_dst,
                         size_t dst_pitch, int32_t height, int32_t width, sobel4_border border,
                         sobel4_format fmt, cudaStream_t stream);

/*
 * Gradient output of one COLOUR image, converted to gray on the fly: the
 * paper prepares grayscale input on the host before the kernel (Section 4.3)
 * without stating the rule; this library reads it as the ITU-R BT.601 luma
 * in 8-bit fixed point, Y = (77 R + 150 G + 29 B + 128) >> 8, and applies
 * Eq. (3) and Eq. (4) to Y.  The conversion happens inside the kernel, as it
 * reads the rows: 3 bytes in and the output's bytes out per pixel.
 *   d_src     : device pointer to height rows of width interleaved RGB pixels
 *               (bytes R, G, B per pixel); any alignment.
 *   src_pitch : bytes between rows; >= 3 * width.
 *   d_dst, dst_pitch, height, width, border, fmt, stream: as for sobel4_run.
 * Runs the TMA-family register-window kernel whatever the handle's variant.
 * Errors: INVALID_ARG (nothing enqueued), UNSUPPORTED (the handle has runtime
 * weights or another operator set), CUDA.
 */
sobel4_status sobel4_run_rgb(sobel4_handle h, const uint8_t *d_src, size_t src_pitch, void *d_dst,
                             size_t dst_pitch, int32_t height, int32_t width, sobel4_border border,
                             sobel4_format fmt, cudaStream_t stream);

/*
 * Many images of uneven sizes in persistent launches whose CTAs pull the
 * tiles of all images from a device-side work queue: one small launch (more
 * for very large batches) carries the image descriptors in its parameters,
 * then one batched kernel for the images whose source rows are 16-byte
 * aligned (staged by tensor copies) and one for the others (staged by bulk
 * row copies) -- at most two batched kernels per call; with the RG_LANECOPY
 * variant, one lane-copy batched kernel.  `h_images` is HOST memory with
 * n >= 1 descriptors (each obeying sobel4_run's rules, all with the batch's
 * `border` and `fmt`); it is copied before the call returns.  No two images
 * may write overlapping output, and no output may overlap any input.
 * Asynchronous on `stream`; calls on one handle must not overlap on the GPU
 * (they share the handle's queue counter).  Each image's output is identical
 * to its output from sobel4_run.
 * Errors: INVALID_ARG (nothing enqueued), OOM (descriptor buffer growth), CUDA.
 */
sobel4_status sobel4_run_batched(sobel4_handle h, const sobel4_image *h_images, int32_t n,
                                 sobel4_border border, sobel4_format fmt, cudaStream_t stream);

/*
 * End-to-end form with HOST buffers (the paper's "runtime including data
 * loading", Table 2): copies h_src to the device, runs, copies the result
 * into h_dst and waits for completion.  Pitches follow sobel4_run.  Device
 * buffers are held by the handle and reused across calls.  Pinned host
 * memory (cudaHostAlloc / cudaHostRegister) gives full link bandwidth;
 * pageable memory works but is slower.  Synchronous.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
sobel4_status sobel4_run_host(sobel4_handle h, const uint8_t *h_src, size_t src_pitch,
                              void *h_dst, size_t dst_pitch, int32_t height, int32_t width,
                              sobel4_border border, sobel4_format fmt);

/* Release the handle (waits for its own internal work only).  NULL is a no-op. */
sobel4_status sobel4_destroy(sobel4_handle h);

/* Static English text for a status code (never NULL). */
const char *sobel4_status_string(sobel4_status s);

/* The cudaError_t of the handle's most recent SOBEL4_ERR_CUDA (0 if none). */
int32_t sobel4_last_cuda_error(sobel4_handle h);

/*
 * Result of the bounded waits inside this handle's kernels.  The TMA-staged
 * kernel waits on shared-memory barriers for its row copies; a wait that runs
 * out (2 s) makes the kernel stop early and set the handle's error word, and
 * the outputs of that launch are then incomplete.  This call synchronises the
 * handle's device, reads and clears the word, and returns TIMEOUT if any wait
 * ran out since the previous call, OK otherwise (CUDA if the device faulted).
 */
sobel4_status sobel4_device_status(sobel4_handle h);

/*
 * Failure injection for tests of the bounded waits: the next single-image
 * launch on this handle that uses TMA staging withholds the row copies of
 * stage `stage` (0-based, 8 rows) of its first work item, so that the warp
 * holding that item waits until its limit (2 s), records the failure and
 * stops; sobel4_device_status then returns TIMEOUT.  The launch's output is
 * incomplete.  No GPU fault is involved and the context stays usable.
 * Errors: INVALID_ARG (h == NULL, stage < 0).
 */
sobel4_status sobel4_inject_stage_loss(sobel4_handle h, int32_t stage);

/*
 * Runtime weights: the generalised operator of Eq. (5) (Section 3.2),
 *   K_x = a (1 n m n 1)^T (-1 -b 0 b 1),  K_y = its transpose,
 *   K_d, K_dt the matching diagonal masks of Eq. (5),
 * replaces the Eq. (3) masks for this handle's later runs (a = 1, b = 2,
 * n = 4, m = 6 restores Eq. 3 and the register-window kernels).  With other
 * weights, single images run on the tensor-core kernel where it applies
 * (VALID, F32, aligned rows, width a multiple of 4) and on the DIRECT kernel
 * otherwise; batches run image by image.  Every weight must be an integer
 * (a a positive integer, b, n, m positive reals).
 * Errors: INVALID_ARG (h == NULL, a weight that is not an integer or exceeds
 * 16 bits, a non-positive parameter), UNSUPPORTED (the largest S = sum of the
 * four squared responses would not fit in int32); later S16X4 runs return
 * UNSUPPORTED when a response can exceed the int16 range.
 */
sobel4_status sobel4_set_weights(sobel4_handle h, double a, double b, double n, double m);

/*
 * Operators (Section 3.1): the four-directional 5x5 of Eq. (3) (the default),
 * the two-directional 5x5 (its K_x and K_y only, S = R_x^2 + R_y^2), and the
 * two-directional 3x3 of Eq. (1)-(2) (whose VALID frame is 1 pixel wide).
 * The two-directional operators run like runtime weights: on the tensor-core
 * kernel where it applies, else on DIRECT; S16X4 writes R_x, R_y and two zero
 * planes.  SOBEL4_OP_4DIR_5X5 restores Eq. (3) (same as sobel4_set_weights
 * with 1, 2, 4, 6).  Errors: INVALID_ARG (h == NULL, unknown operator).
 */
typedef enum {
  SOBEL4_OP_4DIR_5X5 = 0,
  SOBEL4_OP_2DIR_5X5 = 1,
  SOBEL4_OP_2DIR_3X3 = 2
} sobel4_operator;
sobel4_status sobel4_set_operator(sobel4_handle h, int32_t op);

/*
 * Threshold T >= 0 of the EDGE8 output for this handle's later runs
 * (default 128): a pixel is 255 where sqrt(S) >= T.
 * Errors: INVALID_ARG (h == NULL, T negative, not a number, or above 46341).
 */
sobel4_status sobel4_set_threshold(sobel4_handle h, double t);

/* Number of kernels this handle has launched so far (for launch accounting). */
uint64_t sobel4_launch_count(sobel4_handle h);

/* Select the kernel variant for later calls (sobel4_variant); INVALID_ARG if unknown. */
sobel4_status sobel4_set_variant(sobel4_handle h, int32_t variant);

/*
 * Self-check of the magnitude step of Eq. (4) on the device: for every S in
 * [s_begin, s_end) (0 <= s_begin <= s_end; the Eq. (3) operator's whole range
 * of S is [0, 599,270,401), runtime weights may reach up to 2^31 - 2),
 * compares the F32 magnitude with CUDA's IEEE sqrtf((float)S) and the U8
 * magnitude with min(255, round(sqrt(S))); *mismatches receives the number of
 * disagreements (0 expected).  Synchronous; allocates 8 bytes of device
 * memory for the count.  Errors: INVALID_ARG, OOM, CUDA.
 */
sobel4_status sobel4_check_magnitude(sobel4_handle h, int32_t s_begin, int32_t s_end,
                                     uint64_t *mismatches);

/*
 * Allocation-free batched run.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate GPU memory -- plugins inside
 * a host framework that owns every device buffer, services held to a fixed
 * memory budget, latency-critical threads that must not pay for cudaMalloc or
 * cudaFree.  It runs on the CURRENT device, with no handle, and calls no
 * cudaMalloc, cudaFree or other allocating routine.  Its scratch (image
 * descriptors and the work-queue counter) lives in a static device array of
 * SOBEL4_STATIC_SCRATCH_BYTES bytes inside the library, which every GPU that
 * loads the library holds until the process exits.
 *   h_images, n, border, fmt, stream: as for sobel4_run_batched, with
 *   1 <= n <= SOBEL4_STATIC_MAX_IMAGES (a larger n returns UNSUPPORTED) and
 *   fmt F32, U8 or S16X4 (U16 and EDGE8 return UNSUPPORTED).
 * What it enqueues on `stream`: one to three small launches that carry the
 * descriptors in their kernel parameters (the first also zeroes the queue
 * counter), then the lane-copy persistent batched kernel (the batched kernel
 * of the RG_LANECOPY variant) over all n images.  `h_images` is read before
 * the call returns.  Every call looks up the array's device address on the
 * current device; the first call on a device can also load the library's
 * device code there.
 * Every call shares the one array and overwrites it: calls that overlap on
 * the GPU race, so serialise them (for example on one stream).  The call uses
 * about 4 KB of the calling thread's stack.  Results equal
 * sobel4_run_batched's bit for bit.
 * Errors: INVALID_ARG and UNSUPPORTED (nothing enqueued), CUDA.
 */
#define SOBEL4_STATIC_MAX_IMAGES 1024
#define SOBEL4_STATIC_SCRATCH_BYTES (SOBEL4_STATIC_MAX_IMAGES * 64 + 256)
sobel4_status sobel4_run_batched_static(const sobel4_image *h_images, int32_t n,
                                        sobel4_border border, sobel4_format fmt,
                                        cudaStream_t stream);

/*
 * Autotuner: the per-shape form of the paper's block-configuration study
 * (Fig. 5, Section 5.2).  sobel4_tune times, on a height x width image in
 * scratch device buffers it allocates and frees, the tensor-core kernel
 * (where it applies), the TMA-staged register-window kernel at strip heights
 * R = 8, 16, 24 ... 128 (no taller than the image needs) plus its built-in
 * choice, and the lane-copy kernel (2 or 4 columns per thread x R in 8, 16,
 * 32, 64); options that force a variant, columns or R restrict the
 * candidates.  It records the fastest in
 * the handle's table under the bucket (ceil log2 height, ceil log2 width,
 * fmt).  Later sobel4_run calls whose shape falls in that bucket use it.
 * Each candidate is timed as three regions of ten back-to-back launches;
 * *best_us (may be NULL) receives the chosen candidate's time per launch in
 * microseconds (the median of the three regions' means).  On a handle with
 * runtime weights (sobel4_set_weights other than Eq. 3's) it times only the
 * TMA-staged kernel with the weights' coefficients, and answers UNSUPPORTED
 * where those weights do not run on the packed passes (S16X4, the DIRECT
 * variant, weights outside the proven range, the two-directional operators).
 * Synchronous.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA.
 */
sobel4_status sobel4_tune(sobel4_handle h, int32_t height, int32_t width, sobel4_border border,
                          sobel4_format fmt, float *best_us);

/*
 * Autotune the batched kernel on a real batch: the TMA-family batched
 * kernel at strip heights 8, 16, 32, 48, 64, 96, 128 and the lane-copy one
 * (columns per thread 2/4 x strip height 8/16/32 x 2/4/6 CTAs per SM).  Runs
 * sobel4_run_batched repeatedly on `h_images` (their outputs are written)
 * and keeps the fastest for batches of format `fmt`.  Synchronous.  Errors as
 * sobel4_run_batched.
 */
sobel4_status sobel4_tune_batched(sobel4_handle h, const sobel4_image *h_images, int32_t n,
                                  sobel4_border border, sobel4_format fmt, float *best_us);

/* Number of entries in the handle's tuned table. */
int32_t sobel4_tune_entries(sobel4_handle h);

/*
 * The configuration this handle uses for single VALID images of height x
 * width in format fmt whose source and destination rows are 16-byte aligned:
 * *kernel = 2 for the tensor-core kernel, 1 for the TMA-staged register-window
 * kernel, 0 for the lane-copy one; its columns per lane and strip height
 * (tuned if sobel4_tune or a loaded cache covers the shape, else the
 * built-in rule).  Handles that do not run those report 3 for DIRECT (also
 * runtime weights where the tensor-core kernel does not apply) and 4 .. 8
 * for LADDER_SM, LADDER_SM_P, LADDER_RG, LADDER_RG_V1, LADDER_RG_V2, with 1
 * column per lane and the RG ladder's strip height (else 0).
 * Errors: INVALID_ARG.
 */
sobel4_status sobel4_tune_config(sobel4_handle h, int32_t height, int32_t width,
                                 sobel4_format fmt, int32_t *kernel, int32_t *columns_per_lane,
                                 int32_t *rows_per_strip);

/*
 * Write the tuned table to `path` as JSON (written to path.tmp, then renamed
 * over path).  The file records the device name, SM count and library
 * version.  Errors: INVALID_ARG (bad path or write failure).
 */
sobel4_status sobel4_tune_save(sobel4_handle h, const char *path);

/*
 * Merge a table written by sobel4_tune_save into the handle.  A file tuned on
 * another device model returns UNSUPPORTED and changes nothing; a missing,
 * malformed or out-of-range file returns INVALID_ARG and changes nothing.
 * sobel4_create loads the file named by the SOBEL4_TUNE_CACHE environment
 * variable, when set, the same way.
 */
sobel4_status sobel4_tune_load(sobel4_handle h, const char *path);

/*
 * Graph-captured video pipeline: the stream processing the paper proposes for
 * its IO bottleneck (Section 5.2, Section 6).  A pipeline owns `slots` (2..64)
 * frame slots for height x width frames of one border rule and format; each
 * slot has pinned host input and output buffers, device buffers, its own
 * stream and an instantiated CUDA graph of host->device copy and kernel; the
 * kernel stores the result straight into the slot's pinned output (mapped
 * page-locked memory), with no device->host copy.  While one slot's kernel
 * runs, other slots' uploads run.
 * Usage per frame: wait(slot) (its previous frame is done and its output
 * readable), write the frame into the slot's input buffer, submit(slot).
 * Host buffers use the pitches reported by sobel4_pipeline_buffers; S16X4
 * outputs hold 4 planes of `height` rows.  The handle must outlive the
 * pipeline; its kernel configuration at creation time is frozen into the graphs.
 */
typedef struct sobel4_pipeline_ctx *sobel4_pipeline;

/* Errors: INVALID_ARG, OOM, CUDA.  On error *out is NULL. */
sobel4_status sobel4_pipeline_create(sobel4_handle h, int32_t height, int32_t width,
                                     sobel4_border border, sobel4_format fmt, int32_t slots,
                                     sobel4_pipeline *out);

/* The slot's pinned buffers and their row pitches (any pointer may be NULL). */
sobel4_status sobel4_pipeline_buffers(sobel4_pipeline p, int32_t slot, uint8_t **h_in,
                                      void **h_out, size_t *in_pitch, size_t *out_pitch);

/* Launch the slot's graph; INVALID_ARG if the slot's previous frame was not waited for. */
sobel4_status sobel4_pipeline_submit(sobel4_pipeline p, int32_t slot);

/*
 * One frame from caller host buffers: h_in (the frame, height rows at the
 * pipeline's input pitch) is copied to the slot's device buffer and the
 * result goes to h_out (the pipeline's output pitch and planes); NULL keeps
 * the slot's own buffer.  With both NULL (or the slot's own buffers) this is
 * sobel4_pipeline_submit, one graph launch.  Otherwise the slot's stream gets
 * the upload and then either the kernel storing into h_out itself (h_out
 * mapped page-locked memory, as sobel4_host_alloc gives) or a graph of the
 * kernel alone and a download.  h_in should be page-locked for the upload to
 * run asynchronously; both buffers must stay valid until wait(slot) returns.
 * Errors: INVALID_ARG (as submit), CUDA (sobel4_last_cuda_error has the code).
 */
sobel4_status sobel4_pipeline_submit_from(sobel4_pipeline p, int32_t slot, const uint8_t *h_in,
                                          void *h_out);

/* Block until the slot's last submitted frame is complete (OK if none is pending). */
sobel4_status sobel4_pipeline_wait(sobel4_pipeline p, int32_t slot);

/* Wait for all slots and release everything.  NULL is a no-op. */
sobel4_status sobel4_pipeline_destroy(sobel4_pipeline p);

/*
 * Page-locked host memory (cudaHostAlloc, portable to every device) for
 * frames and results that cross the host link, such as a ring of frames fed
 * to sobel4_pipeline_submit_from or the buffers of server requests.  On a
 * Grace host the copy engines stream such memory at the link rate on every
 * pass, where pages locked after allocation (cudaHostRegister) can fall far
 * below it once a ring is larger than the translation caches.  *out receives
 * the buffer, `bytes` long, uninitialised (NULL on error).  Errors:
 * INVALID_ARG (out NULL or bytes 0), OOM, CUDA.
 */
sobel4_status sobel4_host_alloc(size_t bytes, void **out);

/* Release a buffer from sobel4_host_alloc.  NULL is a no-op.  Errors: CUDA. */
sobel4_status sobel4_host_free(void *p);

/*
 * Continuous-batching request server.  A scheduler thread admits submitted
 * requests first-in first-out while a device-memory arena of
 * `memory_budget` bytes (allocated once, at creation) has room for their
 * input (and their output where it is staged, below), uploads them on a copy
 * stream, and packs everything admitted into one persistent batched launch
 * (sobel4_run_batched; at most two batches on the GPU at once, so requests
 * arriving while a batch runs join the next; a batch of up to three runs as
 * sobel4_run launches).  A result buffer that is mapped page-locked host memory
 * (sobel4_host_alloc, cudaHostAlloc, or cudaHostRegister where the device
 * maps it at the same address) with pitch and address multiples of the
 * element size is written by the kernel itself, over the host link; any
 * other result buffer is staged in the arena and downloaded on a third
 * stream.  A completion thread waits on one event per request in order; a
 * request completes when its result is in host memory.  Comparison modes:
 * plain = 1 makes each request its own sobel4_run launch on the same
 * streams; plain = 2 runs one request at a time in arrival order on ONE
 * stream (upload, sobel4_run, download where staged).  Host buffers passed
 * to submit must stay valid, and the result buffer untouched, until wait
 * returns; page-locked input keeps the uploads asynchronous (pageable memory
 * serialises them).  Every result equals sobel4_run's output for that image.
 */
typedef struct sobel4_server_ctx *sobel4_server;

typedef struct {
  int64_t memory_budget; /* device bytes for admitted requests; 0 = 8 GiB */
  int32_t max_batch;     /* images per launch; 0 = 256 */
  int32_t border;        /* sobel4_border of every request */
  int32_t format;        /* sobel4_format of every request */
  int32_t plain;         /* 0 = batched; 1 = one launch per request; 2 = one stream, in order */
} sobel4_server_options;

typedef struct {
  uint64_t submitted, completed, batches, max_batch_seen;
  int64_t device_bytes_in_use, device_bytes_peak;
} sobel4_server_counters;

/* Start a server on the handle's device.  Errors: INVALID_ARG, OOM, CUDA. */
sobel4_status sobel4_server_create(sobel4_handle h, const sobel4_server_options *opt,
                                   sobel4_server *out);

/*
 * Queue one request (host image, host output in the server's format and
 * border).  *ticket identifies it.  Errors: INVALID_ARG, UNSUPPORTED (larger
 * than the whole budget), CUDA (the server has failed).
 */
sobel4_status sobel4_server_submit(sobel4_server s, const uint8_t *h_src, size_t src_pitch,
                                   void *h_dst, size_t dst_pitch, int32_t height, int32_t width,
                                   uint64_t *ticket);

/*
 * Wait for a request (timeout_us < 0: no limit).  On success the output is in
 * h_dst, *latency_us (may be NULL) holds submit-to-completion time, and the
 * ticket is retired.  TIMEOUT if it is still pending (the ticket stays valid).
 */
sobel4_status sobel4_server_wait(sobel4_server s, uint64_t ticket, int64_t timeout_us,
                                 double *latency_us);

/* Counters and the arena's current and peak use. */
sobel4_status sobel4_server_stats(sobel4_server s, sobel4_server_counters *out);

/* Finish every submitted request, stop the scheduler, release the arena. */
sobel4_status sobel4_server_destroy(sobel4_server s);

/* Library version as "major.minor.patch" (static string). */
const char *sobel4_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SOBEL4_H_ */
