// sobel4_launch.h — internal launchers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sobel4.h"
#include "sobel4_device.cuh"

namespace sobel4 {

// RG kernel over one image with nc (2 or 4) columns per lane: CTAs of 4
// independent warps, at most as many as are resident on sm_count SMs, pulling
// items from the device counter pair `pair` (two zero words; the kernel leaves
// them zero again).  No two launches in flight at once may share a pair.
// im.n_seg must be ceil(W / (32 * nc)).
cudaError_t launch_rg_single(const ImageDesc &im, int border, int fmt, int R, int nc,
                             int sm_count, unsigned int *pair, cudaStream_t st);

// Persistent RG kernel over a batch: min(grid, resident CTAs on sm_count SMs)
// CTAs pull warp items from the device counter *d_queue (reset to 0 by the
// caller before the launch).
cudaError_t launch_rg_batched(const ImageDesc *d_descs, int n_img, int64_t total_items,
                              unsigned int *d_queue, int border, int fmt, int R, int nc,
                              int grid, int sm_count, cudaStream_t st);

// TMA-family RG kernel (sobel4_tma.cuh) over one image of any alignment:
// sources whose address and pitch are multiples of 16 bytes (tma_eligible)
// are staged with 2-D tensor copies, others with 1-D bulk copies of each
// row's 16-byte granules.  R must equal tma_round_R(R) (a multiple of the
// kernel's row-step unroll).  One kernel runs (a lean one when every item
// takes the fast path); `pair` points to two zeroed counter words, which the
// kernel leaves zero.  A stage wait that runs out sets bit 0 of *err and the
// kernel returns early.
bool tma_eligible(const uint8_t *src, size_t sp);
int tma_pick_R(int fmt, int sm_count, int32_t H, int32_t W, bool all_fast);
int tma_round_R(int R);
// lose_stage >= 0 (failure injection for tests) withholds that stage's copy
// for the first item, so that one warp's bounded wait runs out.
// cw: runtime-weight coefficients for the packed passes (Coefs, Eq. 5); not
// with S16X4 (INVALID_VALUE).  nullptr: the Eq. (3) passes.
cudaError_t launch_tma_single(const uint8_t *src, size_t sp, void *dst, size_t dp, int32_t H,
                              int32_t W, int border, int fmt, int R, int sm_count,
                              unsigned int *pair, unsigned int *err, cudaStream_t st,
                              int lose_stage = -1, int32_t thr = 0, const Coefs *cw = nullptr);

// The same for an interleaved RGB source (3 bytes per pixel, row pitch sp >=
// 3W, any alignment): the kernel stages RGB rows and turns them into gray
// (Y = (77R + 150G + 29B + 128) >> 8) as it reads them.
cudaError_t launch_tma_single_rgb(const uint8_t *src, size_t sp, void *dst, size_t dp, int32_t H,
                                  int32_t W, int border, int fmt, int R, int sm_count,
                                  unsigned int *pair, unsigned int *err, cudaStream_t st,
                                  int32_t thr = 0);

// TMA-family batches: the host fills one descriptor (tma_batch_desc_bytes
// bytes: with a tensor map for tensor staging, without for bulk staging) per
// image, copies them to the device and launches min(grid, resident CTAs)
// CTAs that pull items from *d_queue (zeroed before the launch).  A launch
// stages every image one way: tensor copies (bulk = false; every source
// tma_eligible) or bulk row copies (bulk = true; any source); R as for
// launch_tma_single.
size_t tma_batch_desc_bytes(bool bulk);
// thr: the EDGE8 threshold on S.  INVALID_VALUE for tensor staging of a
// source that is not tma_eligible.
cudaError_t tma_fill_batch_desc(void *out, bool bulk, const uint8_t *src, size_t sp, void *dst,
                                size_t dp, int32_t H, int32_t W, int R, int64_t item0,
                                int64_t *items, int32_t thr = 0);
// Which batched kernel a batch needs: every item of every image on the fast
// path with vector stores (the lean kernel), every item on the fast path but
// some destination rows not vector-aligned (the fast kernel with split
// stores), or some items on the general path (the kernel that carries both).
// A batch takes the lowest level of its images.
enum BatchFast : int { kBatchGeneral = 0, kBatchFastSplit = 1, kBatchFastVec = 2 };
// d_queue: one zeroed counter; fast: the batch's BatchFast level.
cudaError_t launch_tma_batched(const void *d_descs, int n_img, int64_t total,
                               unsigned int *d_queue, int border, int fmt, int R, int grid,
                               int sm_count, unsigned int *err, cudaStream_t st, int fast,
                               bool bulk);
bool tma_all_fast(int32_t W, int border, int fmt, const uint8_t *src, size_t sp, const void *dst,
                  size_t dp);
// The same with the staging given (bulk: bulk row copies, else tensor copies).
bool tma_all_fast_staged(int32_t W, int border, int fmt, bool bulk, const void *dst, size_t dp);
// One image's BatchFast level under the staging given.
int tma_fast_level(int32_t W, int border, int fmt, bool bulk, const void *dst, size_t dp);
// A 2-D tensor map (uint8 or float32 elements) over `base` with row pitch
// `pitch` bytes, H x W elements, a box of box_w x box_h elements, zero fill,
// and optionally the 128-byte shared-memory swizzle; `map` points to a
// 64-byte aligned CUtensorMap.  base and pitch must be multiples of 16.
cudaError_t tma_encode_2d(void *map, const void *base, bool f32, size_t pitch, int32_t H,
                          int32_t W, int box_w, int box_h, bool swizzle128);

// Tensor-core kernel (sobel4_tc.cuh): VALID, F32, a width that is a multiple
// of 4, a source that is tma_eligible and a destination whose address and
// pitch are multiples of 16 bytes (tc_eligible).  A wait that runs out sets bit 0 of *err;
// lose_tile >= 0 (failure injection for tests) withholds the copy of that
// CTA-local tile so that the waits run out.
bool tc_eligible(const uint8_t *src, size_t sp, const void *dst, size_t dp, int32_t H, int32_t W,
                 int border, int fmt);
// masks = nullptr: Eq. (3).
cudaError_t launch_tc_single(const uint8_t *src, size_t sp, void *dst, size_t dp, int32_t H,
                             int32_t W, int border, int fmt, int sm_count, unsigned int *err,
                             cudaStream_t st, int lose_tile = -1, const Masks4 *masks = nullptr,
                             int radius = 2);

// DIRECT kernel (one thread per output pixel); masks = nullptr: Eq. (3);
// radius: the masks' support radius (VALID leaves a frame that wide at 0).
cudaError_t launch_direct(const ImageDesc &im, int border, int fmt, const Masks4 *masks,
                          int radius, int32_t thr, cudaStream_t st);

// The paper's kernel ladder (Table 1), Eq. (3) masks only: shared-memory tile,
// the same with the next tile prefetched, and the plain register window with
// the diagonals direct (RG), through K_d+ (RG-v1) and fully decomposed
// (RG-v2); `rows`: output rows per warp strip of the RG kernels.
enum LadderKind : int { kLadderSM = 0, kLadderSMP, kLadderRG, kLadderRGv1, kLadderRGv2 };
cudaError_t launch_ladder(const ImageDesc &im, int border, int fmt, int kind, int rows,
                          int32_t thr, cudaStream_t st);

// Masks of the operators besides the four-directional 5x5: op 1 = the
// two-directional 5x5 (K_x, K_y of Eq. 3), op 2 = the two-directional 3x3 of
// Eq. (1) centred in the 5x5 grid; diagonal masks zero.  Returns the support
// radius (2 or 1), or 0 for an unknown op.
int operator_masks(int op, Masks4 *out);

// The four masks of the generalised operator (Eq. 5) for parameters a, b, n,
// m, built from its factored rows; false if a weight is not an integer or
// does not fit in 16 bits.  (a, b, n, m) = (1, 2, 4, 6) gives Eq. (3).
bool eq5_masks(double a, double b, double n, double m, Masks4 *out);

// Self-check of the magnitude step over S in [s0, s1); mismatches added to *d_bad.
cudaError_t launch_check_magnitude(int64_t s0, int64_t s1, unsigned long long *d_bad, int grid,
                                   cudaStream_t st);

// Handle internals shared with the pipeline and server translation units.
struct HandleInfo {
  int device;
};
__attribute__((visibility("hidden"))) HandleInfo handle_info(sobel4_handle h);
__attribute__((visibility("hidden"))) void note_launches(sobel4_handle h, int64_t delta);
// Records a failed CUDA call as the handle's last error (sobel4_last_cuda_error).
__attribute__((visibility("hidden"))) void note_cuda_error(sobel4_handle h, cudaError_t e);
// sobel4_run with caller-owned RG counters (four zeroed words in device
// memory: a launch may use two counter pairs; nullptr takes the handle's next
// block).  A captured graph must own its
// pair, because every replay of the graph reuses it.
__attribute__((visibility("hidden"))) sobel4_status run_with_pair(
    sobel4_handle h, const uint8_t *d_src, size_t src_pitch, void *d_dst, size_t dst_pitch,
    int32_t height, int32_t width, int border, int fmt, cudaStream_t stream, unsigned int *pair);

// True where a kernel can store a result of `rows` rows of `row_bytes` bytes
// at `pitch` straight into host buffer p: the first and the last byte it
// writes are page-locked host memory that the device maps at the same
// addresses, and p and pitch are multiples of the element size `elem`.
__attribute__((visibility("hidden"))) bool host_kernel_writable(const void *p, size_t pitch,
                                                                size_t rows, size_t row_bytes,
                                                                size_t elem);

// Make `dev` current for the lifetime of the guard.
class DeviceScope {
 public:
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
    if (prev_ != dev) cudaSetDevice(dev);
  }
  ~DeviceScope() {
    int cur = -1;
    if (prev_ >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev_) cudaSetDevice(prev_);
  }

 private:
  int prev_ = -1;
};

}  // namespace sobel4
