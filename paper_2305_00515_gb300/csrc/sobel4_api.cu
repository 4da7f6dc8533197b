// sobel4_api.cu — the C ABI of include/sobel4.h: argument validation, handle
// state, batch descriptor staging and kernel selection.  Every step of the
// operator itself runs in the kernels of sobel4_rg_*.cu / sobel4_direct.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "sobel4.h"
#include "sobel4_launch.h"

namespace sobel4 {
cudaError_t launch_rg_single_f32(const ImageDesc &, int, int, int, int, unsigned int *,
                                 cudaStream_t);
cudaError_t launch_rg_single_u8(const ImageDesc &, int, int, int, int, unsigned int *,
                                cudaStream_t);
cudaError_t launch_rg_single_s16(const ImageDesc &, int, int, int, int, unsigned int *,
                                 cudaStream_t);
cudaError_t launch_rg_batched_f32(const ImageDesc *, int, int64_t, unsigned int *, int, int, int,
                                  int, int, cudaStream_t);
cudaError_t launch_rg_batched_u8(const ImageDesc *, int, int64_t, unsigned int *, int, int, int,
                                 int, int, cudaStream_t);
cudaError_t launch_rg_batched_s16(const ImageDesc *, int, int64_t, unsigned int *, int, int, int,
                                  int, int, cudaStream_t);

cudaError_t launch_rg_single(const ImageDesc &im, int border, int fmt, int R, int nc,
                             int sm_count, unsigned int *pair, cudaStream_t st) {
  switch (fmt) {
    case kF32: return launch_rg_single_f32(im, border, R, nc, sm_count, pair, st);
    case kU8: return launch_rg_single_u8(im, border, R, nc, sm_count, pair, st);
    default: return launch_rg_single_s16(im, border, R, nc, sm_count, pair, st);
  }
}

cudaError_t launch_rg_batched(const ImageDesc *d, int n, int64_t total, unsigned int *q,
                              int border, int fmt, int R, int nc, int grid, int sm_count,
                              cudaStream_t st) {
  switch (fmt) {
    case kF32: return launch_rg_batched_f32(d, n, total, q, border, R, nc, grid, sm_count, st);
    case kU8: return launch_rg_batched_u8(d, n, total, q, border, R, nc, grid, sm_count, st);
    default: return launch_rg_batched_s16(d, n, total, q, border, R, nc, grid, sm_count, st);
  }
}
}  // namespace sobel4

using namespace sobel4;

namespace {

#ifndef SOBEL4_DEFAULT_NC
#define SOBEL4_DEFAULT_NC 4
#endif

constexpr int kSlots = 4;           // batch descriptor slots in flight per handle
constexpr int kQueuePairs = 256;    // single-image work-queue counter blocks per handle
constexpr int kQueueWords = 4;      // words per block: one counter pair, padded to 16 bytes
constexpr int kDefaultNC = SOBEL4_DEFAULT_NC;  // RG columns per lane unless the handle says otherwise
constexpr int kDefaultR = 16;       // RG strip height for large images (measured best on 8192^2)
constexpr int kBatchR = 16;         // RG strip height for batches
constexpr int kMaxSide = 1 << 28;   // largest accepted height or width
constexpr uint64_t kMaxPitch = (1ull << 31) - 1;

struct BatchSlot {
  ImageDesc *h_desc = nullptr;      // pinned host staging (lane-copy images)
  ImageDesc *d_desc = nullptr;
  unsigned char *h_tma = nullptr;   // pinned host staging (TMA descriptors)
  unsigned char *d_tma = nullptr;
  unsigned int *d_queue = nullptr;  // work-queue heads: word 0 lane-copy, word 32 TMA
  int cap = 0;
  cudaEvent_t done = nullptr;
  bool pending = false;
};

// Descriptor upload through kernel parameters: each launch carries up to
// kParamChunk bytes of host data in its (large) parameter block and writes
// them to device memory; the first also zeroes the slot's 64 work-queue
// words.  Parameters travel with the launch command, so the upload never waits
// behind bulk copies that the caller has queued on the copy engines (a serving
// loop uploads the next requests while a batch runs).
constexpr int kParamChunk = 31744;  // bytes per launch (the limit is 32764 with the other arguments)
struct ParamChunk {
  uint4 w[kParamChunk / 16];
};

__global__ void param_copy_kernel(const __grid_constant__ ParamChunk chunk, uint4 *dst, int n16,
                                  unsigned int *queue) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  if (queue && t < 64) queue[t] = 0u;
  for (int i = t; i < n16; i += stride) dst[i] = chunk.w[i];
}

ParamChunk g_param_chunk;  // host staging of one launch's parameter block
std::mutex g_param_mu;

// Uploads `bytes` (a multiple of 16) to device `dst`: fill(buf, off, n) writes
// bytes [off, off + n) of the data into buf, one launch's block at a time.
// Zeroes `queue` with the first launch when it is not null.
template <class Fill>
cudaError_t param_upload_fill(size_t bytes, void *dst, unsigned int *queue, cudaStream_t st,
                              Fill fill) {
  std::lock_guard<std::mutex> lock(g_param_mu);
  size_t off = 0;
  do {
    const size_t n = std::min(bytes - off, (size_t)kParamChunk);
    if (n) fill((uint8_t *)&g_param_chunk, off, n);
    (void)cudaGetLastError();
    param_copy_kernel<<<2, 256, 0, st>>>(g_param_chunk, (uint4 *)((uint8_t *)dst + off),
                                         (int)(n / 16), queue);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    queue = nullptr;
    off += n;
  } while (off < bytes);
  return cudaSuccess;
}

// Uploads `bytes` (a multiple of 16) from host `src` to device `dst`.  Zeroes
// `queue` with the first launch when it is not null.
cudaError_t param_upload(const void *src, void *dst, size_t bytes, unsigned int *queue,
                         cudaStream_t st) {
  return param_upload_fill(bytes, dst, queue, st, [src](uint8_t *buf, size_t off, size_t n) {
    memcpy(buf, (const uint8_t *)src + off, n);
  });
}

size_t elem_size(int fmt) { return fmt == kF32 ? 4 : ((fmt == kU8 || fmt == kEdge8) ? 1 : 2); }
int planes(int fmt) { return fmt == kS16x4 ? 4 : 1; }

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
    if (prev_ != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev_ >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev_) cudaSetDevice(prev_);
  }

 private:
  int prev_ = -1;
};

}  // namespace

// One autotuned configuration: kind 0 = single image bucket (hb, wb) =
// (ceil log2 height, ceil log2 width); kind 1 = batches of format fmt.
struct TuneEntry {
  int kind, hb, wb, fmt;
  int nc, R, ctas;
  float us;
  int kernel;  // 0 = lane-copy staging, 1 = TMA staging, 2 = tensor-core kernel (single images)
};

struct sobel4_ctx {
  int device = 0;
  int sm_count = 0;
  int variant = SOBEL4_VARIANT_AUTO;
  int rows_per_strip = 0;
  int ctas_per_sm = 4;
  int nc = kDefaultNC;  // RG columns per lane (2 or 4)
  bool nc_forced = false;  // set by the creation options
  uint64_t launches = 0;
  int32_t last_err = 0;
  BatchSlot slots[kSlots];
  int next_slot = 0;
  // kQueuePairs zeroed counter pairs, handed to single-image launches in turn;
  // each launch leaves its pair zero again when it completes.
  unsigned int *d_pairs = nullptr;
  uint32_t next_pair = 0;
  unsigned int *d_err = nullptr;  // bit 0: a bounded wait in a kernel ran out (inside d_pairs)
  int lose_stage = -1;            // failure injection for the next TMA-staged launch
  bool custom = false;            // runtime masks (Eq. 5 weights, other operators) replace Eq. (3)
  int radius = 2;                 // support radius of the masks (VALID frame width)
  int32_t thr = 16384;            // EDGE8 threshold on S (T = 128 by default)
  bool custom_s16_ok = true;      // every response fits the S16X4 planes
  bool factored = false;          // runtime weights run on the packed passes (coefs)
  Coefs coefs{};
  Masks4 masks{};
  cudaStream_t own_stream = nullptr;
  uint8_t *d_in = nullptr;
  size_t d_in_bytes = 0;
  uint8_t *d_out = nullptr;
  size_t d_out_bytes = 0;
  // Banded host-buffer runs: copy streams, per-band events, output ring.
  cudaStream_t h2d_stream = nullptr, d2h_stream[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> band_events;  // 3 per band: input landed, computed, downloaded
  uint8_t *d_ring = nullptr;
  size_t d_ring_bytes = 0;
  std::vector<TuneEntry> tuned;
  char device_name[256] = {0};
  bool autotune = false;          // tune each new single-image shape bucket on first use
  std::string cache_path;         // tuning cache rewritten after each automatic tune
  std::vector<uint32_t> autotried;  // buckets the automatic tune has already handled
};

namespace sobel4 {
HandleInfo handle_info(sobel4_handle h) { return HandleInfo{h->device}; }
void note_launches(sobel4_handle h, int64_t delta) { h->launches += (uint64_t)delta; }
void note_cuda_error(sobel4_handle h, cudaError_t e) {
  if (h) h->last_err = (int32_t)e;
}
bool host_kernel_writable(const void *p, size_t pitch, size_t rows, size_t row_bytes,
                          size_t elem) {
  if (!p || !rows || !row_bytes || (uintptr_t)p % elem || pitch % elem || pitch > kMaxPitch)
    return false;
  const char *ends[2] = {(const char *)p, (const char *)p + pitch * (rows - 1) + row_bytes - 1};
  for (const char *q : ends) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
      (void)cudaGetLastError();
      return false;
    }
    if (a.type != cudaMemoryTypeHost || a.devicePointer != (const void *)q) return false;
  }
  return true;
}
}  // namespace sobel4

namespace {

sobel4_status cuda_fail(sobel4_ctx *h, cudaError_t e) {
  if (h) h->last_err = (int32_t)e;
  (void)cudaGetLastError();  // a failed call must not be reported again by a later launch
  return e == cudaErrorMemoryAllocation ? SOBEL4_ERR_OOM : SOBEL4_ERR_CUDA;
}

bool valid_enum(int border, int fmt) {
  return border >= SOBEL4_BORDER_VALID && border <= SOBEL4_BORDER_CONSTANT0 &&
         fmt >= SOBEL4_OUT_F32 && fmt <= SOBEL4_OUT_EDGE8;
}

// Shape and pitch rules shared by every entry point (pointers checked separately).
bool valid_shape(size_t src_pitch, size_t dst_pitch, int32_t H, int32_t W, int border, int fmt) {
  if (!valid_enum(border, fmt)) return false;
  if (H < 1 || W < 1 || H > kMaxSide || W > kMaxSide) return false;
  if (border == SOBEL4_BORDER_REFLECT101 && (H < 3 || W < 3)) return false;
  if (src_pitch < (size_t)W || src_pitch > kMaxPitch) return false;
  if (dst_pitch < (size_t)W * elem_size(fmt) || dst_pitch > kMaxPitch) return false;
  if (fmt == kF32 && dst_pitch % 4) return false;
  if ((fmt == kS16x4 || fmt == kU16) && dst_pitch % 2) return false;
  return true;
}

bool valid_dst_ptr(const void *dst, int fmt) {
  if (!dst) return false;
  if (fmt == kF32 && ((uintptr_t)dst % 4)) return false;
  if ((fmt == kS16x4 || fmt == kU16) && ((uintptr_t)dst % 2)) return false;
  return true;
}

// Byte ranges [begin, end) touched by one image's input and output.
void ranges(const uint8_t *src, size_t sp, const void *dst, size_t dp, int32_t H, int32_t W,
            int fmt, uintptr_t r[4]) {
  r[0] = (uintptr_t)src;
  r[1] = (uintptr_t)src + (uintptr_t)(H - 1) * sp + (uintptr_t)W;
  r[2] = (uintptr_t)dst;
  r[3] = (uintptr_t)dst + (uintptr_t)(planes(fmt) * (size_t)H - 1) * dp +
         (uintptr_t)W * elem_size(fmt);
}

bool overlaps(uintptr_t a0, uintptr_t a1, uintptr_t b0, uintptr_t b1) { return a0 < b1 && b0 < a1; }

int seg_cols(int nc) { return 32 * nc; }

int pick_R(const sobel4_ctx *h, int32_t H, int32_t W) {
  if (h->rows_per_strip > 0) return h->rows_per_strip;
  const int64_t n_seg = (W + seg_cols(h->nc) - 1) / seg_cols(h->nc);  // heuristic at the default NC
  const int64_t target = 2ll * h->sm_count * h->ctas_per_sm * kWarpsPerCta;
  int R = kDefaultR;
  while (R > 4 && n_seg * ((H + 2 * R - 1) / (2 * R)) < target) R /= 2;
  return R;
}

int ceil_log2(int64_t v) {
  int b = 0;
  while ((int64_t(1) << b) < v) ++b;
  return b;
}

const TuneEntry *find_tuned(const sobel4_ctx *h, int kind, int32_t H, int32_t W, int fmt) {
  const int hb = kind == 0 ? ceil_log2(H) : 0, wb = kind == 0 ? ceil_log2(W) : 0;
  for (const TuneEntry &t : h->tuned)
    if (t.kind == kind && t.hb == hb && t.wb == wb && t.fmt == fmt) return &t;
  return nullptr;
}

// The RG configuration for one image: which kernel family (the TMA family
// stages any source: tensor copies for 16-byte aligned rows, bulk row copies
// otherwise), columns per lane and strip height.  Explicit options first,
// then the tuned table, then the heuristics.
void rg_config(const sobel4_ctx *h, const uint8_t *src, size_t sp, const void *dst, size_t dp,
               int32_t H, int32_t W, int border, int fmt, bool *use_tma, int *nc, int *R) {
  const TuneEntry *t = find_tuned(h, 0, H, W, fmt);
  // U16 and EDGE8 exist on the TMA family only (no lane-copy instantiation).
  *use_tma = fmt == kU16 || fmt == kEdge8 ||
             (h->variant != SOBEL4_VARIANT_RG_LANECOPY && !h->nc_forced && !(t && t->kernel == 0));
  if (*use_tma) {
    *nc = 4;
    if (h->rows_per_strip > 0) *R = tma_round_R(h->rows_per_strip);
    else if (t && t->kernel == 1) *R = t->R;
    else *R = tma_pick_R(fmt, h->sm_count, H, W, tma_all_fast(W, border, fmt, src, sp, dst, dp));
    return;
  }
  const bool lane_entry = t && t->kernel == 0;
  *nc = h->nc_forced ? h->nc : (lane_entry ? t->nc : h->nc);
  if (h->rows_per_strip > 0) *R = h->rows_per_strip;
  else if (lane_entry) *R = t->R;
  else *R = pick_R(h, H, W);
}

// The tensor-core kernel serves the images it covers on TC handles, and on
// AUTO handles without register-window options where the tuned table names it
// for the shape.
bool use_tc(const sobel4_ctx *h, const uint8_t *src, size_t sp, const void *dst, size_t dp,
            int32_t H, int32_t W, int border, int fmt) {
  if (!tc_eligible(src, sp, dst, dp, H, W, border, fmt)) return false;
  if (h->variant == SOBEL4_VARIANT_TC) return true;
  if (h->variant != SOBEL4_VARIANT_AUTO || h->nc_forced || h->rows_per_strip > 0) return false;
  const TuneEntry *t = find_tuned(h, 0, H, W, fmt);
  return t && t->kernel == 2;
}

int pow2_align(uintptr_t v) {
  int a = 1;
  while (a < 16 && v % (uintptr_t)(2 * a) == 0) a *= 2;
  return a;
}

ImageDesc make_desc(const uint8_t *src, size_t sp, void *dst, size_t dp, int32_t H, int32_t W,
                    int R, int nc) {
  ImageDesc d;
  memset(&d, 0, sizeof(d));
  d.src = src;
  d.dst = dst;
  d.sp = sp;
  d.dp = dp;
  d.H = H;
  d.W = W;
  d.n_seg = (W + seg_cols(nc) - 1) / seg_cols(nc);
  d.n_band = (H + 2 * R - 1) / (2 * R);
  d.item0 = 0;
  d.src_aligned = ((uintptr_t)src % 16 == 0 && sp % 16 == 0) ? 16
                  : (((uintptr_t)src % 4 == 0 && sp % 4 == 0) ? 4 : 1);
  d.dst_align = pow2_align((uintptr_t)dst | (uintptr_t)dp);
  return d;
}

unsigned int *next_pair(sobel4_ctx *h) {
  return h->d_pairs + kQueueWords * (h->next_pair++ % (uint32_t)kQueuePairs);
}

// pair: the RG kernel's counter pair, or nullptr for the handle's next one.
// The paper's kernel ladder (variants LADDER_*): one launch per image.
bool is_ladder(int variant) {
  return variant >= SOBEL4_VARIANT_LADDER_SM && variant <= SOBEL4_VARIANT_LADDER_RG_V2;
}
// Output rows per warp strip of the ladder's RG kernels: up to 64, fewer
// where that leaves under 16 warps per SM (small images).
int ladder_rows(int32_t H, int32_t W, int sm_count) {
  const int64_t cols = (W + 27) / 28, target = (int64_t)sm_count * 16;
  const int64_t rows = (int64_t)H * cols / std::max<int64_t>(1, target);
  return (int)std::max<int64_t>(8, std::min<int64_t>(64, rows));
}

sobel4_status launch_one(sobel4_ctx *h, const uint8_t *src, size_t sp, void *dst, size_t dp,
                         int32_t H, int32_t W, int border, int fmt, cudaStream_t stream,
                         unsigned int *pair = nullptr) {
  cudaError_t e;
  if (h->custom) {
    // Runtime weights: the packed register-window passes with the weights'
    // coefficients where sobel4_set_weights proved them exact, else the
    // tensor-core kernel where it applies, else DIRECT.
    if (fmt == kS16x4 && !h->custom_s16_ok) return SOBEL4_ERR_UNSUPPORTED;
    if (h->factored && fmt != kS16x4 && h->variant != SOBEL4_VARIANT_DIRECT) {
      int nc, R;
      bool use_tma;
      rg_config(h, src, sp, dst, dp, H, W, border, fmt, &use_tma, &nc, &R);
      if (!use_tma)
        R = tma_pick_R(fmt, h->sm_count, H, W, tma_all_fast(W, border, fmt, src, sp, dst, dp));
      e = launch_tma_single(src, sp, dst, dp, H, W, border, fmt, tma_round_R(R), h->sm_count,
                            pair ? pair : next_pair(h), h->d_err, stream, h->lose_stage, h->thr,
                            &h->coefs);
      h->lose_stage = -1;
    } else if (h->variant != SOBEL4_VARIANT_DIRECT &&
               tc_eligible(src, sp, dst, dp, H, W, border, fmt)) {
      e = launch_tc_single(src, sp, dst, dp, H, W, border, fmt, h->sm_count, h->d_err, stream,
                           h->lose_stage, &h->masks, h->radius);
      h->lose_stage = -1;
    } else {
      const ImageDesc im = make_desc(src, sp, dst, dp, H, W, 1, h->nc);
      e = launch_direct(im, border, fmt, &h->masks, h->radius, h->thr, stream);
    }
  } else if (h->variant == SOBEL4_VARIANT_DIRECT) {
    const ImageDesc im = make_desc(src, sp, dst, dp, H, W, 1, h->nc);
    e = launch_direct(im, border, fmt, nullptr, 2, h->thr, stream);
  } else if (is_ladder(h->variant)) {
    const ImageDesc im = make_desc(src, sp, dst, dp, H, W, 1, h->nc);
    e = launch_ladder(im, border, fmt, h->variant - SOBEL4_VARIANT_LADDER_SM,
                      h->rows_per_strip > 0 ? h->rows_per_strip : ladder_rows(H, W, h->sm_count),
                      h->thr, stream);
  } else if (use_tc(h, src, sp, dst, dp, H, W, border, fmt)) {
    e = launch_tc_single(src, sp, dst, dp, H, W, border, fmt, h->sm_count, h->d_err, stream,
                         h->lose_stage);
    h->lose_stage = -1;
  } else {
    int nc, R;
    bool use_tma;
    rg_config(h, src, sp, dst, dp, H, W, border, fmt, &use_tma, &nc, &R);
    if (use_tma) {
      e = launch_tma_single(src, sp, dst, dp, H, W, border, fmt, R, h->sm_count,
                            pair ? pair : next_pair(h), h->d_err, stream, h->lose_stage, h->thr);
      h->lose_stage = -1;
    } else {
      const ImageDesc im = make_desc(src, sp, dst, dp, H, W, R, nc);
      e = launch_rg_single(im, border, fmt, R, nc, h->sm_count, pair ? pair : next_pair(h),
                           stream);
    }
  }
  if (e != cudaSuccess) return cuda_fail(h, e);
  h->launches += 1;
  return SOBEL4_OK;
}

// (Re)allocates a batch slot's descriptor buffers for `cap` images.  Handles
// start with kInitialSlotCap so that batches of ordinary size never allocate
// (freeing device memory waits for the whole device, which a serving loop
// must not do between batches).
constexpr int kInitialSlotCap = 256;

cudaError_t grow_slot(BatchSlot &slot, int cap) {
  if (slot.h_desc) cudaFreeHost(slot.h_desc);
  if (slot.d_desc) cudaFree(slot.d_desc);
  if (slot.h_tma) cudaFreeHost(slot.h_tma);
  if (slot.d_tma) cudaFree(slot.d_tma);
  slot.h_desc = nullptr;
  slot.d_desc = nullptr;
  slot.h_tma = nullptr;
  slot.d_tma = nullptr;
  slot.cap = 0;
  const size_t tb = std::max(tma_batch_desc_bytes(false), tma_batch_desc_bytes(true)) * cap;
  cudaError_t e = cudaHostAlloc((void **)&slot.h_desc, sizeof(ImageDesc) * cap, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaMalloc((void **)&slot.d_desc, sizeof(ImageDesc) * cap);
  if (e == cudaSuccess) e = cudaHostAlloc((void **)&slot.h_tma, tb, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaMalloc((void **)&slot.d_tma, tb);
  if (e == cudaSuccess && !slot.d_queue) e = cudaMalloc((void **)&slot.d_queue, 256);
  if (e == cudaSuccess) slot.cap = cap;
  return e;
}

void free_slot(BatchSlot &s) {
  if (s.done && s.pending) cudaEventSynchronize(s.done);
  if (s.h_desc) cudaFreeHost(s.h_desc);
  if (s.d_desc) cudaFree(s.d_desc);
  if (s.h_tma) cudaFreeHost(s.h_tma);
  if (s.d_tma) cudaFree(s.d_tma);
  if (s.d_queue) cudaFree(s.d_queue);
  if (s.done) cudaEventDestroy(s.done);
  s = BatchSlot();
}

}  // namespace

extern "C" {

const char *sobel4_version(void) { return "0.1.0"; }

const char *sobel4_status_string(sobel4_status s) {
  switch (s) {
    case SOBEL4_OK: return "success";
    case SOBEL4_ERR_INVALID_ARG: return "invalid argument";
    case SOBEL4_ERR_UNSUPPORTED: return "unsupported request";
    case SOBEL4_ERR_OOM: return "out of memory";
    case SOBEL4_ERR_CUDA: return "CUDA error";
    case SOBEL4_ERR_TIMEOUT: return "timeout";
  }
  return "unknown status";
}

sobel4_status sobel4_create(sobel4_handle *out, int32_t device, const sobel4_options *opt) {
  if (!out) return SOBEL4_ERR_INVALID_ARG;
  *out = nullptr;
  if (opt && (opt->autotune < 0 || opt->autotune > 1 ||
              opt->variant < 0 || opt->variant > SOBEL4_VARIANT_LADDER_RG_V2 || opt->rows_per_strip < 0 ||
              opt->rows_per_strip > 4096 || opt->persistent_ctas_per_sm < 0 ||
              opt->persistent_ctas_per_sm > 64 ||
              (opt->columns_per_lane != 0 && opt->columns_per_lane != 2 &&
               opt->columns_per_lane != 4)))
    return SOBEL4_ERR_INVALID_ARG;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return SOBEL4_ERR_CUDA;
  if (device < 0 || device >= count) return SOBEL4_ERR_INVALID_ARG;
  DeviceGuard g(device);
  sobel4_ctx *h = new (std::nothrow) sobel4_ctx();
  if (!h) return SOBEL4_ERR_OOM;
  h->device = device;
  e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) {
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e == cudaSuccess) snprintf(h->device_name, sizeof(h->device_name), "%s", prop.name);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
  // kQueuePairs counter pairs, then the error word (own 256-byte line).
  const size_t pair_bytes = sizeof(unsigned int) * kQueueWords * kQueuePairs + 256;
  if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_pairs, pair_bytes);
  if (e == cudaSuccess) e = cudaMemset(h->d_pairs, 0, pair_bytes);
  if (e == cudaSuccess) h->d_err = h->d_pairs + kQueueWords * kQueuePairs;
  for (int i = 0; i < kSlots && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&h->slots[i].done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = grow_slot(h->slots[i], kInitialSlotCap);
  }
  if (e != cudaSuccess) {
    sobel4_destroy(h);
    return SOBEL4_ERR_CUDA;
  }
  if (opt) {
    h->variant = opt->variant;
    h->rows_per_strip = opt->rows_per_strip;
    if (opt->persistent_ctas_per_sm > 0) h->ctas_per_sm = opt->persistent_ctas_per_sm;
    if (opt->columns_per_lane != 0) {
      h->nc = opt->columns_per_lane;
      h->nc_forced = true;
    }
    h->autotune = opt->autotune == 1;
    if (opt->cache_path && *opt->cache_path) h->cache_path = opt->cache_path;
  }
  const char *cache = h->cache_path.empty() ? getenv("SOBEL4_TUNE_CACHE") : h->cache_path.c_str();
  if (cache && *cache) sobel4_tune_load(h, cache);  // a missing or foreign cache is ignored
  *out = h;
  return SOBEL4_OK;
}

sobel4_status sobel4_destroy(sobel4_handle h) {
  if (!h) return SOBEL4_OK;
  DeviceGuard g(h->device);
  for (int i = 0; i < kSlots; ++i) free_slot(h->slots[i]);
  if (h->own_stream) {
    cudaStreamSynchronize(h->own_stream);
    cudaStreamDestroy(h->own_stream);
  }
  if (h->h2d_stream) {
    cudaStreamSynchronize(h->h2d_stream);
    cudaStreamDestroy(h->h2d_stream);
  }
  for (cudaStream_t st : h->d2h_stream)
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  for (cudaEvent_t ev : h->band_events) cudaEventDestroy(ev);
  if (h->d_in) cudaFree(h->d_in);
  if (h->d_out) cudaFree(h->d_out);
  if (h->d_ring) cudaFree(h->d_ring);
  if (h->d_pairs) cudaFree(h->d_pairs);
  delete h;
  return SOBEL4_OK;
}

int32_t sobel4_last_cuda_error(sobel4_handle h) { return h ? h->last_err : 0; }

sobel4_status sobel4_inject_stage_loss(sobel4_handle h, int32_t stage) {
  if (!h || stage < 0) return SOBEL4_ERR_INVALID_ARG;
  h->lose_stage = stage;
  return SOBEL4_OK;
}

}  // extern "C"

namespace {

// The largest S the F32 magnitude (magnitude_newton) is checked for,
// exhaustively, by the self-check (tests/test_gpu_sqrt.py): all of int32's
// non-negative range but its last value.
constexpr double kMagnitudeCheckedMax = 2147483646.0;

// The runtime-weight passes (column_step_w) for Eq. (5) weights: the integer
// coefficients, or false where a coefficient is not an integer, where the
// masks the passes imply differ from `mk`, or where a returned sum (R_x, R_y,
// P = K_d+ response, M = K_d- response) could leave (-2^15, 2^15), the range
// of a packed half.
bool factored_coefs(double a, double b, double n, double m, const Masks4 &mk, Coefs *out) {
  const double v[20] = {a,         a * b,         n,           m,           a * m,
                        a * (n + b), 2 * a,       a * (n - b), a * m * b,   2 * a * n * b,
                        a * m,     a * (n - b),   a * (n + b), a * m * b,   2 * a,
                        2 * a * n * b, n,         m,           a * b,       a};
  int32_t c[20];
  for (int i = 0; i < 20; ++i) {
    const double r = std::nearbyint(v[i]);
    if (std::fabs(v[i] - r) > 1e-9 || std::fabs(r) > 32767) return false;
    c[i] = (int32_t)r;
  }
  Coefs k = {c[0],  c[1],  c[2],  c[3],  c[4],  c[5],  c[6],  c[7],  c[8],  c[9],
             c[10], c[11], c[12], c[13], c[14], c[15], c[16], c[17], c[18], c[19],
             -c[18], -c[19]};
  // The masks the passes compute, tap by tap (rows i, columns j of p).
  const int64_t hd[5] = {-k.hdE, -k.hdD, 0, k.hdD, k.hdE};
  const int64_t hs[5] = {1, k.hsB, k.hsC, k.hsB, 1};
  const int64_t xv[5] = {1, k.xv1, k.xv2, k.xv1, 1};
  const int64_t yv[5] = {-k.yv2, -k.yv1, 0, k.yv1, k.yv2};
  const int64_t q0[5] = {k.q0A, k.q0B, k.q0C, k.q0B, k.q0A};
  const int64_t q1[5] = {k.q1A, k.q1B, k.q1C, k.q1B, k.q1A};
  const int64_t r0[5] = {-k.r0E, -k.r0D, 0, k.r0D, k.r0E};
  const int64_t r1[5] = {-k.r1E, -k.r1D, 0, k.r1D, k.r1E};
  const int64_t r2[5] = {-k.r2E, -k.r2D, 0, k.r2D, k.r2E};
  const int64_t *prow[5] = {q0, q1, nullptr, q1, q0};
  const int64_t psgn[5] = {-1, -1, 0, 1, 1};
  const int64_t *mrow[5] = {r0, r1, r2, r1, r0};
  int64_t pos[4] = {0, 0, 0, 0}, neg[4] = {0, 0, 0, 0};  // of R_x, R_y, P, M
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      const int64_t kx = xv[i] * hd[j], ky = yv[i] * hs[j];
      const int64_t kp = prow[i] ? psgn[i] * prow[i][j] : 0, km = mrow[i][j];
      if ((kp + km) % 2 != 0 || kx != mk.w[0][i][j] || ky != mk.w[1][i][j] ||
          (kp + km) / 2 != mk.w[2][i][j] || (kp - km) / 2 != mk.w[3][i][j])
        return false;
      const int64_t w[4] = {kx, ky, kp, km};
      for (int q = 0; q < 4; ++q) (w[q] > 0 ? pos[q] : neg[q]) += w[q] > 0 ? w[q] : -w[q];
    }
  for (int q = 0; q < 4; ++q)
    if (255 * std::max(pos[q], neg[q]) > 32767) return false;
  *out = k;
  return true;
}

}  // namespace

extern "C" {

sobel4_status sobel4_set_weights(sobel4_handle h, double a, double b, double n, double m) {
  if (!h) return SOBEL4_ERR_INVALID_ARG;
  Masks4 mk;
  if (!eq5_masks(a, b, n, m, &mk)) return SOBEL4_ERR_INVALID_ARG;
  // Largest |R_k| = 255 x (sum of the positive weights of mask k) (every mask
  // sums to zero); S must stay exact in int32 (and G's conversion exact).
  double s_max = 0.0;
  bool s16 = true;
  for (int k = 0; k < 4; ++k) {
    int64_t pos = 0, sum = 0;
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) {
        pos += mk.w[k][i][j] > 0 ? mk.w[k][i][j] : 0;
        sum += mk.w[k][i][j];
      }
    if (sum != 0) return SOBEL4_ERR_INVALID_ARG;
    const double r = 255.0 * (double)pos;
    s_max += r * r;
    s16 = s16 && r <= 32767.0;
  }
  if (s_max >= 2147483648.0) return SOBEL4_ERR_UNSUPPORTED;
  Masks4 eq3;
  eq5_masks(1, 2, 4, 6, &eq3);
  h->custom = memcmp(&mk, &eq3, sizeof(mk)) != 0;
  h->custom_s16_ok = s16;
  h->masks = mk;
  h->radius = 2;
  h->factored = h->custom && s_max <= kMagnitudeCheckedMax && factored_coefs(a, b, n, m, mk,
                                                                             &h->coefs);
  return SOBEL4_OK;
}

sobel4_status sobel4_set_threshold(sobel4_handle h, double t) {
  if (!h || !(t >= 0.0) || t > 46341.0) return SOBEL4_ERR_INVALID_ARG;
  // Smallest integer k with k >= t^2, decided exactly: fma(t, t, -k) has the
  // sign of t^2 - k (a nonzero difference never rounds to zero here).
  int64_t k = (int64_t)std::ceil(t * t);
  while (k > 0 && std::fma(t, t, -(double)(k - 1)) <= 0.0) --k;
  while (std::fma(t, t, -(double)k) > 0.0) ++k;
  h->thr = (int32_t)std::min<int64_t>(k, INT32_MAX);
  return SOBEL4_OK;
}

sobel4_status sobel4_set_operator(sobel4_handle h, int32_t op) {
  if (!h) return SOBEL4_ERR_INVALID_ARG;
  if (op == SOBEL4_OP_4DIR_5X5) return sobel4_set_weights(h, 1, 2, 4, 6);
  Masks4 mk;
  const int radius = operator_masks(op, &mk);
  if (!radius) return SOBEL4_ERR_INVALID_ARG;
  h->custom = true;
  h->factored = false;  // the two-directional operators run on the mask kernels
  h->custom_s16_ok = true;
  h->masks = mk;
  h->radius = radius;
  return SOBEL4_OK;
}

sobel4_status sobel4_host_alloc(size_t bytes, void **out) {
  if (!out) return SOBEL4_ERR_INVALID_ARG;
  *out = nullptr;
  if (!bytes) return SOBEL4_ERR_INVALID_ARG;
  void *p = nullptr;
  const cudaError_t e = cudaHostAlloc(&p, bytes, cudaHostAllocPortable);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SOBEL4_ERR_OOM : SOBEL4_ERR_CUDA;
  }
  *out = p;
  return SOBEL4_OK;
}

sobel4_status sobel4_host_free(void *p) {
  if (!p) return SOBEL4_OK;
  const cudaError_t e = cudaFreeHost(p);
  if (e != cudaSuccess) (void)cudaGetLastError();
  return e == cudaSuccess ? SOBEL4_OK : SOBEL4_ERR_CUDA;
}

sobel4_status sobel4_device_status(sobel4_handle h) {
  if (!h) return SOBEL4_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  unsigned int word = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&word, h->d_err, sizeof(word), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && word) e = cudaMemset(h->d_err, 0, sizeof(word));
  if (e != cudaSuccess) return cuda_fail(h, e);
  return word ? SOBEL4_ERR_TIMEOUT : SOBEL4_OK;
}

uint64_t sobel4_launch_count(sobel4_handle h) { return h ? h->launches : 0; }

sobel4_status sobel4_set_variant(sobel4_handle h, int32_t variant) {
  if (!h || variant < SOBEL4_VARIANT_AUTO || variant > SOBEL4_VARIANT_LADDER_RG_V2)
    return SOBEL4_ERR_INVALID_ARG;
  h->variant = variant;
  return SOBEL4_OK;
}

sobel4_status sobel4_run(sobel4_handle h, const uint8_t *d_src, size_t src_pitch, void *d_dst,
                         size_t dst_pitch, int32_t height, int32_t width, sobel4_border border,
                         sobel4_format fmt, cudaStream_t stream) {
  if (h && h->autotune && valid_shape(src_pitch, dst_pitch, height, width, border, fmt)) {
    // The creation option autotune: the first run of a shape bucket without a
    // tuned entry tunes it (scratch buffers, the handle's own stream), unless
    // the call's stream is capturing.  A failed tune leaves the defaults.
    const uint32_t key = ((uint32_t)ceil_log2(height) << 16) | ((uint32_t)ceil_log2(width) << 8) |
                         (uint32_t)fmt;
    if (std::find(h->autotried.begin(), h->autotried.end(), key) == h->autotried.end()) {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) {
        (void)cudaGetLastError();
      } else if (cs == cudaStreamCaptureStatusNone) {
        h->autotried.push_back(key);
        if (!find_tuned(h, 0, height, width, fmt) &&
            sobel4_tune(h, height, width, border, fmt, nullptr) == SOBEL4_OK &&
            !h->cache_path.empty())
          sobel4_tune_save(h, h->cache_path.c_str());
      }
    }
  }
  return sobel4::run_with_pair(h, d_src, src_pitch, d_dst, dst_pitch, height, width, border, fmt,
                               stream, nullptr);
}

}  // extern "C"

namespace sobel4 {
// sobel4_run with a caller-owned counter pair (nullptr: the handle's next);
// a captured graph owns its pair, since every replay reuses it.
sobel4_status run_with_pair(sobel4_handle h, const uint8_t *d_src, size_t src_pitch, void *d_dst,
                            size_t dst_pitch, int32_t height, int32_t width, int border, int fmt,
                            cudaStream_t stream, unsigned int *pair) {
  if (!h || !d_src || !valid_dst_ptr(d_dst, fmt)) return SOBEL4_ERR_INVALID_ARG;
  if (!valid_shape(src_pitch, dst_pitch, height, width, border, fmt))
    return SOBEL4_ERR_INVALID_ARG;
  uintptr_t r[4];
  ranges(d_src, src_pitch, d_dst, dst_pitch, height, width, fmt, r);
  if (overlaps(r[0], r[1], r[2], r[3])) return SOBEL4_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  return launch_one(h, d_src, src_pitch, d_dst, dst_pitch, height, width, border, fmt, stream,
                    pair);
}
}  // namespace sobel4

extern "C" {

sobel4_status sobel4_run_rgb(sobel4_handle h, const uint8_t *d_src, size_t src_pitch, void *d_dst,
                             size_t dst_pitch, int32_t height, int32_t width,
                             sobel4_border border, sobel4_format fmt, cudaStream_t stream) {
  if (!h || !d_src || !valid_dst_ptr(d_dst, fmt) || width < 1 || width > kMaxSide ||
      src_pitch < 3 * (size_t)width)
    return SOBEL4_ERR_INVALID_ARG;
  if (!valid_shape(src_pitch, dst_pitch, height, width, border, fmt))
    return SOBEL4_ERR_INVALID_ARG;
  uintptr_t r[4];
  ranges(d_src, src_pitch, d_dst, dst_pitch, height, width, fmt, r);
  r[1] = (uintptr_t)d_src + (uintptr_t)(height - 1) * src_pitch + 3 * (uintptr_t)width;
  if (overlaps(r[0], r[1], r[2], r[3])) return SOBEL4_ERR_INVALID_ARG;
  if (h->custom) return SOBEL4_ERR_UNSUPPORTED;  // runtime masks run on other kernels
  DeviceGuard g(h->device);
  const int R = tma_pick_R(fmt, h->sm_count, height, width,
                           tma_all_fast_staged(width, border, fmt, true, d_dst, dst_pitch));
  const cudaError_t e = launch_tma_single_rgb(d_src, src_pitch, d_dst, dst_pitch, height, width,
                                              border, fmt, R, h->sm_count, next_pair(h),
                                              h->d_err, stream, h->thr);
  if (e != cudaSuccess) return cuda_fail(h, e);
  h->launches += 1;
  return SOBEL4_OK;
}

sobel4_status sobel4_run_batched(sobel4_handle h, const sobel4_image *imgs, int32_t n,
                                 sobel4_border border, sobel4_format fmt, cudaStream_t stream) {
  if (!h || !imgs || n < 1 || !valid_enum(border, fmt)) return SOBEL4_ERR_INVALID_ARG;
  // Validate every descriptor and the pairwise overlap rule (sweep over sorted ranges).
  struct Iv {
    uintptr_t b, e;
    bool out;
  };
  std::vector<Iv> iv;
  iv.reserve((size_t)n * 2);
  for (int32_t i = 0; i < n; ++i) {
    const sobel4_image &m = imgs[i];
    if (!m.src || !valid_dst_ptr(m.dst, fmt) ||
        !valid_shape(m.src_pitch, m.dst_pitch, m.height, m.width, border, fmt))
      return SOBEL4_ERR_INVALID_ARG;
    uintptr_t r[4];
    ranges(m.src, m.src_pitch, m.dst, m.dst_pitch, m.height, m.width, fmt, r);
    iv.push_back({r[0], r[1], false});
    iv.push_back({r[2], r[3], true});
  }
  std::sort(iv.begin(), iv.end(), [](const Iv &a, const Iv &b) { return a.b < b.b; });
  uintptr_t end_out = 0, end_in = 0;
  for (const Iv &v : iv) {
    if (v.out ? (v.b < end_out || v.b < end_in) : (v.b < end_out)) return SOBEL4_ERR_INVALID_ARG;
    if (v.out) end_out = std::max(end_out, v.e);
    else end_in = std::max(end_in, v.e);
  }
  DeviceGuard g(h->device);
  if (h->variant == SOBEL4_VARIANT_DIRECT || is_ladder(h->variant) || h->custom) {
    for (int32_t i = 0; i < n; ++i) {
      const sobel4_image &m = imgs[i];
      sobel4_status s = launch_one(h, m.src, m.src_pitch, m.dst, m.dst_pitch, m.height, m.width,
                                   border, fmt, stream);
      if (s != SOBEL4_OK) return s;
    }
    return SOBEL4_OK;
  }
  // The tuned entry for batches names the kernel family and its parameters.
  const TuneEntry *bt = find_tuned(h, 1, 0, 0, fmt);
  const TuneEntry *bl = bt && bt->kernel == 0 ? bt : nullptr;
  const int R = h->rows_per_strip > 0 ? h->rows_per_strip : (bl ? bl->R : kBatchR);
  const int bnc = h->nc_forced ? h->nc : (bl ? bl->nc : h->nc);
  const int bctas = bl ? bl->ctas : h->ctas_per_sm;
  BatchSlot &slot = h->slots[h->next_slot];
  h->next_slot = (h->next_slot + 1) % kSlots;
  cudaError_t e = cudaSuccess;
  if (slot.pending) {
    e = cudaEventSynchronize(slot.done);  // the slot's previous batch has consumed its buffers
    if (e != cudaSuccess) return cuda_fail(h, e);
    slot.pending = false;
  }
  if (slot.cap < n) {
    e = grow_slot(slot, std::max(n, 2 * slot.cap));
    if (e != cudaSuccess) return cuda_fail(h, e);
  }
  // Every image goes to ONE launch of the TMA-family batched kernel unless
  // the handle asks for lane copies: staged by tensor copies when every
  // source is 16-byte aligned, else all by bulk row copies (which take any
  // alignment), so that a mixed batch is still one persistent launch.
  const bool tma_ok = (int)fmt == kU16 || (int)fmt == kEdge8 ||
                      (h->variant != SOBEL4_VARIANT_RG_LANECOPY && !h->nc_forced && !bl);
  // TMA strip height: explicit option, else the tuned one, else about four
  // items per resident warp (8 .. 128 rows): taller strips spend less on the
  // 4-row window fill (measured on the 512-image ragged batch with tight
  // pitches: 1.34 ms at 32 rows, 1.16 ms at 128).
  int Rt = tma_round_R(R);
  if (tma_ok && h->rows_per_strip <= 0) {
    if (bt && bt->kernel == 1) {
      Rt = bt->R;
    } else {
      int64_t seg_rows = 0;
      for (int32_t i = 0; i < n; ++i)
        seg_rows += (int64_t)((imgs[i].width + 127) / 128) * imgs[i].height;
      const int64_t warps = (int64_t)h->sm_count * 4 * kWarpsPerCta;
      Rt = tma_round_R(
          (int)std::min<int64_t>(128, std::max<int64_t>(8, seg_rows / (8 * warps))));
    }
  }
  int n_lane = 0, n_tma = 0;
  int64_t total = 0, total_tma = 0;
  int fast = kBatchFastVec;
  bool bulk = false;
  if (tma_ok) {
    for (int32_t i = 0; i < n && !bulk; ++i) bulk = !tma_eligible(imgs[i].src, imgs[i].src_pitch);
    const size_t db = tma_batch_desc_bytes(bulk);
    for (int32_t i = 0; i < n; ++i) {
      const sobel4_image &m = imgs[i];
      int64_t items = 0;
      e = tma_fill_batch_desc(slot.h_tma + db * n_tma, bulk, m.src, m.src_pitch, m.dst,
                              m.dst_pitch, m.height, m.width, Rt, total_tma, &items, h->thr);
      if (e != cudaSuccess) return cuda_fail(h, e);
      total_tma += items;
      ++n_tma;
      // the batch runs the kernel its least fast image needs (BatchFast)
      fast = std::min(fast, tma_fast_level(m.width, border, fmt, bulk, m.dst, m.dst_pitch));
    }
  } else {
    for (int32_t i = 0; i < n; ++i) {
      const sobel4_image &m = imgs[i];
      ImageDesc d = make_desc(m.src, m.src_pitch, m.dst, m.dst_pitch, m.height, m.width, R, bnc);
      d.item0 = total;
      total += (int64_t)d.n_seg * d.n_band;
      slot.h_desc[n_lane++] = d;
    }
  }
  if (total >= (1ll << 31) || total_tma >= (1ll << 31)) return SOBEL4_ERR_UNSUPPORTED;
  // The descriptors reach the device in kernel parameters (param_upload), not
  // by a host-to-device copy, which would queue behind the caller's uploads.
  // (n >= 1, so one of the two uploads runs and zeroes the queue.)
  const size_t lane_bytes = sizeof(ImageDesc) * n_lane;
  const size_t tma_bytes = tma_batch_desc_bytes(bulk) * n_tma;
  if (n_lane) e = param_upload(slot.h_desc, slot.d_desc, lane_bytes, slot.d_queue, stream);
  if (e == cudaSuccess && n_tma)
    e = param_upload(slot.h_tma, slot.d_tma, tma_bytes, n_lane ? nullptr : slot.d_queue, stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  h->launches += (lane_bytes + kParamChunk - 1) / kParamChunk +
                 (tma_bytes + kParamChunk - 1) / kParamChunk;
  if (n_tma) {
    const int64_t want = (total_tma + kWarpsPerCta - 1) / kWarpsPerCta;
    const int grid = (int)std::min<int64_t>(want, 1 << 30);  // capped at residency below
    e = launch_tma_batched(slot.d_tma, n_tma, total_tma, slot.d_queue + 32, border, fmt, Rt,
                           std::max(grid, 1), h->sm_count, h->d_err, stream, fast, bulk);
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->launches += 1;
  }
  if (n_lane) {
    const int64_t want = (total + kWarpsPerCta - 1) / kWarpsPerCta;
    const int grid = (int)std::min<int64_t>(want, (int64_t)h->sm_count * bctas);
    e = launch_rg_batched(slot.d_desc, n_lane, total, slot.d_queue, border, fmt, R, bnc,
                          std::max(grid, 1), h->sm_count, stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->launches += 1;
  }
  e = cudaEventRecord(slot.done, stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  slot.pending = true;
  return SOBEL4_OK;
}

sobel4_status sobel4_run_host(sobel4_handle h, const uint8_t *h_src, size_t src_pitch,
                              void *h_dst, size_t dst_pitch, int32_t height, int32_t width,
                              sobel4_border border, sobel4_format fmt) {
  if (!h || !h_src || !h_dst) return SOBEL4_ERR_INVALID_ARG;
  if (!valid_shape(src_pitch, dst_pitch, height, width, border, fmt))
    return SOBEL4_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  const size_t sp = ((size_t)width + 15) & ~(size_t)15;
  const size_t row_out = (size_t)width * elem_size(fmt);
  const size_t dp = (row_out + 15) & ~(size_t)15;
  const size_t in_bytes = sp * (size_t)height;
  const int np = planes(fmt);
  cudaError_t e = cudaSuccess;
  if (h->d_in_bytes < in_bytes) {
    if (h->d_in) cudaFree(h->d_in);
    h->d_in = nullptr;
    h->d_in_bytes = 0;
    e = cudaMalloc((void **)&h->d_in, in_bytes);
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->d_in_bytes = in_bytes;
  }
  // Large images run as row bands through three streams, so that the upload
  // of band k+1, the kernel of band k and the download of band k-1 overlap:
  // the call then takes about as long as its larger copy direction instead
  // of the sum of both copies and the kernel.  Band k computes the sub-image
  // of its rows plus the 2-row halos above and below (the border rule applies
  // at the image's own top and bottom only; a sub-image's halo rows are
  // computed but never downloaded) into one slot of a 3-slot output ring.
  const size_t out_total = dp * (size_t)height * (size_t)np;
  const int32_t kMinBandRows = 256;
  int32_t bands = 1;
  if (out_total >= ((size_t)16 << 20) && height >= 2 * kMinBandRows)
    bands = std::min<int32_t>(16, height / kMinBandRows);
  if (bands == 1) {
    const size_t out_bytes = out_total;
    if (h->d_out_bytes < out_bytes) {
      if (h->d_out) cudaFree(h->d_out);
      h->d_out = nullptr;
      h->d_out_bytes = 0;
      e = cudaMalloc((void **)&h->d_out, out_bytes);
      if (e != cudaSuccess) return cuda_fail(h, e);
      h->d_out_bytes = out_bytes;
    }
    cudaStream_t st = h->own_stream;
    e = cudaMemcpy2DAsync(h->d_in, sp, h_src, src_pitch, (size_t)width, (size_t)height,
                          cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(h, e);
    sobel4_status s = launch_one(h, h->d_in, sp, h->d_out, dp, height, width, border, fmt, st);
    if (s != SOBEL4_OK) return s;
    e = cudaMemcpy2DAsync(h_dst, dst_pitch, h->d_out, dp, row_out, (size_t)height * np,
                          cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e);
    return SOBEL4_OK;
  }
  const int32_t hb = (height + bands - 1) / bands;  // rows per band (the last may be shorter)
  bands = (height + hb - 1) / hb;
  const size_t slot_bytes = dp * (size_t)(hb + 4) * (size_t)np;
  if (h->d_ring_bytes < 3 * slot_bytes) {
    if (h->d_ring) cudaFree(h->d_ring);
    h->d_ring = nullptr;
    h->d_ring_bytes = 0;
    e = cudaMalloc((void **)&h->d_ring, 3 * slot_bytes);
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->d_ring_bytes = 3 * slot_bytes;
  }
  if (!h->h2d_stream) e = cudaStreamCreateWithFlags(&h->h2d_stream, cudaStreamNonBlocking);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i)
    if (!h->d2h_stream[i]) e = cudaStreamCreateWithFlags(&h->d2h_stream[i], cudaStreamNonBlocking);
  while (e == cudaSuccess && h->band_events.size() < (size_t)(3 * bands)) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) h->band_events.push_back(ev);
  }
  if (e != cudaSuccess) return cuda_fail(h, e);
  cudaEvent_t *ev_in = h->band_events.data();
  cudaEvent_t *ev_done = ev_in + bands;
  cudaEvent_t *ev_out = ev_done + bands;
  // Downloads alternate between two streams (bands k and k+1 in flight together).
  const cudaStream_t up = h->h2d_stream, comp = h->own_stream;
  // The caller's earlier work on the handle's stream finishes first.
  e = cudaEventRecord(ev_out[0], comp);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(up, ev_out[0], 0);
  for (int32_t k = 0; k < bands && e == cudaSuccess; ++k) {
    const int32_t r0 = k * hb, r1 = std::min(height, r0 + hb);
    e = cudaMemcpy2DAsync(h->d_in + (size_t)r0 * sp, sp, h_src + (size_t)r0 * src_pitch,
                          src_pitch, (size_t)width, (size_t)(r1 - r0), cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in[k], up);
  }
  for (int32_t k = 0; k < bands && e == cudaSuccess; ++k) {
    const int32_t r0 = k * hb, r1 = std::min(height, r0 + hb);
    const int32_t s0 = std::max(0, r0 - 2), s1 = std::min(height, r1 + 2);
    e = cudaStreamWaitEvent(comp, ev_in[k], 0);
    if (e == cudaSuccess && k + 1 < bands) e = cudaStreamWaitEvent(comp, ev_in[k + 1], 0);
    if (e == cudaSuccess && k >= 3) e = cudaStreamWaitEvent(comp, ev_out[k - 3], 0);
    if (e != cudaSuccess) break;
    uint8_t *slot = h->d_ring + (size_t)(k % 3) * slot_bytes;
    sobel4_status s = launch_one(h, h->d_in + (size_t)s0 * sp, sp, slot, dp, s1 - s0, width,
                                 border, fmt, comp);
    if (s != SOBEL4_OK) {
      cudaStreamSynchronize(up);
      cudaStreamSynchronize(h->d2h_stream[0]);
      cudaStreamSynchronize(h->d2h_stream[1]);
      return s;
    }
    const cudaStream_t down = h->d2h_stream[k & 1];
    e = cudaEventRecord(ev_done[k], comp);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(down, ev_done[k], 0);
    for (int p = 0; p < np && e == cudaSuccess; ++p) {
      const uint8_t *from = slot + ((size_t)p * (size_t)(s1 - s0) + (size_t)(r0 - s0)) * dp;
      uint8_t *to = (uint8_t *)h_dst + ((size_t)p * (size_t)height + (size_t)r0) * dst_pitch;
      e = cudaMemcpy2DAsync(to, dst_pitch, from, dp, row_out, (size_t)(r1 - r0),
                            cudaMemcpyDeviceToHost, down);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev_out[k], down);
  }
  cudaError_t e2 = cudaStreamSynchronize(up);
  cudaError_t e3 = cudaStreamSynchronize(comp);
  cudaError_t e4 = cudaStreamSynchronize(h->d2h_stream[0]);
  cudaError_t e5 = cudaStreamSynchronize(h->d2h_stream[1]);
  if (e4 == cudaSuccess) e4 = e5;
  if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : (e3 != cudaSuccess ? e3 : e4);
  if (e != cudaSuccess) return cuda_fail(h, e);
  return SOBEL4_OK;
}

sobel4_status sobel4_check_magnitude(sobel4_handle h, int32_t s_begin, int32_t s_end,
                                     uint64_t *mismatches) {
  if (!h || !mismatches || s_begin < 0 || s_end < s_begin) return SOBEL4_ERR_INVALID_ARG;
  *mismatches = 0;
  DeviceGuard g(h->device);
  unsigned long long *d_bad = nullptr;
  cudaError_t e = cudaMalloc((void **)&d_bad, sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_fail(h, e);
  unsigned long long bad = 0;
  e = cudaMemsetAsync(d_bad, 0, sizeof(bad), h->own_stream);
  if (e == cudaSuccess)
    e = launch_check_magnitude(s_begin, s_end, d_bad, h->sm_count * 8, h->own_stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, h->own_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->own_stream);
  cudaFree(d_bad);
  if (e != cudaSuccess) return cuda_fail(h, e);
  h->launches += 1;
  *mismatches = bad;
  return SOBEL4_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free batched entry point.  Some callers cannot allocate device
// memory at all: plugins inside a host framework that owns every device
// buffer, services held to a fixed memory budget, latency-critical threads
// that must not pay for cudaMalloc or cudaFree.  For them
// sobel4_run_batched_static runs the lane-copy persistent batched kernel
// without a handle, with its scratch (the image descriptors and the
// work-queue counter) in the file-scope device array below.  The caller still
// owns the images.  The array is part of the library's device image, so every
// GPU that loads the library holds it (about 64 KB) until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int kStaticMaxImages = SOBEL4_STATIC_MAX_IMAGES;
constexpr size_t kStaticDescBytes = sizeof(ImageDesc) * kStaticMaxImages;
constexpr size_t kStaticScratchBytes = kStaticDescBytes + 256;  // descriptors + queue words

static_assert(sizeof(ImageDesc) == 64, "descriptor size is part of SOBEL4_STATIC_SCRATCH_BYTES");
static_assert(kStaticScratchBytes == SOBEL4_STATIC_SCRATCH_BYTES, "scratch size mismatch");
static_assert(kParamChunk % sizeof(ImageDesc) == 0, "descriptors must not straddle uploads");
static_assert(2 * kStaticMaxImages <= 65536, "range indices are 16-bit");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

}  // namespace

extern "C" sobel4_status sobel4_run_batched_static(const sobel4_image *imgs, int32_t n,
                                                   sobel4_border border, sobel4_format fmt,
                                                   cudaStream_t stream) {
  if (!imgs || n < 1 || !valid_enum(border, fmt)) return SOBEL4_ERR_INVALID_ARG;
  if (n > kStaticMaxImages || (int)fmt == kU16 || (int)fmt == kEdge8)
    return SOBEL4_ERR_UNSUPPORTED;  // the lane-copy kernel has no such output
  const int R = kBatchR;
  int64_t total = 0;  // work items of the whole batch
  for (int32_t i = 0; i < n; ++i) {
    const sobel4_image &m = imgs[i];
    if (!m.src || !valid_dst_ptr(m.dst, fmt) ||
        !valid_shape(m.src_pitch, m.dst_pitch, m.height, m.width, border, fmt))
      return SOBEL4_ERR_INVALID_ARG;
    const ImageDesc d = make_desc(m.src, m.src_pitch, m.dst, m.dst_pitch, m.height, m.width, R,
                                  kDefaultNC);
    total += (int64_t)d.n_seg * d.n_band;
  }
  // Overlap rule: a sweep over the 2n byte ranges sorted by their start,
  // through 16-bit indices on the stack (4 KB; no heap).
  auto range_of = [&](int k, uintptr_t *b, uintptr_t *e) {
    const sobel4_image &m = imgs[k >> 1];
    uintptr_t r[4];
    ranges(m.src, m.src_pitch, m.dst, m.dst_pitch, m.height, m.width, fmt, r);
    *b = r[2 * (k & 1)];
    *e = r[2 * (k & 1) + 1];
  };
  uint16_t idx[2 * kStaticMaxImages];
  for (int k = 0; k < 2 * n; ++k) idx[k] = (uint16_t)k;
  std::sort(idx, idx + 2 * n, [&](uint16_t a, uint16_t b) {
    uintptr_t ba, ea, bb, eb;
    range_of(a, &ba, &ea);
    range_of(b, &bb, &eb);
    return ba < bb;
  });
  uintptr_t end_out = 0, end_in = 0;
  for (int k = 0; k < 2 * n; ++k) {
    uintptr_t b, e;
    range_of(idx[k], &b, &e);
    const bool out = idx[k] & 1;  // odd index: an output range
    if (out ? (b < end_out || b < end_in) : (b < end_out)) return SOBEL4_ERR_INVALID_ARG;
    if (out) end_out = std::max(end_out, e);
    else end_in = std::max(end_in, e);
  }
  if (total >= (1ll << 31)) return SOBEL4_ERR_UNSUPPORTED;  // before anything is enqueued
  // The array's device address on the current device: the host-side symbol
  // is only a stand-in and must never reach a kernel.  Looked up on every
  // call (a host-side query once the device code is loaded), so no address
  // outlives a context.
  int dev = 0, sms = 0;
  void *scratch = nullptr;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaGetSymbolAddress(&scratch, g_static_scratch) != cudaSuccess) {
    (void)cudaGetLastError();
    return SOBEL4_ERR_CUDA;
  }
  ImageDesc *d_desc = (ImageDesc *)scratch;
  unsigned int *d_queue = (unsigned int *)((unsigned char *)scratch + kStaticDescBytes);
  // The descriptors travel in the parameters of small copy launches, built in
  // place (no host buffer outlives the call); the first launch also zeroes
  // the queue words.
  int64_t item0 = 0;
  cudaError_t e = param_upload_fill(
      sizeof(ImageDesc) * (size_t)n, d_desc, d_queue, stream,
      [&](uint8_t *buf, size_t off, size_t bytes) {
        ImageDesc *out = (ImageDesc *)buf;
        const size_t i0 = off / sizeof(ImageDesc), cnt = bytes / sizeof(ImageDesc);
        for (size_t j = 0; j < cnt; ++j) {
          const sobel4_image &m = imgs[i0 + j];
          ImageDesc d = make_desc(m.src, m.src_pitch, m.dst, m.dst_pitch, m.height, m.width, R,
                                  kDefaultNC);
          d.item0 = item0;
          item0 += (int64_t)d.n_seg * d.n_band;
          out[j] = d;
        }
      });
  if (e != cudaSuccess) return SOBEL4_ERR_CUDA;
  const int64_t want = (total + kWarpsPerCta - 1) / kWarpsPerCta;
  const int grid = (int)std::min<int64_t>(want, (int64_t)sms * 4);
  e = launch_rg_batched(d_desc, n, total, d_queue, border, fmt, R, kDefaultNC, std::max(grid, 1),
                        sms, stream);
  return e == cudaSuccess ? SOBEL4_OK : SOBEL4_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Autotuner: the per-shape analogue of the paper's block-configuration study
// (Fig. 5, Section 5.2).  Candidates are timed with CUDA events on the
// handle's own stream; the fastest is recorded in the handle's table.
// ---------------------------------------------------------------------------
namespace {

constexpr int kTuneWarmup = 2;
// Each candidate runs kTuneRegions regions of kTuneLaunches back-to-back
// launches between two events (steady-state throughput, as a stream of
// launches sees it: per-launch event pairs add their own gaps); its time is
// the median of the regions' means.
constexpr int kTuneRegions = 3;
constexpr int kTuneLaunches = 10;

template <class Launch>
cudaError_t median_us(cudaStream_t st, Launch launch, float *us) {
  cudaEvent_t ev[kTuneRegions + 1];
  for (int i = 0; i <= kTuneRegions; ++i) ev[i] = nullptr;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i <= kTuneRegions && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
  for (int i = 0; i < kTuneWarmup && e == cudaSuccess; ++i) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
  for (int r = 0; r < kTuneRegions && e == cudaSuccess; ++r) {
    for (int i = 0; i < kTuneLaunches && e == cudaSuccess; ++i) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(ev[r + 1], st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float t[kTuneRegions];
  for (int r = 0; r < kTuneRegions && e == cudaSuccess; ++r) {
    e = cudaEventElapsedTime(&t[r], ev[r], ev[r + 1]);
    t[r] /= (float)kTuneLaunches;
  }
  for (int i = 0; i <= kTuneRegions; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess) return e;
  std::sort(t, t + kTuneRegions);
  *us = 1000.0f * t[kTuneRegions / 2];
  return cudaSuccess;
}

void upsert(sobel4_ctx *h, const TuneEntry &t) {
  for (TuneEntry &u : h->tuned)
    if (u.kind == t.kind && u.hb == t.hb && u.wb == t.wb && u.fmt == t.fmt) {
      u = t;
      return;
    }
  h->tuned.push_back(t);
}

bool valid_entry(const TuneEntry &t) {
  return (t.kind == 0 || t.kind == 1) && t.hb >= 0 && t.hb <= 31 && t.wb >= 0 && t.wb <= 31 &&
         t.fmt >= 0 && t.fmt <= 2 && (t.nc == 2 || t.nc == 4) && t.R >= 1 && t.R <= (1 << 20) &&
         t.ctas >= 1 && t.ctas <= 64 && (t.kernel == 0 || (t.kernel == 1 && t.nc == 4 &&
                                                           t.R == tma_round_R(t.R)) ||
                                         (t.kernel == 2 && t.kind == 0));
}

}  // namespace

extern "C" sobel4_status sobel4_tune(sobel4_handle h, int32_t height, int32_t width,
                                     sobel4_border border, sobel4_format fmt, float *best_us) {
  if (!h) return SOBEL4_ERR_INVALID_ARG;
  const size_t sp = ((size_t)width + 15) & ~(size_t)15;
  const size_t dp = ((size_t)width * elem_size(fmt) + 15) & ~(size_t)15;
  if (!valid_shape(sp, dp, height, width, border, fmt)) return SOBEL4_ERR_INVALID_ARG;
  // Runtime weights that sobel4_set_weights proved exact on the packed passes
  // run on the TMA-staged kernel alone (with their coefficients), so only its
  // strip heights are timed; other runtime weights have nothing to tune.
  const bool weights = h->custom;
  const Coefs *cw = weights && h->factored && (int)fmt != kS16x4 &&
                            h->variant != SOBEL4_VARIANT_DIRECT ? &h->coefs : nullptr;
  if (weights && !cw) return SOBEL4_ERR_UNSUPPORTED;
  DeviceGuard g(h->device);
  uint8_t *src = nullptr, *dst = nullptr;
  cudaError_t e = cudaMalloc((void **)&src, sp * (size_t)height);
  if (e == cudaSuccess) e = cudaMalloc((void **)&dst, dp * (size_t)height * planes(fmt));
  if (e == cudaSuccess) e = cudaMemsetAsync(src, 0x5A, sp * (size_t)height, h->own_stream);
  TuneEntry best = {0, ceil_log2(height), ceil_log2(width), (int)fmt, h->nc, 0, h->ctas_per_sm, 0,
                    0};
  bool have = false;
  auto consider = [&](int kernel, int nc, int R, float us) {
    if (!have || us < best.us) {
      best.kernel = kernel;
      best.nc = nc;
      best.R = R;
      best.us = us;
      have = true;
    }
  };
  // Tensor-core kernel (AUTO and TC handles, the images it covers).
  if (e == cudaSuccess && !weights &&
      (h->variant == SOBEL4_VARIANT_AUTO || h->variant == SOBEL4_VARIANT_TC) && !h->nc_forced &&
      h->rows_per_strip <= 0 && tc_eligible(src, sp, dst, dp, height, width, border, fmt)) {
    float us = 0.f;
    e = median_us(h->own_stream, [&]() {
      h->launches += 1;
      return launch_tc_single(src, sp, dst, dp, height, width, border, fmt, h->sm_count,
                              h->d_err, h->own_stream);
    }, &us);
    if (e == cudaSuccess) consider(2, 4, 8, us);
  }
  // TMA-staged kernel: a few strip heights, including the one that gives every
  // resident warp about one item.
  if (((int)fmt == kU16 || (int)fmt == kEdge8 ||
       (h->variant != SOBEL4_VARIANT_RG_LANECOPY && !h->nc_forced)) &&
      tma_eligible(src, sp)) {
    std::vector<int> cands;
    if (h->rows_per_strip > 0) {
      cands.push_back(tma_round_R(h->rows_per_strip));
    } else {
      // 8, 16, 24, ... 128 rows per strip (no taller than the image needs),
      // plus the heuristic's choice.
      const int top = tma_round_R(std::max(8, (height + 1) / 2));
      for (int R = 8; R <= 128 && R <= top; R += 8) cands.push_back(R);
      const int r0 = tma_pick_R(fmt, h->sm_count, height, width,
                                tma_all_fast(width, border, fmt, src, sp, dst, dp));
      if (std::find(cands.begin(), cands.end(), r0) == cands.end()) cands.push_back(r0);
    }
    for (size_t b = 0; b < cands.size() && e == cudaSuccess; ++b) {
      const int R = cands[b];
      float us = 0.f;
      e = median_us(h->own_stream, [&]() {
        h->launches += 1;
        return launch_tma_single(src, sp, dst, dp, height, width, border, fmt, R, h->sm_count,
                                 next_pair(h), h->d_err, h->own_stream, -1, h->thr, cw);
      }, &us);
      if (e == cudaSuccess) consider(1, 4, R, us);
    }
  }
  const int ncs[2] = {2, 4};
  const int Rs[4] = {8, 16, 32, 64};
  for (int a = 0; a < 2 && e == cudaSuccess && (int)fmt != kU16 && (int)fmt != kEdge8 && !weights; ++a) {
    if (h->nc_forced && ncs[a] != h->nc) continue;
    for (int b = 0; b < 4 && e == cudaSuccess; ++b) {
      if (h->rows_per_strip > 0 && Rs[b] != h->rows_per_strip) continue;
      const ImageDesc im = make_desc(src, sp, dst, dp, height, width, Rs[b], ncs[a]);
      float us = 0.f;
      e = median_us(h->own_stream, [&]() {
        h->launches += 1;
        return launch_rg_single(im, border, fmt, Rs[b], ncs[a], h->sm_count, next_pair(h),
                                h->own_stream);
      }, &us);
      if (e == cudaSuccess) consider(0, ncs[a], Rs[b], us);
    }
  }
  if (e == cudaSuccess && !have) e = cudaErrorInvalidValue;  // no candidate fits the options
  if (src) cudaFree(src);
  if (dst) cudaFree(dst);
  if (e != cudaSuccess) return cuda_fail(h, e);
  upsert(h, best);
  if (best_us) *best_us = best.us;
  return SOBEL4_OK;
}

extern "C" sobel4_status sobel4_tune_batched(sobel4_handle h, const sobel4_image *imgs, int32_t n,
                                             sobel4_border border, sobel4_format fmt,
                                             float *best_us) {
  if (!h || !imgs || n < 1 || !valid_enum(border, fmt)) return SOBEL4_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  const std::vector<TuneEntry> saved = h->tuned;
  TuneEntry best = {1, 0, 0, (int)fmt, h->nc, kBatchR, h->ctas_per_sm, 0, 0};
  bool have = false;
  const int ncs[2] = {2, 4};
  const int Rs[3] = {8, 16, 32};
  const int ctas[3] = {2, 4, 6};
  cudaError_t e = cudaSuccess;
  sobel4_status st = SOBEL4_OK;
  auto try_entry = [&](const TuneEntry &cand) {
    h->tuned = saved;
    upsert(h, cand);
    float us = 0.f;
    e = median_us(h->own_stream, [&]() {
      st = sobel4_run_batched(h, imgs, n, border, fmt, h->own_stream);
      return st == SOBEL4_OK ? cudaSuccess : cudaErrorUnknown;
    }, &us);
    if (st != SOBEL4_OK) return;
    if (e != cudaSuccess) {
      st = cuda_fail(h, e);
      return;
    }
    if (!have || us < best.us) {
      best = cand;
      best.us = us;
      have = true;
    }
  };
  // TMA-family kernel (any alignment): strip heights 8 .. 128.
  if (h->variant != SOBEL4_VARIANT_RG_LANECOPY && !h->nc_forced) {
    const int Rt[7] = {8, 16, 32, 48, 64, 96, 128};
    for (int b = 0; b < 7 && st == SOBEL4_OK; ++b) {
      if (h->rows_per_strip > 0 && Rt[b] != tma_round_R(h->rows_per_strip)) continue;
      try_entry({1, 0, 0, (int)fmt, 4, Rt[b], h->ctas_per_sm, 0, 1});
    }
  }
  // Lane-copy kernel: columns per lane, strip height, CTAs per SM.
  for (int a = 0; a < 2 && st == SOBEL4_OK && (int)fmt != kU16 && (int)fmt != kEdge8; ++a) {
    if (h->nc_forced && ncs[a] != h->nc) continue;
    for (int b = 0; b < 3 && st == SOBEL4_OK; ++b) {
      if (h->rows_per_strip > 0 && Rs[b] != h->rows_per_strip) continue;
      for (int c = 0; c < 3 && st == SOBEL4_OK; ++c) {
        try_entry({1, 0, 0, (int)fmt, ncs[a], Rs[b], ctas[c], 0, 0});
      }
    }
  }
  h->tuned = saved;
  if (st != SOBEL4_OK) return st;
  upsert(h, best);
  if (best_us) *best_us = best.us;
  return SOBEL4_OK;
}

extern "C" int32_t sobel4_tune_entries(sobel4_handle h) { return h ? (int32_t)h->tuned.size() : 0; }

extern "C" sobel4_status sobel4_tune_config(sobel4_handle h, int32_t height, int32_t width,
                                            sobel4_format fmt, int32_t *kernel,
                                            int32_t *columns_per_lane, int32_t *rows_per_strip) {
  if (!h || !kernel || !columns_per_lane || !rows_per_strip || height < 1 || width < 1 ||
      fmt < SOBEL4_OUT_F32 || fmt > SOBEL4_OUT_EDGE8)
    return SOBEL4_ERR_INVALID_ARG;
  // The configuration a VALID launch with 16-byte aligned rows would use.
  static const uint8_t kAligned[16] __attribute__((aligned(16))) = {0};
  bool use_tma = false;
  int nc = 0, R = 0;
  DeviceGuard g(h->device);
  const size_t sp = ((size_t)width + 15) & ~(size_t)15;
  const size_t dp = ((size_t)width * elem_size(fmt) + 15) & ~(size_t)15;
  // The same routing as launch_one: runtime weights, DIRECT, the ladder.
  if (h->custom || h->variant == SOBEL4_VARIANT_DIRECT || is_ladder(h->variant)) {
    *columns_per_lane = 1;
    *rows_per_strip = 0;
    if (h->custom && h->factored && (int)fmt != kS16x4 && h->variant != SOBEL4_VARIANT_DIRECT) {
      rg_config(h, kAligned, sp, kAligned, dp, height, width, SOBEL4_BORDER_VALID, fmt,
                &use_tma, &nc, &R);
      *kernel = 1;
      *columns_per_lane = 4;
      *rows_per_strip = use_tma ? R : tma_pick_R(fmt, h->sm_count, height, width, true);
    } else if (h->custom) {
      *kernel = h->variant != SOBEL4_VARIANT_DIRECT &&
                        tc_eligible(kAligned, sp, kAligned, dp, height, width,
                                    SOBEL4_BORDER_VALID, fmt)
                    ? 2 : 3;
    } else if (h->variant == SOBEL4_VARIANT_DIRECT) {
      *kernel = 3;
    } else {
      *kernel = 4 + (h->variant - SOBEL4_VARIANT_LADDER_SM);
      if (h->variant >= SOBEL4_VARIANT_LADDER_RG)
        *rows_per_strip = h->rows_per_strip > 0 ? h->rows_per_strip
                                                : ladder_rows(height, width, h->sm_count);
    }
    return SOBEL4_OK;
  }
  rg_config(h, kAligned, sp, kAligned, dp, height, width, SOBEL4_BORDER_VALID, fmt, &use_tma, &nc,
            &R);
  *kernel = use_tma ? 1 : 0;
  if (use_tc(h, kAligned, sp, kAligned, dp, height, width, SOBEL4_BORDER_VALID, fmt)) *kernel = 2;
  *columns_per_lane = nc;
  *rows_per_strip = R;
  return SOBEL4_OK;
}

extern "C" sobel4_status sobel4_tune_save(sobel4_handle h, const char *path) {
  if (!h || !path || !*path) return SOBEL4_ERR_INVALID_ARG;
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = fopen(tmp.c_str(), "w");
  if (!f) return SOBEL4_ERR_INVALID_ARG;
  fprintf(f, "{\"sobel4_tune\": 1, \"version\": \"%s\", \"device\": \"%s\", \"sm_count\": %d,\n",
          sobel4_version(), h->device_name, h->sm_count);
  fprintf(f, " \"entries\": [\n");
  for (size_t i = 0; i < h->tuned.size(); ++i) {
    const TuneEntry &t = h->tuned[i];
    fprintf(f,
            "  {\"kind\": %d, \"hb\": %d, \"wb\": %d, \"fmt\": %d, \"nc\": %d, \"R\": %d, "
            "\"ctas\": %d, \"kernel\": %d, \"us\": %.3f}%s\n",
            t.kind, t.hb, t.wb, t.fmt, t.nc, t.R, t.ctas, t.kernel, t.us,
            i + 1 < h->tuned.size() ? "," : "");
  }
  fprintf(f, " ]}\n");
  const bool ok = fclose(f) == 0;
  if (!ok || rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    return SOBEL4_ERR_INVALID_ARG;
  }
  return SOBEL4_OK;
}

extern "C" sobel4_status sobel4_tune_load(sobel4_handle h, const char *path) {
  if (!h || !path) return SOBEL4_ERR_INVALID_ARG;
  FILE *f = fopen(path, "r");
  if (!f) return SOBEL4_ERR_INVALID_ARG;
  char line[512];
  bool header_ok = false, device_ok = false;
  std::vector<TuneEntry> got;
  while (fgets(line, sizeof(line), f)) {
    if (strstr(line, "\"sobel4_tune\": 1")) {
      header_ok = true;
      char want[320];
      snprintf(want, sizeof(want), "\"device\": \"%s\", \"sm_count\": %d,", h->device_name,
               h->sm_count);
      device_ok = strstr(line, want) != nullptr;
      continue;
    }
    TuneEntry t;
    if (sscanf(line,
               " {\"kind\": %d, \"hb\": %d, \"wb\": %d, \"fmt\": %d, \"nc\": %d, \"R\": %d, "
               "\"ctas\": %d, \"kernel\": %d, \"us\": %f}",
               &t.kind, &t.hb, &t.wb, &t.fmt, &t.nc, &t.R, &t.ctas, &t.kernel, &t.us) == 9) {
      if (!valid_entry(t)) {
        fclose(f);
        return SOBEL4_ERR_INVALID_ARG;
      }
      got.push_back(t);
    }
  }
  fclose(f);
  if (!header_ok) return SOBEL4_ERR_INVALID_ARG;
  if (!device_ok) return SOBEL4_ERR_UNSUPPORTED;  // tuned on another device: keep the heuristic
  for (const TuneEntry &t : got) upsert(h, t);
  return SOBEL4_OK;
}
