// sobel4_tma.cu — host side of the TMA-staged kernel: the source tensor map
// (encoded through the driver entry point, so the library needs no -lcuda),
// the strip-height rule and the launch.
#include <cudaTypedefs.h>

#include <algorithm>

#include "sobel4_launch.h"
#include "sobel4_tma.cuh"

#ifndef SOBEL4_TMA_L2PROMO
#define SOBEL4_TMA_L2PROMO 3  // L2 fill granule of the copies: 0 none, 1 64 B, 2 128 B, 3 256 B
#endif

namespace sobel4 {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      (void)cudaGetLastError();
      p = nullptr;
    }
    return (PFN_cuTensorMapEncodeTiled_v12000)p;
  }();
  return fn;
}

template <int FMT, int MODE>
int tma_resident() {
  static const int r = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tma::tma_single_kernel<FMT, MODE>,
                                                      tma::kWarps * 32, 0) != cudaSuccess ||
        b < 1) {
      (void)cudaGetLastError();
      b = 1;
    }
    return b;
  }();
  return r;
}

template <int MODE>
int resident_mode(int fmt) {
  switch (fmt) {
    case kF32: return tma_resident<kF32, MODE>();
    case kU8: return tma_resident<kU8, MODE>();
    default: return tma_resident<kS16x4, MODE>();
  }
}

int resident_for(int fmt) { return resident_mode<tma::kFastOnly>(fmt); }

// Which kernels an image needs: every item on the fast path (one lean
// kernel), none (one general kernel), or both kinds: two launches when the
// image is large enough to fill the GPU twice over, else one kernel that
// carries both paths.
enum Plan { kPlanFast, kPlanGeneral, kPlanBoth, kPlanAll };

Plan plan_for(int32_t W, int border, int fmt, int dst_align, int64_t items, int sm_count) {
  const int vec_need = fmt == kF32 ? 16 : (fmt == kU8 ? 4 : 8);
  if (dst_align < vec_need || W < tma::kCols) return kPlanGeneral;
  if (W % tma::kCols == 0 && (border == kValid || border == kConstant0)) return kPlanFast;
  const int64_t warps = (int64_t)sm_count * resident_for(fmt) * tma::kWarps;
  return items >= 2 * warps ? kPlanBoth : kPlanAll;
}

template <int FMT, int MODE>
void launch_single_mode(const CUtensorMap &map, const tma::TmaImage &im, int border, int R,
                        int items, int sm_count, unsigned int *pair, unsigned int *err,
                        cudaStream_t st) {
  const int64_t cap = (int64_t)sm_count * tma_resident<FMT, MODE>();
  const int64_t grid = std::min<int64_t>((items + tma::kWarps - 1) / tma::kWarps, cap);
  tma::tma_single_kernel<FMT, MODE><<<(unsigned)grid, tma::kWarps * 32, 0, st>>>(
      map, im, border, R, items, pair, err);
}

template <int FMT>
void launch_single_plan(Plan plan, const CUtensorMap &map, const tma::TmaImage &im, int border,
                        int R, int items, int sm_count, unsigned int *pair, unsigned int *err,
                        cudaStream_t st) {
  if (plan == kPlanFast) {
    launch_single_mode<FMT, tma::kFastOnly>(map, im, border, R, items, sm_count, pair, err, st);
  } else if (plan == kPlanGeneral) {
    launch_single_mode<FMT, tma::kGeneralOnly>(map, im, border, R, items, sm_count, pair, err, st);
  } else if (plan == kPlanAll) {
    launch_single_mode<FMT, tma::kAll>(map, im, border, R, items, sm_count, pair, err, st);
  } else {
    launch_single_mode<FMT, tma::kFastOnly>(map, im, border, R, items, sm_count, pair, err, st);
    launch_single_mode<FMT, tma::kGeneralOnly>(map, im, border, R, items, sm_count, pair + 2,
                                               err, st);
  }
}

}  // namespace

bool tma_eligible(const uint8_t *src, size_t sp) {
  return ((uintptr_t)src % 16 == 0) && (sp % 16 == 0) && sp < (1ull << 40) &&
         encode_fn() != nullptr;
}

int tma_round_R(int R) {
  R = std::max(R, tma::kUnroll);
  return (R + tma::kUnroll - 1) / tma::kUnroll * tma::kUnroll;
}

int tma_pick_R(int fmt, int sm_count, int32_t H, int32_t W) {
  const int64_t n_seg = (W + tma::kCols - 1) / tma::kCols;
  // About two items per resident warp: the second round absorbs the spread
  // of per-warp speeds better than one item each (measured on 8192^2).
  const int64_t warps = (int64_t)sm_count * resident_for(fmt) * tma::kWarps;
  const int64_t bands = std::max<int64_t>(1, (2 * warps + n_seg - 1) / n_seg);
  int64_t R = (H + 2 * bands - 1) / (2 * bands);
  R = std::max<int64_t>(R, 8);
  R = (R + tma::kUnroll - 1) / tma::kUnroll * tma::kUnroll;
  return (int)std::min<int64_t>(R, 1 << 20);
}

namespace {

// The source tensor map: 2-D uint8 {W, H}, row stride sp, box 160 x 8,
// zero fill outside the image.
cudaError_t encode_map(CUtensorMap *map, const uint8_t *src, size_t sp, int32_t H, int32_t W) {
  const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
  const cuuint64_t strides[1] = {(cuuint64_t)sp};
  const cuuint32_t box[2] = {(cuuint32_t)tma::kBoxW, (cuuint32_t)tma::kStageRows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult cr = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void *)src, dims,
                                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                  CU_TENSOR_MAP_SWIZZLE_NONE,
                                  (CUtensorMapL2promotion)SOBEL4_TMA_L2PROMO,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return cr == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

tma::TmaImage make_image(const uint8_t *src, size_t sp, void *dst, size_t dp, int32_t H,
                         int32_t W, int R) {
  tma::TmaImage im;
  im.src = src;
  im.sp = sp;
  im.dst = dst;
  im.dp = dp;
  im.H = H;
  im.W = W;
  im.n_seg = (W + tma::kCols - 1) / tma::kCols;
  im.n_band = (H + 2 * R - 1) / (2 * R);
  int a = 1;
  while (a < 16 && (((uintptr_t)dst | (uintptr_t)dp) % (uintptr_t)(2 * a)) == 0) a *= 2;
  im.dst_align = a;
  im.lose_stage = -1;
  return im;
}

}  // namespace

cudaError_t launch_tma_single(const uint8_t *src, size_t sp, void *dst, size_t dp, int32_t H,
                              int32_t W, int border, int fmt, int R, int sm_count,
                              unsigned int *pair, unsigned int *err, cudaStream_t st,
                              int lose_stage) {
  if (R < tma::kUnroll || R % tma::kUnroll) return cudaErrorInvalidValue;
  CUtensorMap map;
  cudaError_t e = encode_map(&map, src, sp, H, W);
  if (e != cudaSuccess) return e;
  tma::TmaImage im = make_image(src, sp, dst, dp, H, W, R);
  im.lose_stage = lose_stage;
  const int64_t items = (int64_t)im.n_seg * im.n_band;
  if (items >= (1ll << 31)) return cudaErrorInvalidValue;
  const Plan plan = plan_for(W, border, fmt, im.dst_align, items, sm_count);
  (void)cudaGetLastError();  // report this launch only, not an earlier failed call
  switch (fmt) {
    case kF32:
      launch_single_plan<kF32>(plan, map, im, border, R, (int)items, sm_count, pair, err, st);
      break;
    case kU8:
      launch_single_plan<kU8>(plan, map, im, border, R, (int)items, sm_count, pair, err, st);
      break;
    default:
      launch_single_plan<kS16x4>(plan, map, im, border, R, (int)items, sm_count, pair, err, st);
      break;
  }
  return cudaGetLastError();
}

int tma_launches(int32_t H, int32_t W, int border, int fmt, const void *dst, size_t dp, int R,
                 int sm_count) {
  const tma::TmaImage im = make_image(nullptr, 0, (void *)dst, dp, H, W, R);
  return plan_for(W, border, fmt, im.dst_align, (int64_t)im.n_seg * im.n_band, sm_count) ==
                 kPlanBoth
             ? 2
             : 1;
}

size_t tma_batch_desc_bytes() { return sizeof(tma::TmaBatchDesc); }

cudaError_t tma_fill_batch_desc(void *out, const uint8_t *src, size_t sp, void *dst, size_t dp,
                                int32_t H, int32_t W, int R, int64_t item0, int64_t *items) {
  tma::TmaBatchDesc *d = (tma::TmaBatchDesc *)out;
  cudaError_t e = encode_map(&d->map, src, sp, H, W);
  if (e != cudaSuccess) return e;
  d->im = make_image(src, sp, dst, dp, H, W, R);
  d->item0 = item0;
  *items = (int64_t)d->im.n_seg * d->im.n_band;
  return cudaSuccess;
}

cudaError_t launch_tma_batched(const void *d_descs, int n_img, int64_t total,
                               unsigned int *d_queue, int border, int fmt, int R, int grid,
                               int sm_count, unsigned int *err, cudaStream_t st, bool all_fast) {
  if (R < tma::kUnroll || R % tma::kUnroll || total >= (1ll << 31)) return cudaErrorInvalidValue;
  const tma::TmaBatchDesc *d = (const tma::TmaBatchDesc *)d_descs;
  (void)cudaGetLastError();  // report this launch only, not an earlier failed call
  auto go = [&](auto kernel, int res, unsigned int *queue) {
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(grid, (int64_t)sm_count * res));
    kernel<<<g, tma::kWarps * 32, 0, st>>>(d, n_img, (int)total, queue, border, R, err);
  };
  switch (fmt) {
    case kF32:
      go(tma::tma_batched_kernel<kF32, tma::kFastOnly>, tma_resident<kF32, tma::kFastOnly>(),
         d_queue);
      if (!all_fast)
        go(tma::tma_batched_kernel<kF32, tma::kGeneralOnly>,
           tma_resident<kF32, tma::kGeneralOnly>(), d_queue + 1);
      break;
    case kU8:
      go(tma::tma_batched_kernel<kU8, tma::kFastOnly>, tma_resident<kU8, tma::kFastOnly>(),
         d_queue);
      if (!all_fast)
        go(tma::tma_batched_kernel<kU8, tma::kGeneralOnly>,
           tma_resident<kU8, tma::kGeneralOnly>(), d_queue + 1);
      break;
    default:
      go(tma::tma_batched_kernel<kS16x4, tma::kFastOnly>,
         tma_resident<kS16x4, tma::kFastOnly>(), d_queue);
      if (!all_fast)
        go(tma::tma_batched_kernel<kS16x4, tma::kGeneralOnly>,
           tma_resident<kS16x4, tma::kGeneralOnly>(), d_queue + 1);
      break;
  }
  return cudaGetLastError();
}

bool tma_batch_all_fast(int32_t W, int border, int fmt, const void *dst, size_t dp) {
  int a = 1;
  while (a < 16 && (((uintptr_t)dst | (uintptr_t)dp) % (uintptr_t)(2 * a)) == 0) a *= 2;
  return plan_for(W, border, fmt, a, 0, 1) == kPlanFast;
}

}  // namespace sobel4
