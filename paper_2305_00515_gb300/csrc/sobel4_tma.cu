// sobel4_tma.cu — host side of the TMA-family kernels: the source tensor map
// (encoded through the driver entry point, so the library needs no -lcuda),
// the choice of staging (tensor copies for 16-byte aligned rows, bulk row
// copies otherwise), the strip-height rule and the launch plan.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "sobel4_launch.h"
#include "sobel4_tma_fmt.cuh"

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

int resident(int fmt, int mode, int st) {
  switch (fmt) {
    case kF32: return TmaFmt<kF32>::resident(mode, st);
    case kU8: return TmaFmt<kU8>::resident(mode, st);
    case kU16: return TmaFmt<kU16>::resident(mode, st);
    case kEdge8: return TmaFmt<kEdge8>::resident(mode, st);
    default: return TmaFmt<kS16x4>::resident(mode, st);
  }
}

int resident_for(int fmt) { return resident(fmt, tma::kFastOnly, tma::kTensor); }

// The tensor staging needs 16-byte aligned rows and the driver's encoder.
bool tensor_ok(const uint8_t *src, size_t sp) {
  return ((uintptr_t)src % 16 == 0) && (sp % 16 == 0) && sp < (1ull << 40) &&
         encode_fn() != nullptr;
}

// Which kernel an image needs: every item on the fast path with vector
// stores (the lean kernel when the width is a multiple of the segment, the
// ragged-width fast kernel otherwise), every item on the fast path with
// destination rows that are not vector-aligned (the one-body fast kernel with
// split stores), none (the general kernel), or anything else (one kernel that
// carries both paths and the split stores, and hands the edge items out
// first).
enum Plan { kPlanFast, kPlanFastPart, kPlanFastRA, kPlanGeneral, kPlanAll };

Plan plan_for(int32_t W, int border, int fmt, int dst_align, int st) {
  const int vec_need = vec_bytes(fmt);
  if (border == kValid || (st == tma::kTensor && border == kConstant0)) {
    if (dst_align < vec_need) return kPlanFastRA;
    return W % tma::kCols == 0 ? kPlanFast : kPlanFastPart;
  }
  if (W < tma::kCols) return kPlanGeneral;
  return kPlanAll;
}

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
  im.thr = 0;
  return im;
}

void single(int fmt, int mode, int st, const CUtensorMap &map, const tma::TmaImage &im,
            int border, int R, int items, int sm_count, unsigned int *pair, unsigned int *err,
            cudaStream_t s, const Coefs *cw = nullptr) {
  const int64_t cap = (int64_t)sm_count * resident(fmt, mode, st);
  const int grid = (int)std::min<int64_t>((items + tma::kWarps - 1) / tma::kWarps, cap);
  switch (fmt) {
    case kF32:
      TmaFmt<kF32>::single(mode, st, map, im, border, R, items, grid, pair, err, s, cw);
      break;
    case kU8:
      TmaFmt<kU8>::single(mode, st, map, im, border, R, items, grid, pair, err, s, cw);
      break;
    case kU16:
      TmaFmt<kU16>::single(mode, st, map, im, border, R, items, grid, pair, err, s, cw);
      break;
    case kEdge8:
      TmaFmt<kEdge8>::single(mode, st, map, im, border, R, items, grid, pair, err, s, cw);
      break;
    default:
      TmaFmt<kS16x4>::single(mode, st, map, im, border, R, items, grid, pair, err, s, cw);
      break;
  }
}

}  // namespace

bool tma_eligible(const uint8_t *src, size_t sp) { return tensor_ok(src, sp); }

cudaError_t tma_encode_2d(void *map, const void *base, bool f32, size_t pitch, int32_t H,
                          int32_t W, int box_w, int box_h, bool swizzle128) {
  if (!base || (uintptr_t)base % 16 || pitch % 16 || pitch >= (1ull << 40) || !encode_fn())
    return cudaErrorInvalidValue;
  const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch};
  const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult cr = encode_fn()(
      (CUtensorMap *)map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
      (void *)base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
      swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
      f32 ? CU_TENSOR_MAP_L2_PROMOTION_NONE : (CUtensorMapL2promotion)SOBEL4_TMA_L2PROMO,
      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return cr == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int tma_round_R(int R) {
  R = std::max(R, tma::kUnroll);
  return (R + tma::kUnroll - 1) / tma::kUnroll * tma::kUnroll;
}

int tma_pick_R(int fmt, int sm_count, int32_t H, int32_t W, bool all_fast) {
  const int64_t n_seg = (W + tma::kCols - 1) / tma::kCols;
  // About two items per resident warp when every item takes the fast path:
  // the second round absorbs the spread of per-warp speeds better than one
  // item each (measured on 8192^2).  About six otherwise, so that the slower
  // edge items, handed out first, stay short beside the rest.
  const int64_t warps = (int64_t)sm_count * resident_for(fmt) * tma::kWarps;
  const int64_t per_warp = all_fast ? 2 : 6;
  const int64_t bands = std::max<int64_t>(1, (per_warp * warps + n_seg - 1) / n_seg);
  int64_t R = (H + 2 * bands - 1) / (2 * bands);
  R = std::max<int64_t>(R, 8);
  R = (R + tma::kUnroll - 1) / tma::kUnroll * tma::kUnroll;
  return (int)std::min<int64_t>(R, 1 << 20);
}

cudaError_t launch_tma_single(const uint8_t *src, size_t sp, void *dst, size_t dp, int32_t H,
                              int32_t W, int border, int fmt, int R, int sm_count,
                              unsigned int *pair, unsigned int *err, cudaStream_t st,
                              int lose_stage, int32_t thr, const Coefs *cw) {
  if (cw && fmt == kS16x4) return cudaErrorInvalidValue;  // its planes need R_d, R_dt
  if (R < tma::kUnroll || R % tma::kUnroll) return cudaErrorInvalidValue;
  const int staging = tensor_ok(src, sp) ? tma::kTensor : tma::kBulk;
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  if (staging == tma::kTensor) {
    const cudaError_t e = encode_map(&map, src, sp, H, W);
    if (e != cudaSuccess) return e;
  }
  tma::TmaImage im = make_image(src, sp, dst, dp, H, W, R);
  im.lose_stage = lose_stage;
  im.thr = thr;
  const int64_t items = (int64_t)im.n_seg * im.n_band;
  if (items >= (1ll << 31)) return cudaErrorInvalidValue;
  const Plan plan = plan_for(W, border, fmt, im.dst_align, staging);
  const int mode = plan == kPlanFast       ? tma::kFastOnly
                   : plan == kPlanFastPart ? tma::kFastPart
                   : plan == kPlanFastRA   ? tma::kFastRA
                   : plan == kPlanGeneral  ? tma::kGeneralOnly
                                           : tma::kAll;
  (void)cudaGetLastError();  // report this launch only, not an earlier failed call
  single(fmt, mode, staging, map, im, border, R, (int)items, sm_count, pair, err, st, cw);
  return cudaGetLastError();
}

cudaError_t launch_tma_single_rgb(const uint8_t *src, size_t sp, void *dst, size_t dp, int32_t H,
                                  int32_t W, int border, int fmt, int R, int sm_count,
                                  unsigned int *pair, unsigned int *err, cudaStream_t st,
                                  int32_t thr) {
  if (R < tma::kUnroll || R % tma::kUnroll) return cudaErrorInvalidValue;
  CUtensorMap map;  // not used by the RGB staging
  memset(&map, 0, sizeof(map));
  tma::TmaImage im = make_image(src, sp, dst, dp, H, W, R);
  im.thr = thr;
  const int64_t items = (int64_t)im.n_seg * im.n_band;
  if (items >= (1ll << 31)) return cudaErrorInvalidValue;
  const Plan plan = plan_for(W, border, fmt, im.dst_align, tma::kBulk);
  const int mode = plan == kPlanFast       ? tma::kFastOnly
                   : plan == kPlanFastPart ? tma::kFastPart
                   : plan == kPlanFastRA   ? tma::kFastRA
                   : plan == kPlanGeneral  ? tma::kGeneralOnly
                                           : tma::kAll;
  (void)cudaGetLastError();  // report this launch only, not an earlier failed call
  single(fmt, mode, tma::kRgbBulk, map, im, border, R, (int)items, sm_count, pair, err, st);
  return cudaGetLastError();
}

size_t tma_batch_desc_bytes(bool bulk) {
  return bulk ? sizeof(tma::TmaBulkDesc) : sizeof(tma::TmaBatchDesc);
}

cudaError_t tma_fill_batch_desc(void *out, bool bulk, const uint8_t *src, size_t sp, void *dst,
                                size_t dp, int32_t H, int32_t W, int R, int64_t item0,
                                int64_t *items, int32_t thr) {
  tma::TmaImage im = make_image(src, sp, dst, dp, H, W, R);
  im.thr = thr;
  if (bulk) {
    tma::TmaBulkDesc *d = (tma::TmaBulkDesc *)out;
    memset(d, 0, sizeof(*d));
    d->im = im;
    d->item0 = item0;
  } else {
    if (!tensor_ok(src, sp)) return cudaErrorInvalidValue;
    tma::TmaBatchDesc *d = (tma::TmaBatchDesc *)out;
    memset(d, 0, sizeof(*d));
    const cudaError_t e = encode_map(&d->map, src, sp, H, W);
    if (e != cudaSuccess) return e;
    d->im = im;
    d->item0 = item0;
  }
  *items = (int64_t)im.n_seg * im.n_band;
  return cudaSuccess;
}

bool tma_all_fast_staged(int32_t W, int border, int fmt, bool bulk, const void *dst, size_t dp) {
  return tma_fast_level(W, border, fmt, bulk, dst, dp) == kBatchFastVec;
}

int tma_fast_level(int32_t W, int border, int fmt, bool bulk, const void *dst, size_t dp) {
  int a = 1;
  while (a < 16 && (((uintptr_t)dst | (uintptr_t)dp) % (uintptr_t)(2 * a)) == 0) a *= 2;
  const Plan plan = plan_for(W, border, fmt, a, bulk ? tma::kBulk : tma::kTensor);
  return plan == kPlanFast || plan == kPlanFastPart ? kBatchFastVec
         : plan == kPlanFastRA                      ? kBatchFastSplit
                                                    : kBatchGeneral;
}

bool tma_all_fast(int32_t W, int border, int fmt, const uint8_t *src, size_t sp,
                        const void *dst, size_t dp) {
  return tma_all_fast_staged(W, border, fmt, !tensor_ok(src, sp), dst, dp);
}

cudaError_t launch_tma_batched(const void *d_descs, int n_img, int64_t total,
                               unsigned int *d_queue, int border, int fmt, int R, int grid,
                               int sm_count, unsigned int *err, cudaStream_t st, int fast,
                               bool bulk) {
  if (R < tma::kUnroll || R % tma::kUnroll || total >= (1ll << 31)) return cudaErrorInvalidValue;
  const void *d = d_descs;
  const int staging = bulk ? tma::kBulk : tma::kTensor;
  (void)cudaGetLastError();  // report this launch only, not an earlier failed call
  auto go = [&](int mode, unsigned int *queue) {
    const int g = (int)std::max<int64_t>(
        1, std::min<int64_t>(grid, (int64_t)sm_count * resident(fmt, mode, staging)));
    switch (fmt) {
      case kF32:
        TmaFmt<kF32>::batched(mode, staging, d, n_img, (int)total, queue, border, R, g, err, st);
        break;
      case kU8:
        TmaFmt<kU8>::batched(mode, staging, d, n_img, (int)total, queue, border, R, g, err, st);
        break;
      case kU16:
        TmaFmt<kU16>::batched(mode, staging, d, n_img, (int)total, queue, border, R, g, err, st);
        break;
      case kEdge8:
        TmaFmt<kEdge8>::batched(mode, staging, d, n_img, (int)total, queue, border, R, g, err,
                                st);
        break;
      default:
        TmaFmt<kS16x4>::batched(mode, staging, d, n_img, (int)total, queue, border, R, g, err,
                                st);
        break;
    }
  };
  go(fast == kBatchFastVec ? tma::kFastOnly : fast == kBatchFastSplit ? tma::kFastRA : tma::kAll,
     d_queue);
  return cudaGetLastError();
}

}  // namespace sobel4
