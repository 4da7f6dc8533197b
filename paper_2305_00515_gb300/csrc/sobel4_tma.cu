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

template <int FMT>
int tma_resident() {
  static const int r = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tma::tma_single_kernel<FMT>,
                                                      tma::kWarps * 32, 0) != cudaSuccess ||
        b < 1) {
      (void)cudaGetLastError();
      b = 1;
    }
    return b;
  }();
  return r;
}

int resident_for(int fmt) {
  switch (fmt) {
    case kF32: return tma_resident<kF32>();
    case kU8: return tma_resident<kU8>();
    default: return tma_resident<kS16x4>();
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
  const int64_t cap = (int64_t)sm_count * resident_for(fmt);
  const int64_t grid = std::min<int64_t>((items + tma::kWarps - 1) / tma::kWarps, cap);
  (void)cudaGetLastError();  // report this launch only, not an earlier failed call
  const dim3 g((unsigned)grid), b(tma::kWarps * 32);
  switch (fmt) {
    case kF32:
      tma::tma_single_kernel<kF32><<<g, b, 0, st>>>(map, im, border, R, (int)items, pair, err);
      break;
    case kU8:
      tma::tma_single_kernel<kU8><<<g, b, 0, st>>>(map, im, border, R, (int)items, pair, err);
      break;
    default:
      tma::tma_single_kernel<kS16x4><<<g, b, 0, st>>>(map, im, border, R, (int)items, pair, err);
      break;
  }
  return cudaGetLastError();
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
                               int sm_count, unsigned int *err, cudaStream_t st) {
  if (R < tma::kUnroll || R % tma::kUnroll || total >= (1ll << 31)) return cudaErrorInvalidValue;
  const int64_t cap = (int64_t)sm_count * resident_for(fmt);
  grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, cap));
  const tma::TmaBatchDesc *d = (const tma::TmaBatchDesc *)d_descs;
  (void)cudaGetLastError();  // report this launch only, not an earlier failed call
  const dim3 g((unsigned)grid), b(tma::kWarps * 32);
  switch (fmt) {
    case kF32:
      tma::tma_batched_kernel<kF32><<<g, b, 0, st>>>(d, n_img, (int)total, d_queue, border, R, err);
      break;
    case kU8:
      tma::tma_batched_kernel<kU8><<<g, b, 0, st>>>(d, n_img, (int)total, d_queue, border, R, err);
      break;
    default:
      tma::tma_batched_kernel<kS16x4><<<g, b, 0, st>>>(d, n_img, (int)total, d_queue, border, R,
                                                      err);
      break;
  }
  return cudaGetLastError();
}

}  // namespace sobel4
