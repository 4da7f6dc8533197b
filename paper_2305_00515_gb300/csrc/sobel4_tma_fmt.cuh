// sobel4_tma_fmt.cuh — launch helpers of the TMA-family kernels for one
// output format, explicitly instantiated once per format in
// sobel4_tma_{f32,u8,s16,u16,edge8}.cu so the kernel variants compile in parallel.
#pragma once

#include <algorithm>

#include "sobel4_tma.cuh"

namespace sobel4 {

template <int FMT>
struct TmaFmt {
  // Resident CTAs per SM of the single-image kernel (mode, staging).
  static int resident(int mode, int st);
  // cw: runtime-weight coefficients (nullptr: Eq. 3); not with S16X4 or RGB staging.
  static void single(int mode, int st, const CUtensorMap &map, const tma::TmaImage &im,
                     int border, int R, int items, int grid, unsigned int *pair,
                     unsigned int *err, cudaStream_t s, const Coefs *cw);
  // d: TmaBatchDesc array (tensor staging) or TmaBulkDesc array (bulk staging).
  static void batched(int mode, int st, const void *d, int n_img, int total,
                      unsigned int *queue, int border, int R, int grid, unsigned int *err,
                      cudaStream_t s);
};

namespace tma_detail {

template <typename K>
int occupancy(K kernel) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, tma::kWarps * 32, 0) !=
          cudaSuccess ||
      b < 1) {
    (void)cudaGetLastError();
    b = 1;
  }
  return b;
}

template <int FMT, int MODE, int ST>
int resident_of() {
  static const int r = occupancy(tma::tma_single_kernel<FMT, MODE, ST>);
  return r;
}

}  // namespace tma_detail

#define SOBEL4_TMA_SWITCH(MODE_, ST_, CALL)                                         \
  do {                                                                              \
    if ((ST_) == tma::kTensor) {                                                    \
      if ((MODE_) == tma::kFastOnly) { CALL(tma::kFastOnly, tma::kTensor); }        \
      else if ((MODE_) == tma::kFastRA) { CALL(tma::kFastRA, tma::kTensor); }      \
      else if ((MODE_) == tma::kGeneralOnly) { CALL(tma::kGeneralOnly, tma::kTensor); } \
      else { CALL(tma::kAll, tma::kTensor); }                                       \
    } else {                                                                        \
      if ((MODE_) == tma::kFastOnly) { CALL(tma::kFastOnly, tma::kBulk); }          \
      else if ((MODE_) == tma::kFastRA) { CALL(tma::kFastRA, tma::kBulk); }        \
      else if ((MODE_) == tma::kGeneralOnly) { CALL(tma::kGeneralOnly, tma::kBulk); } \
      else { CALL(tma::kAll, tma::kBulk); }                                         \
    }                                                                               \
  } while (0)

// The single-image kernel has two more modes (fast items of a ragged width;
// fast items with unaligned destination rows) and one more staging (RGB
// sources).
#define SOBEL4_TMA_SWITCH_SINGLE(MODE_, ST_, CALL)                                  \
  do {                                                                              \
    if ((ST_) == tma::kRgbBulk) {                                                   \
      if ((MODE_) == tma::kFastOnly) { CALL(tma::kFastOnly, tma::kRgbBulk); }       \
      else if ((MODE_) == tma::kFastPart) { CALL(tma::kFastPart, tma::kRgbBulk); }  \
      else if ((MODE_) == tma::kFastRA) { CALL(tma::kFastRA, tma::kRgbBulk); }      \
      else if ((MODE_) == tma::kGeneralOnly) { CALL(tma::kGeneralOnly, tma::kRgbBulk); } \
      else { CALL(tma::kAll, tma::kRgbBulk); }                                      \
    } else if ((MODE_) == tma::kFastPart) {                                         \
      if ((ST_) == tma::kTensor) { CALL(tma::kFastPart, tma::kTensor); }            \
      else { CALL(tma::kFastPart, tma::kBulk); }                                    \
    } else {                                                                        \
      SOBEL4_TMA_SWITCH(MODE_, ST_, CALL);                                          \
    }                                                                               \
  } while (0)

template <int FMT>
int TmaFmt<FMT>::resident(int mode, int st) {
#define SOBEL4_RES(M, S) return tma_detail::resident_of<FMT, M, S>()
  SOBEL4_TMA_SWITCH_SINGLE(mode, st, SOBEL4_RES);
#undef SOBEL4_RES
}

#if SOBEL4_PDL
// Launch with the programmatic-stream-serialization attribute (the kernel
// waits for the previous grid itself, in grid_dependency_wait).
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), int grid, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(tma::kWarps * 32);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  (void)cudaLaunchKernelEx(&cfg, kernel, args...);
}
#endif

template <int FMT, int M, int S, bool CW>
void single_launch(const CUtensorMap &map, const tma::TmaImage &im, int border, int R, int items,
                   int grid, unsigned int *pair, unsigned int *err, cudaStream_t s,
                   const Coefs &cw) {
#if SOBEL4_PDL
  launch_pdl(tma::tma_single_kernel<FMT, M, S, CW>, grid, s, map, im, border, R, items, pair, err,
             cw);
#else
  tma::tma_single_kernel<FMT, M, S, CW><<<(unsigned)grid, tma::kWarps * 32, 0, s>>>(
      map, im, border, R, items, pair, err, cw);
#endif
}

template <int FMT>
void TmaFmt<FMT>::single(int mode, int st, const CUtensorMap &map, const tma::TmaImage &im,
                         int border, int R, int items, int grid, unsigned int *pair,
                         unsigned int *err, cudaStream_t s, const Coefs *cw) {
  const Coefs none = {};
#define SOBEL4_SINGLE(M, S)                                                                   \
  do {                                                                                        \
    if constexpr (FMT != kS16x4 && (S) != tma::kRgbBulk) {                                    \
      if (cw) {                                                                               \
        single_launch<FMT, M, S, true>(map, im, border, R, items, grid, pair, err, s, *cw);   \
        break;                                                                                \
      }                                                                                       \
    }                                                                                         \
    single_launch<FMT, M, S, false>(map, im, border, R, items, grid, pair, err, s, none);     \
  } while (0)
  SOBEL4_TMA_SWITCH_SINGLE(mode, st, SOBEL4_SINGLE);
#undef SOBEL4_SINGLE
}

template <int FMT>
void TmaFmt<FMT>::batched(int mode, int st, const void *d, int n_img, int total,
                          unsigned int *queue, int border, int R, int grid, unsigned int *err,
                          cudaStream_t s) {
#if SOBEL4_PDL
#define SOBEL4_BATCH(M, S)                                                                     \
  launch_pdl(tma::tma_batched_kernel<FMT, M, S>, grid, s,                                      \
             (const typename tma::BatchDescOf<S>::type *)d, n_img, total, queue, border, R, err)
#else
#define SOBEL4_BATCH(M, S)                                                                     \
  tma::tma_batched_kernel<FMT, M, S><<<(unsigned)grid, tma::kWarps * 32, 0, s>>>(              \
      (const typename tma::BatchDescOf<S>::type *)d, n_img, total, queue, border, R, err)
#endif
  SOBEL4_TMA_SWITCH(mode, st, SOBEL4_BATCH);
#undef SOBEL4_BATCH
}

extern template struct TmaFmt<kF32>;
extern template struct TmaFmt<kU8>;
extern template struct TmaFmt<kS16x4>;
extern template struct TmaFmt<kU16>;
extern template struct TmaFmt<kEdge8>;

}  // namespace sobel4
