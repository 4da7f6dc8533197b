// sobel4_rg.cuh — RG kernels (single image and persistent batch), instantiated
// per output format by sobel4_rg_<fmt>.cu for NC = 2 and 4 columns per lane.
#pragma once

#include "sobel4_launch.h"

#ifndef SOBEL4_RG_MIN_CTAS
#define SOBEL4_RG_MIN_CTAS 4
#endif
#ifndef SOBEL4_RG2_MIN_CTAS
#define SOBEL4_RG2_MIN_CTAS 6
#endif

namespace sobel4 {

template <int NC>
constexpr int rg_min_ctas() { return NC == 4 ? SOBEL4_RG_MIN_CTAS : SOBEL4_RG2_MIN_CTAS; }

template <int NC, int FMT>
__global__ void __launch_bounds__(kWarpsPerCta * 32, rg_min_ctas<NC>())
    rg_single_kernel(ImageDesc im, int border, int R, int n_items) {
  __shared__ WarpRing<NC> rings[kWarpsPerCta];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * kWarpsPerCta + warp;
  if (item >= n_items) return;
  const int band = item / im.n_seg;
  const int seg = item - band * im.n_seg;
  rg_dispatch<NC, FMT>(im, border, seg, band, R, lane, rings[warp]);
}

template <int NC, int FMT>
__global__ void __launch_bounds__(kWarpsPerCta * 32, rg_min_ctas<NC>())
    rg_batched_kernel(const ImageDesc *__restrict__ descs, int n_img, int64_t total,
                      unsigned int *queue, int border, int R) {
  __shared__ WarpRing<NC> rings[kWarpsPerCta];
  const int lane = threadIdx.x & 31;
  WarpRing<NC> &ring = rings[threadIdx.x >> 5];
  for (;;) {
    unsigned int got = 0;
    if (lane == 0) got = atomicAdd(queue, 1u);
    const int64_t item = (int64_t)__shfl_sync(0xffffffffu, got, 0);
    if (item >= total) break;
    // Largest image index whose first item is <= item.
    int lo = 0, hi = n_img - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(&descs[mid].item0) <= item) lo = mid;
      else hi = mid - 1;
    }
    const ImageDesc im = descs[lo];
    const int64_t local = item - im.item0;
    const int band = (int)(local / im.n_seg);
    const int seg = (int)(local - (int64_t)band * im.n_seg);
    rg_dispatch<NC, FMT>(im, border, seg, band, R, lane, ring);
  }
}

template <int FMT>
cudaError_t launch_rg_single_fmt(const ImageDesc &im, int border, int R, int nc,
                                 cudaStream_t st) {
  const int64_t items = (int64_t)im.n_seg * im.n_band;
  if (items <= 0) return cudaSuccess;
  const int64_t grid = (items + kWarpsPerCta - 1) / kWarpsPerCta;
  (void)cudaGetLastError();  // report this launch only, not an earlier failed call
  if (nc == 2)
    rg_single_kernel<2, FMT><<<(unsigned)grid, kWarpsPerCta * 32, 0, st>>>(im, border, R,
                                                                          (int)items);
  else
    rg_single_kernel<4, FMT><<<(unsigned)grid, kWarpsPerCta * 32, 0, st>>>(im, border, R,
                                                                          (int)items);
  return cudaGetLastError();
}

template <int FMT>
cudaError_t launch_rg_batched_fmt(const ImageDesc *d_descs, int n_img, int64_t total,
                                  unsigned int *d_queue, int border, int R, int nc, int grid,
                                  cudaStream_t st) {
  (void)cudaGetLastError();  // report this launch only, not an earlier failed call
  if (nc == 2)
    rg_batched_kernel<2, FMT><<<grid, kWarpsPerCta * 32, 0, st>>>(d_descs, n_img, total,
                                                                 d_queue, border, R);
  else
    rg_batched_kernel<4, FMT><<<grid, kWarpsPerCta * 32, 0, st>>>(d_descs, n_img, total,
                                                                 d_queue, border, R);
  return cudaGetLastError();
}

}  // namespace sobel4
