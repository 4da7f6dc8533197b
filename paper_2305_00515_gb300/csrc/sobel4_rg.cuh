// sobel4_rg.cuh — RG kernels (single image and persistent batch), instantiated
// per output format by sobel4_rg_<fmt>.cu for NC = 2 and 4 columns per lane.
#pragma once

#include <algorithm>

#include "sobel4_launch.h"

#ifndef SOBEL4_RG_MIN_CTAS
#define SOBEL4_RG_MIN_CTAS 3
#endif
#ifndef SOBEL4_RG2_MIN_CTAS
#define SOBEL4_RG2_MIN_CTAS 6
#endif

namespace sobel4 {

template <int NC>
constexpr int rg_min_ctas() { return NC == 4 ? SOBEL4_RG_MIN_CTAS : SOBEL4_RG2_MIN_CTAS; }

// One image; a grid of at most the resident CTAs whose warps pull items
// (band-major, so the warps in flight work on neighbouring bands) from the
// counter pair[0].  Items differ in cost (edge segments and border bands take
// the general path), so the queue, not a fixed stride, balances the warps.
// The last warp out returns the pair to zero for the next launch that uses it:
// every other warp has made its final fetch before counting itself out in
// pair[1].
template <int NC, int FMT>
__global__ void __launch_bounds__(kWarpsPerCta * 32, rg_min_ctas<NC>())
    rg_single_kernel(ImageDesc im, int border, int R, int n_items, unsigned int *pair) {
  __shared__ WarpRing<NC> rings[kWarpsPerCta];
  const int lane = threadIdx.x & 31;
  WarpRing<NC> &ring = rings[threadIdx.x >> 5];
  for (;;) {
    unsigned int got = 0;
    if (lane == 0) got = atomicAdd(&pair[0], 1u);
    got = __shfl_sync(0xffffffffu, got, 0);
    if (got >= (unsigned int)n_items) break;
    const int item = (int)got;
    const int band = item / im.n_seg;
    const int seg = item - band * im.n_seg;
    rg_dispatch<NC, FMT>(im, border, seg, band, R, lane, ring);
  }
  if (lane == 0) {
    __threadfence();  // this warp's last fetch is performed before it counts out
    const unsigned int warps = gridDim.x * kWarpsPerCta;
    if (atomicAdd(&pair[1], 1u) == warps - 1u) {
      atomicExch(&pair[0], 0u);
      atomicExch(&pair[1], 0u);
    }
  }
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

// CTAs of `kernel` that fit on one SM at once (queried once per kernel).
template <typename Kernel>
int resident_ctas(Kernel kernel) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kWarpsPerCta * 32, 0) !=
          cudaSuccess ||
      b < 1) {
    (void)cudaGetLastError();
    b = 1;
  }
  return b;
}

template <int NC, int FMT>
int single_resident() {
  static const int r = resident_ctas(rg_single_kernel<NC, FMT>);
  return r;
}

template <int NC, int FMT>
int batched_resident() {
  static const int r = resident_ctas(rg_batched_kernel<NC, FMT>);
  return r;
}

template <int FMT>
cudaError_t launch_rg_single_fmt(const ImageDesc &im, int border, int R, int nc, int sm_count,
                                 unsigned int *pair, cudaStream_t st) {
  const int64_t items = (int64_t)im.n_seg * im.n_band;
  if (items <= 0) return cudaSuccess;
  const int64_t cap =
      (int64_t)sm_count * (nc == 2 ? single_resident<2, FMT>() : single_resident<4, FMT>());
  const int64_t grid = std::min<int64_t>((items + kWarpsPerCta - 1) / kWarpsPerCta, cap);
  (void)cudaGetLastError();  // report this launch only, not an earlier failed call
  if (nc == 2)
    rg_single_kernel<2, FMT><<<(unsigned)grid, kWarpsPerCta * 32, 0, st>>>(im, border, R,
                                                                          (int)items, pair);
  else
    rg_single_kernel<4, FMT><<<(unsigned)grid, kWarpsPerCta * 32, 0, st>>>(im, border, R,
                                                                          (int)items, pair);
  return cudaGetLastError();
}

template <int FMT>
cudaError_t launch_rg_batched_fmt(const ImageDesc *d_descs, int n_img, int64_t total,
                                  unsigned int *d_queue, int border, int R, int nc, int grid,
                                  int sm_count, cudaStream_t st) {
  // CTAs beyond the resident ones would only find the queue drained.
  const int64_t cap =
      (int64_t)sm_count * (nc == 2 ? batched_resident<2, FMT>() : batched_resident<4, FMT>());
  grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, cap));
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
