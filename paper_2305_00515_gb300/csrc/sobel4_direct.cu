// sobel4_direct.cu — the DIRECT kernel: Eq. (3) summed tap by tap per output
// pixel straight from global memory (the paper's "GM" baseline, Section 5.2).
#include <algorithm>
#include <cstring>

#include "sobel4_launch.h"

namespace sobel4 {

// One output pixel: the 25 taps of each mask, then S and the format's rule.
template <int FMT, bool CUSTOM>
__device__ __forceinline__ void direct_px(const ImageDesc &im, int border, const Masks4 &m,
                                          int fr, int32_t thr, int x, int y) {
  const int H = im.H, W = im.W;
  int32_t r[4] = {0, 0, 0, 0};
  const bool computed =
      border != kValid || (y >= fr && y <= H - 1 - fr && x >= fr && x <= W - 1 - fr);
  if (computed) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      bool zr;
      const int yy = map_index(y + i - 2, H, border, &zr);
      const uint8_t *row = im.src + (uint64_t)(uint32_t)yy * im.sp;
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        bool zc;
        const int xx = map_index(x + j - 2, W, border, &zc);
        const int32_t v = (zr || zc) ? 0 : (int32_t)__ldg(row + xx);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          r[k] += (CUSTOM ? (int32_t)m.w[k][i][j] : (int32_t)kMasks[k][i][j]) * v;
      }
    }
  }
  store_px<FMT>(im, x, y, r, computed, thr);
}

// CUSTOM: the masks come from `m` (runtime weights, Eq. 5) instead of the
// Eq. (3) table.
// fr: the support radius of the masks (2 for 5x5, 1 for a 3x3 operator),
// the width of the frame the paper's rule leaves at 0.
// y0: first row of this launch (images taller than one grid of 65,535 blocks
// of 8 rows take several launches).
template <int FMT, bool CUSTOM>
__global__ void __launch_bounds__(256) direct_kernel(ImageDesc im, int border, Masks4 m, int fr,
                                                     int32_t thr, int y0) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = y0 + blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= im.W || y >= im.H) return;
  direct_px<FMT, CUSTOM>(im, border, m, fr, thr, x, y);
}

cudaError_t launch_direct(const ImageDesc &im, int border, int fmt, const Masks4 *masks,
                          int radius, int32_t thr, cudaStream_t st) {
  const dim3 block(32, 8);
  constexpr int kRowsPerGrid = 65535 * 8;
  Masks4 m;
  if (masks) m = *masks;
  else memset(&m, 0, sizeof(m));
  (void)cudaGetLastError();  // report this launch only, not an earlier failed call
#define SOBEL4_DIRECT(F)                                                                  \
  (masks ? direct_kernel<F, true><<<grid, block, 0, st>>>(im, border, m, radius, thr, y0)   \
         : direct_kernel<F, false><<<grid, block, 0, st>>>(im, border, m, radius, thr, y0))
  for (int y0 = 0; y0 < im.H; y0 += kRowsPerGrid) {
    const dim3 grid((im.W + 31) / 32, (unsigned)((std::min(im.H - y0, kRowsPerGrid) + 7) / 8));
    switch (fmt) {
      case kF32: SOBEL4_DIRECT(kF32); break;
      case kU8: SOBEL4_DIRECT(kU8); break;
      case kU16: SOBEL4_DIRECT(kU16); break;
      case kEdge8: SOBEL4_DIRECT(kEdge8); break;
      default: SOBEL4_DIRECT(kS16x4); break;
    }
  }
#undef SOBEL4_DIRECT
  return cudaGetLastError();
}

}  // namespace sobel4
