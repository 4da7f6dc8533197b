// sobel4_direct.cu — the DIRECT kernel: Eq. (3) summed tap by tap per output
// pixel straight from global memory (the paper's "GM" baseline, Section 5.2).
#include <cstring>

#include "sobel4_launch.h"

namespace sobel4 {

// CUSTOM: the masks come from `m` (runtime weights, Eq. 5) instead of the
// Eq. (3) table.
// fr: the support radius of the masks (2 for 5x5, 1 for a 3x3 operator),
// the width of the frame the paper's rule leaves at 0.
template <int FMT, bool CUSTOM>
__global__ void __launch_bounds__(256) direct_kernel(ImageDesc im, int border, Masks4 m, int fr,
                                                     int32_t thr) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int H = im.H, W = im.W;
  if (x >= W || y >= H) return;
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
  const int32_t s = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3];
  uint8_t *row = (uint8_t *)im.dst + (uint64_t)(uint32_t)y * im.dp;
  if (FMT == kF32) {
    ((float *)row)[x] = magnitude_f32(s);
  } else if (FMT == kU8) {
    row[x] = (uint8_t)magnitude_u8(s);
  } else if (FMT == kU16) {
    ((uint16_t *)row)[x] = (uint16_t)magnitude_u16(s);
  } else if (FMT == kEdge8) {
    row[x] = (computed && s >= thr) ? 255 : 0;
  } else {
    const uint64_t plane = (uint64_t)(uint32_t)H * im.dp;
#pragma unroll
    for (int k = 0; k < 4; ++k) ((int16_t *)(row + k * plane))[x] = (int16_t)r[k];
  }
}

cudaError_t launch_direct(const ImageDesc &im, int border, int fmt, const Masks4 *masks,
                          int radius, int32_t thr, cudaStream_t st) {
  const dim3 block(32, 8);
  const dim3 grid((im.W + 31) / 32, (im.H + 7) / 8);
  Masks4 m;
  if (masks) m = *masks;
  else memset(&m, 0, sizeof(m));
  (void)cudaGetLastError();  // report this launch only, not an earlier failed call
#define SOBEL4_DIRECT(F)                                                          \
  (masks ? direct_kernel<F, true><<<grid, block, 0, st>>>(im, border, m, radius, thr)  \
         : direct_kernel<F, false><<<grid, block, 0, st>>>(im, border, m, radius, thr))
  switch (fmt) {
    case kF32: SOBEL4_DIRECT(kF32); break;
    case kU8: SOBEL4_DIRECT(kU8); break;
    case kU16: SOBEL4_DIRECT(kU16); break;
    case kEdge8: SOBEL4_DIRECT(kEdge8); break;
    default: SOBEL4_DIRECT(kS16x4); break;
  }
#undef SOBEL4_DIRECT
  return cudaGetLastError();
}

}  // namespace sobel4
