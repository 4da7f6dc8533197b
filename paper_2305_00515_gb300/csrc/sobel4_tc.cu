// sobel4_tc.cu — host side of the tensor-core kernel: eligibility, the tensor
// maps (source: uint8 box 96 x 132; destination: float32 box 32 x 128 with the
// 128-byte swizzle), the tile grid and the launch.
#include <algorithm>
#include <cstring>

#include "sobel4_launch.h"
#include "sobel4_tc.cuh"

namespace sobel4 {

bool tc_eligible(const uint8_t *src, size_t sp, const void *dst, size_t dp, int32_t H, int32_t W,
                 int border, int fmt) {
  // W % 4: the store copies write whole 16-byte units, so a row must end on one.
  return fmt == kF32 && border == kValid && H >= 1 && W >= 8 && W % 4 == 0 &&
         tma_eligible(src, sp) && (uintptr_t)dst % 16 == 0 && dp % 16 == 0;
}

cudaError_t launch_tc_single(const uint8_t *src, size_t sp, void *dst, size_t dp, int32_t H,
                             int32_t W, int border, int fmt, int sm_count, unsigned int *err,
                             cudaStream_t st, int lose_tile) {
  if (!tc_eligible(src, sp, dst, dp, H, W, border, fmt)) return cudaErrorInvalidValue;
  alignas(64) CUtensorMap in_map, out_map;
  memset(&in_map, 0, sizeof(in_map));
  memset(&out_map, 0, sizeof(out_map));
  cudaError_t e = tma_encode_2d(&in_map, src, false, sp, H, W, tc::kBoxW, tc::kInRows, false);
  if (e == cudaSuccess) e = tma_encode_2d(&out_map, dst, true, dp, H, W, 32, tc::kM, true);
  if (e != cudaSuccess) return e;
  static const cudaError_t attr = cudaFuncSetAttribute(
      tc::tc_single_kernel<kF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)tc::kSmemBytes);
  if (attr != cudaSuccess) return attr;
  tc::TcImage im;
  im.H = H;
  im.W = W;
  im.n_tx = (W + tc::kTileCols - 1) / tc::kTileCols;
  const int64_t n_ty = (H + tc::kM - 1) / tc::kM;
  const int64_t n_tiles = n_ty * im.n_tx;
  if (n_tiles >= (1ll << 31)) return cudaErrorInvalidValue;
  im.n_tiles = (int32_t)n_tiles;
  im.lose_tile = lose_tile;
  const int grid = (int)std::min<int64_t>(n_tiles, std::max(sm_count, 1));
  (void)cudaGetLastError();  // report this launch only, not an earlier failed call
  tc::tc_single_kernel<kF32><<<grid, tc::kThreads, tc::kSmemBytes, st>>>(in_map, out_map, im, err);
  return cudaGetLastError();
}

}  // namespace sobel4
