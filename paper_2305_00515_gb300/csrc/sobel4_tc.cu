// sobel4_tc.cu — host side of the tensor-core kernel: eligibility, the tensor
// maps (source: uint8 box 96 x 132; destination: float32 box 32 x 128 with the
// 128-byte swizzle), the tile grid and the launch.
#include <algorithm>
#include <cmath>
#include <cstdlib>
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

bool eq5_masks(double a, double b, double n, double m, Masks4 *out) {
  if (!(a > 0) || !(b > 0) || !(n > 0) || !(m > 0) || a != std::floor(a)) return false;
  // Factored rows: K_x = a (v x h), K_y = a (h x v) with v = (1 n m n 1),
  // h = (-1 -b 0 b 1); the diagonal pair through K_d+ = K_d + K_dt (rows
  // -q0, -q1, 0, q1, q0) and K_d- = K_d - K_dt (rows r0, r1, r2, r1, r0), so
  // that K_d = a (K_d+ + K_d-) / 2 and K_dt = a (K_d+ - K_d-) / 2.
  const double v[5] = {1, n, m, n, 1}, h[5] = {-1, -b, 0, b, 1};
  const double q0[5] = {m, n + b, 2, n + b, m};
  const double q1[5] = {n - b, m * b, 2 * n * b, m * b, n - b};
  const double r0[5] = {-m, b - n, 0, n - b, m};
  const double r1[5] = {-(n + b), -m * b, 0, m * b, n + b};
  const double r2[5] = {-2, -2 * n * b, 0, 2 * n * b, 2};
  const double *dp_rows[5] = {q0, q1, nullptr, q1, q0};
  const double dp_sign[5] = {-1, -1, 0, 1, 1};
  const double *dm_rows[5] = {r0, r1, r2, r1, r0};
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      const double kdp = dp_rows[i] ? dp_sign[i] * dp_rows[i][j] : 0.0;
      const double kdm = dm_rows[i][j];
      const double w[4] = {a * v[i] * h[j], a * h[i] * v[j], a * (kdp + kdm) / 2,
                           a * (kdp - kdm) / 2};
      for (int k = 0; k < 4; ++k) {
        const double r = std::nearbyint(w[k]);
        if (std::fabs(w[k] - r) > 1e-9 * std::max(1.0, std::fabs(w[k])) || std::fabs(r) > 32767)
          return false;
        out->w[k][i][j] = (int16_t)r;
      }
    }
  return true;
}

int operator_masks(int op, Masks4 *out) {
  memset(out, 0, sizeof(*out));
  if (op == 1) {  // two-directional 5x5: the x and y masks of the four-directional one
    eq5_masks(1, 2, 4, 6, out);
    memset(out->w[2], 0, sizeof(out->w[2]));
    memset(out->w[3], 0, sizeof(out->w[3]));
    return 2;
  }
  if (op == 2) {  // two-directional 3x3 (Eq. 1): (1 2 1)^T (-1 0 1) and its transpose
    const int v[3] = {1, 2, 1}, d[3] = {-1, 0, 1};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        out->w[0][1 + i][1 + j] = (int16_t)(v[i] * d[j]);
        out->w[1][1 + i][1 + j] = (int16_t)(d[i] * v[j]);
      }
    return 1;
  }
  return 0;
}

cudaError_t launch_tc_single(const uint8_t *src, size_t sp, void *dst, size_t dp, int32_t H,
                             int32_t W, int border, int fmt, int sm_count, unsigned int *err,
                             cudaStream_t st, int lose_tile, const Masks4 *masks, int radius) {
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
  if (radius != 1 && radius != 2) return cudaErrorInvalidValue;
  tc::TcImage im;
  im.fr = radius;
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
  static const Masks4 eq3 = [] {
    Masks4 m;
    eq5_masks(1, 2, 4, 6, &m);
    return m;
  }();
  for (int k = 0; k < 4; ++k)  // the products hold weights up to 2048 exactly (f16)
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j)
        if (masks && std::abs((int)masks->w[k][i][j]) > 2048) return cudaErrorInvalidValue;
  tc::tc_single_kernel<kF32><<<grid, tc::kThreads, tc::kSmemBytes, st>>>(
      in_map, out_map, im, masks ? *masks : eq3, err);
  return cudaGetLastError();
}

}  // namespace sobel4
