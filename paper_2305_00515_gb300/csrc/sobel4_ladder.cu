// sobel4_ladder.cu — the paper's kernel ladder (Section 5.2, Table 1) as
// product variants, so that its ablation can be re-measured on GB300:
//
//  * SM:    each CTA stages a 32 x 8 output tile plus its 2-pixel halo in
//           shared memory, then every thread sums the 25 taps of the four
//           masks of Eq. (3) from there.
//  * SM-P:  SM with prefetching (Section 4.2): a CTA walks 8 tiles down a
//           column strip, and the global loads of the next tile are issued
//           into registers before the current tile is computed, then written
//           to the other half of a double-buffered tile.
//  * RG:    the register window of Section 4.3 in the paper's plain form: one
//           column per lane, 32 lanes load 32 columns and the first 28 produce
//           output (neighbours by __shfl_down_sync, the 2r overlap of the task
//           assignment), rows walked sequentially with the 1x5 passes of K_x
//           and K_y kept in a 5-row register ring (Eq. 6-9); the diagonals
//           K_d and K_dt summed over a 5x5 window of raw pixels in registers.
//  * RG-v1: RG with the diagonals transformed into K_d+ and K_d- (Eq. 10-11):
//           K_d+ through its two distinct row vectors (Eq. 12-15), K_d- still
//           over the raw window; G_d = (P + M) / 2, G_dt = (P - M) / 2.
//  * RG-v2: RG-v1 with K_d- decomposed as well (Eq. 16-19): its rows are
//           r0 = [-6 -2 0 2 6], 6 x [-1 -2 0 2 1] and r2 = [-2 -16 0 16 2].
//
// Arithmetic is scalar int32 (no packing), every border rule goes through
// map_index on each load, and all five output formats share store_px with the
// DIRECT kernel, so every variant is exact against the same oracle.  The
// GB300 design (TMA-staged packed register window, sobel4_tma.cuh) is the
// product path; these kernels exist for the ablation.
#include <algorithm>

#include "sobel4_launch.h"

namespace sobel4 {
namespace {

// Pixel (y, x) under the border rule (0 where CONSTANT0 reads outside; VALID
// clamps, and its frame outputs are zeroed anyway).
__device__ __forceinline__ int32_t load_px(const ImageDesc &im, int y, int x, int border) {
  bool zr, zc;
  const int my = map_index(y, im.H, border, &zr);
  const int mx = map_index(x, im.W, border, &zc);
  if (zr || zc) return 0;
  return (int32_t)__ldg(im.src + (uint64_t)(uint32_t)my * im.sp + mx);
}

__device__ __forceinline__ bool computed_px(const ImageDesc &im, int border, int y, int x) {
  return border != kValid || (y >= 2 && y <= im.H - 3 && x >= 2 && x <= im.W - 3);
}

// The four responses of Eq. (3) at tile position (ty, tx) of a staged tile
// whose row pitch is TW + 4 (the masks as compile-time constants, so zero taps
// cost nothing).
template <int TW>
__device__ __forceinline__ void taps25(const uint8_t *t, int ty, int tx, int32_t r[4]) {
  constexpr int8_t K[4][5][5] = SOBEL4_EQ3_MASKS;
#pragma unroll
  for (int k = 0; k < 4; ++k) r[k] = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const int32_t v = t[(ty + i) * (TW + 4) + tx + j];
#pragma unroll
      for (int k = 0; k < 4; ++k) r[k] += (int32_t)K[k][i][j] * v;
    }
}

constexpr int kTileW = 32, kTileH = 8;          // output tile of one CTA (one thread per pixel)
constexpr int kTileElems = (kTileW + 4) * (kTileH + 4);
constexpr int kSmpTiles = 8;                    // tiles per CTA down a column strip (SM-P)

template <int FMT>
__global__ void __launch_bounds__(kTileW * kTileH) sm_kernel(ImageDesc im, int border,
                                                            int32_t thr) {
  __shared__ uint8_t tile[kTileElems];
  const int tid = threadIdx.y * kTileW + threadIdx.x;
  const int x0 = blockIdx.x * kTileW;
  const int n_ty = (im.H + kTileH - 1) / kTileH;
  for (int tyi = blockIdx.y; tyi < n_ty; tyi += gridDim.y) {  // uniform across the CTA
    const int y0 = tyi * kTileH;
    __syncthreads();  // the previous tile has been read
    for (int e = tid; e < kTileElems; e += kTileW * kTileH)
      tile[e] = (uint8_t)load_px(im, y0 - 2 + e / (kTileW + 4), x0 - 2 + e % (kTileW + 4), border);
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x < im.W && y < im.H) {
      int32_t r[4] = {0, 0, 0, 0};
      const bool comp = computed_px(im, border, y, x);
      if (comp) taps25<kTileW>(tile, threadIdx.y, threadIdx.x, r);
      store_px<FMT>(im, x, y, r, comp, thr);
    }
  }
}

template <int FMT>
__global__ void __launch_bounds__(kTileW * kTileH) smp_kernel(ImageDesc im, int border,
                                                             int32_t thr) {
  __shared__ uint8_t tile[2][kTileElems];
  constexpr int kPer = (kTileElems + kTileW * kTileH - 1) / (kTileW * kTileH);  // 2
  const int tid = threadIdx.y * kTileW + threadIdx.x;
  const int x0 = blockIdx.x * kTileW;
  const int n_strips = (im.H + kTileH * kSmpTiles - 1) / (kTileH * kSmpTiles);
  int32_t pre[kPer];
  auto fetch = [&](int y0) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = tid + q * kTileW * kTileH;
      pre[q] = e < kTileElems
                   ? load_px(im, y0 - 2 + e / (kTileW + 4), x0 - 2 + e % (kTileW + 4), border)
                   : 0;
    }
  };
  auto put = [&](int buf) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = tid + q * kTileW * kTileH;
      if (e < kTileElems) tile[buf][e] = (uint8_t)pre[q];
    }
  };
  for (int si = blockIdx.y; si < n_strips; si += gridDim.y) {  // uniform across the CTA
    const int ys = si * kTileH * kSmpTiles;
    __syncthreads();  // the previous strip's last tile has been read
    fetch(ys);
    put(0);
    __syncthreads();
    for (int t = 0; t < kSmpTiles; ++t) {
      const int y0 = ys + t * kTileH;
      if (y0 >= im.H) break;  // uniform
      const bool more = t + 1 < kSmpTiles && y0 + kTileH < im.H;
      if (more) fetch(y0 + kTileH);  // the next tile's loads overlap this tile's sums
      const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
      if (x < im.W && y < im.H) {
        int32_t r[4] = {0, 0, 0, 0};
        const bool comp = computed_px(im, border, y, x);
        if (comp) taps25<kTileW>(tile[t & 1], threadIdx.y, threadIdx.x, r);
        store_px<FMT>(im, x, y, r, comp, thr);
      }
      if (more) put((t + 1) & 1);
      __syncthreads();
    }
  }
}

constexpr int kRgOut = 28;    // output columns per warp (32 lanes - 2r)
constexpr int kRgWarps = 4;   // warps per CTA

// LEVEL 0: RG, 1: RG-v1, 2: RG-v2.  Each warp walks `rows` output rows of a
// 28-column strip; the rings hold the horizontal results of input rows
// y-2 .. y+2 (index 0 = y-2) of the output row y being finished.
template <int LEVEL, int FMT>
__global__ void __launch_bounds__(32 * kRgWarps) rg_ladder_kernel(ImageDesc im, int border,
                                                                 int rows, int32_t thr) {
  constexpr int8_t K[4][5][5] = SOBEL4_EQ3_MASKS;
  const int lane = threadIdx.x & 31;
  const int wcol = (blockIdx.x * kRgWarps + (threadIdx.x >> 5)) * kRgOut;
  if (wcol >= im.W) return;  // whole warp
  const int xl = wcol - 2 + lane;  // column this lane loads
  const int x = wcol + lane;       // column this lane outputs (lanes 0..27)
  const bool out_lane = lane < kRgOut && x < im.W;
  bool zc;
  const int mx = map_index(xl, im.W, border, &zc);
  const int n_strips = (im.H + rows - 1) / rows;
  for (int si = blockIdx.y; si < n_strips; si += gridDim.y) {
    const int y0 = si * rows, y1 = min(y0 + rows, im.H);
    int32_t hd[5], hs[5], q0[5], q1[5], r0[5], r2[5], raw[5][5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      hd[i] = hs[i] = q0[i] = q1[i] = r0[i] = r2[i] = 0;
#pragma unroll
      for (int j = 0; j < 5; ++j) raw[i][j] = 0;
    }
    for (int yr = y0 - 2; yr < y1 + 2; ++yr) {
      bool zr;
      const int my = map_index(yr, im.H, border, &zr);
      const int32_t v =
          (zr || zc) ? 0 : (int32_t)__ldg(im.src + (uint64_t)(uint32_t)my * im.sp + mx);
      int32_t p[5];
      p[0] = v;
#pragma unroll
      for (int j = 1; j < 5; ++j) p[j] = __shfl_down_sync(0xffffffffu, v, j);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        hd[i] = hd[i + 1];
        hs[i] = hs[i + 1];
        q0[i] = q0[i + 1];
        q1[i] = q1[i + 1];
        r0[i] = r0[i + 1];
        r2[i] = r2[i + 1];
#pragma unroll
        for (int j = 0; j < 5; ++j) raw[i][j] = raw[i + 1][j];
      }
      // The 1x5 row passes: K_x's row [-1 -2 0 2 1] (Eq. 6) and K_y's [1 4 6 4 1].
      hd[4] = (p[4] - p[0]) + 2 * (p[3] - p[1]);
      hs[4] = (p[0] + p[4]) + 4 * (p[1] + p[3]) + 6 * p[2];
      if (LEVEL >= 1) {  // K_d+ rows (Eq. 12): [6 6 2 6 6] and [2 12 16 12 2]
        q0[4] = 6 * (p[0] + p[1] + p[3] + p[4]) + 2 * p[2];
        q1[4] = 2 * (p[0] + p[4]) + 12 * (p[1] + p[3]) + 16 * p[2];
      }
      if (LEVEL >= 2) {  // K_d- rows (Eq. 16-18): 6E + 2D and 2E + 16D
        const int32_t E = p[4] - p[0], D = p[3] - p[1];
        r0[4] = 6 * E + 2 * D;
        r2[4] = 2 * E + 16 * D;
      }
      if (LEVEL <= 1) {
#pragma unroll
        for (int j = 0; j < 5; ++j) raw[4][j] = p[j];
      }
      const int y = yr - 2;
      if (y < y0) continue;  // the window is still filling (uniform)
      int32_t r[4];
      r[0] = hd[0] + 4 * hd[1] + 6 * hd[2] + 4 * hd[3] + hd[4];  // Eq. 7
      r[1] = (hs[4] - hs[0]) + 2 * (hs[3] - hs[1]);
      if (LEVEL == 0) {
        r[2] = r[3] = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
          for (int j = 0; j < 5; ++j) {
            r[2] += (int32_t)K[2][i][j] * raw[i][j];
            r[3] += (int32_t)K[3][i][j] * raw[i][j];
          }
      } else {
        const int32_t P = (q0[4] - q0[0]) + (q1[3] - q1[1]);  // K_d+ (Eq. 15)
        int32_t M = 0;
        if (LEVEL == 1) {
#pragma unroll
          for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = 0; j < 5; ++j) M += (int32_t)(K[2][i][j] - K[3][i][j]) * raw[i][j];
        } else {
          M = (r0[0] + r0[4]) + 6 * (hd[1] + hd[3]) + r2[2];  // K_d- (Eq. 19)
        }
        r[2] = (P + M) >> 1;  // Eq. 11; P + M and P - M are even
        r[3] = (P - M) >> 1;
      }
      const bool comp = computed_px(im, border, y, x);
      if (!comp) r[0] = r[1] = r[2] = r[3] = 0;
      if (out_lane) store_px<FMT>(im, x, y, r, comp, thr);
    }
  }
}

template <int FMT>
void launch_fmt(const ImageDesc &im, int border, int kind, int rows, int32_t thr,
                cudaStream_t st) {
  if (kind == kLadderSM || kind == kLadderSMP) {
    const dim3 block(kTileW, kTileH);
    const int ny = kind == kLadderSM ? (im.H + kTileH - 1) / kTileH
                                     : (im.H + kTileH * kSmpTiles - 1) / (kTileH * kSmpTiles);
    const dim3 grid((im.W + kTileW - 1) / kTileW, (unsigned)std::min(ny, 65535));
    if (kind == kLadderSM) sm_kernel<FMT><<<grid, block, 0, st>>>(im, border, thr);
    else smp_kernel<FMT><<<grid, block, 0, st>>>(im, border, thr);
    return;
  }
  const int per_cta = kRgOut * kRgWarps;
  const int ny = (im.H + rows - 1) / rows;
  const dim3 grid((im.W + per_cta - 1) / per_cta, (unsigned)std::min(ny, 65535));
  if (kind == kLadderRG)
    rg_ladder_kernel<0, FMT><<<grid, 32 * kRgWarps, 0, st>>>(im, border, rows, thr);
  else if (kind == kLadderRGv1)
    rg_ladder_kernel<1, FMT><<<grid, 32 * kRgWarps, 0, st>>>(im, border, rows, thr);
  else
    rg_ladder_kernel<2, FMT><<<grid, 32 * kRgWarps, 0, st>>>(im, border, rows, thr);
}

}  // namespace

cudaError_t launch_ladder(const ImageDesc &im, int border, int fmt, int kind, int rows,
                          int32_t thr, cudaStream_t st) {
  if (kind < kLadderSM || kind > kLadderRGv2 || rows < 1) return cudaErrorInvalidValue;
  (void)cudaGetLastError();  // report this launch only, not an earlier failed call
  switch (fmt) {
    case kF32: launch_fmt<kF32>(im, border, kind, rows, thr, st); break;
    case kU8: launch_fmt<kU8>(im, border, kind, rows, thr, st); break;
    case kU16: launch_fmt<kU16>(im, border, kind, rows, thr, st); break;
    case kEdge8: launch_fmt<kEdge8>(im, border, kind, rows, thr, st); break;
    default: launch_fmt<kS16x4>(im, border, kind, rows, thr, st); break;
  }
  return cudaGetLastError();
}

}  // namespace sobel4
