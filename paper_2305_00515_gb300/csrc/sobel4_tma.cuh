// sobel4_tma.cuh — TMA-staged register-window kernel for single images whose
// rows start on 16-byte boundaries (sm_103a).
//
// The operator is that of sobel4_device.cuh (Section 3.1, Eq. 3 and Eq. 4);
// the schedule is the paper's register-window design (Section 4.3) rebuilt
// around the Blackwell memory path:
//
//  * Work item = one warp: a 128-column segment and a band of 2R rows, split
//    into two strips of R rows that travel together in the two 16-bit halves
//    of every register (v = lo + 65536 * hi, lo = strip a, hi = strip b).  The
//    host sizes R so that the items fill every resident warp about once, which
//    keeps the 4-row window fill of each strip (Section 4.3.2) near 3 % of
//    the rows.
//  * Staging: lane 0 of each warp issues 2-D tensor copies (cp.async.bulk.tensor,
//    TMA) of 8 rows x 160 bytes per strip into a 3-slot shared-memory ring,
//    completing on one mbarrier per slot; rows and columns outside the image
//    arrive as zeros from the copy engine, which is the CONSTANT0 rule and
//    harmless under VALID.  Under REPLICATE / REFLECT101 the lanes whose
//    columns cross the left or right edge read their bytes from the staged row
//    at the mapped columns, and rows outside the image are gathered from the
//    mapped rows in global memory.  This is the prefetch of Section 4.3.4, two
//    stages (16 rows) ahead.
//  * Per new row each column runs the packed passes of sobel4_arith.cuh
//    (Eq. 6-19), then the squares (Eq. 4) and the square root, and each lane
//    stores four results per strip row with one vector store.
//  * Border rules on the fast path: the copy engine's zero fill is the
//    CONSTANT0 rule; under VALID the lane that stored a frame element
//    overwrites it with 0 after the row loop.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sobel4_arith.cuh"
#include "sobel4_device.cuh"

namespace sobel4 {
namespace tma {

constexpr int kNC = 4;                        // columns per lane
constexpr int kCols = 32 * kNC;               // columns per warp segment
constexpr int kBoxW = 160;                    // staged bytes per row: columns x0-16 .. x0+143
constexpr int kStageRows = 8;                 // rows per stage and strip
constexpr int kSlots = 3;                     // ring slots per warp
constexpr int kStripBytes = kStageRows * kBoxW;     // 1280
constexpr int kSlotBytes = 2 * kStripBytes;         // 2560 (strip a, then strip b)
constexpr int kWarps = 4;                     // warps per CTA
#ifndef SOBEL4_TMA_UNROLL
#define SOBEL4_TMA_UNROLL 4
#endif
constexpr int kUnroll = SOBEL4_TMA_UNROLL;    // row steps per main-loop trip (2 or 4)
static_assert(kUnroll == 2 || kUnroll == 4, "the stage length must be a multiple of the unroll");

#ifndef SOBEL4_TMA_CLD
#define SOBEL4_TMA_CLD 1  // ring reads on the fast path: 1 = plain loads, 0 = volatile asm loads
#endif

#ifndef SOBEL4_TMA_MIN_CTAS
#define SOBEL4_TMA_MIN_CTAS 4
#endif
#ifndef SOBEL4_TMA_FAST_CTAS
#define SOBEL4_TMA_FAST_CTAS 4
#endif
// Kernel modes: every item, only fast-path items, only the other items.  A
// kernel without the general path needs fewer registers and no spills.
enum Mode : int { kAll = 0, kFastOnly = 1, kGeneralOnly = 2 };
template <int MODE>
constexpr int min_ctas() { return MODE == kFastOnly ? SOBEL4_TMA_FAST_CTAS : SOBEL4_TMA_MIN_CTAS; }

// Upper bound on one mbarrier wait (globaltimer nanoseconds) before the
// kernel gives up, records the failure and leaves.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

struct __align__(128) WarpRing {
  uint8_t slot[kSlots][kSlotBytes];
  uint64_t bar[kSlots];
};

// One image as the TMA kernel sees it (the source is staged through the
// tensor map; src/sp serve only the edge-rule gathers).
struct TmaImage {
  const uint8_t *src;  // read directly only for rows outside the image (edge rules)
  uint64_t sp;
  void *dst;
  uint64_t dp;
  int32_t H, W;
  int32_t n_seg, n_band;
  int32_t dst_align;  // largest power of two (<= 16) dividing dst and dp
  int32_t lose_stage; // failure injection (tests): stage of item 0 never copied; -1 = off
};

// One image of a TMA-staged batch: its tensor map (written by the host before
// the launch), its geometry and its first work item in the batch.
struct __align__(64) TmaBatchDesc {
  CUtensorMap map;
  TmaImage im;
  int64_t item0;
};

// ---------------------------------------------------------------------------
// PTX wrappers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Acquire a tensor map in global memory for the copy engine (tensor-map
// proxy) before its first use by this thread.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

// Orders this thread's earlier shared-memory accesses (generic proxy) before
// later copies into shared memory by the copy engine (async proxy).
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 2-D tile load: box at element coordinates (x, y) of `map` into shared
// memory at `dst`, completing `bar` with the box's byte count.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ uint32_t lds_u16(uint32_t a) {
  uint16_t v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t lds_u8(uint32_t a) {
  uint16_t v;
  asm volatile("ld.shared.u8 %0, [%1];" : "=h"(v) : "r"(a));
  return v;
}

// Packed columns c[0..7] (columns x-2 .. x+5 of both strips) from the staged
// rows: column x-2 of strip a at shared address `a`, of strip b at a + kStripBytes.
__device__ __forceinline__ void read_cols(uint32_t a, uint32_t c[8]) {
  const uint32_t b = a + kStripBytes;
  const uint32_t a0 = lds_u16(a), a1 = lds_u32(a + 2), a2 = lds_u16(a + 6);
  const uint32_t b0 = lds_u16(b), b1 = lds_u32(b + 2), b2 = lds_u16(b + 6);
  c[0] = __byte_perm(a0, b0, 0x6420);
  c[1] = __byte_perm(a0, b0, 0x7531);
  const uint32_t t1 = __byte_perm(a1, b1, 0x5140);
  const uint32_t t2 = __byte_perm(a1, b1, 0x7362);
  c[2] = __byte_perm(t1, 0u, 0x4140);
  c[3] = __byte_perm(t1, 0u, 0x4342);
  c[4] = __byte_perm(t2, 0u, 0x4140);
  c[5] = __byte_perm(t2, 0u, 0x4342);
  c[6] = __byte_perm(a2, b2, 0x6420);
  c[7] = __byte_perm(a2, b2, 0x7531);
}

// The same through a generic pointer into the ring (plain loads the compiler
// may schedule freely after the stage's barrier wait).
__device__ __forceinline__ void read_cols_p(const uint8_t *a, uint32_t c[8]) {
  const uint8_t *b = a + kStripBytes;
  const uint32_t a0 = *(const uint16_t *)a, a1 = *(const uint32_t *)(a + 2);
  const uint32_t a2 = *(const uint16_t *)(a + 6);
  const uint32_t b0 = *(const uint16_t *)b, b1 = *(const uint32_t *)(b + 2);
  const uint32_t b2 = *(const uint16_t *)(b + 6);
  c[0] = __byte_perm(a0, b0, 0x6420);
  c[1] = __byte_perm(a0, b0, 0x7531);
  const uint32_t t1 = __byte_perm(a1, b1, 0x5140);
  const uint32_t t2 = __byte_perm(a1, b1, 0x7362);
  c[2] = __byte_perm(t1, 0u, 0x4140);
  c[3] = __byte_perm(t1, 0u, 0x4342);
  c[4] = __byte_perm(t2, 0u, 0x4140);
  c[5] = __byte_perm(t2, 0u, 0x4342);
  c[6] = __byte_perm(a2, b2, 0x6420);
  c[7] = __byte_perm(a2, b2, 0x7531);
}

// Edge lanes under REPLICATE / REFLECT101: column j comes from staged byte
// offset off[j] of the row (the mapped column).
__device__ __forceinline__ void read_cols_mapped(uint32_t row_a, const uint32_t off[8],
                                                 uint32_t c[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j)
    c[j] = lds_u8(row_a + off[j]) | (lds_u8(row_a + kStripBytes + off[j]) << 16);
}

// Rows outside the image under REPLICATE / REFLECT101: the strip's bytes come
// from the mapped row (and mapped columns) in global memory; the other strip
// reads its staged row.
__device__ __forceinline__ void gather_cols(const TmaImage &im, uint32_t row_a,
                                            const uint32_t off[8], int x, int ra, int rb,
                                            bool out_a, bool out_b, int border, uint32_t c[8]) {
  bool z;
  const uint8_t *ga = im.src + (uint64_t)(uint32_t)map_index(ra, im.H, border, &z) * im.sp;
  const uint8_t *gb = im.src + (uint64_t)(uint32_t)map_index(rb, im.H, border, &z) * im.sp;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int col = map_index(x - 2 + j, im.W, border, &z);
    const uint32_t va = out_a ? (uint32_t)__ldg(ga + col) : lds_u8(row_a + off[j]);
    const uint32_t vb = out_b ? (uint32_t)__ldg(gb + col) : lds_u8(row_a + kStripBytes + off[j]);
    c[j] = va | (vb << 16);
  }
}

// ---------------------------------------------------------------------------
// Stores of one output row pair (strip a row, strip b row) for columns
// x..x+3.  GEN: per-column and per-row masks (edge items); otherwise four
// columns of both rows, vector stores.
// ---------------------------------------------------------------------------
template <int FMT, bool GEN>
__device__ __forceinline__ void store_rows(const TmaImage &im, uint8_t *row_a, uint8_t *row_b,
                                           int x, const uint32_t vx[4], const uint32_t vy[4],
                                           const uint32_t vd[4], const uint32_t vt[4],
                                           bool st_a, bool st_b, bool zero_a, bool zero_b,
                                           uint32_t colmask, uint32_t framemask, bool vec) {
  if constexpr (FMT == kS16x4) {
    const uint64_t plane = (uint64_t)(uint32_t)im.H * im.dp;
    const uint32_t *vals[4] = {vx, vy, vd, vt};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t *v = vals[q];
      int16_t *pa = (int16_t *)(row_a + q * plane) + x;
      int16_t *pb = (int16_t *)(row_b + q * plane) + x;
      if (!GEN) {
        const uint2 la = make_uint2(__byte_perm(v[0], v[1], 0x5410) ^ 0x80008000u,
                                    __byte_perm(v[2], v[3], 0x5410) ^ 0x80008000u);
        const uint2 lb = make_uint2(__byte_perm(v[0], v[1], 0x7632),
                                    __byte_perm(v[2], v[3], 0x7632));
        if (st_a) *(uint2 *)pa = la;
        if (st_b) *(uint2 *)pb = lb;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (!((colmask >> k) & 1u)) continue;
          const bool fk = (framemask >> k) & 1u;
          if (st_a) pa[k] = (int16_t)((zero_a || fk) ? 0 : lo_of(v[k]));
          if (st_b) pb[k] = (int16_t)((zero_b || fk) ? 0 : hi_of(v[k]));
        }
      }
    }
  } else {
  int32_t sa[4], sb[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) squares(vx[k], vy[k], vd[k], vt[k], sa[k], sb[k]);
  if constexpr (FMT == kF32) {
    float ga[4], gb[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) magnitude_f32x2(sa[k], sb[k], ga[k], gb[k]);
    float *pa = (float *)row_a + x, *pb = (float *)row_b + x;
    if (!GEN) {
      if (st_a) *(float4 *)pa = make_float4(ga[0], ga[1], ga[2], ga[3]);
      if (st_b) *(float4 *)pb = make_float4(gb[0], gb[1], gb[2], gb[3]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool fk = (framemask >> k) & 1u;
        if (zero_a || fk) ga[k] = 0.0f;
        if (zero_b || fk) gb[k] = 0.0f;
      }
      if (vec && colmask == 0xFu) {
        if (st_a) *(float4 *)pa = make_float4(ga[0], ga[1], ga[2], ga[3]);
        if (st_b) *(float4 *)pb = make_float4(gb[0], gb[1], gb[2], gb[3]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (!((colmask >> k) & 1u)) continue;
          if (st_a) pa[k] = ga[k];
          if (st_b) pb[k] = gb[k];
        }
      }
    }
  } else {
    uint32_t ua[4], ub[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) magnitude_u8x2(sa[k], sb[k], ua[k], ub[k]);
    uint8_t *pa = row_a + x, *pb = row_b + x;
    if (GEN) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool fk = (framemask >> k) & 1u;
        if (zero_a || fk) ua[k] = 0u;
        if (zero_b || fk) ub[k] = 0u;
      }
    }
    const uint32_t wa = ua[0] | (ua[1] << 8) | (ua[2] << 16) | (ua[3] << 24);
    const uint32_t wb = ub[0] | (ub[1] << 8) | (ub[2] << 16) | (ub[3] << 24);
    if (!GEN) {
      if (st_a) *(uint32_t *)pa = wa;
      if (st_b) *(uint32_t *)pb = wb;
    } else if (vec && colmask == 0xFu) {
      if (st_a) *(uint32_t *)pa = wa;
      if (st_b) *(uint32_t *)pb = wb;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!((colmask >> k) & 1u)) continue;
        if (st_a) pa[k] = (uint8_t)ua[k];
        if (st_b) pb[k] = (uint8_t)ub[k];
      }
    }
  }
  }
}

// Zero output element (y, x) in every plane of the format.
template <int FMT>
__device__ __forceinline__ void zero_px(const TmaImage &im, int y, int x) {
  uint8_t *row = (uint8_t *)im.dst + (uint64_t)(uint32_t)y * im.dp;
  if constexpr (FMT == kF32) {
    ((float *)row)[x] = 0.0f;
  } else if constexpr (FMT == kU8) {
    row[x] = 0;
  } else {
    const uint64_t plane = (uint64_t)(uint32_t)im.H * im.dp;
#pragma unroll
    for (int q = 0; q < 4; ++q) ((int16_t *)(row + q * plane))[x] = 0;
  }
}

// Zero output elements (y, x..x+3) with vector stores (the destination is
// vector-aligned on the fast path).
template <int FMT>
__device__ __forceinline__ void zero_row4(const TmaImage &im, int y, int x) {
  uint8_t *row = (uint8_t *)im.dst + (uint64_t)(uint32_t)y * im.dp;
  if constexpr (FMT == kF32) {
    *(float4 *)((float *)row + x) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  } else if constexpr (FMT == kU8) {
    *(uint32_t *)(row + x) = 0u;
  } else {
    const uint64_t plane = (uint64_t)(uint32_t)im.H * im.dp;
#pragma unroll
    for (int q = 0; q < 4; ++q) *(uint2 *)((int16_t *)(row + q * plane) + x) = make_uint2(0u, 0u);
  }
}

// ---------------------------------------------------------------------------
// One warp item.  Returns false when a stage wait ran out (recorded in *err).
// ---------------------------------------------------------------------------
struct ItemCtx {
  const CUtensorMap *map;   // source image, box 160 x 8
  const uint8_t *ringp;     // the same ring as a generic pointer
  int lose_stage;           // stage of this item whose copy is withheld (-1: none)
  uint32_t ring;            // shared address of this warp's ring
  uint32_t gstage;          // stages this warp has used so far (slot / parity counter)
};

// Waits until stage counter g has landed (all lanes agree on the outcome).
__device__ __forceinline__ bool wait_stage(const ItemCtx &cx, uint32_t g, unsigned int *err) {
  const uint32_t bar = cx.ring + (uint32_t)(kSlots * kSlotBytes + 8 * (g % kSlots));
  const uint32_t parity = (g / kSlots) & 1u;
  if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
    if (__any_sync(0xffffffffu, global_ns() - t0 > kWaitLimitNs)) {
      if ((threadIdx.x & 31) == 0) atomicOr(err, 1u);
      return false;
    }
  }
}

// After a failed wait: let the copies this warp still has in flight land
// (bounded), so that none writes into shared memory after the CTA is gone.
__device__ __forceinline__ void drain_stages(const ItemCtx &cx, uint32_t g_from, uint32_t g_to) {
  for (uint32_t g = g_from; g < g_to; ++g) {
    const uint32_t bar = cx.ring + (uint32_t)(kSlots * kSlotBytes + 8 * (g % kSlots));
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, (g / kSlots) & 1u) && global_ns() - t0 < kWaitLimitNs) {
    }
  }
}

// FULL: every output row of both strips lies inside the image (no row checks).
template <int FMT, bool GEN, bool FULL>
__device__ __forceinline__ bool tma_item(const TmaImage &im, int border, int seg, int band,
                                         int R, int lane, ItemCtx &cx, unsigned int *err) {
  const int H = im.H, W = im.W;
  const int x0 = seg * kCols;
  const int x = x0 + kNC * lane;
  const int ya = band * 2 * R;
  const int yb = ya + R;
  const int steps = R + 4;
  const int n_stages = (steps + kStageRows - 1) / kStageRows;
  const uint32_t g0 = cx.gstage;
  const bool map_rows = GEN && (border == kReplicate || border == kReflect101);

  // Producer: lane 0 copies stage j (rows 8j .. 8j+7 of both strips).
  auto issue = [&](int j) {
    if (j == cx.lose_stage) return;  // injected loss: this stage's wait must run out
    const uint32_t g = g0 + (uint32_t)j;
    const uint32_t slot = cx.ring + (uint32_t)(kSlotBytes * (g % kSlots));
    const uint32_t bar = cx.ring + (uint32_t)(kSlots * kSlotBytes + 8 * (g % kSlots));
    mbar_expect_tx(bar, (uint32_t)kSlotBytes);
#pragma unroll
    for (int s = 0; s < 2; ++s)
      tma_load_2d(slot + (uint32_t)(s * kStripBytes), cx.map, x0 - 16,
                  (s ? yb : ya) - 2 + kStageRows * j, bar);
  };

  __syncwarp();  // every lane is done with the ring slots about to be refilled
  if (lane == 0) {
    fence_proxy_async();
    for (int j = 0; j < kSlots && j < n_stages; ++j) issue(j);
  }

  // Edge-item bookkeeping.
  uint32_t colmask = 0xFu, framemask = 0u;
  bool mapped_lane = false;
  uint32_t off[8];
  const int na = min(R, H - ya);           // output rows of strip a inside the image
  const int nb = max(0, min(R, H - yb));   // ... of strip b
  bool vec = true;
  if (GEN) {
    colmask = 0u;
#pragma unroll
    for (int k = 0; k < kNC; ++k) {
      if (x + k < W) colmask |= 1u << k;
      if (border == kValid && (x + k < 2 || x + k > W - 3)) framemask |= 1u << k;
    }
    mapped_lane = (border == kReplicate || border == kReflect101) && (x - 2 < 0 || x + 5 >= W);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      bool z;
      const int m = map_index(x - 2 + j, W, border, &z);
      const int o = m - (x0 - 16);
      off[j] = (uint32_t)(o < 0 ? 0 : (o > kBoxW - 1 ? kBoxW - 1 : o));
    }
    const int vec_need = FMT == kF32 ? 16 : (FMT == kU8 ? 4 : 8);
    vec = im.dst_align >= vec_need;
  }

  Col st[kNC];
#pragma unroll
  for (int k = 0; k < kNC; ++k) st[k] = col_zero();
  uint8_t *row_a = (uint8_t *)im.dst + (uint64_t)(uint32_t)ya * im.dp;
  uint8_t *row_b = (uint8_t *)im.dst + (uint64_t)(uint32_t)min(yb, H - 1) * im.dp;
  const uint32_t lane_off = (uint32_t)(14 + kNC * lane);  // column x-2 in a staged row

  auto step = [&](uint32_t rd, int s, bool tail) {
    const int i = s - 4;  // output row of this step within each strip
    uint32_t c[8];
    if (GEN) {
      const int ra = ya - 2 + s, rb = yb - 2 + s;  // input rows of this step
      const bool out_a = map_rows && (ra < 0 || ra >= H);
      const bool out_b = map_rows && (rb < 0 || rb >= H);
      if (out_a || out_b) gather_cols(im, rd - lane_off, off, x, ra, rb, out_a, out_b, border, c);
      else if (mapped_lane) read_cols_mapped(rd - lane_off, off, c);
      else read_cols(rd, c);
    } else {
#if SOBEL4_TMA_CLD
      read_cols_p(cx.ringp + (rd - cx.ring), c);
#else
      read_cols(rd, c);
#endif
    }
    uint32_t vx[kNC], vy[kNC], vd[kNC], vt[kNC];
    if (tail) {
#pragma unroll
      for (int k = 0; k < kNC; ++k)
        column_step<true>(c[k], c[k + 1], c[k + 2], c[k + 3], c[k + 4], st[k], vx[k], vy[k],
                          vd[k], vt[k]);
      const bool st_a = FULL || i < na, st_b = FULL || i < nb;
      bool zero_a = false, zero_b = false;
      if (GEN) {
        if (border == kValid) {
          zero_a = ya + i < 2 || ya + i > H - 3;
          zero_b = yb + i < 2 || yb + i > H - 3;
        }
      }
      store_rows<FMT, GEN>(im, row_a, row_b, x, vx, vy, vd, vt, st_a, st_b, zero_a, zero_b,
                           colmask, framemask, vec);
      row_a += im.dp;
      row_b += im.dp;
    } else {
#pragma unroll
      for (int k = 0; k < kNC; ++k)
        column_step<false>(c[k], c[k + 1], c[k + 2], c[k + 3], c[k + 4], st[k], vx[k], vy[k],
                           vd[k], vt[k]);
    }
  };

  if (!wait_stage(cx, g0, err)) {
    drain_stages(cx, g0 + 1, g0 + (uint32_t)min(kSlots, n_stages));
    return false;
  }
  uint32_t rd = cx.ring + (uint32_t)(kSlotBytes * (g0 % kSlots)) + lane_off;
#pragma unroll
  for (int s = 0; s < 4; ++s)  // rows 0..3 only fill the window
    step(rd + (uint32_t)(s * kBoxW), s, false);
  rd += 4 * kBoxW;
  // Main loop: kUnroll row steps per trip (R is a multiple of kUnroll, so the
  // trips tile the steps and the stage boundaries fall on trip boundaries).
#pragma unroll 1
  for (int s = 4; s < steps; s += kUnroll) {
    if ((s & (kStageRows - 1)) == 0) {
      const int j = s / kStageRows;
      __syncwarp();  // stage j-1 has been read by every lane
      if (lane == 0 && j - 1 + kSlots < n_stages) {
        fence_proxy_async();
        issue(j - 1 + kSlots);
      }
      if (!wait_stage(cx, g0 + (uint32_t)j, err)) {
        drain_stages(cx, g0 + (uint32_t)j + 1, g0 + (uint32_t)min(j - 1 + kSlots + 1, n_stages));
        return false;
      }
      rd = cx.ring + (uint32_t)(kSlotBytes * ((g0 + (uint32_t)j) % kSlots)) + lane_off;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) step(rd + (uint32_t)(u * kBoxW), s + u, true);
    rd += kUnroll * kBoxW;
  }
  cx.gstage = g0 + (uint32_t)n_stages;
  if (!GEN && border == kValid) {
    // The paper's rule leaves the 2-pixel frame at 0.  The fast path computed
    // it from zero-filled halos; the lane that stored each frame element now
    // overwrites it (same thread, later store).
    const int yr[2] = {ya, yb}, nr[2] = {na, nb};
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int f[4] = {0, 1, H - 2, H - 1};
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (f[q] >= yr[t] && f[q] < yr[t] + nr[t] && (q < 2 || f[q] > 1)) zero_row4<FMT>(im, f[q], x);
    }
    // Frame columns {0, 1, W-2, W-1} inside the segment: all lanes share the
    // rows; the barrier orders the stores of the lanes that computed them.
    if (x0 < 2 || x0 + kCols > W - 2) {
      __syncwarp();
      const int fc[4] = {0, 1, W - 2, W - 1};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = fc[q];
        if (c < x0 || c >= x0 + kCols || (q >= 2 && c < 2)) continue;
        for (int r = lane; r < na + nb; r += 32) zero_px<FMT>(im, r < na ? ya + r : yb + r - na, c);
      }
    }
  }
  return true;
}

// An item for the fast path: every lane's four columns inside the image, a
// destination that takes one vector store per lane and row, and either a
// border rule the copy engine's zero fill serves (CONSTANT0; VALID with the
// frame zeroed afterwards) or every input row and column inside the image.
__device__ __forceinline__ bool fast_item(const TmaImage &im, int border, int seg, int band,
                                          int R, int fmt) {
  const int x0 = seg * kCols;
  const int ya = band * 2 * R;
  const int vec_need = fmt == kF32 ? 16 : (fmt == kU8 ? 4 : 8);
  if (im.dst_align < vec_need || x0 + kCols > im.W) return false;
  if (border == kValid || border == kConstant0) return true;
  return x0 >= 2 && x0 + kCols + 2 <= im.W && ya >= 2 && ya + 2 * R + 2 <= im.H;
}

// Runs one item through the variant its geometry needs; a kernel that runs
// only fast items (or only the others) carries only that code.
template <int FMT, int MODE>
__device__ __forceinline__ bool run_item(const TmaImage &im, int border, int seg, int band, int R,
                                         int lane, ItemCtx &cx, unsigned int *err, bool fast) {
  if (MODE != kFastOnly && !fast)
    return tma_item<FMT, true, false>(im, border, seg, band, R, lane, cx, err);
  if constexpr (MODE != kGeneralOnly) {
    if (band * 2 * R + 2 * R <= im.H)
      return tma_item<FMT, false, true>(im, border, seg, band, R, lane, cx, err);
    return tma_item<FMT, false, false>(im, border, seg, band, R, lane, cx, err);
  }
  return false;
}

// The single-image kernel: persistent CTAs of 4 warps; each warp pulls items
// (band-major) from the counter pair[0]; the last warp out resets the pair.
template <int FMT, int MODE>
__global__ void __launch_bounds__(kWarps * 32, min_ctas<MODE>())
    tma_single_kernel(const __grid_constant__ CUtensorMap map, TmaImage im, int border, int R,
                      int n_items, unsigned int *pair, unsigned int *err) {
  __shared__ WarpRing rings[kWarps];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  ItemCtx cx;
  cx.map = &map;
  cx.ring = smem_addr(&rings[warp]);
  cx.ringp = &rings[warp].slot[0][0];
  cx.gstage = 0;
  if (lane == 0) {
    for (int i = 0; i < kSlots; ++i)
      mbar_init(cx.ring + (uint32_t)(kSlots * kSlotBytes + 8 * i), 1u);
    mbar_init_fence();
  }
  __syncwarp();
  for (;;) {
    unsigned int got = 0;
    if (lane == 0) got = atomicAdd(&pair[0], 1u);
    got = __shfl_sync(0xffffffffu, got, 0);
    if (got >= (unsigned int)n_items) break;
    const int item = (int)got;
    const int band = item / im.n_seg;
    const int seg = item - band * im.n_seg;
    cx.lose_stage = item == 0 ? im.lose_stage : -1;
    const bool fast = fast_item(im, border, seg, band, R, FMT);
    if ((MODE == kFastOnly && !fast) || (MODE == kGeneralOnly && fast)) continue;
    if (!run_item<FMT, MODE>(im, border, seg, band, R, lane, cx, err, fast)) break;
  }
  if (lane == 0) {
    __threadfence();  // this warp's last fetch is performed before it counts out
    const unsigned int warps = gridDim.x * kWarps;
    if (atomicAdd(&pair[1], 1u) == warps - 1u) {
      atomicExch(&pair[0], 0u);
      atomicExch(&pair[1], 0u);
    }
  }
}


// The batched kernel: persistent CTAs of 4 warps pull items (image by image,
// band-major) from *queue (zeroed by the host before the launch); a warp
// finds an item's image by binary search over the descriptors' first items.
template <int FMT, int MODE>
__global__ void __launch_bounds__(kWarps * 32, min_ctas<MODE>())
    tma_batched_kernel(const TmaBatchDesc *__restrict__ descs, int n_img, int total,
                       unsigned int *queue, int border, int R, unsigned int *err) {
  __shared__ WarpRing rings[kWarps];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  ItemCtx cx;
  cx.ring = smem_addr(&rings[warp]);
  cx.ringp = &rings[warp].slot[0][0];
  cx.gstage = 0;
  if (lane == 0) {
    for (int i = 0; i < kSlots; ++i)
      mbar_init(cx.ring + (uint32_t)(kSlots * kSlotBytes + 8 * i), 1u);
    mbar_init_fence();
  }
  __syncwarp();
  int cur = -1;
  for (;;) {
    unsigned int got = 0;
    if (lane == 0) got = atomicAdd(queue, 1u);
    got = __shfl_sync(0xffffffffu, got, 0);
    if (got >= (unsigned int)total) break;
    const int64_t item = (int64_t)got;
    int lo = 0, hi = n_img - 1;  // largest image whose first item is <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(&descs[mid].item0) <= item) lo = mid;
      else hi = mid - 1;
    }
    const TmaBatchDesc *d = descs + lo;
    const TmaImage im = d->im;
    const int local = (int)(item - d->item0);
    const int band = local / im.n_seg;
    const int seg = local - band * im.n_seg;
    const bool fast = fast_item(im, border, seg, band, R, FMT);
    if ((MODE == kFastOnly && !fast) || (MODE == kGeneralOnly && fast)) continue;
    if (lo != cur) {
      if (lane == 0) tensormap_acquire(&d->map);
      cur = lo;
    }
    cx.map = &d->map;
    cx.lose_stage = -1;
    if (!run_item<FMT, MODE>(im, border, seg, band, R, lane, cx, err, fast)) break;
  }
}

}  // namespace tma
}  // namespace sobel4
