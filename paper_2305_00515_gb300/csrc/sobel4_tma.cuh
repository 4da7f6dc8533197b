// sobel4_tma.cuh — TMA-family register-window kernels (sm_103a): single
// images and batches, any row alignment.
//
// The operator is that of sobel4_device.cuh (Section 3.1, Eq. 3 and Eq. 4);
// the schedule is the paper's register-window design (Section 4.3) rebuilt
// around the Blackwell memory path:
//
//  * Work item = one warp: a 128-column segment and a band of 2R rows, split
//    into two strips of R rows that travel together in the two 16-bit halves
//    of every register (v = lo + 65536 * hi, lo = strip a, hi = strip b).  The
//    host sizes R (about two items per resident warp for images whose items
//    all take the fast path, more otherwise; or the tuned value); a last band
//    with fewer than 2R rows is split evenly between its strips.  Items are
//    handed out edge items first (item_coords).
//  * Staging into a 3-slot per-warp shared-memory ring completed by one
//    mbarrier per slot, two stages (16 rows) ahead: the prefetch of Section
//    4.3.4.  Tensor staging (rows on 16-byte boundaries): lane 0 issues 2-D
//    tensor copies (cp.async.bulk.tensor, TMA) of 8 rows x 160 bytes per
//    strip; rows and columns outside the image arrive as zeros.  Bulk staging
//    (any other source): 16 lanes each copy the 16-byte granules of one row
//    (cp.async.bulk) and record that row's byte offset.
//  * Per new row each column runs the packed passes of sobel4_arith.cuh
//    (Eq. 6-19), then the squares (Eq. 4) and the magnitude, and each lane
//    stores four results per strip row with one vector store (lane-shifted
//    aligned stores when the destination rows are not vector-aligned).
//  * Border rules: on the fast path the zero fill is the CONSTANT0 rule and,
//    under VALID, the lane that stored a frame element overwrites it with 0
//    after the row loop; edge items of REPLICATE / REFLECT101 (and of bulk
//    staging) read the mapped columns from the staged row and gather rows
//    outside the image from their mapped rows.
//  * Kernel modes: fast items only (the lean kernel, widths that are a
//    multiple of the segment), fast items of a ragged width (one body whose
//    stores stop at column W), general items only, or both in one kernel.
//    A batched launch sends all its fast items through one body (see
//    run_item: several live bodies thrash the instruction cache).
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
constexpr int kBoxW = 160;                    // tensor box width: columns x0-16 .. x0+143
constexpr int kStageRows = 8;                 // rows per stage and strip
constexpr int kSlots = 3;                     // ring slots per warp
constexpr int kWarps = 4;                     // warps per CTA

// Three stagings share the kernel.  kTensor: 2-D tensor copies (TMA) of a box
// of 160 x 8 bytes per strip; needs 16-byte aligned rows.  kBulk: 1-D bulk
// copies (cp.async.bulk), one per row, of the 16-byte granules that hold the
// row's bytes for columns x0-2 .. x0+129 (at most 176 bytes), for rows of any
// alignment; each row slot keeps a 16-byte pad in front of the data and the
// slot keeps, per row, the byte offset of column x0-2 from the copied data.
// kRgbBulk: an interleaved RGB source (3 bytes per pixel, any alignment),
// staged like kBulk -- one 1-D bulk copy per row of the 16-byte granules that
// hold the bytes of columns x0-2 .. x0+129 (at most 432 bytes) behind a
// 32-byte pad -- in stages of 4 rows; the ring reads turn each pixel into gray
// (rgb_cols below).
enum Staging : int { kTensor = 0, kBulk = 1, kRgbBulk = 2 };
template <int ST>
struct Geo {
  static constexpr bool kRows = ST != kTensor;  // per-row copies with per-row offsets
  static constexpr int kBpp = ST == kRgbBulk ? 3 : 1;           // source bytes per pixel
  static constexpr int kStageRows = ST == kRgbBulk ? 4 : 8;     // rows per stage and strip
  static constexpr int kSlots = 3;                              // ring slots per warp
  static constexpr int kRowPitch =                              // bytes per staged row
      ST == kBulk ? 192 : (ST == kRgbBulk ? 480 : kBoxW);
  static constexpr int kRowData = ST == kBulk ? 16 : (ST == kRgbBulk ? 32 : 0);
  static constexpr int kStrip = kStageRows * kRowPitch;
  static constexpr int kHdr = 2 * kStrip;                      // per-row offsets
  static constexpr int kSlot = 2 * kStrip + (kRows ? 64 : 0);
};
constexpr int kStripBytes = Geo<kTensor>::kStrip;    // 1280
constexpr int kSlotBytes = Geo<kTensor>::kSlot;      // 2560 (strip a, then strip b)
#ifndef SOBEL4_TMA_UNROLL
#define SOBEL4_TMA_UNROLL 4
#endif
constexpr int kUnroll = SOBEL4_TMA_UNROLL;    // row steps per main-loop trip (2 or 4)
static_assert(kUnroll == 2 || kUnroll == 4, "the stage length must be a multiple of the unroll");

#ifndef SOBEL4_RA_SPLIT
#define SOBEL4_RA_SPLIT 1  // unaligned destination rows: 1 = each lane's own elements in
                           // at most three aligned stores, 0 = lane-shifted vector stores
#endif

#ifndef SOBEL4_TMA_CLD
#define SOBEL4_TMA_CLD 1  // ring reads on the fast path: 1 = plain loads, 0 = volatile asm loads
#endif

#ifndef SOBEL4_PDL
#define SOBEL4_PDL 1  // 1: launched as programmatic dependents (prologue overlaps the previous grid)
#endif

#ifndef SOBEL4_TMA_MIN_CTAS
#define SOBEL4_TMA_MIN_CTAS 4
#endif
#ifndef SOBEL4_TMA_FAST_CTAS
#define SOBEL4_TMA_FAST_CTAS 4
#endif
// Kernel modes: every item, only fast-path items, only the other items, and
// (single images) only fast-path items of a width that is not a multiple of
// the segment, and only fast-path items with destination rows that are not
// vector-aligned.  A kernel without the general path needs fewer registers
// and no spills.
enum Mode : int { kAll = 0, kFastOnly = 1, kGeneralOnly = 2, kFastPart = 3, kFastRA = 4 };
template <int MODE>
__host__ __device__ constexpr bool fast_mode() {
  return MODE == kFastOnly || MODE == kFastPart || MODE == kFastRA;
}
template <int MODE>
constexpr int min_ctas() { return fast_mode<MODE>() ? SOBEL4_TMA_FAST_CTAS : SOBEL4_TMA_MIN_CTAS; }

// Upper bound on one mbarrier wait (globaltimer nanoseconds) before the
// kernel gives up, records the failure and leaves.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

template <int ST>
struct __align__(128) WarpRing {
  uint8_t slot[Geo<ST>::kSlots][Geo<ST>::kSlot];
  uint64_t bar[Geo<ST>::kSlots];
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
  int32_t thr;        // EDGE8: an output pixel is 255 where S >= thr, else 0
};

// One image of a TMA-staged batch: its tensor map (written by the host before
// the launch), its geometry and its first work item in the batch.
struct __align__(64) TmaBatchDesc {
  CUtensorMap map;
  TmaImage im;
  int64_t item0;
};

// One image of a bulk-staged batch: no tensor map.
struct __align__(16) TmaBulkDesc {
  TmaImage im;
  int64_t item0;
};

template <int ST>
struct BatchDescOf {
  using type = TmaBatchDesc;
};
template <>
struct BatchDescOf<kBulk> {
  using type = TmaBulkDesc;
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

// Programmatic dependent launch: the grid may start while the previous grid
// on the stream is finishing; it waits here for that grid's completion and
// memory before its first global access, and lets the next grid start its
// own prologue on SMs this grid has left.
__device__ __forceinline__ void grid_dependency_wait() {
#if SOBEL4_PDL
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
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

// 1-D bulk copy of `bytes` (a multiple of 16) from 16-byte aligned global
// `src` into 16-byte aligned shared `dst`, completing `bar`.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ int32_t lds_s32(uint32_t a) {
  int32_t v;
  asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
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
template <int STRIP = kStripBytes>
__device__ __forceinline__ void read_cols(uint32_t a, uint32_t c[8]) {
  const uint32_t b = a + STRIP;
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
  const uint8_t *b = a + kStripBytes;  // tensor staging
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

// Packed columns from rows staged at any byte offset (bulk staging): column
// x-2 of strip a at shared address `a`, of strip b at `b`; the 8 bytes of each
// are funnel-shifted out of three aligned words (the shift is the same for
// every lane of a row).
__device__ __forceinline__ void read_cols_any(uint32_t a, uint32_t b, uint32_t c[8]) {
  const uint32_t qa = a & ~3u, qb = b & ~3u;
  const uint32_t sa = (a & 3u) * 8u, sb = (b & 3u) * 8u;
  const uint32_t a0 = lds_u32(qa), a1 = lds_u32(qa + 4), a2 = lds_u32(qa + 8);
  const uint32_t b0 = lds_u32(qb), b1 = lds_u32(qb + 4), b2 = lds_u32(qb + 8);
  const uint32_t la0 = __funnelshift_r(a0, a1, sa), la1 = __funnelshift_r(a1, a2, sa);
  const uint32_t lb0 = __funnelshift_r(b0, b1, sb), lb1 = __funnelshift_r(b1, b2, sb);
  const uint32_t t0 = __byte_perm(la0, lb0, 0x5140), t1 = __byte_perm(la0, lb0, 0x7362);
  const uint32_t t2 = __byte_perm(la1, lb1, 0x5140), t3 = __byte_perm(la1, lb1, 0x7362);
  c[0] = __byte_perm(t0, 0u, 0x4140);
  c[1] = __byte_perm(t0, 0u, 0x4342);
  c[2] = __byte_perm(t1, 0u, 0x4140);
  c[3] = __byte_perm(t1, 0u, 0x4342);
  c[4] = __byte_perm(t2, 0u, 0x4140);
  c[5] = __byte_perm(t2, 0u, 0x4342);
  c[6] = __byte_perm(t3, 0u, 0x4140);
  c[7] = __byte_perm(t3, 0u, 0x4342);
}

// Gray of interleaved RGB pixels (the host preparation of Section 4.3; the
// rule read for it): Y = (77 R + 150 G + 29 B + 128) >> 8, as 4-way byte dot
// products whose weight bytes sit where the pixel's bytes sit in a word.  The
// result is Y * 256 + (fraction), below 2^16, so Y is its byte 1.
__device__ __forceinline__ uint32_t dp4(uint32_t w, uint32_t k, uint32_t c) {
  return __dp4a(w, k, c);
}
constexpr uint32_t kRgbW0 = 0x001D964Du;  // R, G, B weights at bytes 0, 1, 2

// Packed gray columns c[0..7] (columns x-2 .. x+5 of both strips) from RGB
// rows at any byte offset: pixel x-2 of strip a at shared address `a`, of
// strip b at `b`.  The 24 bytes of each strip are funnel-shifted out of seven
// aligned words (the shift is the same for every lane of a row) into six
// words in which pixel j starts at byte 3j, then each pixel is one dot product
// (within a word) or two (across two words).
__device__ __forceinline__ void rgb_words(uint32_t a, uint32_t n[6]) {
  const uint32_t q = a & ~3u, sh = (a & 3u) * 8u;
  uint32_t w[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) w[i] = lds_u32(q + 4 * i);
#pragma unroll
  for (int i = 0; i < 6; ++i) n[i] = __funnelshift_r(w[i], w[i + 1], sh);
}
__device__ __forceinline__ void rgb_gray6(const uint32_t n[6], uint32_t y[8]) {
  y[0] = dp4(n[0], kRgbW0, 128u);                                   // bytes 0-2
  y[1] = dp4(n[1], 0x00001D96u, dp4(n[0], 0x4D000000u, 128u));      // bytes 3 | 4-5
  y[2] = dp4(n[2], 0x0000001Du, dp4(n[1], 0x964D0000u, 128u));      // bytes 6-7 | 8
  y[3] = dp4(n[2], kRgbW0 << 8, 128u);                              // bytes 9-11
  y[4] = dp4(n[3], kRgbW0, 128u);                                   // bytes 12-14
  y[5] = dp4(n[4], 0x00001D96u, dp4(n[3], 0x4D000000u, 128u));      // bytes 15 | 16-17
  y[6] = dp4(n[5], 0x0000001Du, dp4(n[4], 0x964D0000u, 128u));      // bytes 18-19 | 20
  y[7] = dp4(n[5], kRgbW0 << 8, 128u);                              // bytes 21-23
}
__device__ __forceinline__ void read_cols_rgb(uint32_t a, uint32_t b, uint32_t c[8]) {
  uint32_t na[6], nb[6], ya[8], yb[8];
  rgb_words(a, na);
  rgb_words(b, nb);
  rgb_gray6(na, ya);
  rgb_gray6(nb, yb);
#pragma unroll
  for (int j = 0; j < 8; ++j) c[j] = __byte_perm(ya[j], yb[j], 0x6521);  // (Y_a, Y_b)
}

// The gray of one RGB pixel from three bytes (edge items).
__device__ __forceinline__ uint32_t rgb_gray1(uint32_t r, uint32_t g, uint32_t b) {
  return (77u * r + 150u * g + 29u * b + 128u) >> 8;
}

// Edge lanes under REPLICATE / REFLECT101: column j comes from staged byte
// offset off[j] (relative to column x0-2) of each strip's row.
__device__ __forceinline__ void read_cols_mapped(uint32_t base_a, uint32_t base_b,
                                                 const int32_t off[8], uint32_t c[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j)
    c[j] = lds_u8(base_a + off[j]) | (lds_u8(base_b + off[j]) << 16);
}

// Edge items of the general path: each strip's byte for column x-2+j is the
// staged byte at the mapped column (off[j], relative to column x0-2) when the
// strip's row is inside the image, else the mapped row's byte in global
// memory (REPLICATE / REFLECT101) or 0 (CONSTANT0, VALID); zmask marks
// columns outside the image that read 0 (CONSTANT0).
// BPP = 3: RGB pixels, turned into gray.
template <int BPP = 1>
__device__ __forceinline__ void gather_cols(const TmaImage &im, uint32_t base_a, uint32_t base_b,
                                            const int32_t off[8], uint32_t zmask, int x, int ra,
                                            int rb, bool out_a, bool out_b, int border,
                                            uint32_t c[8]) {
  bool z;
  const bool mapped = border == kReplicate || border == kReflect101;
  const uint8_t *ga = im.src + (uint64_t)(uint32_t)map_index(ra, im.H, border, &z) * im.sp;
  const uint8_t *gb = im.src + (uint64_t)(uint32_t)map_index(rb, im.H, border, &z) * im.sp;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int col = map_index(x - 2 + j, im.W, border, &z);
    uint32_t va, vb;
    if constexpr (BPP == 3) {
      const uint8_t *pa = ga + 3 * col, *pb = gb + 3 * col;
      const uint32_t sa = base_a + 3 * off[j], sb = base_b + 3 * off[j];
      va = out_a ? (mapped ? rgb_gray1(__ldg(pa), __ldg(pa + 1), __ldg(pa + 2)) : 0u)
                 : rgb_gray1(lds_u8(sa), lds_u8(sa + 1), lds_u8(sa + 2));
      vb = out_b ? (mapped ? rgb_gray1(__ldg(pb), __ldg(pb + 1), __ldg(pb + 2)) : 0u)
                 : rgb_gray1(lds_u8(sb), lds_u8(sb + 1), lds_u8(sb + 2));
    } else {
      va = out_a ? (mapped ? (uint32_t)__ldg(ga + col) : 0u) : lds_u8(base_a + off[j]);
      vb = out_b ? (mapped ? (uint32_t)__ldg(gb + col) : 0u) : lds_u8(base_b + off[j]);
    }
    if ((zmask >> j) & 1u) va = vb = 0u;
    c[j] = va | (vb << 16);
  }
}

// ---------------------------------------------------------------------------
// Stores of one output row pair (strip a row, strip b row) for columns
// x..x+3.  GEN: per-column and per-row masks (edge items); otherwise four
// columns of both rows, vector stores.
// ---------------------------------------------------------------------------
// Stores of one row's four elements per lane into a destination row that is
// not vector-aligned.  Every lane's run starts at the same offset m from an
// aligned chunk (runs are one chunk wide), so the warp shifts its elements up
// by one lane: lanes 1..31 each write one whole aligned chunk made of the
// previous lane's last m elements and their own first 4-m; lane 0 writes the
// head of the first chunk and lane 31 the tail of the last element by element,
// so that no store touches another segment's columns.  Every lane calls these
// (they shuffle); `on` and m are warp-uniform, and an aligned row (m = 0)
// takes plain vector stores without shuffling.
//
// PART: the segment runs past the image's last column; `wl` = W - x is the
// number of this lane's four columns inside the image (may be <= 0 or > 4),
// and no element at column >= W is written: a chunk that crosses column W is
// written element by element up to it.
// ---------------------------------------------------------------------------
// SOBEL4_RA_SPLIT: the misalignment m of a row is the same for every lane, and
// each lane stores its own four elements in at most three naturally aligned
// pieces (m = 0: one 16-byte store; m = 2: two 8-byte stores; m odd: 4, 8 and
// 4 bytes), so no lane touches another lane's elements and no shuffles are
// needed.  U8 and 16-bit formats split the same way at their scale.
template <bool PART>
__device__ __forceinline__ void st4_f32_split(float *p, const float v[4], bool on, int wl) {
  if (!on) return;
  if (PART && wl < 4) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < wl) p[k] = v[k];
    return;
  }
  const uint32_t m = ((uint32_t)(uintptr_t)p >> 2) & 3u;
  if (m == 0) {
    *(float4 *)p = make_float4(v[0], v[1], v[2], v[3]);
  } else if (m == 2) {
    *(float2 *)p = make_float2(v[0], v[1]);
    *(float2 *)(p + 2) = make_float2(v[2], v[3]);
  } else {
    p[0] = v[0];
    *(float2 *)(p + 1) = make_float2(v[1], v[2]);
    p[3] = v[3];
  }
}

template <bool PART>
__device__ __forceinline__ void st4_u8_split(uint8_t *p, uint32_t w, bool on, int wl) {
  if (!on) return;
  if (PART && wl < 4) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < wl) p[k] = (uint8_t)(w >> (8 * k));
    return;
  }
  const uint32_t m = (uint32_t)(uintptr_t)p & 3u;
  if (m == 0) {
    *(uint32_t *)p = w;
  } else if (m == 2) {
    *(uint16_t *)p = (uint16_t)w;
    *(uint16_t *)(p + 2) = (uint16_t)(w >> 16);
  } else {
    p[0] = (uint8_t)w;
    *(uint16_t *)(p + 1) = (uint16_t)(w >> 8);
    p[3] = (uint8_t)(w >> 24);
  }
}

// w0 holds elements 0, 1 and w1 elements 2, 3 (little-endian 16-bit pairs).
template <bool PART>
__device__ __forceinline__ void st4_s16_split(int16_t *p, uint32_t w0, uint32_t w1, bool on,
                                              int wl) {
  if (!on) return;
  if (PART && wl < 4) {
    const uint64_t cur = ((uint64_t)w1 << 32) | w0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < wl) p[k] = (int16_t)(cur >> (16 * k));
    return;
  }
  const uint32_t m = ((uint32_t)(uintptr_t)p >> 1) & 3u;
  if (m == 0) {
    *(uint2 *)p = make_uint2(w0, w1);
  } else if (m == 2) {
    *(uint32_t *)p = w0;
    *(uint32_t *)(p + 2) = w1;
  } else {
    p[0] = (int16_t)w0;
    *(uint32_t *)(p + 1) = __funnelshift_r(w0, w1, 16);
    p[3] = (int16_t)(w1 >> 16);
  }
}

template <bool PART>
__device__ __forceinline__ void st4_f32_realigned(float *p, const float v[4], bool on, int wl) {
#if SOBEL4_RA_SPLIT
  st4_f32_split<PART>(p, v, on, wl);
  return;
#endif
  const int lane = threadIdx.x & 31;
  const uint32_t m = ((uint32_t)(uintptr_t)p >> 2) & 3u;  // elements past the chunk start
  if (m == 0) {  // an aligned row (m is the same for every lane): plain stores
    if (!on) return;
    if (!PART || wl >= 4) {
      *(float4 *)p = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < wl) p[k] = v[k];
    }
    return;
  }
  const float p1 = __shfl_up_sync(0xffffffffu, v[1], 1);
  const float p2 = __shfl_up_sync(0xffffffffu, v[2], 1);
  const float p3 = __shfl_up_sync(0xffffffffu, v[3], 1);
  if (!on) return;
  const float o[4] = {m == 1 ? p3 : (m == 2 ? p2 : p1), m == 1 ? v[0] : (m == 2 ? p3 : p2),
                      m == 1 ? v[1] : (m == 2 ? v[0] : p3), m == 1 ? v[2] : (m == 2 ? v[1] : v[0])};
  if (lane > 0) {
    if (!PART || wl + (int)m >= 4) {
      *(float4 *)(p - m) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j < wl + (int)m) (p - m)[j] = o[j];
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < 4 - (int)m && (!PART || k < wl)) p[k] = v[k];
  }
  if (lane == 31) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k >= 4 - (int)m && (!PART || k < wl)) p[k] = v[k];
  }
}

template <bool PART>
__device__ __forceinline__ void st4_u8_realigned(uint8_t *p, uint32_t w, bool on, int wl) {
#if SOBEL4_RA_SPLIT
  st4_u8_split<PART>(p, w, on, wl);
  return;
#endif
  const int lane = threadIdx.x & 31;
  const uint32_t m = (uint32_t)(uintptr_t)p & 3u;
  if (m == 0) {  // an aligned row: plain stores
    if (!on) return;
    if (!PART || wl >= 4) {
      *(uint32_t *)p = w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < wl) p[k] = (uint8_t)(w >> (8 * k));
    }
    return;
  }
  const uint32_t prev = __shfl_up_sync(0xffffffffu, w, 1);
  if (!on) return;
  if (lane > 0) {
    const uint32_t o = __funnelshift_l(prev, w, 8u * m);
    if (!PART || wl + (int)m >= 4) {
      *(uint32_t *)(p - m) = o;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j < wl + (int)m) (p - m)[j] = (uint8_t)(o >> (8 * j));
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < 4 - (int)m && (!PART || k < wl)) p[k] = (uint8_t)(w >> (8 * k));
  }
  if (lane == 31) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k >= 4 - (int)m && (!PART || k < wl)) p[k] = (uint8_t)(w >> (8 * k));
  }
}

// w0 holds elements 0, 1 and w1 elements 2, 3 (little-endian int16 pairs).
template <bool PART>
__device__ __forceinline__ void st4_s16_realigned(int16_t *p, uint32_t w0, uint32_t w1, bool on,
                                                  int wl) {
#if SOBEL4_RA_SPLIT
  st4_s16_split<PART>(p, w0, w1, on, wl);
  return;
#endif
  const int lane = threadIdx.x & 31;
  const uint32_t m = ((uint32_t)(uintptr_t)p >> 1) & 3u;
  const uint64_t cur = ((uint64_t)w1 << 32) | w0;
  if (m == 0) {  // an aligned row: plain stores
    if (!on) return;
    if (!PART || wl >= 4) {
      *(uint2 *)p = make_uint2(w0, w1);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < wl) p[k] = (int16_t)(cur >> (16 * k));
    }
    return;
  }
  const uint32_t q0 = __shfl_up_sync(0xffffffffu, w0, 1);
  const uint32_t q1 = __shfl_up_sync(0xffffffffu, w1, 1);
  if (!on) return;
  const uint64_t prev = ((uint64_t)q1 << 32) | q0;
  const uint64_t out = (cur << (16u * m)) | (prev >> (64u - 16u * m));
  if (lane > 0) {
    if (!PART || wl + (int)m >= 4) {
      *(uint2 *)(p - m) = make_uint2((uint32_t)out, (uint32_t)(out >> 32));
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j < wl + (int)m) (p - m)[j] = (int16_t)(out >> (16 * j));
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < 4 - (int)m && (!PART || k < wl)) p[k] = (int16_t)(cur >> (16 * k));
  }
  if (lane == 31) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k >= 4 - (int)m && (!PART || k < wl)) p[k] = (int16_t)(cur >> (16 * k));
  }
}

// ---------------------------------------------------------------------------
// RA (fast path only): the destination rows are not vector-aligned; the
// realigned stores above take the place of the vector stores.  PART (fast
// path only): only the wl = W - x first of the lane's columns are stored.
// CW: the responses are R_x, R_y, P, M of the runtime-weight passes
// (column_step_w), whose S is squares_w's; never with S16X4.
template <int FMT, bool GEN, bool RA, bool PART, bool CW = false>
__device__ __forceinline__ void store_rows(const TmaImage &im, uint8_t *row_a, uint8_t *row_b,
                                           int x, const uint32_t vx[4], const uint32_t vy[4],
                                           const uint32_t vd[4], const uint32_t vt[4],
                                           bool st_a, bool st_b, bool zero_a, bool zero_b,
                                           uint32_t colmask, uint32_t framemask, bool vec,
                                           int wl) {
  if constexpr (FMT == kS16x4) {
    static_assert(!CW, "runtime-weight passes carry P and M, not the S16X4 planes");
    const uint64_t plane = (uint64_t)(uint32_t)im.H * im.dp;
    const uint32_t *vals[4] = {vx, vy, vd, vt};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t *v = vals[q];
      int16_t *pa = (int16_t *)(row_a + q * plane) + x;
      int16_t *pb = (int16_t *)(row_b + q * plane) + x;
      if (!GEN) {
        const uint2 la = make_uint2(__byte_perm(v[0], v[1], 0x5410) ^ (kBias * 0x10001u),
                                    __byte_perm(v[2], v[3], 0x5410) ^ (kBias * 0x10001u));
        const uint2 lb = make_uint2(__byte_perm(hi_ready(v[0]), hi_ready(v[1]), 0x7632),
                                    __byte_perm(hi_ready(v[2]), hi_ready(v[3]), 0x7632));
        if constexpr (RA) {
          st4_s16_realigned<PART>(pa, la.x, la.y, st_a, wl);
          st4_s16_realigned<PART>(pb, lb.x, lb.y, st_b, wl);
        } else if (!PART || wl >= 4) {
          if (st_a) *(uint2 *)pa = la;
          if (st_b) *(uint2 *)pb = lb;
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (k >= wl) continue;
            const uint32_t wa = k < 2 ? la.x : la.y, wb = k < 2 ? lb.x : lb.y;
            if (st_a) pa[k] = (int16_t)(wa >> (16 * (k & 1)));
            if (st_b) pb[k] = (int16_t)(wb >> (16 * (k & 1)));
          }
        }
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
  if constexpr (CW) {
#pragma unroll
    for (int k = 0; k < 4; ++k) squares_w(vx[k], vy[k], vd[k], vt[k], sa[k], sb[k]);
  } else
#if SOBEL4_SQW == 2
  // F32: strip b's S stays negated (the square root folds the sign in).
  if constexpr (FMT == kF32) {
#pragma unroll
    for (int k = 0; k < 4; ++k) squares_wide(vx[k], vy[k], vd[k], vt[k], sa[k], sb[k]);
  } else
#endif
  {
    constexpr bool kSqb = (RA || GEN) ? (SOBEL4_SQB_RA != 0) : (SOBEL4_SQB != 0);
#pragma unroll
    for (int k = 0; k < 4; ++k) squares<kSqb>(vx[k], vy[k], vd[k], vt[k], sa[k], sb[k]);
  }
  if constexpr (FMT == kF32) {
    float ga[4], gb[4];
#if SOBEL4_SQW == 2
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ga[k] = magnitude_newton(sa[k]);
      gb[k] = CW ? magnitude_newton(sb[k]) : magnitude_newton_neg(sb[k]);
    }
#else
#pragma unroll
    for (int k = 0; k < 4; ++k) magnitude_f32x2(sa[k], sb[k], ga[k], gb[k]);
#endif
    float *pa = (float *)row_a + x, *pb = (float *)row_b + x;
    if (!GEN) {
      if constexpr (RA) {
        st4_f32_realigned<PART>(pa, ga, st_a, wl);
        st4_f32_realigned<PART>(pb, gb, st_b, wl);
      } else if (!PART || wl >= 4) {
        if (st_a) *(float4 *)pa = make_float4(ga[0], ga[1], ga[2], ga[3]);
        if (st_b) *(float4 *)pb = make_float4(gb[0], gb[1], gb[2], gb[3]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (k >= wl) continue;
          if (st_a) pa[k] = ga[k];
          if (st_b) pb[k] = gb[k];
        }
      }
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
  } else if constexpr (FMT == kU16) {
    uint32_t ua[4], ub[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ua[k] = magnitude_u16(sa[k]);
      ub[k] = magnitude_u16(sb[k]);
    }
    uint16_t *pa = (uint16_t *)row_a + x, *pb = (uint16_t *)row_b + x;
    if (GEN) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool fk = (framemask >> k) & 1u;
        if (zero_a || fk) ua[k] = 0u;
        if (zero_b || fk) ub[k] = 0u;
      }
    }
    const uint2 wa = make_uint2(ua[0] | (ua[1] << 16), ua[2] | (ua[3] << 16));
    const uint2 wb = make_uint2(ub[0] | (ub[1] << 16), ub[2] | (ub[3] << 16));
    if (!GEN) {
      if constexpr (RA) {
        st4_s16_realigned<PART>((int16_t *)pa, wa.x, wa.y, st_a, wl);
        st4_s16_realigned<PART>((int16_t *)pb, wb.x, wb.y, st_b, wl);
      } else if (!PART || wl >= 4) {
        if (st_a) *(uint2 *)pa = wa;
        if (st_b) *(uint2 *)pb = wb;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (k >= wl) continue;
          if (st_a) pa[k] = (uint16_t)ua[k];
          if (st_b) pb[k] = (uint16_t)ub[k];
        }
      }
    } else if (vec && colmask == 0xFu) {
      if (st_a) *(uint2 *)pa = wa;
      if (st_b) *(uint2 *)pb = wb;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!((colmask >> k) & 1u)) continue;
        if (st_a) pa[k] = (uint16_t)ua[k];
        if (st_b) pb[k] = (uint16_t)ub[k];
      }
    }
  } else {
    uint32_t ua[4], ub[4];
    if constexpr (FMT == kEdge8) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        ua[k] = sa[k] >= im.thr ? 255u : 0u;
        ub[k] = sb[k] >= im.thr ? 255u : 0u;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) magnitude_u8x2(sa[k], sb[k], ua[k], ub[k]);
    }
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
      if constexpr (RA) {
        st4_u8_realigned<PART>(pa, wa, st_a, wl);
        st4_u8_realigned<PART>(pb, wb, st_b, wl);
      } else if (!PART || wl >= 4) {
        if (st_a) *(uint32_t *)pa = wa;
        if (st_b) *(uint32_t *)pb = wb;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (k >= wl) continue;
          if (st_a) pa[k] = (uint8_t)ua[k];
          if (st_b) pb[k] = (uint8_t)ub[k];
        }
      }
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
  } else if constexpr (FMT == kU8 || FMT == kEdge8) {
    row[x] = 0;
  } else if constexpr (FMT == kU16) {
    ((uint16_t *)row)[x] = 0;
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
  } else if constexpr (FMT == kU8 || FMT == kEdge8) {
    *(uint32_t *)(row + x) = 0u;
  } else if constexpr (FMT == kU16) {
    *(uint2 *)((uint16_t *)row + x) = make_uint2(0u, 0u);
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
  const CUtensorMap *map;   // source image (tensor staging), box 160 x 8
  const uint8_t *ringp;     // the same ring as a generic pointer
  int lose_stage;           // stage of this item whose copy is withheld (-1: none)
  uint32_t ring;            // shared address of this warp's ring
  uint32_t gstage;          // stages this warp has used so far (slot / parity counter)
};

template <int ST>
__device__ __forceinline__ uint32_t bar_addr(const ItemCtx &cx, uint32_t g) {
  return cx.ring + (uint32_t)(Geo<ST>::kSlots * Geo<ST>::kSlot + 8 * (g % Geo<ST>::kSlots));
}

// Waits until stage counter g has landed (all lanes agree on the outcome).
template <int ST>
__device__ __forceinline__ bool wait_stage(const ItemCtx &cx, uint32_t g, unsigned int *err) {
  const uint32_t bar = bar_addr<ST>(cx, g);
  const uint32_t parity = (g / Geo<ST>::kSlots) & 1u;
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
template <int ST>
__device__ __forceinline__ void drain_stages(const ItemCtx &cx, uint32_t g_from, uint32_t g_to) {
  for (uint32_t g = g_from; g < g_to; ++g) {
    const uint32_t bar = bar_addr<ST>(cx, g);
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, (g / Geo<ST>::kSlots) & 1u) && global_ns() - t0 < kWaitLimitNs) {
    }
  }
}

// Copies stage j of an item (rows 8j .. 8j+7 of both strips) into ring slot
// g % Geo<ST>::kSlots.  All lanes call it after a warp barrier.  Tensor staging: lane
// 0 issues two box copies.  Bulk staging: lane 8s+k copies row k of strip s
// (the granules that hold columns x0-2 .. x0+129 of an image row; rows outside
// the image are not copied) and records the offset of column x0-2 from the
// copied data; lane 0 arms the barrier with the stage's total byte count
// before any copy is issued.
template <int ST>
__device__ __forceinline__ void issue_stage(const TmaImage &im, const ItemCtx &cx, int x0, int ya,
                                            int yb, int j, uint32_t g, int lane) {
  using G = Geo<ST>;
  const uint32_t slot = cx.ring + (uint32_t)(G::kSlot * (g % Geo<ST>::kSlots));
  const uint32_t bar = bar_addr<ST>(cx, g);
  if (j == cx.lose_stage) return;  // injected loss: this stage's wait must run out
  if constexpr (ST == kTensor) {
    if (lane == 0) {
      fence_proxy_async();
      mbar_expect_tx(bar, (uint32_t)G::kSlot);
      tma_load_2d(slot, cx.map, x0 - 16, ya - 2 + Geo<ST>::kStageRows * j, bar);
      tma_load_2d(slot + (uint32_t)G::kStrip, cx.map, x0 - 16, yb - 2 + Geo<ST>::kStageRows * j, bar);
    }
  } else {
    uint32_t bytes = 0;
    const uint8_t *from = nullptr;
    uint32_t to = 0;
    if (lane < 2 * Geo<ST>::kStageRows) {
      constexpr int B = G::kBpp;
      const int s = lane / Geo<ST>::kStageRows, k = lane % Geo<ST>::kStageRows;
      const int y = (s ? yb : ya) - 2 + Geo<ST>::kStageRows * j + k;
      to = slot + (uint32_t)(s * G::kStrip + k * G::kRowPitch + G::kRowData);
      int32_t hdr = 0;
      if (y >= 0 && y < im.H) {
        const uintptr_t row = (uintptr_t)im.src + (uintptr_t)(uint32_t)y * im.sp;
        const uintptr_t lo = row + (uintptr_t)(B * max(x0 - 2, 0));
        const uintptr_t hi = row + (uintptr_t)(B * min(x0 + kCols + 2, im.W));
        const uintptr_t g0 = lo & ~(uintptr_t)15;
        from = (const uint8_t *)g0;
        bytes = (uint32_t)(((hi + 15) & ~(uintptr_t)15) - g0);
        hdr = (int32_t)((intptr_t)row + (intptr_t)(B * (x0 - 2)) - (intptr_t)g0);
      }
      *(int32_t *)(cx.ringp + (slot - cx.ring) + G::kHdr + 4 * lane) = hdr;
    }
    const uint32_t total = __reduce_add_sync(0xffffffffu, bytes);
    if (lane == 0) mbar_expect_tx(bar, total);
    __syncwarp();
    if (bytes) {
      fence_proxy_async();
      bulk_load(to, from, bytes, bar);
    }
  }
}

// FULL: every output row of both strips lies inside the image (no row checks).
// RA (fast path): realigned stores for a destination that is not vector-aligned.
// PART (fast path): the segment runs past column W-1; stores stop at column W.
// CW: runtime-weight passes with the coefficients cw (else Eq. 3's, and cw unused).
template <int FMT, bool GEN, bool FULL, int ST, bool RA, bool PART, bool CW = false>
// ya: first row of strip a; R: this item's strip height (see strip_rows).
__device__ __forceinline__ bool tma_item(const TmaImage &im, int border, int seg, int ya,
                                         int R, int lane, ItemCtx &cx, unsigned int *err,
                                         const Coefs &cw) {
  using G = Geo<ST>;
  const int H = im.H, W = im.W;
  const int x0 = seg * kCols;
  const int x = x0 + kNC * lane;
  const int wl = W - x;  // this lane's columns inside the image (PART)
  const int yb = ya + R;
  const int steps = R + 4;
  const int n_stages = (steps + Geo<ST>::kStageRows - 1) / Geo<ST>::kStageRows;
  const uint32_t g0 = cx.gstage;
  const bool mapped_rule = border == kReplicate || border == kReflect101;

  __syncwarp();  // every lane is done with the ring slots about to be refilled
  for (int j = 0; j < Geo<ST>::kSlots && j < n_stages; ++j)
    issue_stage<ST>(im, cx, x0, ya, yb, j, g0 + (uint32_t)j, lane);

  // Edge-item bookkeeping.
  uint32_t colmask = 0xFu, framemask = 0u, zmask = 0u;
  bool edge_lane = false;
  int32_t off[8];
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
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = x - 2 + j;
      bool z;
      const int m = map_index(col, W, border, &z);
      const int o = m - (x0 - 2);  // staged offset relative to column x0-2
      off[j] = o < 0 ? 0 : (o > kCols + 3 ? kCols + 3 : o);
      if (G::kRows && border != kReplicate && border != kReflect101 && (col < 0 || col >= W))
        zmask |= 1u << j;
    }
    // Lanes whose columns cross an image edge read through the mapping (the
    // bulk staging also for CONSTANT0, whose outside columns read 0).
    edge_lane = (mapped_rule || (G::kRows && border == kConstant0)) &&
                (x - 2 < 0 || x + 5 >= W);
    const int vec_need = vec_bytes(FMT);
    vec = im.dst_align >= vec_need;
  }

  Col st[kNC];
#pragma unroll
  for (int k = 0; k < kNC; ++k) st[k] = col_zero();
  uint8_t *row_a = (uint8_t *)im.dst + (uint64_t)(uint32_t)ya * im.dp;
  uint8_t *row_b = (uint8_t *)im.dst + (uint64_t)(uint32_t)min(yb, H - 1) * im.dp;

  // rd: shared address of staged row k (data start) of strip a in the stage.
  auto step = [&](uint32_t rd, int k, int s, bool tail) {
    const int i = s - 4;  // output row of this step within each strip
    // Shared addresses of column x0-2 in strip a's and strip b's row.
    uint32_t base_a, base_b;
    if constexpr (ST == kTensor) {
      base_a = rd + 14;
      base_b = base_a + G::kStrip;
    } else {
      const uint32_t slot = rd - (uint32_t)(k * G::kRowPitch + G::kRowData);
      base_a = rd + (uint32_t)lds_s32(slot + G::kHdr + 4 * k);
      base_b = rd + (uint32_t)G::kStrip + (uint32_t)lds_s32(slot + G::kHdr + 4 * (Geo<ST>::kStageRows + k));
    }
    uint32_t c[8];
    if (GEN) {
      const int ra = ya - 2 + s, rb = yb - 2 + s;  // input rows of this step
      const bool out_a = ra < 0 || ra >= H, out_b = rb < 0 || rb >= H;
      if (((mapped_rule || G::kRows) && (out_a || out_b)) || edge_lane)
        gather_cols<G::kBpp>(im, base_a, base_b, off, zmask, x, ra, rb, out_a, out_b, border, c);
      else if constexpr (ST == kTensor)
        read_cols<G::kStrip>(base_a + kNC * lane, c);
      else if constexpr (ST == kRgbBulk)
        read_cols_rgb(base_a + 3 * kNC * lane, base_b + 3 * kNC * lane, c);
      else
        read_cols_any(base_a + kNC * lane, base_b + kNC * lane, c);
    } else if constexpr (ST == kTensor) {
#if SOBEL4_TMA_CLD
      read_cols_p(cx.ringp + (base_a + kNC * lane - cx.ring), c);
#else
      read_cols<G::kStrip>(base_a + kNC * lane, c);
#endif
    } else if constexpr (ST == kRgbBulk) {
      read_cols_rgb(base_a + 3 * kNC * lane, base_b + 3 * kNC * lane, c);
    } else {
      read_cols_any(base_a + kNC * lane, base_b + kNC * lane, c);
    }
    uint32_t vx[kNC], vy[kNC], vd[kNC], vt[kNC];
    if (tail) {
#pragma unroll
      for (int q = 0; q < kNC; ++q) {
        if constexpr (CW)
          column_step_w<true>(cw, c[q], c[q + 1], c[q + 2], c[q + 3], c[q + 4], st[q], vx[q],
                              vy[q], vd[q], vt[q]);
        else
          column_step<true>(c[q], c[q + 1], c[q + 2], c[q + 3], c[q + 4], st[q], vx[q], vy[q],
                            vd[q], vt[q]);
      }
      const bool st_a = FULL || i < na, st_b = FULL || i < nb;
      bool zero_a = false, zero_b = false;
      if (GEN) {
        if (border == kValid) {
          zero_a = ya + i < 2 || ya + i > H - 3;
          zero_b = yb + i < 2 || yb + i > H - 3;
        }
      }
      store_rows<FMT, GEN, RA, PART, CW>(im, row_a, row_b, x, vx, vy, vd, vt, st_a, st_b, zero_a,
                                     zero_b, colmask, framemask, vec, wl);
      row_a += im.dp;
      row_b += im.dp;
    } else {
#pragma unroll
      for (int q = 0; q < kNC; ++q) {
        if constexpr (CW)
          column_step_w<false>(cw, c[q], c[q + 1], c[q + 2], c[q + 3], c[q + 4], st[q], vx[q],
                               vy[q], vd[q], vt[q]);
        else
          column_step<false>(c[q], c[q + 1], c[q + 2], c[q + 3], c[q + 4], st[q], vx[q], vy[q],
                             vd[q], vt[q]);
      }
    }
  };

  if (!wait_stage<ST>(cx, g0, err)) {
    drain_stages<ST>(cx, g0 + 1, g0 + (uint32_t)min(Geo<ST>::kSlots, n_stages));
    return false;
  }
  uint32_t rd = cx.ring + (uint32_t)(G::kSlot * (g0 % Geo<ST>::kSlots) + G::kRowData);
#pragma unroll
  for (int s = 0; s < 4; ++s)  // rows 0..3 only fill the window
    step(rd + (uint32_t)(s * G::kRowPitch), s, s, false);
  rd += 4 * G::kRowPitch;
  // Main loop: kUnroll row steps per trip (R is a multiple of kUnroll, so the
  // trips tile the steps and the stage boundaries fall on trip boundaries).
#pragma unroll 1
  for (int s = 4; s < steps; s += kUnroll) {
    if ((s & (Geo<ST>::kStageRows - 1)) == 0) {
      const int j = s / Geo<ST>::kStageRows;
      __syncwarp();  // stage j-1 has been read by every lane
      if (j - 1 + Geo<ST>::kSlots < n_stages)
        issue_stage<ST>(im, cx, x0, ya, yb, j - 1 + Geo<ST>::kSlots, g0 + (uint32_t)(j - 1 + Geo<ST>::kSlots),
                        lane);
      if (!wait_stage<ST>(cx, g0 + (uint32_t)j, err)) {
        drain_stages<ST>(cx, g0 + (uint32_t)j + 1,
                         g0 + (uint32_t)min(j - 1 + Geo<ST>::kSlots + 1, n_stages));
        return false;
      }
      rd = cx.ring + (uint32_t)(G::kSlot * ((g0 + (uint32_t)j) % Geo<ST>::kSlots) + G::kRowData);
    }
    const int k0 = s & (Geo<ST>::kStageRows - 1);
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) step(rd + (uint32_t)(u * G::kRowPitch), k0 + u, s + u, true);
    rd += kUnroll * G::kRowPitch;
  }
  cx.gstage = g0 + (uint32_t)n_stages;
  if (!GEN && border == kValid) {
    // The paper's rule leaves the 2-pixel frame at 0.  The fast path computed
    // it from halos that may hold anything outside the image; the lane that
    // stored each frame element now overwrites it (same thread, later store;
    // with realigned stores a neighbouring lane stored it, and the warp
    // barrier orders the two).
    if constexpr (RA) __syncwarp();
    const int yr[2] = {ya, yb}, nr[2] = {na, nb};
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int f[4] = {0, 1, H - 2, H - 1};
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (f[q] >= yr[t] && f[q] < yr[t] + nr[t] && (q < 2 || f[q] > 1)) {
          if constexpr (RA || PART) {
#pragma unroll
            for (int k = 0; k < kNC; ++k)
              if (!PART || k < wl) zero_px<FMT>(im, f[q], x + k);
          } else {
            zero_row4<FMT>(im, f[q], x);
          }
        }
    }
    // Frame columns {0, 1, W-2, W-1} inside the segment: all lanes share the
    // rows; the barrier orders the stores of the lanes that computed them.
    if (x0 < 2 || x0 + kCols > W - 2) {
      __syncwarp();
      const int fc[4] = {0, 1, W - 2, W - 1};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = fc[q];
        if (c < x0 || c >= x0 + kCols || c >= W || (q >= 2 && c < 2)) continue;
        for (int r = lane; r < na + nb; r += 32) zero_px<FMT>(im, r < na ? ya + r : yb + r - na, c);
      }
    }
  }
  return true;
}

// An item for the fast path: a border rule the staging serves as is (VALID,
// frame zeroed afterwards; CONSTANT0 with tensor staging, whose copies
// zero-fill), with any segment, the last one of a ragged width included
// (PART); or every input row and column inside the image.
template <int ST>
__device__ __forceinline__ bool fast_item(const TmaImage &im, int border, int seg, int ya,
                                          int R, int fmt) {
  const int x0 = seg * kCols;
  (void)fmt;
  if (border == kValid || (ST == kTensor && border == kConstant0)) return true;
  return x0 >= 2 && x0 + kCols + 2 <= im.W && ya >= 2 && ya + 2 * R + 2 <= im.H;
}

// Item order: the frame of edge items first, then the interior.  Edge items
// take the general path, whose steps cost more than the fast path's; handing
// them out first lets the fast items fill in around them instead of leaving
// them as the tail of the launch.  The fast items form the rectangle of bands
// [bl, bh) x segments [sl, sh) (the complement of fast_item's rules without
// the destination test); item i maps to (seg, band) by taking, in turn, the
// frame bands x all segments, the inner bands x frame segments, and the
// inner rectangle band-major.  The mapping is a bijection on [0, n_seg *
// n_band) for any bounds, so it never decides correctness.
template <int ST>
__device__ __forceinline__ void item_coords(const TmaImage &im, int border, int R, int i,
                                            int *seg, int *band) {
  const int S = im.n_seg, B = im.n_band;
  const bool inner_rule = !(border == kValid || (ST == kTensor && border == kConstant0));
  int sl = 0, sh = im.W / kCols, bl = 0, bh = B;
  if (inner_rule) {
    sl = 1;
    sh = im.W >= kCols + 2 ? (im.W - kCols - 2) / kCols + 1 : 0;
    bl = 1;
    bh = im.H >= 2 * R + 2 ? (im.H - 2 * R - 2) / (2 * R) + 1 : 0;
  }
  sh = max(sh, sl);
  bh = max(bh, bl);
  const int nb_in = bh - bl, ns_in = sh - sl;
  const int nA = (B - nb_in) * S;
  if (i < nA) {
    const int k = i / S;
    *band = k < bl ? k : bh + (k - bl);
    *seg = i - k * S;
    return;
  }
  i -= nA;
  const int ns_edge = S - ns_in;
  if (i < nb_in * ns_edge) {
    const int b = i / ns_edge, k = i - b * ns_edge;
    *band = bl + b;
    *seg = k < sl ? k : sh + (k - sl);
    return;
  }
  i -= nb_in * ns_edge;
  const int b = i / ns_in;
  *band = bl + b;
  *seg = sl + (i - b * ns_in);
}

// Strip height of the items of a band: R, except in a last band with fewer
// than 2R rows, whose rows are split evenly between the two strips (rounded
// up to the row-step unroll), so that no strip runs far past the image.
__device__ __forceinline__ int strip_rows(const TmaImage &im, int band, int R) {
  const int left = im.H - band * 2 * R;
  if (left >= 2 * R) return R;
  const int half = (left + 1) / 2;
  return min(R, (half + kUnroll - 1) / kUnroll * kUnroll);
}

// Runs one item through the variant its geometry needs; a kernel that runs
// only fast items (or only the others) carries only that code.  Each variant
// is a large unrolled body, and warps of one SM running several of them at
// once miss in the instruction cache (measured on ragged batches: 56 % hits
// with three fast variants live, 98 % with one).  So the batched kernel
// (ONE) and the single-image kernels of a ragged width (kFastPart) or of
// unaligned destination rows (kFastRA) send every fast item through a single
// body: row checks, stores that stop at column W, and, in a kernel that may
// meet unaligned destinations (kAll, kFastRA), the realigned stores, which
// fall through to plain vector stores on an aligned row.  The
// lean single-image kernel (kFastOnly, width a multiple of the segment) keeps
// the check-free body for full bands and carries no other.
template <int FMT, int MODE, int ST, bool ONE, bool CW = false>
__device__ __forceinline__ bool run_item(const TmaImage &im, int border, int seg, int ya, int R,
                                         int lane, ItemCtx &cx, unsigned int *err, bool fast,
                                         const Coefs &cw) {
  if (!fast_mode<MODE>() && !fast)
    return tma_item<FMT, true, false, ST, false, false, CW>(im, border, seg, ya, R, lane, cx, err, cw);
  constexpr bool kRA = MODE == kAll || MODE == kFastRA;  // realigned stores possible
  if constexpr (ONE || MODE == kFastPart || MODE == kFastRA) {
    return tma_item<FMT, false, false, ST, kRA, true, CW>(im, border, seg, ya, R, lane, cx, err, cw);
  } else if constexpr (MODE == kFastOnly) {
    // The host plans this kernel only for widths that are a multiple of kCols.
    if (ya + 2 * R <= im.H)
      return tma_item<FMT, false, true, ST, false, false, CW>(im, border, seg, ya, R, lane, cx, err, cw);
    return tma_item<FMT, false, false, ST, false, false, CW>(im, border, seg, ya, R, lane, cx, err, cw);
  } else {
    if (im.dst_align < vec_bytes(FMT))
      return tma_item<FMT, false, false, ST, true, true, CW>(im, border, seg, ya, R, lane, cx, err, cw);
    if (im.W % kCols != 0)
      return tma_item<FMT, false, false, ST, false, true, CW>(im, border, seg, ya, R, lane, cx, err, cw);
    if (ya + 2 * R <= im.H)
      return tma_item<FMT, false, true, ST, false, false, CW>(im, border, seg, ya, R, lane, cx, err, cw);
    return tma_item<FMT, false, false, ST, false, false, CW>(im, border, seg, ya, R, lane, cx, err, cw);
  }
}

template <int ST>
__device__ __forceinline__ void init_ring(ItemCtx &cx, WarpRing<ST> &ring, int lane) {
  cx.ring = smem_addr(&ring);
  cx.ringp = &ring.slot[0][0];
  cx.gstage = 0;
  cx.lose_stage = -1;
  if (lane == 0) {
    for (int i = 0; i < Geo<ST>::kSlots; ++i)
      mbar_init(cx.ring + (uint32_t)(Geo<ST>::kSlots * Geo<ST>::kSlot + 8 * i), 1u);
    mbar_init_fence();
  }
  if constexpr (Geo<ST>::kRows) {
    // Zero the pads and offsets once so that no read of the ring ever meets
    // uninitialised bytes.
    for (int i = lane; i < Geo<ST>::kSlots * Geo<ST>::kSlot / 4; i += 32)
      ((uint32_t *)&ring.slot[0][0])[i] = 0u;
  }
  __syncwarp();
}

// The single-image kernel: persistent CTAs of 4 warps; each warp pulls items
// (band-major) from the counter pair[0]; the last warp out resets the pair.
// `map` is used by the tensor staging only.
// CW: runtime-weight passes with the coefficients cw, a __grid_constant__
// kernel parameter: the multiply-adds read them from the constant bank as
// operands (as a plain parameter they cost 13 more registers per thread and
// 3.0 M more warp instructions on 8192 x 8192).
template <int FMT, int MODE, int ST, bool CW = false>
__global__ void __launch_bounds__(kWarps * 32, min_ctas<MODE>())
    tma_single_kernel(const __grid_constant__ CUtensorMap map, TmaImage im, int border, int R,
                      int n_items, unsigned int *pair, unsigned int *err,
                      const __grid_constant__ Coefs cw) {
  __shared__ WarpRing<ST> rings[kWarps];
  const int lane = threadIdx.x & 31;
  ItemCtx cx;
  init_ring<ST>(cx, rings[threadIdx.x >> 5], lane);
  cx.map = &map;
  grid_dependency_wait();
  for (;;) {
    unsigned int got = 0;
    if (lane == 0) got = atomicAdd(&pair[0], 1u);
    got = __shfl_sync(0xffffffffu, got, 0);
    if (got >= (unsigned int)n_items) break;
    const int item = (int)got;
    int seg, band;
    item_coords<ST>(im, border, R, item, &seg, &band);
    cx.lose_stage = item == 0 ? im.lose_stage : -1;
    const int ya = band * 2 * R, Ri = strip_rows(im, band, R);
    const bool fast = fast_item<ST>(im, border, seg, ya, Ri, FMT);
    if ((fast_mode<MODE>() && !fast) || (MODE == kGeneralOnly && fast)) continue;
    if (!run_item<FMT, MODE, ST, false, CW>(im, border, seg, ya, Ri, lane, cx, err, fast, cw))
      break;
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

// Coefficients of the batched kernel, which runs Eq. (3) only (unused).
__device__ const Coefs kNoCoefs = {};

// The batched kernel: persistent CTAs of 4 warps pull items (image by image,
// band-major) from *queue (zeroed by the host before the launch); a warp
// finds an item's image by binary search over the descriptors' first items.
template <int FMT, int MODE, int ST>
__global__ void __launch_bounds__(kWarps * 32, min_ctas<MODE>())
    tma_batched_kernel(const typename BatchDescOf<ST>::type *__restrict__ descs, int n_img,
                       int total, unsigned int *queue, int border, int R, unsigned int *err) {
  __shared__ WarpRing<ST> rings[kWarps];
  const int lane = threadIdx.x & 31;
  ItemCtx cx;
  init_ring<ST>(cx, rings[threadIdx.x >> 5], lane);
  grid_dependency_wait();
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
    const typename BatchDescOf<ST>::type *d = descs + lo;
    const TmaImage im = d->im;
    int seg, band;
    item_coords<ST>(im, border, R, (int)(item - d->item0), &seg, &band);
    const int ya = band * 2 * R, Ri = strip_rows(im, band, R);
    const bool fast = fast_item<ST>(im, border, seg, ya, Ri, FMT);
    if ((fast_mode<MODE>() && !fast) || (MODE == kGeneralOnly && fast)) continue;
    if constexpr (ST == kTensor) {
      if (lo != cur) {
        if (lane == 0) tensormap_acquire(&d->map);
        cur = lo;
      }
      cx.map = &d->map;
    } else {
      cx.map = nullptr;  // bulk staging reads rows through im.src
    }
    cx.lose_stage = -1;
    if (!run_item<FMT, MODE, ST, true>(im, border, seg, ya, Ri, lane, cx, err, fast, kNoCoefs))
      break;
  }
}

}  // namespace tma
}  // namespace sobel4
