// sobel4_tc.cuh — tensor-core kernel for the paper's border rule (VALID):
// the four 5x5 masks of Eq. (3) as banded matrix products on the fifth-
// generation tensor cores (tcgen05.mma, accumulators in tensor memory), the
// squares of Eq. (4) and the square root on the CUDA cores.
//
// Why a matrix product.  The register-window kernel (sobel4_tma.cuh) spends
// about 37 integer and float instructions per pixel, and its run time is set
// by instruction issue, not by HBM.  The four responses are linear in the 25
// input pixels around each output: R_k(y, x) = sum_{dy,dx} K_k[dy][dx] *
// I(y+dy-2, x+dx-2).  For one mask row dy that is a product of the image rows
// with a banded matrix, so a tile of 128 output rows x 8 output columns
// takes five accumulating products D += A_dy * B_dy with
//   A_dy[i, k] = I(y0 - 2 + dy + i, x0 - 2 + k)   (128 x 16, f16)
//   B_dy[n, k] = K_r[dy][k - j] for n = 4j + r, 0 <= k - j <= 4, else 0
// (N = 8 columns x 4 responses = 32, K = 16 input columns of which 12 are
// used).  All five A_dy are views of one staged tile at row offsets dy: the
// staged operand keeps its 8-row core matrices back to back (16 bytes per
// row), so a view dy rows down is the same descriptor 16*dy bytes later.
//
// Exactness.  Inputs are staged as the f16 value 1024 + p (exact; the bias
// cancels because every mask sums to zero: true of Eq. 3 and of every
// operator of Eq. 5), weights are integers of at most 2048 in magnitude, and
// each accumulator is preset to 1.5 * 2^23 (a tensor-memory store of the bit
// pattern 0x4B400000), so every partial sum is an integer in [2^23, 2^24),
// exact in fp32, and the final bits are 0x4B400000 + R.  The squares are
// taken from the bits in int32, modulo 2^32:
//   S = sum (b_r - C)^2 = sum b_r^2 - 2C * sum b_r   (4C^2 = 0 mod 2^32),
// exact because S < 2^31, and G = sqrtf((float)S) as in the other kernels.
//
// Schedule.  Persistent CTAs, one per SM (tensor memory: two accumulator
// buffers of 256 columns), over tiles of 128 output rows x 64 output columns:
//   * warp 16 lane 0: 2-D tensor copies (TMA) of the 132 x 96 input box
//     (columns x0-16 .. x0+79) into a ring of six shared buffers;
//   * warps 0..15: convert a landed box into the f16 operand (9 column groups
//     x 132 rows, double-buffered), then read a finished accumulator buffer
//     (thread = output row, 2 x-tiles per warp), preset it again for its next
//     use, form S and G, and write them into a 128-byte-swizzled staging tile;
//   * warp 17 lane 0: 40 products per tile (5 mask rows, each over the 8
//     x-tiles) into the free accumulator buffer, then a commit to an mbarrier;
//   * warp 18 lane 0: 2-D tensor stores (TMA) of the staging tile (two 32 x
//     128 boxes; the copy engine clips at the image edge).
// Every wait is bounded (2 s of global time); a wait that runs out sets bit 0
// of *err, raises the CTA's abort flag, and all roles leave after letting
// their copies and products in flight land.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sobel4_arith.cuh"
#include "sobel4_tma.cuh"

namespace sobel4 {
namespace tc {

constexpr int kM = 128;                // output rows per tile: MMA M, tensor-memory lanes
constexpr int kInRows = kM + 4;        // staged input rows
constexpr int kXT = 8;                 // x-tiles (8 output columns each) per tile
constexpr int kTileCols = 8 * kXT;     // 64
constexpr int kBoxW = 96;              // input box width (bytes): columns x0-16 .. x0+79
constexpr int kKG = kXT + 1;           // 8-column groups of the f16 operand
constexpr int kN = 32;                 // MMA N: 8 columns x 4 responses
constexpr int kEpiWarps = 16;
constexpr int kLoadWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1, kStoreWarp = kEpiWarps + 2;
constexpr int kThreads = (kEpiWarps + 3) * 32;
constexpr uint32_t kTmemCols = 512;    // two buffers of kXT * kN columns
// Input boxes in flight per CTA: enough bytes outstanding per SM to cover the
// HBM latency (two were not).
constexpr int kUStages = 6;
constexpr uint32_t kUBytes = kBoxW * kInRows;            // 12672
// Bytes between the operand's 8-column groups: 132 rows of 16 bytes plus 16,
// which puts the groups of one row on distinct bank quads for the converters.
constexpr uint32_t kALbo = kInRows * 16 + 16;
constexpr uint32_t kABytes = kKG * kALbo;                // 19152
constexpr uint32_t kBMat = 2 * kN * 16;                  // one 32 x 16 weight matrix
constexpr uint32_t kOBox = kM * 128;                     // one 32-column output box
constexpr uint32_t kMagic = 0x4B400000u;                 // bits of 1.5 * 2^23

constexpr uint32_t align_up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }
// Shared-memory map (offsets from a 1024-byte aligned base).
constexpr uint32_t kOffO = 0;                              // 2 staging tiles x 2 boxes (swizzled)
constexpr uint32_t kOffU = kOffO + 4 * kOBox;
constexpr uint32_t kUStride = align_up(kUBytes, 128);
constexpr uint32_t kOffA = kOffU + kUStages * kUStride;
constexpr uint32_t kAStride = align_up(kABytes, 128);
constexpr uint32_t kOffB = kOffA + 2 * kAStride;           // 5 matrices: mask rows dy = 0..4
constexpr int kNumBars = 2 * kUStages + 10;
constexpr uint32_t kOffBar = kOffB + 5 * kBMat;
constexpr uint32_t kOffMisc = kOffBar + kNumBars * 8;      // tmem base, abort, last loads/commits
constexpr uint32_t kSmemUsed = kOffMisc + 64;
constexpr uint32_t kSmemBytes = align_up(kSmemUsed, 1024) + 1024;  // + room to align the base
static_assert(kSmemBytes > 114 * 1024, "one CTA per SM: each allocates all tensor memory");
static_assert(kSmemBytes <= 227 * 1024, "shared-memory map");

// One per input stage (full, empty), two of each of the others (one per buffer).
enum Bar {
  kUFull = 0,
  kUEmpty = kUStages,
  kAFull = 2 * kUStages,
  kTFull = 2 * kUStages + 2,
  kTEmpty = 2 * kUStages + 4,
  kOFull = 2 * kUStages + 6,
  kOEmpty = 2 * kUStages + 8
};

struct TcImage {
  int32_t H, W;
  int32_t fr;  // support radius of the masks: the VALID frame width
  int32_t n_tx, n_tiles;
  int32_t lose_tile;  // failure injection (tests): this CTA-local tile's copy is never issued
};

// ---------------------------------------------------------------------------
// tcgen05 wrappers.
// ---------------------------------------------------------------------------
// Shared-memory matrix descriptor, no swizzle: start address, the byte
// distance between 8-element column groups (leading) and between 8-row core
// matrices (stride), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: f16 A and B (K-major), f32 accumulator.
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kN >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);

// D += A * B (the accumulators are always preset).
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, 1, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

#define SOBEL4_W32(r)                                                                          \
  "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),          \
      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),  \
      "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),            \
      "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),            \
      "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
// 32 consecutive accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : SOBEL4_W32(r)
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Presets 32 consecutive accumulator columns of this thread's lane to
// 1.5 * 2^23 (two stores of 16 columns from 16 registers holding the pattern).
__device__ __forceinline__ void tmem_preset32(uint32_t taddr, const uint32_t (&m)[16]) {
#pragma unroll
  for (int h = 0; h < 2; ++h)
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16};" ::"r"(taddr + 16u * h),
        "r"(m[0]), "r"(m[1]), "r"(m[2]), "r"(m[3]), "r"(m[4]), "r"(m[5]), "r"(m[6]), "r"(m[7]),
        "r"(m[8]), "r"(m[9]), "r"(m[10]), "r"(m[11]), "r"(m[12]), "r"(m[13]), "r"(m[14]),
        "r"(m[15])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// 2-D tensor store of a shared box to global memory (bulk group).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, uint32_t src, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
          (uint64_t)map),
      "r"(x), "r"(y), "r"(src)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Waits until the committed stores have read their shared source.
__device__ __forceinline__ void bulk_wait_read0() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// Waits until the committed stores are complete.
__device__ __forceinline__ void bulk_wait0() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Bounded waits.  Single-thread form (copy, product and store issuers) and
// warp form (all lanes agree).  Both give up early once another role raised
// the abort flag.  Each probe lets the hardware suspend the thread for up to
// kSuspendNs until the phase completes, so waiting warps do not spin on the
// issue slots the working warps need.
// ---------------------------------------------------------------------------
constexpr uint32_t kSuspendNs = 20000;

__device__ __forceinline__ bool try_wait_suspend(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool wait_one(uint32_t bar, uint32_t parity, volatile uint32_t *abort,
                                         unsigned int *err) {
  if (tma::mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = tma::global_ns();
  for (;;) {
    if (try_wait_suspend(bar, parity)) return true;
    if (*abort) return false;
    if (tma::global_ns() - t0 > tma::kWaitLimitNs) {
      atomicOr(err, 1u);
      *abort = 1u;
      return false;
    }
  }
}

__device__ __forceinline__ bool wait_warp(uint32_t bar, uint32_t parity, volatile uint32_t *abort,
                                          unsigned int *err) {
  if (__all_sync(0xffffffffu, tma::mbar_try_wait(bar, parity))) return true;
  const uint64_t t0 = tma::global_ns();
  for (;;) {
    if (__all_sync(0xffffffffu, try_wait_suspend(bar, parity))) return true;
    if (__any_sync(0xffffffffu, *abort != 0u)) return false;
    if (__any_sync(0xffffffffu, tma::global_ns() - t0 > tma::kWaitLimitNs)) {
      if ((threadIdx.x & 31) == 0) {
        atomicOr(err, 1u);
        *abort = 1u;
      }
      return false;
    }
  }
}

// Waits (bounded, ignoring the abort flag) until phase `parity` of `bar` has
// completed: used on the way out so that no copy or product still targets
// this CTA's shared or tensor memory.
__device__ __forceinline__ void drain(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = tma::global_ns();
  while (!tma::mbar_try_wait(bar, parity) && tma::global_ns() - t0 < tma::kWaitLimitNs) {
  }
}

// Byte offset of element (row, k) in a K-major no-swizzle operand whose rows
// are 16 bytes apart and whose 8-column groups are `lbo` bytes apart.
__device__ __forceinline__ uint32_t op_off(int row, int k, uint32_t lbo) {
  return (uint32_t)(k >> 3) * lbo + (uint32_t)row * 16u + (uint32_t)(k & 7) * 2u;
}

// The five banded weight matrices B_dy[n = 4j + r][k] = K_r[dy][k - j].
__device__ __forceinline__ void fill_weights(uint8_t *smem, const Masks4 &m) {
  for (int e = threadIdx.x; e < 5 * kN * 16; e += blockDim.x) {
    const int dy = e / (kN * 16), n = (e / 16) % kN, k = e % 16;
    const int j = n >> 2, r = n & 3, dx = k - j;
    const float w = (dx >= 0 && dx <= 4) ? (float)m.w[r][dy][dx] : 0.0f;
    *(__half *)(smem + kOffB + dy * kBMat + op_off(n, k, kN * 16)) = __float2half_rn(w);
  }
}

// Converts a landed input box (u8, 96 bytes per row, column c = x0 - 16 + c)
// into the f16 operand: staged column k = image column x0 - 2 + k = box
// byte k + 14, value 1024 + p (half bit pattern 0x64pp).
__device__ __forceinline__ void convert_box(const uint8_t *u, uint8_t *a, int tid) {
  for (int e = tid; e < kKG * kInRows; e += kEpiWarps * 32) {
    const int r = e / kKG, g = e - r * kKG;  // consecutive threads: consecutive groups of a row
    const uint8_t *row = u + r * kBoxW + 8 * g;
    const uint2 w0 = *(const uint2 *)(row + 8);   // bytes 8g+8 .. 8g+15
    const uint2 w1 = *(const uint2 *)(row + 16);  // bytes 8g+16 .. 8g+23
    uint4 h;
    h.x = __byte_perm(w0.y, 0x64u, 0x4342);  // bytes 8g+14, 8g+15
    h.y = __byte_perm(w1.x, 0x64u, 0x4140);  // bytes 8g+16, 8g+17
    h.z = __byte_perm(w1.x, 0x64u, 0x4342);  // bytes 8g+18, 8g+19
    h.w = __byte_perm(w1.y, 0x64u, 0x4140);  // bytes 8g+20, 8g+21
    *(uint4 *)(a + (uint32_t)g * kALbo + (uint32_t)r * 16u) = h;
  }
}

// S of one output pixel from the accumulator bits of its four responses.
__device__ __forceinline__ int32_t s_from_bits(uint32_t b0, uint32_t b1, uint32_t b2, uint32_t b3) {
  const uint32_t sum = b0 + b1 + b2 + b3;
  uint32_t s = sum * (0u - 2u * kMagic);
  s += b0 * b0;
  s += b1 * b1;
  s += b2 * b2;
  s += b3 * b3;
  return (int32_t)s;
}

// The eight magnitudes of one x-tile row into the staging tile (16-byte
// chunks c and c+1 of row `row` of a 128-byte-swizzled box).  MASK: the tile
// touches the frame, whose pixels the paper's rule leaves at 0.
template <bool MASK>
__device__ __forceinline__ void stage_xtile(uint8_t *box, int row, int c, bool frame_row, int x,
                                            int W, int fr, const uint32_t (&r)[32]) {
  float g[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int32_t s = s_from_bits(r[4 * j], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
    const float v = magnitude_newton(s);
    g[j] = MASK && (frame_row || x + j < fr || x + j > W - 1 - fr) ? 0.0f : v;
  }
  uint8_t *line = box + row * 128;
  const int sw = row & 7;
  *(float4 *)(line + ((c ^ sw) << 4)) = make_float4(g[0], g[1], g[2], g[3]);
  *(float4 *)(line + (((c + 1) ^ sw) << 4)) = make_float4(g[4], g[5], g[6], g[7]);
}

template <int FMT>
__global__ void __launch_bounds__(kThreads, 1)
    tc_single_kernel(const __grid_constant__ CUtensorMap in_map,
                     const __grid_constant__ CUtensorMap out_map, TcImage im,
                     const __grid_constant__ Masks4 masks, unsigned int *err) {
  static_assert(FMT == kF32, "tensor-core kernel: F32 output");
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned base (the swizzled staging boxes need it).
  uint8_t *smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = smem_addr(smem);
  const uint32_t bar0 = sbase + kOffBar;
  // misc: [0] tmem base, [1] abort, [2, 2+kUStages) last load per input stage,
  // [2+kUStages, 4+kUStages) last commit per accumulator buffer
  uint32_t *misc = (uint32_t *)(smem + kOffMisc);
  volatile uint32_t *abort = misc + 1;
  auto bar = [&](int which, int b) { return bar0 + 8u * (uint32_t)(which + b); };

  fill_weights(smem, masks);
  if (tid == 0) {
    for (int u = 0; u < kUStages; ++u) {
      tma::mbar_init(bar(kUFull, u), 1);
      tma::mbar_init(bar(kUEmpty, u), kEpiWarps);
    }
    for (int b = 0; b < 2; ++b) {
      tma::mbar_init(bar(kAFull, b), kEpiWarps);
      tma::mbar_init(bar(kTFull, b), 1);
      tma::mbar_init(bar(kTEmpty, b), kEpiWarps);
      tma::mbar_init(bar(kOFull, b), kEpiWarps);
      tma::mbar_init(bar(kOEmpty, b), 1);
    }
    misc[1] = 0u;
    for (int i = 2; i < 4 + kUStages; ++i) misc[i] = 0xFFFFFFFFu;
    tma::mbar_init_fence();
  }
  tma::fence_proxy_async();  // weights written by the generic proxy, read by the MMA
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     sbase + kOffMisc),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = misc[0];

  const int n_local = (int)(((uint32_t)im.n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
  auto tile_of = [&](int li) { return (int)blockIdx.x + li * (int)gridDim.x; };

  if (warp == kLoadWarp) {
    if (lane == 0) {
      for (int li = 0; li < n_local; ++li) {
        const int u = li % kUStages, k = li / kUStages;
        if (li >= kUStages && !wait_one(bar(kUEmpty, u), (uint32_t)(k - 1) & 1u, abort, err))
          break;
        if (*abort) break;
        if (li == im.lose_tile) continue;  // injected loss: the converters' wait must run out
        const int t = tile_of(li), ty = t / im.n_tx, tx = t - ty * im.n_tx;
        tma::fence_proxy_async();
        tma::mbar_expect_tx(bar(kUFull, u), kUBytes);
        tma::tma_load_2d(sbase + kOffU + (uint32_t)u * kUStride, &in_map, kTileCols * tx - 16,
                         kM * ty - 2, bar(kUFull, u));
        misc[2 + u] = (uint32_t)li;
      }
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      for (int li = 0; li < n_local; ++li) {
        const int b = li & 1, k = li >> 1;
        if (!wait_one(bar(kAFull, b), (uint32_t)k & 1u, abort, err)) break;
        if (li >= 2 && !wait_one(bar(kTEmpty, b), (uint32_t)(k - 1) & 1u, abort, err)) break;
        tc_fence_after();
        const uint32_t a0 = sbase + kOffA + (uint32_t)b * kAStride;
        const uint32_t d0 = tmem + (uint32_t)b * (kXT * kN);
        // Mask row by mask row, each over the eight x-tiles: consecutive
        // products write different accumulators.
#pragma unroll 1
        for (int dy = 0; dy < 5; ++dy) {
          const uint64_t bd = smem_desc(sbase + kOffB + (uint32_t)dy * kBMat, kN * 16, 128);
#pragma unroll
          for (int t = 0; t < kXT; ++t)
            mma_f16(d0 + (uint32_t)(t * kN),
                    smem_desc(a0 + (uint32_t)t * kALbo + 16u * dy, kALbo, 128), bd);
        }
        mma_commit(bar(kTFull, b));
        misc[2 + kUStages + b] = (uint32_t)li;
      }
    }
  } else if (warp == kStoreWarp) {
    if (lane == 0) {
      for (int li = 0; li < n_local; ++li) {
        const int ob = li & 1;
        if (!wait_one(bar(kOFull, ob), (uint32_t)(li >> 1) & 1u, abort, err)) break;
        const int t = tile_of(li), ty = t / im.n_tx, tx = t - ty * im.n_tx;
        for (int q = 0; q < 2; ++q) {
          const int x = kTileCols * tx + 32 * q;
          if (x < im.W)
            tma_store_2d(&out_map, sbase + kOffO + (uint32_t)(2 * ob + q) * kOBox, x, kM * ty);
        }
        bulk_commit();
        bulk_wait_read0();
        mbar_arrive(bar(kOEmpty, ob));
      }
      bulk_wait0();
    }
  } else {
    // Converters and epilogue: warps 0..15.
    const int g4 = warp >> 2;                 // x-tiles 2*g4, 2*g4 + 1
    const int lrow = 32 * (warp & 3) + lane;  // accumulator lane = output row in the tile
    const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    uint32_t magic[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) magic[i] = kMagic;
    // Preset both accumulator buffers before their first products.
#pragma unroll 1
    for (int b = 0; b < 2; ++b)
      for (int q = 0; q < 2; ++q)
        tmem_preset32(tl + (uint32_t)(b * kXT * kN + (2 * g4 + q) * kN), magic);
    tmem_wait_st();
    tc_fence_before();
    auto convert = [&](int li) -> bool {
      const int b = li & 1, k = li >> 1, u = li % kUStages;
      if (!wait_warp(bar(kUFull, u), (uint32_t)(li / kUStages) & 1u, abort, err)) return false;
      if (li >= 2 && !wait_warp(bar(kTFull, b), (uint32_t)(k - 1) & 1u, abort, err)) return false;
      convert_box(smem + kOffU + u * kUStride, smem + kOffA + b * kAStride, tid);
      tma::fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(bar(kAFull, b));
        mbar_arrive(bar(kUEmpty, u));
      }
      return true;
    };
    bool ok = n_local > 0 ? convert(0) : true;
    for (int li = 0; ok && li < n_local; ++li) {
      if (li + 1 < n_local && !convert(li + 1)) break;
      const int b = li & 1, k = li >> 1, ob = li & 1;
      if (!wait_warp(bar(kTFull, b), (uint32_t)k & 1u, abort, err)) break;
      // The staging tile is free once its previous boxes were read out.
      if (li >= 2 && !wait_warp(bar(kOEmpty, ob), (uint32_t)(k - 1) & 1u, abort, err)) break;
      tc_fence_after();
      const int t = tile_of(li), ty = t / im.n_tx, tx = t - ty * im.n_tx;
      const int y = kM * ty + lrow;
      const bool frame_row = y < im.fr || y > im.H - 1 - im.fr;
      const bool mask = tx == 0 || kTileCols * tx + kTileCols > im.W - im.fr;
#pragma unroll 1
      for (int q = 0; q < 2; ++q) {
        const int xt = 2 * g4 + q;
        const uint32_t ta = tl + (uint32_t)(b * kXT * kN + xt * kN);
        uint32_t r[32];
        tmem_ld32(ta, r);
        tmem_preset32(ta, magic);  // ready for this buffer's next tile
        uint8_t *box = smem + kOffO + (2 * ob + (xt >> 2)) * kOBox;
        const int x = kTileCols * tx + 8 * xt;
        if (mask || frame_row)
          stage_xtile<true>(box, lrow, 2 * (xt & 3), frame_row, x, im.W, im.fr, r);
        else
          stage_xtile<false>(box, lrow, 2 * (xt & 3), frame_row, x, im.W, im.fr, r);
      }
      tmem_wait_st();
      tc_fence_before();
      tma::fence_proxy_async();  // staging writes, read next by the store copies
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(bar(kTEmpty, b));  // the accumulator buffer is free (and preset)
        mbar_arrive(bar(kOFull, ob));
      }
    }
  }

  // Leave: let this CTA's last copies and products land, then free the
  // tensor memory.
  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    for (int u = 0; u < kUStages; ++u)
      if (misc[2 + u] != 0xFFFFFFFFu) drain(bar(kUFull, u), (misc[2 + u] / kUStages) & 1u);
    for (int b = 0; b < 2; ++b)
      if (misc[2 + kUStages + b] != 0xFFFFFFFFu)
        drain(bar(kTFull, b), (misc[2 + kUStages + b] >> 1) & 1u);
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

}  // namespace tc
}  // namespace sobel4
