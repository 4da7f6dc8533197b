// sobel4_selftest.cu — on-device self-check of the magnitude step: the
// library's F32 magnitudes (the one of the direct kernel, the two-strip one
// of the register-window kernels, and the one that takes S negated) against
// CUDA's IEEE
// sqrtf((float)S), and its U8 magnitudes against the exact rule
// min(255, round(sqrt(S))), for every S in a range (the operator's whole
// domain is 0 .. 599,270,400).
#include "sobel4_launch.h"

namespace sobel4 {

// exact rule: u = round(sqrt(S)) <=> (2u-1)^2 <= 4S < (2u+1)^2, saturated at 255
__device__ __forceinline__ bool u8_ok(uint32_t u, int32_t s) {
  const int64_t q = 4 * (int64_t)s;
  return u == 255u ? q >= 509ll * 509ll
                   : ((u == 0u || (int64_t)(2 * u - 1) * (2 * u - 1) <= q) &&
                      q < (int64_t)(2 * u + 1) * (2 * u + 1));
}

__global__ void check_magnitude_kernel(int64_t s0, int64_t s1, unsigned long long *bad) {
  unsigned long long nb = 0;
  for (int64_t i = s0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s1;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = (int32_t)i;
    const float want = sqrtf((float)s);
    if (__float_as_uint(magnitude_f32(s)) != __float_as_uint(want)) ++nb;
    if (__float_as_uint(magnitude_newton_neg(-s)) != __float_as_uint(want)) ++nb;
    if (!u8_ok(magnitude_u8(s), s)) ++nb;
    // packed pair: s in the low lane, its mirror s1 - 1 - (s - s0) in the high lane
    const int32_t m = (int32_t)(s1 - 1 - (i - s0));
    float ga, gb;
    magnitude_f32x2(s, m, ga, gb);
    if (__float_as_uint(ga) != __float_as_uint(want)) ++nb;
    if (__float_as_uint(gb) != __float_as_uint(sqrtf((float)m))) ++nb;
    uint32_t ua, ub;
    magnitude_u8x2(s, m, ua, ub);
    if (!u8_ok(ua, s) || !u8_ok(ub, m)) ++nb;
  }
  if (nb) atomicAdd(bad, nb);
}

cudaError_t launch_check_magnitude(int64_t s0, int64_t s1, unsigned long long *d_bad, int grid,
                                   cudaStream_t st) {
  (void)cudaGetLastError();  // report this launch only, not an earlier failed call
  check_magnitude_kernel<<<grid, 256, 0, st>>>(s0, s1, d_bad);
  return cudaGetLastError();
}

}  // namespace sobel4
