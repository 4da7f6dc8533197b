// sobel4_selftest.cu — on-device self-check of the magnitude step: the
// library's F32 magnitude against CUDA's IEEE sqrtf((float)S), and its U8
// magnitude against the exact rule min(255, round(sqrt(S))), for every S in
// a range (the operator's whole domain is 0 .. 599,270,400).
#include "sobel4_launch.h"

namespace sobel4 {

__global__ void check_magnitude_kernel(int64_t s0, int64_t s1, unsigned long long *bad) {
  unsigned long long nb = 0;
  for (int64_t i = s0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s1;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = (int32_t)i;
    const float want = sqrtf((float)s);
    if (__float_as_uint(magnitude_f32(s)) != __float_as_uint(want)) ++nb;
    // exact rule: u = round(sqrt(S)) <=> (2u-1)^2 <= 4S < (2u+1)^2, saturated at 255
    const uint32_t u = magnitude_u8(s);
    const int64_t q = 4 * (int64_t)s;
    const bool ok = u == 255u ? q >= 509ll * 509ll
                              : ((u == 0u || (int64_t)(2 * u - 1) * (2 * u - 1) <= q) &&
                                 q < (int64_t)(2 * u + 1) * (2 * u + 1));
    if (!ok) ++nb;
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
