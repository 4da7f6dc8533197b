// RG kernels instantiated for the u8 output format.
#include "sobel4_rg.cuh"

namespace sobel4 {
cudaError_t launch_rg_single_u8(const ImageDesc &im, int border, int R, int nc, int sm_count,
                               unsigned int *pair, cudaStream_t st) {
  return launch_rg_single_fmt<kU8>(im, border, R, nc, sm_count, pair, st);
}
cudaError_t launch_rg_batched_u8(const ImageDesc *d, int n, int64_t total, unsigned int *q,
                                int border, int R, int nc, int grid, int sm_count,
                                cudaStream_t st) {
  return launch_rg_batched_fmt<kU8>(d, n, total, q, border, R, nc, grid, sm_count, st);
}
}  // namespace sobel4
