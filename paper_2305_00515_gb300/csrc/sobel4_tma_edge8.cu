// TMA-family kernels (tensor and bulk staging, every item mode) instantiated
// for one output format.
#include "sobel4_tma_fmt.cuh"

namespace sobel4 {
template struct TmaFmt<kEdge8>;
}  // namespace sobel4
