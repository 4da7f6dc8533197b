// sobel4_ptx.cuh — inline-PTX wrappers used by the RG kernel (sm_80+ async
// copies into shared memory; available on sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sobel4 {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// 4-byte global -> shared copy; bytes beyond `nbytes` (0 or 4) are zero-filled.
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src, uint32_t nbytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(nbytes)
               : "memory");
}

// 16-byte global -> shared copy (both addresses 16-byte aligned); bytes beyond
// `nbytes` (0 or 16) are zero-filled.  Bypasses L1 (.cg).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t nbytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(nbytes)
               : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Wait until at most N of this thread's committed copy groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace sobel4
