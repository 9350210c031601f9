// Asynchronous global -> shared copies (cp.async, sm_80 and later) shared by
// the convolution kernels: every copy a thread issues is in flight at once
// until cp_async_wait_all, instead of one load-store round trip each.
#pragma once

#include <cstdint>

namespace lt {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16 bytes from src to the shared address dst; with valid == false it writes
// zeros and reads nothing (src must still be a mapped address).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace lt
