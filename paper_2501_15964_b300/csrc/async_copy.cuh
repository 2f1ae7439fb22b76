// Asynchronous global-to-shared copies (cp.async, LSU path) for sm_103a.
//
// Each thread moves 16 bytes per cp.async and groups its copies with
// commit_group / wait_group, so a thread that reads only the shared memory it
// filled itself needs no barrier and no spin-wait: wait_group returns once the
// thread's own older groups have landed. L2 eviction-priority policies mark
// rows read once per launch (evict_first) and rows gathered many times
// (evict_last).
#pragma once

#include <stdint.h>

namespace ccm {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint64_t policy) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(dst),
               "l"(src), "l"(policy)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copy this lane's quads of one row (quads lane, lane + LANES, ...: the layout
// of row_load) from global to shared memory, 16 bytes per cp.async.
template <int LANES, int CH, typename T>
__device__ __forceinline__ void row_copy_async(T* dst, const T* src, int ld, int lane,
                                               uint64_t policy) {
  constexpr int kPieces = (int)(4 * sizeof(T) / 16);  // 16-byte pieces per quad
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int q = c * LANES + lane;
    if (4 * q < ld) {
#pragma unroll
      for (int h = 0; h < kPieces; ++h)
        cp_async16(smem_u32(dst + 4 * q + h * (16 / sizeof(T))),
                   src + 4 * q + h * (16 / sizeof(T)), policy);
    }
  }
}

}  // namespace ccm
