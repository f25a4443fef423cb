// hq_cp_async.cuh -- global -> shared copies that bypass registers
// (cp.async, sm_80 and later): a thread issues many copies, commits them as a
// group and waits once, instead of stalling on each load.
#pragma once

#include <cuda_runtime.h>

namespace hq {

// 16 bytes; both addresses 16-byte aligned
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    const unsigned d = unsigned(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
// 8 bytes; both addresses 8-byte aligned
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    const unsigned d = unsigned(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's committed groups are still in flight
template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace hq
