// k_copy.cu -- host -> device state uploads read by the SMs (hq_state_upload).
//
// A pinned host buffer is addressable from the GPU; the kernel reads it over
// the CPU-GPU link in 16-byte loads, eight per thread in flight, and writes
// the device state with streaming stores.  Pageable host memory is copied by
// the driver (cudaMemcpyAsync).
#include "hq_internal.cuh"

namespace hq {

namespace {

constexpr int kCopyThreads = 256;
constexpr int kCopyUnroll = 8;

__global__ void __launch_bounds__(kCopyThreads) k_upload(const uint4 *__restrict__ src, uint4 *__restrict__ dst,
                                                         int64_t n16)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    for (; i + (kCopyUnroll - 1) * stride < n16; i += kCopyUnroll * stride) {
        uint4 v[kCopyUnroll];
#pragma unroll
        for (int u = 0; u < kCopyUnroll; ++u) v[u] = src[i + u * stride];
#pragma unroll
        for (int u = 0; u < kCopyUnroll; ++u) __stcs(dst + i + u * stride, v[u]);
    }
    for (; i < n16; i += stride) __stcs(dst + i, src[i]);
}

}  // namespace

hq_status launch_upload(void *state, const void *host, size_t bytes, cudaStream_t s)
{
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, host);
    if (e != cudaSuccess) {
        cudaGetLastError();  // an unregistered pointer may leave an error behind on older runtimes
        at.type = cudaMemoryTypeUnregistered;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer)
        return cuda_status("upload (pageable)", cudaMemcpyAsync(state, host, bytes, cudaMemcpyHostToDevice, s));
    const int64_t n16 = int64_t(bytes / 16);
    const int grid = sm_count() * 4;
    k_upload<<<grid, kCopyThreads, 0, s>>>(static_cast<const uint4 *>(at.devicePointer), static_cast<uint4 *>(state),
                                           n16);
    return cuda_status("k_upload", cudaGetLastError());
}

}  // namespace hq
