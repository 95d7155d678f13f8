// Staging of host frames on the device (reg_scan, reg_scan_batch with host frames).
#include <cstdint>

#include "reg_internal.h"

namespace reg {

// 16-byte words of mapped page-locked host memory, read by the SMs over the CPU-GPU link, four in
// flight per thread, grid-stride.  (On GB300 a copy-engine transfer that follows an idle spell of
// the engine ran 4-9x below the link's rate for its first ~100 ms; this kernel ran at the link's
// rate in the same place.)
__global__ void __launch_bounds__(256) stage_copy_kernel(uint4 *__restrict__ dst, const uint4 *__restrict__ src,
                                                         size_t n)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
        dst[i] = a;
        dst[i + stride] = b;
        dst[i + 2 * stride] = c;
        dst[i + 3 * stride] = d;
    }
    for (; i < n; i += stride) dst[i] = src[i];
}

cudaError_t launch_stage_copy(void *dst, const void *src, size_t bytes, int blocks, cudaStream_t s)
{
    if (bytes == 0) return cudaSuccess;
    if (bytes % 16 || (uintptr_t)dst % 16 || (uintptr_t)src % 16 || blocks <= 0) return cudaErrorInvalidValue;
    stage_copy_kernel<<<blocks, 256, 0, s>>>((uint4 *)dst, (const uint4 *)src, bytes / 16);
    return cudaGetLastError();
}

}  // namespace reg
