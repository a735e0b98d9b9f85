// Kernel launch helper, dynamic shared memory declaration and the process-wide
// launch counter of libngf_b300.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

namespace ngf {

std::atomic<int64_t>& launch_counter();

// Launch `kern` on `stream` and count it.  Returns the launch error (the
// kernel itself runs asynchronously).
template <class Kern, class... Args>
inline cudaError_t launch(Kern kern, dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                          Args... args) {
    kern<<<grid, block, smem, stream>>>(args...);
    launch_counter().fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace ngf

// Dynamic shared memory of the calling kernel, 16-byte aligned.
#define NGF_DYNAMIC_SMEM(name) extern __shared__ __align__(16) unsigned char name[]
