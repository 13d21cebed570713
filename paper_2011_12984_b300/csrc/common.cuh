// common.cuh - shared helpers of libbdfb (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bdfb.h"

#define BDFB_VERSION_INT 100  // 0.1.0

namespace bdfb {

// Remember the last CUDA error for bdfb_strerror (per thread).
void note_cuda_error(cudaError_t e);

#define BDFB_CUDA(call)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) {                             \
      ::bdfb::note_cuda_error(e_);                       \
      return BDFB_CUDA_FAIL;                             \
    }                                                    \
  } while (0)

// Streaming-multiprocessor count of the current device (cached per device).
int sm_count();

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

constexpr unsigned FULL_MASK = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
  return v;
}

}  // namespace bdfb
