// util.cu - error strings, device queries.
#include <cstdio>

#include "common.cuh"

namespace bdfb {

static thread_local cudaError_t g_last_cuda = cudaSuccess;

void note_cuda_error(cudaError_t e) { g_last_cuda = e; }

int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (cache[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
    cache[dev] = v;
  }
  return cache[dev];
}

}  // namespace bdfb

extern "C" int bdfb_version(void) { return BDFB_VERSION_INT; }

extern "C" const char* bdfb_strerror(int code) {
  static thread_local char buf[256];
  switch (code) {
    case BDFB_SUCCESS: return "success";
    case BDFB_TOO_MUCH_WORK: return "too much work: mxstep steps taken before tout";
    case BDFB_ERR_FAILURE: return "error test failed repeatedly or the step size underflowed";
    case BDFB_CONV_FAILURE: return "Newton iteration failed repeatedly";
    case BDFB_LSETUP_FAIL: return "linear solver setup failed";
    case BDFB_LSOLVE_FAIL: return "linear solve failed";
    case BDFB_RHSFUNC_FAIL: return "right-hand side evaluation failed";
    case BDFB_MEM_FAIL: return "memory allocation failed";
    case BDFB_CUDA_FAIL:
      std::snprintf(buf, sizeof buf, "CUDA runtime error: %s",
                    cudaGetErrorString(bdfb::g_last_cuda));
      return buf;
    case BDFB_ILL_INPUT: return "illegal input";
    default: return "unknown error code";
  }
}
