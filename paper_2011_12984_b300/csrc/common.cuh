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

// FP64 <-> FP32 conversions on the integer pipe, from the IEEE-754 binary64
// and binary32 layouts (B300 issues FP64 instructions, conversions that
// involve FP64 among them, at 2 per cycle per SM; the integer pipe at 64).
// to_f32 truncates the significand (round toward zero), flushes magnitudes
// below 2^-126 to a signed zero and maps magnitudes from 2^128 up,
// infinities and NaN to infinity or NaN; to_f64 is exact for every normal
// binary32 and zero.
__device__ __forceinline__ float to_f32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);          // top 23 significand bits
  unsigned bits;
  if (e == 0x7ff) bits = sign | 0x7f800000u | (m != 0u || (lo & 0x1fffffffu) != 0u ? 0x400000u : 0u);
  else if (e - 896 >= 255) bits = sign | 0x7f800000u;
  else if (e - 896 <= 0) bits = sign;
  else bits = sign | ((unsigned)(e - 896) << 23) | m;
  return __uint_as_float(bits);
}

__device__ __forceinline__ double to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u;
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned m = b & 0x7fffffu;
  if (e == 0u) return __hiloint2double((int)sign, 0);                 // zero (subnormals flushed)
  const unsigned e64 = e == 0xffu ? 0x7ffu : e + 896u;
  return __hiloint2double((int)(sign | (e64 << 20) | (m >> 3)), (int)(m << 29));
}

// 1 / s for a positive normal double: FP32 reciprocal as the seed (24 bits),
// then two Newton-Raphson steps x <- x + x (1 - s x), each doubling the
// correct bits (the textbook iteration for reciprocals); the last FMA rounds
// once, so the result lies within about half an ulp of the quotient (an
// exact-arithmetic check of 6000 seeds over [1e-10, 1e10] found at most
// 0.49991 ulp), for four FP64 FMAs instead of a full-precision division.
// Magnitudes outside [2^-99, 2^101) (and zero, negative or non-finite s) take
// the division; the range test reads the exponent bits on the integer pipe.
__device__ __forceinline__ double recip_nr(double s) {
  const long long b = __double_as_longlong(s);
  if ((unsigned long long)(b - (924LL << 52)) >= (200ULL << 52)) return 1.0 / s;
  double x = to_f64(__frcp_rn(to_f32(s)));
  double e = fma(-s, x, 1.0);
  x = fma(x, e, x);
  e = fma(-s, x, 1.0);
  return fma(x, e, x);
}

}  // namespace bdfb
