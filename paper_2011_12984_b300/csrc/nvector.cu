// nvector.cu - fused NVECTOR operations on FP64 device vectors (Sec. 4 of the
// paper: streaming operations run asynchronously; reductions return a scalar).
//
// B300 design: every kernel is HBM-bound, so each thread moves 16-byte
// (double2) words with streaming cache hints, the grid is a multiple of the SM
// count with several loads in flight per thread, and the multi-vector forms
// read their shared operand once per element.  Reductions are deterministic:
// per-block partial sums (warp shuffles, then shared memory) go to a
// caller-owned workspace, and the last block to finish adds the partials in
// a fixed order and resets the arrival counter.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"

namespace bdfb {

constexpr int NV_MAX = 16;
constexpr int ST_THREADS = 256;   // streaming kernels
constexpr int RD_THREADS = 256;   // reductions
constexpr int RD_MAX_BLOCKS = 1024;
constexpr int UNROLL = 4;

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// blocks for `items` work items, each thread taking UNROLL per sweep; at most
// `per_sm` resident blocks on every SM
static int grid_for(int64_t items, int threads, int per_sm) {
  int64_t want = (items + (int64_t)threads * UNROLL - 1) / ((int64_t)threads * UNROLL);
  int64_t cap = (int64_t)sm_count() * per_sm;
  if (want > cap) want = cap;
  return want < 1 ? 1 : (int)want;
}

// Blocks of `kernel` (at `threads` threads) that fit on one SM at once, from
// the occupancy calculator, cached per kernel and device.  A grid-stride
// kernel whose grid exceeds what is resident runs a second, partial wave of
// equally loaded blocks: its grid is capped at the resident count instead.
static int resident_per_sm(const void* kernel, int threads) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(kernel, dev);
  const auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, 0) != cudaSuccess || b < 1) b = 1;
  cache[key] = b;
  return b;
}
template <typename K>
static int grid_of(K kernel, int64_t items, int threads, int per_sm) {
  return grid_for(items, threads, std::min(per_sm, resident_per_sm(reinterpret_cast<const void*>(kernel), threads)));
}

// ------------------------------------------------------------ LinearSum
// z = a x + b y.  On B300 FP64 issues at 1/64 of FP32, so even this op is
// co-limited by the FP64 pipe (two operations per 24 bytes); a coefficient of
// +-1 (the sums and differences the integrators form) needs one: SB folds
// b = +-1 into a fused multiply-add, SA folds a = +-1 (0: general).
template <int SA, int SB>
__device__ __forceinline__ double lsum(double a, double x, double b, double y) {
  if (SB) return fma(a, x, SB > 0 ? y : -y);
  if (SA) return fma(b, y, SA > 0 ? x : -x);
  return fma(a, x, b * y);
}

template <int SA, int SB>
__global__ void k_linear_sum2(int64_t n2, double a, const double2* x, double b, const double2* y,
                              double2* z) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (UNROLL - 1) * stride < n2; i += UNROLL * stride) {
    double2 xv[UNROLL], yv[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) { xv[u] = __ldcs(x + i + u * stride); yv[u] = __ldcs(y + i + u * stride); }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u)
      __stcs(z + i + u * stride, make_double2(lsum<SA, SB>(a, xv[u].x, b, yv[u].x),
                                              lsum<SA, SB>(a, xv[u].y, b, yv[u].y)));
  }
  for (; i < n2; i += stride) {
    double2 xv = __ldcs(x + i), yv = __ldcs(y + i);
    __stcs(z + i, make_double2(lsum<SA, SB>(a, xv.x, b, yv.x), lsum<SA, SB>(a, xv.y, b, yv.y)));
  }
}

__global__ void k_linear_sum1(int64_t n, double a, const double* x, double b, const double* y,
                              double* z) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    z[i] = a * x[i] + b * y[i];
}

// ------------------------------------------------------------ support ops
// z = op(x) elementwise: Scale (a x), Const (a), Abs, Inv (1 / x), AddConst
// (x + a), and the fused error weight 1 / (a |x| + b) (a = rtol, b = atol)
enum { UOP_SCALE = 0, UOP_CONST, UOP_ABS, UOP_INV, UOP_ADDCONST, UOP_EWT };

template <int OP>
__device__ __forceinline__ double uop(double x, double a, double b) {
  if (OP == UOP_SCALE) return a * x;
  if (OP == UOP_CONST) return a;
  if (OP == UOP_ABS) return fabs(x);
  if (OP == UOP_INV) return 1.0 / x;
  if (OP == UOP_ADDCONST) return x + a;
  return recip_nr(a * fabs(x) + b);     // error weights without an FP64 division
}

template <int OP>
__global__ void k_unary2(int64_t n2, const double2* x, double a, double b, double2* z) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (UNROLL - 1) * stride < n2; i += UNROLL * stride) {
    double2 v[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) v[u] = OP == UOP_CONST ? make_double2(0.0, 0.0) : __ldcs(x + i + u * stride);
#pragma unroll
    for (int u = 0; u < UNROLL; ++u)
      __stcs(z + i + u * stride, make_double2(uop<OP>(v[u].x, a, b), uop<OP>(v[u].y, a, b)));
  }
  for (; i < n2; i += stride) {
    const double2 v = OP == UOP_CONST ? make_double2(0.0, 0.0) : __ldcs(x + i);
    __stcs(z + i, make_double2(uop<OP>(v.x, a, b), uop<OP>(v.y, a, b)));
  }
}

template <int OP>
__global__ void k_unary1(int64_t n, const double* x, double a, double b, double* z) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    z[i] = uop<OP>(OP == UOP_CONST ? 0.0 : x[i], a, b);
}

template <int OP>
static int launch_unary(int64_t n, const double* x, double a, double b, double* z, cudaStream_t s) {
  const bool al = aligned16(z) && (OP == UOP_CONST || aligned16(x));
  const int64_t n2 = n >> 1;
  if (al && n2) {
    k_unary2<OP><<<grid_of(k_unary2<OP>, n2, ST_THREADS, 8), ST_THREADS, 0, s>>>(
        n2, reinterpret_cast<const double2*>(x), a, b, reinterpret_cast<double2*>(z));
    if (n & 1) k_unary1<OP><<<1, 32, 0, s>>>(1, OP == UOP_CONST ? x : x + n - 1, a, b, z + n - 1);
  } else {
    k_unary1<OP><<<grid_of(k_unary1<OP>, n, ST_THREADS, 8), ST_THREADS, 0, s>>>(n, x, a, b, z);
  }
  BDFB_CUDA(cudaGetLastError());
  return BDFB_SUCCESS;
}

// ------------------------------------------------------------ LinearCombination
struct LCArgs {
  const double* x[NV_MAX];
  double c[NV_MAX];
};

// sweeps per loop trip: few operands get more independent loads in flight
template <int NV>
struct Sweeps {
  static constexpr int U = NV <= 2 ? 4 : (NV <= 4 ? 2 : 1);
};

template <int NV>
__global__ void k_linear_combination2(int64_t n2, LCArgs A, double2* z) {
  constexpr int U = Sweeps<NV>::U;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (U - 1) * stride < n2; i += U * stride) {
    double2 v[U][NV];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < NV; ++j) v[u][j] = __ldcs(reinterpret_cast<const double2*>(A.x[j]) + i + u * stride);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      double sx = A.c[0] * v[u][0].x, sy = A.c[0] * v[u][0].y;
#pragma unroll
      for (int j = 1; j < NV; ++j) { sx = fma(A.c[j], v[u][j].x, sx); sy = fma(A.c[j], v[u][j].y, sy); }
      __stcs(z + i + u * stride, make_double2(sx, sy));
    }
  }
  for (; i < n2; i += stride) {
    double2 v[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = __ldcs(reinterpret_cast<const double2*>(A.x[j]) + i);
    double sx = A.c[0] * v[0].x, sy = A.c[0] * v[0].y;
#pragma unroll
    for (int j = 1; j < NV; ++j) { sx = fma(A.c[j], v[j].x, sx); sy = fma(A.c[j], v[j].y, sy); }
    __stcs(z + i, make_double2(sx, sy));
  }
}

__global__ void k_linear_combination1(int64_t n, int nv, LCArgs A, double* z) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double s = A.c[0] * A.x[0][i];
    for (int j = 1; j < nv; ++j) s = fma(A.c[j], A.x[j][i], s);
    z[i] = s;
  }
}

// ------------------------------------------------------------ ScaleAddMulti
struct SAMArgs {
  const double* y[NV_MAX];
  double* z[NV_MAX];
  double a[NV_MAX];
};

template <int NV>
__global__ void k_scale_add_multi2(int64_t n2, const double2* x, SAMArgs A) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
    double2 xv = __ldcs(x + i);
    double2 yv[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) yv[j] = __ldcs(reinterpret_cast<const double2*>(A.y[j]) + i);
#pragma unroll
    for (int j = 0; j < NV; ++j)
      __stcs(reinterpret_cast<double2*>(A.z[j]) + i,
             make_double2(fma(A.a[j], xv.x, yv[j].x), fma(A.a[j], xv.y, yv[j].y)));
  }
}

__global__ void k_scale_add_multi1(int64_t n, int nv, const double* x, SAMArgs A) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double xv = x[i];
    for (int j = 0; j < nv; ++j) A.z[j][i] = fma(A.a[j], xv, A.y[j][i]);
  }
}

// ------------------------------------------------------------ reductions
struct RedArgs {
  const double* y[NV_MAX];   // DotProdMulti operands, or y[0] = weights for WRMS
};

// Block-wide sum of NV values per thread; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*sh)[RD_THREADS / 32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double s = warp_sum(v[j]);
    if (lane == 0) sh[j][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double s = lane < RD_THREADS / 32 ? sh[j][lane] : 0.0;
      v[j] = warp_sum(s);
    }
  }
}

// MODE 0: out[j] = x . y_j;  MODE 1: out[0] = sqrt(sum (x w)^2 / n)
// resident blocks per SM a reduction is compiled for (bounds its registers:
// enough warps must be resident to keep the loads of all operands in flight)
template <int NV>
struct RedBlocks {
  static constexpr int value = NV <= 6 ? 4 : 2;
};

template <int NV, int MODE>
__global__ void __launch_bounds__(RD_THREADS, RedBlocks<NV>::value) k_reduce(int64_t n, const double* x, RedArgs A,
                                                       double* work, double* out, int vec) {
  __shared__ double sh[NV][RD_THREADS / 32];
  __shared__ int is_last;
  double acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (vec) {
    const int64_t n2 = n >> 1;
    const double2* x2 = reinterpret_cast<const double2*>(x);
    constexpr int U = Sweeps<NV>::U;
    int64_t i = i0;
    for (; i + (U - 1) * stride < n2; i += U * stride) {
      double2 xv[U], yv[U][NV];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        xv[u] = __ldcs(x2 + i + u * stride);
#pragma unroll
        for (int j = 0; j < NV; ++j) yv[u][j] = __ldcs(reinterpret_cast<const double2*>(A.y[j]) + i + u * stride);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int j = 0; j < NV; ++j) {
          if (MODE == 0) {
            acc[j] = fma(xv[u].x, yv[u][j].x, acc[j]);
            acc[j] = fma(xv[u].y, yv[u][j].y, acc[j]);
          } else {
            double p = xv[u].x * yv[u][j].x, q = xv[u].y * yv[u][j].y;
            acc[j] = fma(p, p, acc[j]);
            acc[j] = fma(q, q, acc[j]);
          }
        }
    }
    for (; i < n2; i += stride) {
      double2 xv = __ldcs(x2 + i);
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        double2 yv = __ldcs(reinterpret_cast<const double2*>(A.y[j]) + i);
        if (MODE == 0) {
          acc[j] = fma(xv.x, yv.x, acc[j]);
          acc[j] = fma(xv.y, yv.y, acc[j]);
        } else {
          double p = xv.x * yv.x, q = xv.y * yv.y;
          acc[j] = fma(p, p, acc[j]);
          acc[j] = fma(q, q, acc[j]);
        }
      }
    }
    if ((n & 1) && i0 == 0) {
      const int64_t t = n - 1;
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        double p = x[t] * A.y[j][t];
        acc[j] = MODE == 0 ? acc[j] + p : fma(p, p, acc[j]);
      }
    }
  } else {
    for (int64_t i = i0; i < n; i += stride) {
      double xv = x[i];
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        double p = xv * A.y[j][i];
        acc[j] = MODE == 0 ? acc[j] + p : fma(p, p, acc[j]);
      }
    }
  }
  block_sum<NV>(acc, sh);
  unsigned* counter = reinterpret_cast<unsigned*>(work + (int64_t)RD_MAX_BLOCKS * NV_MAX);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) work[(int64_t)blockIdx.x * NV + j] = acc[j];
    __threadfence();
    unsigned prev = atomicAdd(counter, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double s[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) s[j] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int j = 0; j < NV; ++j) s[j] += __ldcg(work + (int64_t)b * NV + j);
  }
  __syncthreads();   // sh reused
  block_sum<NV>(s, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) out[j] = MODE == 0 ? s[j] : (n > 0 ? sqrt(s[j] / (double)n) : 0.0);
    *counter = 0u;
  }
}

}  // namespace bdfb

using namespace bdfb;

extern "C" int64_t bdfb_nv_work_doubles(int64_t n, int nv) {
  (void)n;
  (void)nv;
  return (int64_t)RD_MAX_BLOCKS * NV_MAX + 2;
}

extern "C" int bdfb_nv_scale(int64_t n, double c, const double* x, double* z, void* stream) {
  if (n < 0 || (n > 0 && (!x || !z))) return BDFB_ILL_INPUT;
  return n ? launch_unary<UOP_SCALE>(n, x, c, 0.0, z, as_stream(stream)) : BDFB_SUCCESS;
}

extern "C" int bdfb_nv_const(int64_t n, double c, double* z, void* stream) {
  if (n < 0 || (n > 0 && !z)) return BDFB_ILL_INPUT;
  return n ? launch_unary<UOP_CONST>(n, nullptr, c, 0.0, z, as_stream(stream)) : BDFB_SUCCESS;
}

extern "C" int bdfb_nv_abs(int64_t n, const double* x, double* z, void* stream) {
  if (n < 0 || (n > 0 && (!x || !z))) return BDFB_ILL_INPUT;
  return n ? launch_unary<UOP_ABS>(n, x, 0.0, 0.0, z, as_stream(stream)) : BDFB_SUCCESS;
}

extern "C" int bdfb_nv_inv(int64_t n, const double* x, double* z, void* stream) {
  if (n < 0 || (n > 0 && (!x || !z))) return BDFB_ILL_INPUT;
  return n ? launch_unary<UOP_INV>(n, x, 0.0, 0.0, z, as_stream(stream)) : BDFB_SUCCESS;
}

extern "C" int bdfb_nv_add_const(int64_t n, const double* x, double b, double* z, void* stream) {
  if (n < 0 || (n > 0 && (!x || !z))) return BDFB_ILL_INPUT;
  return n ? launch_unary<UOP_ADDCONST>(n, x, b, 0.0, z, as_stream(stream)) : BDFB_SUCCESS;
}

extern "C" int bdfb_nv_error_weights(int64_t n, double rtol, double atol, const double* y, double* w,
                                     void* stream) {
  if (n < 0 || (n > 0 && (!y || !w)) || !(rtol >= 0.0) || !(atol > 0.0)) return BDFB_ILL_INPUT;
  return n ? launch_unary<UOP_EWT>(n, y, rtol, atol, w, as_stream(stream)) : BDFB_SUCCESS;
}

extern "C" int bdfb_nv_linear_sum(int64_t n, double a, const double* x, double b, const double* y,
                                  double* z, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y || !z))) return BDFB_ILL_INPUT;
  if (n == 0) return BDFB_SUCCESS;
  cudaStream_t s = as_stream(stream);
  if (aligned16(x) && aligned16(y) && aligned16(z)) {
    int64_t n2 = n >> 1;
    if (n2) {
      const double2 *x2 = reinterpret_cast<const double2*>(x), *y2 = reinterpret_cast<const double2*>(y);
      double2* z2 = reinterpret_cast<double2*>(z);
#define LS_CALL(SA, SB) \
  k_linear_sum2<SA, SB><<<grid_of(k_linear_sum2<SA, SB>, n2, ST_THREADS, 8), ST_THREADS, 0, s>>>(n2, a, x2, b, y2, z2)
      if (b == 1.0) LS_CALL(0, 1);
      else if (b == -1.0) LS_CALL(0, -1);
      else if (a == 1.0) LS_CALL(1, 0);
      else if (a == -1.0) LS_CALL(-1, 0);
      else LS_CALL(0, 0);
#undef LS_CALL
    }
    if (n & 1) k_linear_sum1<<<1, 32, 0, s>>>(1, a, x + n - 1, b, y + n - 1, z + n - 1);
  } else {
    k_linear_sum1<<<grid_of(k_linear_sum1, n, ST_THREADS, 8), ST_THREADS, 0, s>>>(n, a, x, b, y, z);
  }
  BDFB_CUDA(cudaGetLastError());
  return BDFB_SUCCESS;
}

#define BDFB_NV_SWITCH(NV, CALL) \
  switch (NV) {                  \
    case 1: CALL(1); break;      \
    case 2: CALL(2); break;      \
    case 3: CALL(3); break;      \
    case 4: CALL(4); break;      \
    case 5: CALL(5); break;      \
    case 6: CALL(6); break;      \
    case 7: CALL(7); break;      \
    case 8: CALL(8); break;      \
    case 9: CALL(9); break;      \
    case 10: CALL(10); break;    \
    case 11: CALL(11); break;    \
    case 12: CALL(12); break;    \
    case 13: CALL(13); break;    \
    case 14: CALL(14); break;    \
    case 15: CALL(15); break;    \
    default: CALL(16); break;    \
  }

extern "C" int bdfb_nv_linear_combination(int64_t n, int nv, const double* c,
                                          const double* const* x, double* z, void* stream) {
  if (n < 0 || nv < 1 || nv > NV_MAX || !c || !x || (n > 0 && !z)) return BDFB_ILL_INPUT;
  if (n == 0) return BDFB_SUCCESS;
  LCArgs A;
  std::memset(&A, 0, sizeof A);
  bool al = aligned16(z);
  for (int j = 0; j < nv; ++j) {
    if (!x[j]) return BDFB_ILL_INPUT;
    A.x[j] = x[j];
    A.c[j] = c[j];
    al = al && aligned16(x[j]);
  }
  cudaStream_t s = as_stream(stream);
  int64_t n2 = n >> 1;
  if (al && n2) {
    double2* z2 = reinterpret_cast<double2*>(z);
#define LC_CALL(K) \
  k_linear_combination2<K><<<grid_of(k_linear_combination2<K>, n2, ST_THREADS, 8), ST_THREADS, 0, s>>>(n2, A, z2)
    BDFB_NV_SWITCH(nv, LC_CALL)
#undef LC_CALL
    if (n & 1) {
      LCArgs T = A;
      for (int j = 0; j < nv; ++j) T.x[j] = A.x[j] + (n - 1);
      k_linear_combination1<<<1, 32, 0, s>>>(1, nv, T, z + n - 1);
    }
  } else {
    k_linear_combination1<<<grid_of(k_linear_combination1, n, ST_THREADS, 8), ST_THREADS, 0, s>>>(n, nv, A, z);
  }
  BDFB_CUDA(cudaGetLastError());
  return BDFB_SUCCESS;
}

extern "C" int bdfb_nv_scale_add_multi(int64_t n, int nv, const double* a, const double* x,
                                       const double* const* y, double* const* z, void* stream) {
  if (n < 0 || nv < 1 || nv > NV_MAX || !a || !y || !z || (n > 0 && !x)) return BDFB_ILL_INPUT;
  if (n == 0) return BDFB_SUCCESS;
  SAMArgs A;
  std::memset(&A, 0, sizeof A);
  bool al = aligned16(x);
  for (int j = 0; j < nv; ++j) {
    if (!y[j] || !z[j]) return BDFB_ILL_INPUT;
    A.y[j] = y[j];
    A.z[j] = z[j];
    A.a[j] = a[j];
    al = al && aligned16(y[j]) && aligned16(z[j]);
  }
  cudaStream_t s = as_stream(stream);
  int64_t n2 = n >> 1;
  if (al && n2) {
    const double2* x2 = reinterpret_cast<const double2*>(x);
#define SAM_CALL(K) \
  k_scale_add_multi2<K><<<grid_of(k_scale_add_multi2<K>, n2, ST_THREADS, 8), ST_THREADS, 0, s>>>(n2, x2, A)
    BDFB_NV_SWITCH(nv, SAM_CALL)
#undef SAM_CALL
    if (n & 1) {
      SAMArgs T = A;
      for (int j = 0; j < nv; ++j) { T.y[j] = A.y[j] + (n - 1); T.z[j] = A.z[j] + (n - 1); }
      k_scale_add_multi1<<<1, 32, 0, s>>>(1, nv, x + n - 1, T);
    }
  } else {
    k_scale_add_multi1<<<grid_of(k_scale_add_multi1, n, ST_THREADS, 8), ST_THREADS, 0, s>>>(n, nv, x, A);
  }
  BDFB_CUDA(cudaGetLastError());
  return BDFB_SUCCESS;
}

static int launch_reduce(int mode, int64_t n, int nv, const double* x, const RedArgs& A, bool al,
                         double* work, double* out, cudaStream_t s) {
  int g = grid_for(al ? (n >> 1) : n, RD_THREADS, nv <= 6 ? 4 : 2);
  if (g > RD_MAX_BLOCKS) g = RD_MAX_BLOCKS;
  int vec = al ? 1 : 0;
  if (mode == 1) {
    k_reduce<1, 1><<<g, RD_THREADS, 0, s>>>(n, x, A, work, out, vec);
  } else {
#define RD_CALL(K) k_reduce<K, 0><<<g, RD_THREADS, 0, s>>>(n, x, A, work, out, vec)
    BDFB_NV_SWITCH(nv, RD_CALL)
#undef RD_CALL
  }
  BDFB_CUDA(cudaGetLastError());
  return BDFB_SUCCESS;
}

extern "C" int bdfb_nv_dot_prod_multi(int64_t n, int nv, const double* x, const double* const* y,
                                      double* out, double* work, void* stream) {
  if (n < 0 || nv < 1 || nv > NV_MAX || !y || !out || !work || (n > 0 && !x)) return BDFB_ILL_INPUT;
  RedArgs A;
  std::memset(&A, 0, sizeof A);
  bool al = aligned16(x);
  for (int j = 0; j < nv; ++j) {
    if (!y[j] && n > 0) return BDFB_ILL_INPUT;
    A.y[j] = y[j];
    al = al && aligned16(y[j]);
  }
  return launch_reduce(0, n, nv, x, A, al, work, out, as_stream(stream));
}

extern "C" int bdfb_nv_wrms_norm(int64_t n, const double* x, const double* w, double* out,
                                 double* work, void* stream) {
  if (n < 0 || !out || !work || (n > 0 && (!x || !w))) return BDFB_ILL_INPUT;
  RedArgs A;
  std::memset(&A, 0, sizeof A);
  A.y[0] = w;
  bool al = aligned16(x) && aligned16(w);
  return launch_reduce(1, n, 1, x, A, al, work, out, as_stream(stream));
}

// ---------------------------------------------------------------------------
// Multi-dot product that allocates nothing.
//
// Some callers cannot hand the library a workspace or let it call cudaMalloc:
// applications whose own memory manager or pool owns every device byte, code
// that must not trigger the implicit device synchronisation a device
// allocation can cause, and code that runs where allocating is not allowed.
// For them the reduction scratch (block partial sums and the arrival counter)
// lives in a fixed array in the library's device image instead.  Every GPU
// that loads the library holds it until the process exits.  All calls on a
// device share it, so calls that overlap on that GPU (other streams, other
// host threads) race and must be serialised by the caller.  The kernel is the
// same k_reduce the allocating entry point launches.
// ---------------------------------------------------------------------------
namespace bdfb {

constexpr int64_t NOALLOC_SCRATCH_DOUBLES = (int64_t)RD_MAX_BLOCKS * NV_MAX + 2;   // 128 KiB + 16 B
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};
static std::mutex g_noalloc_mu;

// Device address of the scratch on the current device.  The host-side name
// g_noalloc_scratch is only a stand-in, so the address is looked up once per
// device (with that device current) and cached for the process's life; a
// cudaDeviceReset reloads the module and leaves the cached address stale
// (the entry point's documentation rules that use out).
static int noalloc_scratch(double** out) {
  int dev = 0;
  BDFB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return BDFB_ILL_INPUT;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    BDFB_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return BDFB_SUCCESS;
}

}  // namespace bdfb

extern "C" int64_t bdfb_nv_noalloc_max_nv(void) { return NV_MAX; }

extern "C" int bdfb_nv_dot_prod_multi_noalloc(int64_t n, int nv, const double* x,
                                              const double* const* y, double* out, void* stream) {
  if (n < 0 || !y || !out || (n > 0 && !x)) return BDFB_ILL_INPUT;
  if (nv < 1 || nv > NV_MAX) return BDFB_ILL_INPUT;   // the fixed scratch holds at most NV_MAX results per block
  RedArgs A;
  std::memset(&A, 0, sizeof A);
  bool al = aligned16(x);
  for (int j = 0; j < nv; ++j) {
    if (!y[j] && n > 0) return BDFB_ILL_INPUT;
    A.y[j] = y[j];
    al = al && aligned16(y[j]);
  }
  double* scratch = nullptr;
  int r = noalloc_scratch(&scratch);
  if (r) return r;
  cudaStream_t s = as_stream(stream);
  // the arrival counter must start at zero (the kernel also leaves it zero)
  BDFB_CUDA(cudaMemsetAsync(scratch + (int64_t)RD_MAX_BLOCKS * NV_MAX, 0, 2 * sizeof(double), s));
  return launch_reduce(0, n, nv, x, A, al, scratch, out, s);
}
