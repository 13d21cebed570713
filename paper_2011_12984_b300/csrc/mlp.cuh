// mlp.cuh - the learned Newton initial guess: a 12 -> 64 -> 64 -> 10 ReLU
// network evaluated with BF16 tensor-core MMAs (m16n8k16, FP32 accumulate).
// The paper has no learned component; this is the build's extension.
//
// Parameters (FP32 master, 5642 values): W1[64][12], b1[64], W2[64][64],
// b2[64], W3[10][64], b3[10], W[out][in].  The packed device form holds BF16
// copies laid out for the MMA operand fragments: W1b[64][16], W2b[64][64],
// W3b[16][64] (forward, row = output) and W2T[64][64], W3T[64][16] (backward,
// row = input), then FP32 biases b1[64], b2[64], b3[16].
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace bdfb {

constexpr int MLP_NI = 12, MLP_NH = 64, MLP_NO = 10;
constexpr int MLP_NPARAM = MLP_NH * MLP_NI + MLP_NH + MLP_NH * MLP_NH + MLP_NH + MLP_NO * MLP_NH + MLP_NO;
constexpr int P_W1 = 0, P_B1 = P_W1 + MLP_NH * MLP_NI, P_W2 = P_B1 + MLP_NH, P_B2 = P_W2 + MLP_NH * MLP_NH,
              P_W3 = P_B2 + MLP_NH, P_B3 = P_W3 + MLP_NO * MLP_NH;

// packed layout (element offsets in bf16 units for the matrices)
constexpr int K_W1B = 0, K_W2B = K_W1B + 64 * 16, K_W3B = K_W2B + 64 * 64, K_W2T = K_W3B + 16 * 64,
              K_W3T = K_W2T + 64 * 64, K_BF16_END = K_W3T + 64 * 16;
constexpr int PACKED_BYTES = K_BF16_END * 2 + (64 + 64 + 16) * 4;

struct MlpW {
  const __nv_bfloat16* W1b;
  const __nv_bfloat16* W2b;
  const __nv_bfloat16* W3b;
  const __nv_bfloat16* W2T;
  const __nv_bfloat16* W3T;
  const float* b1;
  const float* b2;
  const float* b3;
};

__host__ __device__ inline MlpW mlp_view(const void* packed) {
  const __nv_bfloat16* b = static_cast<const __nv_bfloat16*>(packed);
  const float* f = reinterpret_cast<const float*>(b + K_BF16_END);
  MlpW w;
  w.W1b = b + K_W1B;
  w.W2b = b + K_W2B;
  w.W3b = b + K_W3B;
  w.W2T = b + K_W2T;
  w.W3T = b + K_W3T;
  w.b1 = f;
  w.b2 = f + 64;
  w.b3 = f + 128;
  return w;
}

// D = A (16x16 bf16, row) * B (16x8 bf16, col) + C, FP32 accumulate
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// B fragment of W^T for n-tile t, k-tile m, from a row-major [rows = n][ld] bf16 matrix:
// b0b1 = W[8t + g][16m + 2c .. +1], b2b3 = W[8t + g][16m + 2c + 8 .. +9]
__device__ __forceinline__ void bfrag(uint32_t (&b)[2], const __nv_bfloat16* W, int ld, int t, int m) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  const __nv_bfloat16* r = W + (8 * t + g) * ld + 16 * m + 2 * c;
  b[0] = ld32(r);
  b[1] = ld32(r + 8);
}

// A fragments of the next layer from the FP32 accumulators of the previous
// one (16 rows x 64 columns as 8 n-tiles): bias, ReLU, round to BF16.
__device__ __forceinline__ void act_to_afrag(const float (&acc)[8][4], const float* bias, uint32_t (&a)[4][4],
                                             bool relu) {
  const int c = threadIdx.x & 3;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {          // n-tile 2m + h covers columns 16m + 8h ..
      const int t = 2 * m + h;
      const float b0 = bias[8 * t + 2 * c], b1 = bias[8 * t + 2 * c + 1];
      float v0 = acc[t][0] + b0, v1 = acc[t][1] + b1, v2 = acc[t][2] + b0, v3 = acc[t][3] + b1;
      if (relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); v2 = fmaxf(v2, 0.f); v3 = fmaxf(v3, 0.f); }
      a[m][2 * h] = pack_bf16(v0, v1);       // row g
      a[m][2 * h + 1] = pack_bf16(v2, v3);   // row g + 8
    }
  }
}

// Forward pass of one 16-row tile whose layer-1 A fragment is given; out[t]
// holds the FP32 outputs for n-tiles t = 0, 1 (columns 0..15, 10 used).
// The hidden activations stay in registers (accumulator -> operand layout).
__device__ __forceinline__ void mlp_tile_forward(const MlpW& W, const uint32_t (&a1)[4], float (&out)[2][4]) {
  float acc[8][4];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
    uint32_t b[2];
    bfrag(b, W.W1b, 16, t, 0);
    mma_bf16(acc[t], a1, b);
  }
  uint32_t a[4][4];
  act_to_afrag(acc, W.b1, a, true);
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      uint32_t b[2];
      bfrag(b, W.W2b, 64, t, m);
      uint32_t am[4] = {a[m][0], a[m][1], a[m][2], a[m][3]};
      mma_bf16(acc[t], am, b);
    }
  }
  act_to_afrag(acc, W.b2, a, true);
  const int c = threadIdx.x & 3;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    out[t][0] = out[t][1] = out[t][2] = out[t][3] = 0.f;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      uint32_t b[2];
      bfrag(b, W.W3b, 64, t, m);
      uint32_t am[4] = {a[m][0], a[m][1], a[m][2], a[m][3]};
      mma_bf16(out[t], am, b);
    }
    const float b0 = W.b3[8 * t + 2 * c], b1 = W.b3[8 * t + 2 * c + 1];
    out[t][0] += b0; out[t][1] += b1; out[t][2] += b0; out[t][3] += b1;
  }
}

// A fragment of a 16 x 16 input tile from a row-major FP32 array (ld floats
// per row), rows >= nrows and columns >= ncols read as zero
__device__ __forceinline__ void afrag_from_f32(uint32_t (&a)[4], const float* X, int ld, int nrows, int ncols) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  auto at = [&](int r, int k) -> float { return (r < nrows && k < ncols) ? X[r * ld + k] : 0.f; };
  a[0] = pack_bf16(at(g, 2 * c), at(g, 2 * c + 1));
  a[1] = pack_bf16(at(g + 8, 2 * c), at(g + 8, 2 * c + 1));
  a[2] = pack_bf16(at(g, 2 * c + 8), at(g, 2 * c + 9));
  a[3] = pack_bf16(at(g + 8, 2 * c + 8), at(g + 8, 2 * c + 9));
}

}  // namespace bdfb
