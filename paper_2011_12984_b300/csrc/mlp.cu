// mlp.cu - BF16 tensor-core training and inference of the learned Newton
// initial guess (mlp.cuh).  One warp owns a 16-row tile: forward pass with
// the hidden activations kept in registers, backward pass with the three
// weight-gradient products (dY^T H2, dH2^T H1, dH1^T X) and the two input
// gradients (dY W3, dH2 W2) as m16n8k16 MMAs, FP32 accumulation throughout.
// Per-CTA gradients gather in shared memory (FP32) and reach global memory
// with one atomic add per parameter per CTA; Adam updates the FP32 master
// weights and repacks the BF16 operand copies.
#include <cmath>

#include "mlp.cuh"

namespace bdfb {

constexpr int MLP_WARPS = 4;

struct WarpBufs {               // per-warp tile buffers (BF16, row-major)
  __nv_bfloat16 X[16][16];
  __nv_bfloat16 H1[16][64];
  __nv_bfloat16 H2[16][64];
  __nv_bfloat16 dY[16][16];
  __nv_bfloat16 dH2[16][64];
  __nv_bfloat16 dH1[16][64];
};

__device__ __forceinline__ void store_afrag(__nv_bfloat16 (*H)[64], const uint32_t (&a)[4][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    *reinterpret_cast<uint32_t*>(&H[g][16 * m + 2 * c]) = a[m][0];
    *reinterpret_cast<uint32_t*>(&H[g + 8][16 * m + 2 * c]) = a[m][1];
    *reinterpret_cast<uint32_t*>(&H[g][16 * m + 8 + 2 * c]) = a[m][2];
    *reinterpret_cast<uint32_t*>(&H[g + 8][16 * m + 8 + 2 * c]) = a[m][3];
  }
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  __nv_bfloat162 v;
  v.x = lo;
  v.y = hi;
  return *reinterpret_cast<uint32_t*>(&v);
}

// A fragment of S^T for m-tile mt, S row-major [16 rows][ld] (A[m][k] = S[k][m])
template <int LD>
__device__ __forceinline__ void afrag_T(uint32_t (&a)[4], const __nv_bfloat16 (*S)[LD], int mt) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  const int m0 = 16 * mt + g, m1 = m0 + 8;
  a[0] = pack2(S[2 * c][m0], S[2 * c + 1][m0]);
  a[1] = pack2(S[2 * c][m1], S[2 * c + 1][m1]);
  a[2] = pack2(S[2 * c + 8][m0], S[2 * c + 9][m0]);
  a[3] = pack2(S[2 * c + 8][m1], S[2 * c + 9][m1]);
}

// B fragment with B[k][n] = S[k][n] (k = tile row), n-tile t
template <int LD>
__device__ __forceinline__ void bfrag_rows(uint32_t (&b)[2], const __nv_bfloat16 (*S)[LD], int t) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  const int n = 8 * t + g;
  b[0] = pack2(S[2 * c][n], S[2 * c + 1][n]);
  b[1] = pack2(S[2 * c + 8][n], S[2 * c + 9][n]);
}

// add a C fragment (rows = outputs o0 + g / + 8, cols = inputs i0 + 2c / + 1)
// into the shared gradient of a [rows][ld] weight block
__device__ __forceinline__ void acc_grad(float* G, int ld, int nrow, int o0, int i0, int ncol, const float (&d)[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  const int r0 = o0 + g, r1 = r0 + 8, k0 = i0 + 2 * c;
  if (r0 < nrow) {
    if (k0 < ncol) atomicAdd(&G[r0 * ld + k0], d[0]);
    if (k0 + 1 < ncol) atomicAdd(&G[r0 * ld + k0 + 1], d[1]);
  }
  if (r1 < nrow) {
    if (k0 < ncol) atomicAdd(&G[r1 * ld + k0], d[2]);
    if (k0 + 1 < ncol) atomicAdd(&G[r1 * ld + k0 + 1], d[3]);
  }
}

// forward + backward over rows [0, nrows): grad (FP32, oracle layout) and
// loss (mean over rows and outputs of the squared error) are accumulated
__global__ void __launch_bounds__(32 * MLP_WARPS) k_mlp_grad(int64_t nrows, const float* __restrict__ X,
                                                             const float* __restrict__ T, const void* packed,
                                                             float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* G = reinterpret_cast<float*>(smem_raw);                       // MLP_NPARAM floats
  WarpBufs* WB = reinterpret_cast<WarpBufs*>(smem_raw + ((MLP_NPARAM * 4 + 15) / 16) * 16);
  const MlpW W = mlp_view(packed);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  WarpBufs& B = WB[warp];
  for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) G[i] = 0.f;
  __syncthreads();
  const float scale = 1.0f / (float)((double)nrows * MLP_NO);
  float lsum = 0.f;
  const int64_t ntiles = (nrows + 15) / 16;
  for (int64_t tile = (int64_t)blockIdx.x * MLP_WARPS + warp; tile < ntiles; tile += (int64_t)gridDim.x * MLP_WARPS) {
    const int64_t r0 = tile * 16;
    const int nr = (int)(nrows - r0 < 16 ? nrows - r0 : 16);
    const float* Xt = X + r0 * MLP_NI;
    // input tile: registers (A fragment) and shared memory (for dW1)
    uint32_t a1[4];
    afrag_from_f32(a1, Xt, MLP_NI, nr, MLP_NI);
    *reinterpret_cast<uint32_t*>(&B.X[g][2 * c]) = a1[0];
    *reinterpret_cast<uint32_t*>(&B.X[g + 8][2 * c]) = a1[1];
    *reinterpret_cast<uint32_t*>(&B.X[g][8 + 2 * c]) = a1[2];
    *reinterpret_cast<uint32_t*>(&B.X[g + 8][8 + 2 * c]) = a1[3];
    // ---- forward, keeping H1 and H2
    float acc[8][4];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
      uint32_t b[2];
      bfrag(b, W.W1b, 16, t, 0);
      mma_bf16(acc[t], a1, b);
    }
    uint32_t h[4][4];
    act_to_afrag(acc, W.b1, h, true);
    store_afrag(B.H1, h);
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        uint32_t b[2];
        bfrag(b, W.W2b, 64, t, m);
        uint32_t am[4] = {h[m][0], h[m][1], h[m][2], h[m][3]};
        mma_bf16(acc[t], am, b);
      }
    }
    act_to_afrag(acc, W.b2, h, true);
    store_afrag(B.H2, h);
    float out[2][4];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      out[t][0] = out[t][1] = out[t][2] = out[t][3] = 0.f;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        uint32_t b[2];
        bfrag(b, W.W3b, 64, t, m);
        uint32_t am[4] = {h[m][0], h[m][1], h[m][2], h[m][3]};
        mma_bf16(out[t], am, b);
      }
    }
    // ---- dY = 2 (Y - T) / (rows * 10) on valid rows and outputs
    float dy[2][4];
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int row = g + 8 * (e >> 1), col = 8 * t + 2 * c + (e & 1);
        float v = 0.f;
        if (row < nr && col < MLP_NO) {
          const float y = out[t][e] + W.b3[col];
          const float err = y - T[(r0 + row) * MLP_NO + col];
          lsum += err * err * scale;
          v = 2.0f * err * scale;
        }
        dy[t][e] = v;
      }
    uint32_t ady[4] = {pack_bf16(dy[0][0], dy[0][1]), pack_bf16(dy[0][2], dy[0][3]),
                       pack_bf16(dy[1][0], dy[1][1]), pack_bf16(dy[1][2], dy[1][3])};
    *reinterpret_cast<uint32_t*>(&B.dY[g][2 * c]) = ady[0];
    *reinterpret_cast<uint32_t*>(&B.dY[g + 8][2 * c]) = ady[1];
    *reinterpret_cast<uint32_t*>(&B.dY[g][8 + 2 * c]) = ady[2];
    *reinterpret_cast<uint32_t*>(&B.dY[g + 8][8 + 2 * c]) = ady[3];
    __syncwarp();
    // ---- dH2 = (dY W3) * [H2 > 0]
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
      uint32_t b[2];
      bfrag(b, W.W3T, 16, t, 0);
      mma_bf16(acc[t], ady, b);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int row = g + 8 * (e >> 1), col = 8 * t + 2 * c + (e & 1);
        if (!(__bfloat162float(B.H2[row][col]) > 0.f)) acc[t][e] = 0.f;
      }
    }
    // accumulator -> operand layout, no bias and no activation
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int t = 2 * m + hh;
        h[m][2 * hh] = pack_bf16(acc[t][0], acc[t][1]);
        h[m][2 * hh + 1] = pack_bf16(acc[t][2], acc[t][3]);
      }
    store_afrag(B.dH2, h);
    // ---- dH1 = (dH2 W2) * [H1 > 0]
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        uint32_t b[2];
        bfrag(b, W.W2T, 64, t, m);
        uint32_t am[4] = {h[m][0], h[m][1], h[m][2], h[m][3]};
        mma_bf16(acc[t], am, b);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int row = g + 8 * (e >> 1), col = 8 * t + 2 * c + (e & 1);
        if (!(__bfloat162float(B.H1[row][col]) > 0.f)) acc[t][e] = 0.f;
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int t = 2 * m + hh;
        h[m][2 * hh] = pack_bf16(acc[t][0], acc[t][1]);
        h[m][2 * hh + 1] = pack_bf16(acc[t][2], acc[t][3]);
      }
    store_afrag(B.dH1, h);
    __syncwarp();
    // ---- weight gradients: dW3 = dY^T H2, dW2 = dH2^T H1, dW1 = dH1^T X
    {
      uint32_t a[4];
      afrag_T<16>(a, B.dY, 0);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        uint32_t b[2];
        bfrag_rows<64>(b, B.H2, t);
        mma_bf16(d, a, b);
        acc_grad(G + P_W3, MLP_NH, MLP_NO, 0, 8 * t, MLP_NH, d);
      }
    }
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
      uint32_t a[4];
      afrag_T<64>(a, B.dH2, mt);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        uint32_t b[2];
        bfrag_rows<64>(b, B.H1, t);
        mma_bf16(d, a, b);
        acc_grad(G + P_W2, MLP_NH, MLP_NH, 16 * mt, 8 * t, MLP_NH, d);
      }
      afrag_T<64>(a, B.dH1, mt);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        uint32_t b[2];
        bfrag_rows<16>(b, B.X, t);
        mma_bf16(d, a, b);
        acc_grad(G + P_W1, MLP_NI, MLP_NH, 16 * mt, 8 * t, MLP_NI, d);
      }
    }
    // ---- bias gradients: column sums of dY, dH2, dH1 over the tile rows
    for (int col = lane; col < 64; col += 32) {
      float s2 = 0.f, s1 = 0.f;
      for (int r = 0; r < 16; ++r) {
        s2 += __bfloat162float(B.dH2[r][col]);
        s1 += __bfloat162float(B.dH1[r][col]);
      }
      atomicAdd(&G[P_B2 + col], s2);
      atomicAdd(&G[P_B1 + col], s1);
    }
    if (lane < MLP_NO) {
      float s3 = 0.f;
      for (int r = 0; r < 16; ++r) s3 += __bfloat162float(B.dY[r][lane]);
      atomicAdd(&G[P_B3 + lane], s3);
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(FULL_MASK, lsum, o);
  if (lane == 0 && lsum != 0.f) atomicAdd(loss, lsum);
  __syncthreads();
  for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x)
    if (G[i] != 0.f) atomicAdd(&grad[i], G[i]);
}

// Y[r][0..9] for rows r < nrows (BF16 MMAs, FP32 outputs)
__global__ void __launch_bounds__(32 * MLP_WARPS) k_mlp_forward(int64_t nrows, const float* __restrict__ X,
                                                                const void* packed, float* __restrict__ Y) {
  const MlpW W = mlp_view(packed);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  const int64_t ntiles = (nrows + 15) / 16;
  for (int64_t tile = (int64_t)blockIdx.x * MLP_WARPS + warp; tile < ntiles; tile += (int64_t)gridDim.x * MLP_WARPS) {
    const int64_t r0 = tile * 16;
    const int nr = (int)(nrows - r0 < 16 ? nrows - r0 : 16);
    uint32_t a1[4];
    afrag_from_f32(a1, X + r0 * MLP_NI, MLP_NI, nr, MLP_NI);
    float out[2][4];
    mlp_tile_forward(W, a1, out);
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int row = g + 8 * (e >> 1), col = 8 * t + 2 * c + (e & 1);
        if (row < nr && col < MLP_NO) Y[(r0 + row) * MLP_NO + col] = out[t][e];
      }
  }
}

// FP32 master parameters (oracle layout) -> packed BF16 operands + biases
__global__ void k_mlp_pack(const float* __restrict__ p, void* packed) {
  __nv_bfloat16* b = static_cast<__nv_bfloat16*>(packed);
  float* f = reinterpret_cast<float*>(b + K_BF16_END);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K_BF16_END + 144; e += gridDim.x * blockDim.x) {
    if (e < K_W2B) {                              // W1b[64][16]
      const int o = (e - K_W1B) / 16, i = (e - K_W1B) % 16;
      b[e] = __float2bfloat16(i < MLP_NI ? p[P_W1 + o * MLP_NI + i] : 0.f);
    } else if (e < K_W3B) {                       // W2b[64][64]
      const int o = (e - K_W2B) / 64, i = (e - K_W2B) % 64;
      b[e] = __float2bfloat16(p[P_W2 + o * MLP_NH + i]);
    } else if (e < K_W2T) {                       // W3b[16][64]
      const int o = (e - K_W3B) / 64, i = (e - K_W3B) % 64;
      b[e] = __float2bfloat16(o < MLP_NO ? p[P_W3 + o * MLP_NH + i] : 0.f);
    } else if (e < K_W3T) {                       // W2T[64 in][64 out]
      const int i = (e - K_W2T) / 64, o = (e - K_W2T) % 64;
      b[e] = __float2bfloat16(p[P_W2 + o * MLP_NH + i]);
    } else if (e < K_BF16_END) {                  // W3T[64 in][16 out]
      const int i = (e - K_W3T) / 16, o = (e - K_W3T) % 16;
      b[e] = __float2bfloat16(o < MLP_NO ? p[P_W3 + o * MLP_NH + i] : 0.f);
    } else {
      const int k = e - K_BF16_END;               // b1[64], b2[64], b3[16]
      float v = 0.f;
      if (k < 64) v = p[P_B1 + k];
      else if (k < 128) v = p[P_B2 + k - 64];
      else if (k - 128 < MLP_NO) v = p[P_B3 + k - 128];
      f[k] = v;
    }
  }
}

// Adam (Kingma & Ba) on the FP32 master weights; grad is zeroed for the next step
__global__ void k_mlp_adam(float* __restrict__ p, float* __restrict__ grad, float* __restrict__ m,
                           float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MLP_NPARAM; i += gridDim.x * blockDim.x) {
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    grad[i] = 0.f;
  }
}

static int grad_smem() { return ((MLP_NPARAM * 4 + 15) / 16) * 16 + MLP_WARPS * (int)sizeof(WarpBufs); }

}  // namespace bdfb

using namespace bdfb;

extern "C" int64_t bdfb_mlp_nparam(void) { return MLP_NPARAM; }
extern "C" int64_t bdfb_mlp_packed_bytes(void) { return PACKED_BYTES; }

extern "C" int bdfb_mlp_pack(const float* params, void* packed, void* stream) {
  if (!params || !packed) return BDFB_ILL_INPUT;
  k_mlp_pack<<<16, 256, 0, as_stream(stream)>>>(params, packed);
  BDFB_CUDA(cudaGetLastError());
  return BDFB_SUCCESS;
}

extern "C" int bdfb_mlp_forward(int64_t nrows, const float* X, const void* packed, float* Y, void* stream) {
  if (nrows < 0 || (nrows > 0 && (!X || !packed || !Y))) return BDFB_ILL_INPUT;
  if (nrows == 0) return BDFB_SUCCESS;
  const int64_t tiles = (nrows + 15) / 16;
  const int grid = (int)std::min<int64_t>((tiles + MLP_WARPS - 1) / MLP_WARPS, (int64_t)sm_count() * 8);
  k_mlp_forward<<<grid, 32 * MLP_WARPS, 0, as_stream(stream)>>>(nrows, X, packed, Y);
  BDFB_CUDA(cudaGetLastError());
  return BDFB_SUCCESS;
}

extern "C" int bdfb_mlp_loss_grad(int64_t nrows, const float* X, const float* T, const void* packed,
                                  float* grad, float* loss, void* stream) {
  if (nrows < 1 || !X || !T || !packed || !grad || !loss) return BDFB_ILL_INPUT;
  const int smem = grad_smem();
  BDFB_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int64_t tiles = (nrows + 15) / 16;
  const int grid = (int)std::min<int64_t>((tiles + MLP_WARPS - 1) / MLP_WARPS, (int64_t)sm_count() * 2);
  k_mlp_grad<<<grid, 32 * MLP_WARPS, smem, as_stream(stream)>>>(nrows, X, T, packed, grad, loss);
  BDFB_CUDA(cudaGetLastError());
  return BDFB_SUCCESS;
}

extern "C" int bdfb_mlp_adam(float* params, float* grad, float* m, float* v, int64_t t, float lr, void* stream) {
  if (!params || !grad || !m || !v || t < 1 || !(lr > 0.f)) return BDFB_ILL_INPUT;
  const double b1 = 0.9, b2 = 0.999;
  k_mlp_adam<<<8, 256, 0, as_stream(stream)>>>(params, grad, m, v, lr, (float)b1, (float)b2, 1e-8f,
                                              (float)(1.0 - std::pow(b1, (double)t)),
                                              (float)(1.0 - std::pow(b2, (double)t)));
  BDFB_CUDA(cudaGetLastError());
  return BDFB_SUCCESS;
}

extern "C" int bdfb_mlp_train(int64_t nrows, const float* X, const float* T, float* params, float* m, float* v,
                              void* packed, float* grad, float* loss_hist, int batch, int nsteps, int64_t t0,
                              float lr, void* stream) {
  if (nrows < 1 || batch < 1 || nsteps < 0 || t0 < 0 || !X || !T || !params || !m || !v || !packed || !grad ||
      !loss_hist || !(lr > 0.f))
    return BDFB_ILL_INPUT;
  cudaStream_t s = as_stream(stream);
  BDFB_CUDA(cudaMemsetAsync(grad, 0, MLP_NPARAM * sizeof(float), s));
  if (nsteps > 0) BDFB_CUDA(cudaMemsetAsync(loss_hist, 0, nsteps * sizeof(float), s));
  int r = bdfb_mlp_pack(params, packed, stream);
  if (r) return r;
  const int64_t nb = std::max<int64_t>(1, nrows / batch);
  for (int st = 0; st < nsteps; ++st) {
    const int64_t b = (t0 + st) % nb;
    const int64_t rows = std::min<int64_t>(batch, nrows - b * batch);
    r = bdfb_mlp_loss_grad(rows, X + b * batch * MLP_NI, T + b * batch * MLP_NO, packed, grad, loss_hist + st, stream);
    if (r) return r;
    r = bdfb_mlp_adam(params, grad, m, v, t0 + st + 1, lr, stream);
    if (r) return r;
    r = bdfb_mlp_pack(params, packed, stream);
    if (r) return r;
  }
  return BDFB_SUCCESS;
}
