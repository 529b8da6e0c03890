// Learned surrogate of the local upscaled quantities.
//
// It takes the place of the paper's random-interpolation model of
// S^m(xi_m), b^m(xi_m) (Sec. 3.1, Algs. 1-2): the cell problem of Eq. MsFEB2
// depends on the cell's few local parameters xi_m only, so per patch family
// (cells whose local bumps sit at the same relative offsets) a multilayer
// perceptron maps xi_m to K_e / abar_cell and to the load, trained on pairs
// from the plain upscaler; unreliable predictions fall back to the plain
// upscaler (the out-of-range fallback of the paper's Remark in Sec. 3.1).
//
// Network: x (16, zero padded) -> 128 -> 128 -> 128 -> 16, GELU (erf form)
// on the hidden layers; FP32 master weights, BF16 matrix products with FP32
// accumulation.  Weights are stored [out][in] per layer.
//
// Targets (13 of the 16 outputs): K_e / abar - K_ref (10 packed entries)
// and b_l / (f H^2) - 1/4 for l = 0..2; abar = arithmetic mean of a over the
// cell's fine elements.  Prediction: K = abar (K_ref + Pi y), Pi the
// orthogonal projector onto packed zero-row-sum symmetric matrices;
// b_l = f H^2 (1/4 + y_{10+l}), b_3 = f H^2 - b_0 - b_1 - b_2.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstring>
#include <map>
#include <vector>

#include "ckpt.cuh"
#include "common.cuh"
#include "stomsfem.h"
#include "tc_gemm.cuh"

namespace stomsfem {

constexpr int kIn = 16, kHid = 128, kOut = 16, kOutUsed = 13;
constexpr int kParams = kHid * kIn + kHid + 2 * (kHid * kHid + kHid) + kOut * kHid + kOut;  // 37264
constexpr int oW1 = 0, oB1 = oW1 + kHid * kIn, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid,
              oW3 = oB2 + kHid, oB3 = oW3 + kHid * kHid, oW4 = oB3 + kHid, oB4 = oW4 + kOut * kHid;
constexpr int kBatch = 64;

// ---------------------------------------------------------------- math

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C tile (16 x 8 at m0, n0) += A(m, k) B(k, n) over k < K; the accessors
// return floats read from shared memory (any layout, transposes included).
// Thread layout of m16n8k16: g = lane / 4, t = lane % 4; c[0..1] at
// (m0+g, n0+2t+{0,1}), c[2..3] at (m0+g+8, n0+2t+{0,1}).
template <class FA, class FB>
__device__ __forceinline__ void mma_tile(const FA& A, const FB& B, int m0, int n0, int K, float c[4], int lane) {
  const int g = lane >> 2, t = lane & 3;
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[4], b[2];
    a[0] = pack_bf16(A(m0 + g, k0 + 2 * t), A(m0 + g, k0 + 2 * t + 1));
    a[1] = pack_bf16(A(m0 + g + 8, k0 + 2 * t), A(m0 + g + 8, k0 + 2 * t + 1));
    a[2] = pack_bf16(A(m0 + g, k0 + 8 + 2 * t), A(m0 + g, k0 + 8 + 2 * t + 1));
    a[3] = pack_bf16(A(m0 + g + 8, k0 + 8 + 2 * t), A(m0 + g + 8, k0 + 8 + 2 * t + 1));
    b[0] = pack_bf16(B(k0 + 2 * t, n0 + g), B(k0 + 2 * t + 1, n0 + g));
    b[1] = pack_bf16(B(k0 + 8 + 2 * t, n0 + g), B(k0 + 8 + 2 * t + 1, n0 + g));
    mma16816(c, a, b);
  }
}

struct RowMajor {  // element (i, k) = p[i * ld + k]
  const __nv_bfloat16* p;
  int ld;
  __device__ __forceinline__ float operator()(int i, int k) const { return __bfloat162float(p[i * ld + k]); }
};
struct ColMajor {  // element (i, k) = p[k * ld + i]
  const __nv_bfloat16* p;
  int ld;
  __device__ __forceinline__ float operator()(int i, int k) const { return __bfloat162float(p[k * ld + i]); }
};

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// ---------------------------------------------------------------- training

// Shared memory of one family's training CTA.  BF16 products: BF16
// copies of the weights and every activation.  FP32 products: FP32
// activations, the weights read from the FP32 master copy in global memory,
// and GELU(Z) recomputed from Z where it is an operand (the stored H of the
// BF16 mode would not fit next to FP32 Z and dZ).
template <bool F32>
struct TrainSmemT;
template <>
struct TrainSmemT<false> {
  __nv_bfloat16 W1[kHid * kIn], W2[kHid * kHid], W3[kHid * kHid], W4[kOut * kHid];  // [out][in]
  __nv_bfloat16 X[kBatch * kIn];
  __nv_bfloat16 Z1[kBatch * kHid], Z2[kBatch * kHid], Z3[kBatch * kHid];  // pre-activations
  __nv_bfloat16 H1[kBatch * kHid], H2[kBatch * kHid], H3[kBatch * kHid];  // GELU(Z)
  __nv_bfloat16 D1[kBatch * kHid], D2[kBatch * kHid];                     // dZ ping-pong
  __nv_bfloat16 DY[kBatch * kOut];
  float T[kBatch * kOut];
  float gb[2][kHid];  // bias gradients: the layer being applied and the next
  float loss;
  int rows[kBatch];
};
template <>
struct TrainSmemT<true> {
  float X[kBatch * kIn];
  float Z1[kBatch * kHid], Z2[kBatch * kHid], Z3[kBatch * kHid];
  float D1[kBatch * kHid], D2[kBatch * kHid];
  float DY[kBatch * kOut];
  float T[kBatch * kOut];
  float gb[2][kHid];
  float loss;
  int rows[kBatch];
};

struct TrainArgs {
  int nfam;
  const int* fam_row0;   // [nfam + 1] row ranges of each family in X/Y, or NULL: rows [row_lo, row_hi)
  int row_lo, row_hi;
  const float* X;        // [N][kIn]
  const float* Y;        // [N][kOut]
  float* W;              // [nfam][kParams] FP32 master weights
  float* m;              // Adam moments
  float* v;
  float* grad_out;       // [nfam][kParams] (grad-only mode) or NULL
  float* loss_out;       // [nfam][steps]
  int steps, step0;
  float lr, lr_min, beta1, beta2, eps;
  uint64_t seed;
  int grad_only;         // 1: one step on rows [row0, row0 + kBatch), gradients out, no update
};

// Bias-corrected Adam on one parameter.
__device__ __forceinline__ float adam(float& w, float& m, float& v, float g, float lr, float b1, float b2, float eps,
                                      float c1, float c2) {
  m = b1 * m + (1.f - b1) * g;
  v = b2 * v + (1.f - b2) * g * g;
  w -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  return w;
}

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename E>
__device__ __forceinline__ E from_f(float v) {
  if constexpr (std::is_same<E, float>::value)
    return v;
  else
    return __float2bfloat16_rn(v);
}
template <typename E>
struct RowM {  // element (i, k) = p[i * ld + k]
  const E* p;
  int ld;
  __device__ __forceinline__ float operator()(int i, int k) const { return to_f(p[i * ld + k]); }
};
template <typename E>
struct ColM {  // element (i, k) = p[k * ld + i]
  const E* p;
  int ld;
  __device__ __forceinline__ float operator()(int i, int k) const { return to_f(p[k * ld + i]); }
};
struct GeluRowM {  // element (i, k) = GELU(z[i * ld + k])
  const float* z;
  int ld;
  __device__ __forceinline__ float operator()(int i, int k) const { return gelu(z[i * ld + k]); }
};

// The same 16 x 8 tile as mma_tile (same lane layout) with FP32 products
// and FP32 sums in k order.
template <class FA, class FB>
__device__ __forceinline__ void fma_tile(const FA& A, const FB& B, int m0, int n0, int K, float c[4], int lane) {
  const int g = lane >> 2, t = lane & 3;
  const int r0 = m0 + g, r1 = m0 + g + 8, c0 = n0 + 2 * t, c1 = n0 + 2 * t + 1;
  for (int k = 0; k < K; ++k) {
    const float a0 = A(r0, k), a1 = A(r1, k), b0 = B(k, c0), b1 = B(k, c1);
    c[0] = fmaf(a0, b0, c[0]);
    c[1] = fmaf(a0, b1, c[1]);
    c[2] = fmaf(a1, b0, c[2]);
    c[3] = fmaf(a1, b1, c[3]);
  }
}
template <bool F32, class FA, class FB>
__device__ __forceinline__ void tile_op(const FA& A, const FB& B, int m0, int n0, int K, float c[4], int lane) {
  if constexpr (F32)
    fma_tile(A, B, m0, n0, K, c, lane);
  else
    mma_tile(A, B, m0, n0, K, c, lane);
}

// One CTA (8 warps) per family: minibatch of 64 rows, forward, backward and
// Adam (bias corrected, cosine learning-rate decay over the call's steps),
// every step.  F32: FP32 products and activations (the check mode of the
// gradients); otherwise BF16 products with FP32 accumulation.
template <bool F32>
__global__ void __launch_bounds__(256) surrogate_train_kernel(TrainArgs A) {
  using E = typename std::conditional<F32, float, __nv_bfloat16>::type;
  using HAcc = typename std::conditional<F32, GeluRowM, RowM<__nv_bfloat16>>::type;
  extern __shared__ __align__(16) unsigned char tsm_raw[];
  TrainSmemT<F32>& S = *reinterpret_cast<TrainSmemT<F32>*>(tsm_raw);
  const int fam = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  float* Wm = A.W + (size_t)fam * kParams;
  float* Mm = A.m + (size_t)fam * kParams;
  float* Vm = A.v + (size_t)fam * kParams;
  const int r0 = A.fam_row0 ? A.fam_row0[fam] : A.row_lo, r1 = A.fam_row0 ? A.fam_row0[fam + 1] : A.row_hi;
  const int nrows = r1 - r0;
  if (nrows <= 0) return;
  // weight operands: the BF16 copies, or the FP32 master weights
  const E *pW1, *pW2, *pW3, *pW4;
  HAcc H1, H2, H3;
  if constexpr (F32) {
    pW1 = Wm + oW1;
    pW2 = Wm + oW2;
    pW3 = Wm + oW3;
    pW4 = Wm + oW4;
    H1 = GeluRowM{S.Z1, kHid};
    H2 = GeluRowM{S.Z2, kHid};
    H3 = GeluRowM{S.Z3, kHid};
  } else {
    for (int i = tid; i < kHid * kIn; i += 256) S.W1[i] = __float2bfloat16_rn(Wm[oW1 + i]);
    for (int i = tid; i < kHid * kHid; i += 256) {
      S.W2[i] = __float2bfloat16_rn(Wm[oW2 + i]);
      S.W3[i] = __float2bfloat16_rn(Wm[oW3 + i]);
    }
    for (int i = tid; i < kOut * kHid; i += 256) S.W4[i] = __float2bfloat16_rn(Wm[oW4 + i]);
    pW1 = S.W1;
    pW2 = S.W2;
    pW3 = S.W3;
    pW4 = S.W4;
    H1 = RowM<__nv_bfloat16>{S.H1, kHid};
    H2 = RowM<__nv_bfloat16>{S.H2, kHid};
    H3 = RowM<__nv_bfloat16>{S.H3, kHid};
  }
  // refresh of a BF16 weight copy after its update (the FP32 mode reads the
  // master weights directly)
  auto refresh = [&](__nv_bfloat16* dst, int off, int n) {
    if constexpr (!F32) {
      if (!A.grad_only)
        for (int i = tid; i < n; i += 256) dst[i] = __float2bfloat16_rn(Wm[off + i]);
    }
  };
  const int steps = A.grad_only ? 1 : A.steps;
  for (int step = 0; step < steps; ++step) {
    const int gstep = A.step0 + step;
    // ---- minibatch (every 10th row of a family is held out for validation)
    if (tid < kBatch) {
      int r;
      if (A.grad_only) {
        r = tid % nrows;
      } else {
        r = (int)(splitmix64(A.seed ^ ((uint64_t)fam << 40) ^ ((uint64_t)gstep << 16) ^ (uint64_t)tid) %
                  (uint64_t)nrows);
        if (r % 10 == 9 && nrows > 1) r -= 1;
      }
      S.rows[tid] = r0 + r;
    }
    if (tid == 0) S.loss = 0.f;
    __syncthreads();
    for (int i = tid; i < kBatch * kIn; i += 256) S.X[i] = from_f<E>(A.X[(size_t)S.rows[i / kIn] * kIn + i % kIn]);
    for (int i = tid; i < kBatch * kOut; i += 256) S.T[i] = A.Y[(size_t)S.rows[i / kOut] * kOut + i % kOut];
    __syncthreads();
    // ---- forward: hidden layers [64 x 128]; warp w owns columns [16w, 16w+16)
    auto fwd_layer = [&](const auto& Ain, int KIN, const E* WS, int BOFF, E* ZOUT, __nv_bfloat16* HOUT) {
      for (int mt = 0; mt < kBatch / 16; ++mt)
        for (int nt = 0; nt < 2; ++nt) {
          const int m0 = mt * 16, n0 = warp * 16 + nt * 8;
          float c[4] = {0, 0, 0, 0};
          tile_op<F32>(Ain, ColM<E>{WS, KIN}, m0, n0, KIN, c, lane);
          for (int q = 0; q < 4; ++q) {
            const int row = m0 + g + (q >> 1) * 8, col = n0 + 2 * t4 + (q & 1);
            const float z = c[q] + Wm[BOFF + col];
            ZOUT[row * kHid + col] = from_f<E>(z);
            if constexpr (!F32) HOUT[row * kHid + col] = __float2bfloat16_rn(gelu(z));
          }
        }
      __syncthreads();
    };
    __nv_bfloat16 *h1 = nullptr, *h2 = nullptr, *h3 = nullptr;
    if constexpr (!F32) {
      h1 = S.H1;
      h2 = S.H2;
      h3 = S.H3;
    }
    fwd_layer(RowM<E>{S.X, kIn}, kIn, pW1, oB1, S.Z1, h1);
    fwd_layer(H1, kHid, pW2, oB2, S.Z2, h2);
    fwd_layer(H2, kHid, pW3, oB3, S.Z3, h3);
    // ---- output layer [64 x 16]: 8 tiles, one per warp; dY = 2 (Y - T) / (B * 13)
    {
      const int m0 = (warp >> 1) * 16, n0 = (warp & 1) * 8;
      float c[4] = {0, 0, 0, 0};
      tile_op<F32>(H3, ColM<E>{pW4, kHid}, m0, n0, kHid, c, lane);
      float ls = 0.f;
      for (int q = 0; q < 4; ++q) {
        const int row = m0 + g + (q >> 1) * 8, col = n0 + 2 * t4 + (q & 1);
        const float y = c[q] + Wm[oB4 + col];
        const float d = (col < kOutUsed) ? (y - S.T[row * kOut + col]) : 0.f;
        ls += d * d;
        S.DY[row * kOut + col] = from_f<E>(2.f * d / (kBatch * kOutUsed));
      }
      ls = warp_sum(ls);
      if (lane == 0) atomicAdd(&S.loss, ls / (kBatch * kOutUsed));
    }
    if (tid < kHid) S.gb[0][tid] = 0.f;
    __syncthreads();
    if (tid == 0 && A.loss_out) A.loss_out[(size_t)fam * A.steps + step] = S.loss;
    const float lr = A.lr_min + 0.5f * (A.lr - A.lr_min) * (1.f + cosf(3.14159265358979f * gstep / fmaxf(1.f, (float)(A.step0 + A.steps))));
    const float c1 = 1.f - powf(A.beta1, (float)(gstep + 1)), c2 = 1.f - powf(A.beta2, (float)(gstep + 1));
    // gradient sink: update in place, or write out (grad-only mode)
    auto apply = [&](int off, float gr) {
      if (A.grad_only) {
        A.grad_out[(size_t)fam * kParams + off] = gr;
      } else {
        adam(Wm[off], Mm[off], Vm[off], gr, lr, A.beta1, A.beta2, A.eps, c1, c2);
      }
    };
    // dZ_in = (dZ W) * gelu'(Z_in) with the layer's weights before their
    // update, and the column sums of dZ_in (the next bias gradient) into gb
    auto back_in = [&](const auto& DZa, int KD, const auto& Wa, const E* ZIN, E* DZOUT, float* gb) {
      for (int mt = 0; mt < kBatch / 16; ++mt)
        for (int nt = 0; nt < 2; ++nt) {
          const int m0 = mt * 16, n0 = warp * 16 + nt * 8;
          float c[4] = {0, 0, 0, 0};
          tile_op<F32>(DZa, Wa, m0, n0, KD, c, lane);
          float cs0 = 0.f, cs1 = 0.f;
          for (int q = 0; q < 4; ++q) {
            const int row = m0 + g + (q >> 1) * 8, col = n0 + 2 * t4 + (q & 1);
            const float dz = c[q] * gelu_grad(to_f(ZIN[row * kHid + col]));
            DZOUT[row * kHid + col] = from_f<E>(dz);
            if (q & 1) cs1 += dz; else cs0 += dz;
          }
          // column sums over the 16 rows of this tile: reduce over g (lanes with equal t4)
          for (int o = 4; o < 32; o <<= 1) {
            cs0 += __shfl_xor_sync(0xffffffffu, cs0, o);
            cs1 += __shfl_xor_sync(0xffffffffu, cs1, o);
          }
          if (g == 0) {
            atomicAdd(&gb[n0 + 2 * t4], cs0);
            atomicAdd(&gb[n0 + 2 * t4 + 1], cs1);
          }
        }
      __syncthreads();
    };
    // ---- layer 4: dZ3 = (dY W4) * gelu'(Z3) (W4 [out][in]: B(k = o, n = i) = W4[o][i]), then dW4 = dY^T H3, db4
    back_in(RowM<E>{S.DY, kOut}, kOut, RowM<E>{pW4, kHid}, S.Z3, S.D1, S.gb[0]);
    for (int tt = warp; tt < 16; tt += 8) {
      const int n0 = tt * 8;
      float c[4] = {0, 0, 0, 0};
      tile_op<F32>(ColM<E>{S.DY, kOut}, H3, 0, n0, kBatch, c, lane);
      for (int q = 0; q < 4; ++q) {
        const int o = g + (q >> 1) * 8, i = n0 + 2 * t4 + (q & 1);
        apply(oW4 + o * kHid + i, c[q]);
      }
    }
    if (tid < kOut) {
      float sacc = 0.f;
      for (int b = 0; b < kBatch; ++b) sacc += to_f(S.DY[b * kOut + tid]);
      apply(oB4 + tid, sacc);
    }
    __syncthreads();
    if constexpr (!F32) refresh(S.W4, oW4, kOut * kHid);
    // ---- hidden layers 3, 2, 1: dZ_in first (old weights), then dW = dZ^T H_in and db
    auto back_w = [&](const E* DZ, const auto& HIN, int KIN, int WOFF, int BOFF, const float* gb) {
      // dW [128 x KIN]: warp w owns rows [16w, 16w + 16)
      for (int nt = 0; nt < KIN / 8; ++nt) {
        const int m0 = warp * 16, n0 = nt * 8;
        float c[4] = {0, 0, 0, 0};
        tile_op<F32>(ColM<E>{DZ, kHid}, HIN, m0, n0, kBatch, c, lane);
        for (int q = 0; q < 4; ++q) {
          const int o = m0 + g + (q >> 1) * 8, i = n0 + 2 * t4 + (q & 1);
          apply(WOFF + o * KIN + i, c[q]);
        }
      }
      if (tid < kHid) apply(BOFF + tid, gb[tid]);
      __syncthreads();
    };
    // layer 3 (dZ3 in D1, its bias gradient in gb[0])
    if (tid < kHid) S.gb[1][tid] = 0.f;
    __syncthreads();
    back_in(RowM<E>{S.D1, kHid}, kHid, RowM<E>{pW3, kHid}, S.Z2, S.D2, S.gb[1]);
    back_w(S.D1, H2, kHid, oW3, oB3, S.gb[0]);
    if constexpr (!F32) refresh(S.W3, oW3, kHid * kHid);
    // layer 2 (dZ2 in D2, bias gradient in gb[1])
    if (tid < kHid) S.gb[0][tid] = 0.f;
    __syncthreads();
    back_in(RowM<E>{S.D2, kHid}, kHid, RowM<E>{pW2, kHid}, S.Z1, S.D1, S.gb[0]);
    back_w(S.D2, H1, kHid, oW2, oB2, S.gb[1]);
    if constexpr (!F32) refresh(S.W2, oW2, kHid * kHid);
    // layer 1 (dZ1 in D1, bias gradient in gb[0]; its input is X)
    back_w(S.D1, RowM<E>{S.X, kIn}, kIn, oW1, oB1, S.gb[0]);
    if constexpr (!F32) refresh(S.W1, oW1, kHid * kIn);
    __syncthreads();
  }
}

// Training rows: X[row][kIn] = xi of the cell's local variables (zero
// padded), Y[row][kOut] = scaled targets; row = fam_row0[f] + s * ncf + pos.
__global__ void surrogate_prepare_kernel(int S, int nc, int rho, int nf, double f, int K,
                                         const double* __restrict__ xi, const double* __restrict__ a,
                                         const double* __restrict__ Ke, const double* __restrict__ be,
                                         const int* __restrict__ var_ids, const int* __restrict__ cell_fam,
                                         const int* __restrict__ cell_pos, const int* __restrict__ fam_row0,
                                         const int* __restrict__ fam_ncell, float* __restrict__ X,
                                         float* __restrict__ Y) {
  const int ncell = nc * nc;
  const long long units = (long long)S * ncell;
  const double kref[10] = {4.0 / 6, -1.0 / 6, -2.0 / 6, -1.0 / 6, 4.0 / 6, -1.0 / 6, -2.0 / 6, 4.0 / 6, -1.0 / 6, 4.0 / 6};
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < units;
       u += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(u / ncell), cell = (int)(u % ncell);
    const int fm = cell_fam[cell];
    const long long row = fam_row0[fm] + (long long)s * fam_ncell[fm] + cell_pos[cell];
    for (int j = 0; j < kIn; ++j) {
      const int id = var_ids[cell * kIn + j];
      X[row * kIn + j] = id >= 0 ? (float)xi[(size_t)s * K + id] : 0.f;
    }
    const int cx = cell % nc, cy = cell / nc;
    double sa = 0.0;
    for (int ey = 0; ey < rho; ++ey)
      for (int ex = 0; ex < rho; ++ex) sa += a[((size_t)s * nf + cy * rho + ey) * nf + cx * rho + ex];
    const double abar = sa / (rho * rho);
    const double H = (double)rho / nf;
    for (int q = 0; q < 10; ++q) Y[row * kOut + q] = (float)(Ke[u * 10 + q] / abar - kref[q]);
    for (int l = 0; l < 3; ++l) Y[row * kOut + 10 + l] = (float)(be[u * 4 + l] / (f * H * H) - 0.25);
    for (int q = kOutUsed; q < kOut; ++q) Y[row * kOut + q] = 0.f;
  }
}

// Per family and input feature: range of the training inputs.
__global__ void surrogate_box_kernel(const int* __restrict__ fam_row0, const float* __restrict__ X,
                                     float* __restrict__ box) {
  const int fm = blockIdx.x, j = threadIdx.x;
  if (j >= kIn) return;
  float lo = 3.4e38f, hi = -3.4e38f;
  for (int r = fam_row0[fm]; r < fam_row0[fm + 1]; ++r) {
    const float v = X[(size_t)r * kIn + j];
    lo = fminf(lo, v);
    hi = fmaxf(hi, v);
  }
  box[(fm * kIn + j) * 2] = lo;
  box[(fm * kIn + j) * 2 + 1] = hi;
}

// ---------------------------------------------------------------- inference

constexpr int kInPad = 64;    // input features padded to one 128-byte K row
constexpr int kTile = 128;    // rows (units) per CTA
// BF16 weights of one family, K-major rows ready for the tensor core:
// W1 [128][64], W2 [128][128], W3 [128][128], W4 [16][128]
constexpr int kWb1 = 0, kWb2 = kWb1 + kHid * kInPad, kWb3 = kWb2 + kHid * kHid, kWb4 = kWb3 + kHid * kHid,
              kWbSize = kWb4 + kOut * kHid;

__global__ void surrogate_pack_kernel(int nfam, const float* __restrict__ W, __nv_bfloat16* __restrict__ Wb) {
  const long long total = (long long)nfam * kWbSize;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(idx / kWbSize), e = (int)(idx % kWbSize);
    const float* w = W + (size_t)f * kParams;
    float v;
    if (e < kWb2) {
      const int o = e / kInPad, i = e % kInPad;
      v = i < kIn ? w[oW1 + o * kIn + i] : 0.f;
    } else if (e < kWb3) {
      v = w[oW2 + (e - kWb2)];
    } else if (e < kWb4) {
      v = w[oW3 + (e - kWb3)];
    } else {
      v = w[oW4 + (e - kWb4)];
    }
    Wb[idx] = __float2bfloat16_rn(v);
  }
}

// Rows of the inference batch grouped by family (each family padded to
// whole 128-row tiles): X[row][64] BF16, unit_of_row[row]; per unit the
// cell means abar (arithmetic) and ahar (harmonic) of a.
__global__ void surrogate_infer_prepare_kernel(int S, int nc, int rho, int nf, int K, const double* __restrict__ xi,
                                               const double* __restrict__ a, const int* __restrict__ var_ids,
                                               const int* __restrict__ cell_fam, const int* __restrict__ cell_pos,
                                               const int* __restrict__ fam_row0, const int* __restrict__ fam_ncell,
                                               __nv_bfloat16* __restrict__ X, int* __restrict__ unit_of_row,
                                               float* __restrict__ Xf, double* __restrict__ abar,
                                               double* __restrict__ ahar) {
  const int ncell = nc * nc;
  const long long units = (long long)S * ncell;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < units;
       u += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(u / ncell), cell = (int)(u % ncell);
    const int fm = cell_fam[cell];
    const long long row = fam_row0[fm] + (long long)s * fam_ncell[fm] + cell_pos[cell];
    // the unit's 16 inputs: one 128-byte BF16 row (zero padded) and 64
    // bytes of FP32, written as 16-byte vectors
    float v[kIn];
#pragma unroll
    for (int j = 0; j < kIn; ++j) {
      const int id = var_ids[cell * kIn + j];
      v[j] = id >= 0 ? (float)xi[(size_t)s * K + id] : 0.f;
    }
    uint4* xr = reinterpret_cast<uint4*>(X + row * kInPad);
    xr[0] = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    xr[1] = make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]), pack_bf16(v[12], v[13]),
                       pack_bf16(v[14], v[15]));
#pragma unroll
    for (int c = 2; c < kInPad / 8; ++c) xr[c] = make_uint4(0u, 0u, 0u, 0u);
    float4* xf = reinterpret_cast<float4*>(Xf + u * kIn);
#pragma unroll
    for (int c = 0; c < kIn / 4; ++c) xf[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
    unit_of_row[row] = (int)u;
    const int cx = cell % nc, cy = cell / nc;
    // arithmetic mean in FP64 (it scales K_e); the harmonic mean only bounds
    // the indicator's energy test, so its reciprocals are FP32 (summed in FP64)
    double sa = 0.0, si = 0.0;
    for (int ey = 0; ey < rho; ++ey)
      for (int ex = 0; ex < rho; ++ex) {
        const double av = a[((size_t)s * nf + cy * rho + ey) * nf + cx * rho + ex];
        sa += av;
        si += (double)__frcp_rn((float)av);
      }
    abar[u] = sa / (rho * rho);
    ahar[u] = (rho * rho) / si;
  }
}

// Orthogonal projector, in the packed coordinates of a symmetric 4x4
// matrix, onto the matrices with zero row sums (row-major [10][10]); set
// by the host before each inference launch.
__constant__ float kZeroRowSumProj[100];

// P = B (B^T B)^{-1} B^T with B [10][6]: a zero-row-sum symmetric matrix is
// fixed by its 6 off-diagonal entries o, its diagonal being -(row sums).
static void zero_row_sum_projector(float* P) {
  const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {1, 2, 3, 2, 3, 3};
  auto packed = [](int l, int lp) { return l * 4 - (l * (l - 1)) / 2 + (lp - l); };
  double B[10][6] = {};
  for (int j = 0; j < 6; ++j) {
    B[packed(pa[j], pb[j])][j] = 1.0;
    B[packed(pa[j], pa[j])][j] = -1.0;
    B[packed(pb[j], pb[j])][j] = -1.0;
  }
  double G[6][16] = {};  // [B^T B | B^T]
  for (int i = 0; i < 6; ++i) {
    for (int j = 0; j < 6; ++j)
      for (int q = 0; q < 10; ++q) G[i][j] += B[q][i] * B[q][j];
    for (int q = 0; q < 10; ++q) G[i][6 + q] = B[q][i];
  }
  for (int c = 0; c < 6; ++c) {  // Gauss-Jordan, B^T B is SPD
    const double inv = 1.0 / G[c][c];
    for (int k = 0; k < 16; ++k) G[c][k] *= inv;
    for (int r = 0; r < 6; ++r)
      if (r != c) {
        const double f = G[r][c];
        for (int k = 0; k < 16; ++k) G[r][k] -= f * G[c][k];
      }
  }
  for (int q = 0; q < 10; ++q)
    for (int r = 0; r < 10; ++r) {
      double t = 0.0;
      for (int j = 0; j < 6; ++j) t += B[q][j] * G[j][6 + r];
      P[q * 10 + r] = (float)t;
    }
}

// Zero inputs for the padding rows of every family's last tile (the
// prepare kernel writes every unit's row; a padding row only feeds its own,
// discarded output row).
__global__ void surrogate_zero_pad_kernel(const int* __restrict__ fam_row0, const int* __restrict__ fam_ncell, int S,
                                          __nv_bfloat16* __restrict__ X) {
  const int f = blockIdx.x;
  const long long r0 = fam_row0[f] + (long long)S * fam_ncell[f], r1 = fam_row0[f + 1];
  uint4* x = reinterpret_cast<uint4*>(X);
  for (long long i = r0 * (kInPad / 8) + threadIdx.x; i < r1 * (kInPad / 8); i += blockDim.x)
    x[i] = make_uint4(0u, 0u, 0u, 0u);
}

// Row and tile starts of every family for S samples (each family padded to
// whole tiles of kTile rows), computed on the device so that a call copies
// nothing from the host.
__global__ void surrogate_tiles_kernel(int nfam, const int* __restrict__ fam_ncell, int S, int* __restrict__ row0,
                                       int* __restrict__ tile0) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int t = 0;
  for (int f = 0; f < nfam; ++f) {
    row0[f] = t * kTile;
    tile0[f] = t;
    t += (int)(((long long)S * fam_ncell[f] + kTile - 1) / kTile);
  }
  row0[nfam] = t * kTile;
  tile0[nfam] = t;
}

struct InferArgs {
  const __nv_bfloat16* X;
  const int* unit_of_row;
  const int* tile0;       // [nfam + 1] first tile of every family (rows of 128 units)
  int nfam;
  const __nv_bfloat16* Wb;
  const float* W;         // FP32 master (biases)
  const float* box;       // [nfam][16][2]
  const float* Xf;        // [units][16] inputs (FP32) for the range check
  const double* abar;
  const double* ahar;
  double f, H, delta, margin;
  double* Ke;
  double* be;
  uint8_t* flag;
  int32_t* err;
};

// Threads of the inference CTA: kInferSplit warps per TMEM lane quadrant,
// each taking kHid / kInferSplit of the hidden columns in the epilogues.
constexpr int kInferSplit = 4;
constexpr int kInferThreads = 128 * kInferSplit;

__device__ __forceinline__ void stage_rows(unsigned char* dst, const __nv_bfloat16* src, int rows, int kblocks,
                                           int ld, int tid) {
  // src rows of ld BF16 (ld = 64 * kblocks) -> kblocks swizzled [rows][64]
  // blocks, by 16-byte asynchronous copies (the caller waits for them)
  const int chunks = rows * kblocks * 8;
  for (int c = tid; c < chunks; c += kInferThreads) {
    const int row = c / (kblocks * 8), rem = c % (kblocks * 8), kb = rem / 8, ch = rem % 8;
    tc::cp_async16(dst + (size_t)kb * rows * 128 + tc::sw128_offset(row, ch * 8),
                   reinterpret_cast<const uint4*>(src + (size_t)row * ld + kb * 64) + ch);
  }
}

__global__ void __launch_bounds__(kInferThreads, 1) surrogate_infer_kernel(InferArgs A) {
  extern __shared__ __align__(1024) unsigned char ism_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(ism_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sX = sm;                          // [128][64]            16 KB
  unsigned char* sH = sX + kTile * 128;            // 2 x [128][64]        32 KB
  unsigned char* sW1 = sH + 2 * kTile * 128;       // [128][64]            16 KB
  unsigned char* sW2 = sW1 + kHid * 128;           // 2 x [128][64]        32 KB
  unsigned char* sW3 = sW2 + 2 * kHid * 128;       // 2 x [128][64]        32 KB
  unsigned char* sW4 = sW3 + 2 * kHid * 128;       // 2 x [16][64]          4 KB
  __shared__ uint64_t mbar;
  __shared__ uint32_t taddr_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x;
  int lo = 0, hi = A.nfam;  // tile0[lo] <= tile < tile0[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (A.tile0[mid] <= tile) lo = mid;
    else hi = mid;
  }
  const int fam = lo;
  const float* Wm = A.W + (size_t)fam * kParams;
  if (warp == 0) tc::tmem_alloc(&taddr_s, 128);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  const __nv_bfloat16* Wb = A.Wb + (size_t)fam * kWbSize;
  stage_rows(sX, A.X + (size_t)tile * kTile * kInPad, kTile, 1, kInPad, tid);
  stage_rows(sW1, Wb + kWb1, kHid, 1, kInPad, tid);
  stage_rows(sW2, Wb + kWb2, kHid, 2, kHid, tid);
  stage_rows(sW3, Wb + kWb3, kHid, 2, kHid, tid);
  stage_rows(sW4, Wb + kWb4, kOut, 2, kHid, tid);
  tc::cp_async_wait_all();
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = taddr_s;
  const uint32_t aX = tc::smem_u32(sX), aH = tc::smem_u32(sH);
  const uint32_t aW[4] = {tc::smem_u32(sW1), tc::smem_u32(sW2), tc::smem_u32(sW3), tc::smem_u32(sW4)};
  const int quad = warp & 3, half = warp >> 2;  // TMEM lane quadrant, share of the hidden columns
  const int row = quad * 32 + lane;
  const uint32_t tlane = (uint32_t)(quad * 32) << 16;
  bool ok = true;
  uint32_t phase = 0;
  for (int layer = 0; layer < 4 && ok; ++layer) {
    const int N = layer == 3 ? kOut : kHid;
    const int ksteps = layer == 0 ? kInPad / 16 : kHid / 16;
    if (tid == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(kTile, N);
      for (int kk = 0; kk < ksteps; ++kk) {
        const int kb = kk >> 2, ki = kk & 3;
        const uint32_t a_addr = (layer == 0 ? aX : aH) + kb * (kTile * 128) + ki * 32;
        const uint32_t b_addr = aW[layer] + kb * (N * 128) + ki * 32;
        tc::mma_bf16(taddr, tc::sdesc_sw128(a_addr), tc::sdesc_sw128(b_addr), idesc, kk > 0 ? 1u : 0u);
      }
      tc::mma_commit(&mbar);
    }
    __syncwarp();
    ok = tc::mbar_wait_bounded(&mbar, phase, 1u << 24);
    phase ^= 1u;
    tc::fence_after_sync();
    if (!ok) break;
    if (layer < 3) {
      const int boff = layer == 0 ? oB1 : (layer == 1 ? oB2 : oB3);
      for (int col = half * (kHid / kInferSplit); col < (half + 1) * (kHid / kInferSplit); col += 16) {
        float v[16];
        tc::tmem_ld16(taddr + tlane + col, v);
        uint32_t pk[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          pk[q] = pack_bf16(gelu(v[2 * q] + Wm[boff + col + 2 * q]), gelu(v[2 * q + 1] + Wm[boff + col + 2 * q + 1]));
        unsigned char* blk = sH + (col >> 6) * (kTile * 128);
        const int k0 = col & 63;
        *reinterpret_cast<uint4*>(blk + tc::sw128_offset(row, k0)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        *reinterpret_cast<uint4*>(blk + tc::sw128_offset(row, k0 + 8)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      }
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
    }
  }
  if (!ok) {
    if (lane == 0) atomicOr(A.err, 2);
  } else if (half == 0) {
    float y[16];
    tc::tmem_ld16(taddr + tlane, y);
    const int u = A.unit_of_row[tile * kTile + row];
    if (u >= 0) {
      float yf[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) yf[q] = y[q] + Wm[oB4 + q];
      // projection onto symmetric zero-row-sum 4x4 matrices (packed): the
      // orthogonal projector of the packed coordinates, a constant 10x10
      // matrix built on the host (FP32 suffices next to the BF16 network)
      const double kref[10] = {4.0 / 6, -1.0 / 6, -2.0 / 6, -1.0 / 6, 4.0 / 6, -1.0 / 6, -2.0 / 6, 4.0 / 6, -1.0 / 6, 4.0 / 6};
      float Kp[10];
#pragma unroll
      for (int q = 0; q < 10; ++q) {
        float t = 0.f;
#pragma unroll
        for (int r = 0; r < 10; ++r) t = fmaf(kZeroRowSumProj[q * 10 + r], yf[r], t);
        Kp[q] = t;
      }
      const double ab = A.abar[u], ah = A.ahar[u];
      double K[10];
      for (int q = 0; q < 10; ++q) K[q] = ab * (kref[q] + (double)Kp[q]);
      const double fH2 = A.f * A.H * A.H;
      double b[4];
      for (int l = 0; l < 3; ++l) b[l] = fH2 * (0.25 + (double)yf[10 + l]);
      b[3] = fH2 - b[0] - b[1] - b[2];
      // error indicator
      bool bad = false;
      const float* box = A.box + (size_t)fam * kIn * 2;
      for (int j = 0; j < kIn; ++j) {
        const float x = A.Xf[(size_t)u * kIn + j];
        const float lo = box[2 * j], hi = box[2 * j + 1], m = (float)A.margin * (hi - lo);
        if (x < lo - m || x > hi + m) bad = true;
      }
      // v = x-linear (0,1,1,0) and y-linear (0,0,1,1): harmonic <= v^T K v <= arithmetic mean
      const double ex = K[4] + 2 * K[5] + K[7];
      const double ey = K[7] + 2 * K[8] + K[9];
      if (!(ex >= ah * (1 - A.delta) && ex <= ab * (1 + A.delta))) bad = true;
      if (!(ey >= ah * (1 - A.delta) && ey <= ab * (1 + A.delta))) bad = true;
      // positive definite on the complement of the constants: leading minors of rows/cols 0..2
      const double m1 = K[0], m2 = K[0] * K[4] - K[1] * K[1];
      const double m3 = K[0] * (K[4] * K[7] - K[5] * K[5]) - K[1] * (K[1] * K[7] - K[5] * K[2]) +
                        K[2] * (K[1] * K[5] - K[4] * K[2]);
      if (!(m1 > 0 && m2 > 0 && m3 > 0)) bad = true;
      for (int q = 0; q < 10; ++q) A.Ke[(size_t)u * 10 + q] = K[q];
      for (int l = 0; l < 4; ++l) A.be[(size_t)u * 4 + l] = b[l];
      A.flag[u] = bad ? 1 : 0;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, 128);
}

// Units whose indicator fired (or every unit after a device-side failure).
// Ensemble indicator: a unit the rules accepted falls back (flag 2) when the
// two networks' K_e differ by more than tol relative (Euclidean norm over the
// 10 packed entries, FP64 from the stored outputs).
__global__ void surrogate_ensemble_kernel(long long units, const double* __restrict__ K1, const double* __restrict__ K2,
                                          double tol, uint8_t* __restrict__ flag) {
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < units;
       u += (long long)gridDim.x * blockDim.x) {
    if (flag[u]) continue;
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int q = 0; q < 10; ++q) {
      const double x = K1[u * 10 + q], y = K2[u * 10 + q];
      num += (x - y) * (x - y);
      den += x * x;
    }
    if (!(num <= tol * tol * den)) flag[u] = 2;
  }
}

__global__ void surrogate_compact_kernel(long long units, uint8_t* __restrict__ flag, const int32_t* __restrict__ err,
                                         int32_t* __restrict__ list, int32_t* __restrict__ count) {
  const bool all = err[0] != 0;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < units;
       u += (long long)gridDim.x * blockDim.x) {
    if (all) flag[u] = 1;
    if (flag[u]) list[atomicAdd(count, 1)] = (int32_t)u;
  }
}

}  // namespace stomsfem

using namespace stomsfem;

struct stomsfem_surrogate {
  stomsfem_grid grid;
  stomsfem_field field;
  double tau;
  int ncell = 0, nfam = 0, K = 0;
  std::vector<int> k_cell, fam_cell, pos_cell, var_ids, fam_ncell;
  int *var_ids_d = nullptr, *cell_fam_d = nullptr, *cell_pos_d = nullptr, *fam_ncell_d = nullptr;
  float *W = nullptr, *m = nullptr, *v = nullptr, *box = nullptr;
  int step = 0;
  // ensemble indicator: a second network on the same families (not owned)
  // and the relative K_e disagreement above which a unit falls back
  const stomsfem_surrogate* partner = nullptr;
  double ens_tol = 0.0;
};

static void sg_free(stomsfem_surrogate* h) {
  if (!h) return;
  cudaFree(h->var_ids_d);
  cudaFree(h->cell_fam_d);
  cudaFree(h->cell_pos_d);
  cudaFree(h->fam_ncell_d);
  cudaFree(h->W);
  cudaFree(h->m);
  cudaFree(h->v);
  cudaFree(h->box);
  delete h;
}

// Local variables of every cell (no oversampling): bump i is local to the
// cell when exp(-d^2 / w^2) >= tau, d the distance from its centre to the
// closed cell rectangle; sorted by the centre's offset from the cell's
// south-west corner (y, then x).  Cells whose local bumps have the same
// offsets form one family.
static int local_vars(const stomsfem_grid* g, const stomsfem_field* fd, double tau,
                      std::vector<int>& k_cell, std::vector<int>& fam_cell, std::vector<int>& pos_cell,
                      std::vector<int>& var_ids, std::vector<int>& fam_ncell, int& nfam) {
  const int nc = g->nc, ncell = nc * nc;
  const double H = 1.0 / nc;
  k_cell.assign(ncell, 0);
  fam_cell.assign(ncell, -1);
  pos_cell.assign(ncell, 0);
  var_ids.assign((size_t)ncell * kIn, -1);
  fam_ncell.clear();
  std::map<std::vector<long long>, int> fam_of;
  for (int cell = 0; cell < ncell; ++cell) {
    const int cx = cell % nc, cy = cell / nc;
    const double x0 = cx * H, x1 = (cx + 1) * H, y0 = cy * H, y1 = (cy + 1) * H;
    std::vector<std::pair<std::pair<long long, long long>, int>> loc;
    for (int by = 0; by < fd->nby; ++by)
      for (int bx = 0; bx < fd->nbx; ++bx) {
        const double px = (bx + 0.5) / fd->nbx, py = (by + 0.5) / fd->nby;
        const double dx = std::max(std::max(x0 - px, 0.0), px - x1);
        const double dy = std::max(std::max(y0 - py, 0.0), py - y1);
        if (std::exp(-(dx * dx + dy * dy) / (fd->width * fd->width)) >= tau) {
          const long long oy = std::llround((py - y0) * g->nf * 1e6), ox = std::llround((px - x0) * g->nf * 1e6);
          loc.push_back({{oy, ox}, by * fd->nbx + bx});
        }
      }
    std::sort(loc.begin(), loc.end());
    if ((int)loc.size() > kIn)
      return set_error(STOMSFEM_EINVAL, "cell %d has %zu local variables > %d (raise tau)", cell, loc.size(), kIn);
    std::vector<long long> key;
    for (size_t j = 0; j < loc.size(); ++j) {
      key.push_back(loc[j].first.first);
      key.push_back(loc[j].first.second);
      var_ids[(size_t)cell * kIn + j] = loc[j].second;
    }
    k_cell[cell] = (int)loc.size();
    auto it = fam_of.find(key);
    int fm;
    if (it == fam_of.end()) {
      fm = (int)fam_ncell.size();
      fam_of[key] = fm;
      fam_ncell.push_back(0);
    } else {
      fm = it->second;
    }
    fam_cell[cell] = fm;
    pos_cell[cell] = fam_ncell[fm]++;
  }
  nfam = (int)fam_ncell.size();
  return STOMSFEM_OK;
}

extern "C" int stomsfem_local_vars(const stomsfem_grid* grid, const stomsfem_field* field, double tau,
                                   int32_t* k_per_cell, int32_t* var_ids, int32_t* family,
                                   int32_t* n_families) {
  if (!grid || !field || grid->nc <= 0 || !(tau > 0.0) || !(tau < 1.0))
    return set_error(STOMSFEM_EINVAL, "bad grid/field/tau");
  std::vector<int> k, fm, pos, ids, fn;
  int nfam = 0;
  const int rc = local_vars(grid, field, tau, k, fm, pos, ids, fn, nfam);
  if (rc) return rc;
  const int ncell = grid->nc * grid->nc;
  for (int c = 0; c < ncell; ++c) {
    if (k_per_cell) k_per_cell[c] = k[c];
    if (family) family[c] = fm[c];
    if (var_ids)
      for (int j = 0; j < kIn; ++j) var_ids[c * kIn + j] = ids[(size_t)c * kIn + j];
  }
  if (n_families) *n_families = nfam;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_surrogate_create(const stomsfem_grid* grid, const stomsfem_field* field,
                                         double tau, const float* init_weights, stomsfem_surrogate** out,
                                         int32_t* n_families) {
  if (!grid || !field || !out || grid->nf <= 0 || grid->nc <= 0 || grid->nf % grid->nc)
    return set_error(STOMSFEM_EINVAL, "bad grid/field/out");
  if (!init_weights) return set_error(STOMSFEM_EINVAL, "init_weights (host) required");
  *out = nullptr;
  auto* h = new stomsfem_surrogate();
  h->grid = *grid;
  h->field = *field;
  h->tau = tau;
  h->ncell = grid->nc * grid->nc;
  h->K = field->nbx * field->nby;
  int rc = local_vars(grid, field, tau, h->k_cell, h->fam_cell, h->pos_cell, h->var_ids, h->fam_ncell, h->nfam);
  if (rc) {
    sg_free(h);
    return rc;
  }
#define TRY(x)                                          \
  if ((rc = check_cuda((x), #x)) != STOMSFEM_OK) {      \
    sg_free(h);                                         \
    return rc;                                          \
  }
  const size_t np = (size_t)h->nfam * kParams;
  TRY(cudaMalloc(&h->var_ids_d, sizeof(int) * h->ncell * kIn));
  TRY(cudaMalloc(&h->cell_fam_d, sizeof(int) * h->ncell));
  TRY(cudaMalloc(&h->cell_pos_d, sizeof(int) * h->ncell));
  TRY(cudaMalloc(&h->fam_ncell_d, sizeof(int) * h->nfam));
  TRY(cudaMalloc(&h->W, sizeof(float) * np));
  TRY(cudaMalloc(&h->m, sizeof(float) * np));
  TRY(cudaMalloc(&h->v, sizeof(float) * np));
  TRY(cudaMalloc(&h->box, sizeof(float) * h->nfam * kIn * 2));
  TRY(cudaMemcpy(h->var_ids_d, h->var_ids.data(), sizeof(int) * h->ncell * kIn, cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(h->cell_fam_d, h->fam_cell.data(), sizeof(int) * h->ncell, cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(h->cell_pos_d, h->pos_cell.data(), sizeof(int) * h->ncell, cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(h->fam_ncell_d, h->fam_ncell.data(), sizeof(int) * h->nfam, cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(h->W, init_weights, sizeof(float) * np, cudaMemcpyHostToDevice));
  TRY(cudaMemset(h->m, 0, sizeof(float) * np));
  TRY(cudaMemset(h->v, 0, sizeof(float) * np));
  TRY(cudaMemset(h->box, 0, sizeof(float) * h->nfam * kIn * 2));
#undef TRY
  if (n_families) *n_families = h->nfam;
  *out = h;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_surrogate_destroy(stomsfem_surrogate* h) {
  sg_free(h);
  return STOMSFEM_OK;
}

extern "C" int stomsfem_surrogate_weights(const stomsfem_surrogate* h, float* w_host) {
  if (!h || !w_host) return set_error(STOMSFEM_EINVAL, "NULL argument");
  STOMSFEM_TRY_CUDA(cudaMemcpy(w_host, h->W, sizeof(float) * h->nfam * kParams, cudaMemcpyDeviceToHost));
  return STOMSFEM_OK;
}

static const char kSgMagic[8] = {'S', 'T', 'M', 'F', 'S', 'U', 'R', '1'};

extern "C" int stomsfem_surrogate_save(const stomsfem_surrogate* h, void* host_buf, size_t buf_bytes,
                                       size_t* bytes) {
  if (!h || !bytes) return set_error(STOMSFEM_EINVAL, "NULL surrogate / bytes");
  const size_t np = (size_t)h->nfam * kParams, nb = (size_t)h->nfam * kIn * 2;
  std::vector<float> W, m, v, box;
  if (host_buf) {
    W.resize(np);
    m.resize(np);
    v.resize(np);
    box.resize(nb);
    STOMSFEM_TRY_CUDA(cudaMemcpy(W.data(), h->W, sizeof(float) * np, cudaMemcpyDeviceToHost));
    STOMSFEM_TRY_CUDA(cudaMemcpy(m.data(), h->m, sizeof(float) * np, cudaMemcpyDeviceToHost));
    STOMSFEM_TRY_CUDA(cudaMemcpy(v.data(), h->v, sizeof(float) * np, cudaMemcpyDeviceToHost));
    STOMSFEM_TRY_CUDA(cudaMemcpy(box.data(), h->box, sizeof(float) * nb, cudaMemcpyDeviceToHost));
  }
  CkptWriter w(host_buf, buf_bytes);
  ckpt_header(w, kSgMagic);
  w.val<int32_t>(h->grid.nf);
  w.val<int32_t>(h->grid.nc);
  w.val<double>(h->grid.f);
  w.val<int32_t>(h->field.kind);
  w.val<int32_t>(h->field.nbx);
  w.val<int32_t>(h->field.nby);
  w.val<double>(h->field.width);
  w.val<double>(h->field.scale);
  w.val<double>(h->field.contrast_log);
  w.val<double>(h->field.gain);
  w.val<double>(h->tau);
  w.val<int32_t>(h->nfam);
  w.val<int32_t>(kParams);
  w.val<int32_t>(h->step);
  w.put(host_buf ? (const void*)W.data() : nullptr, sizeof(float) * np);
  w.put(host_buf ? (const void*)m.data() : nullptr, sizeof(float) * np);
  w.put(host_buf ? (const void*)v.data() : nullptr, sizeof(float) * np);
  w.put(host_buf ? (const void*)box.data() : nullptr, sizeof(float) * nb);
  *bytes = w.pos;
  if (host_buf && !w.fits()) return set_error(STOMSFEM_ENOMEM, "checkpoint buffer %zu < %zu bytes", buf_bytes, w.pos);
  return STOMSFEM_OK;
}

extern "C" int stomsfem_surrogate_load(const void* host_buf, size_t buf_bytes, stomsfem_surrogate** out,
                                       int32_t* n_families) {
  if (!host_buf || !out) return set_error(STOMSFEM_EINVAL, "NULL buffer / out");
  *out = nullptr;
  CkptReader r(host_buf, buf_bytes);
  const int hc = ckpt_check_header(r, kSgMagic);
  if (hc == 1) return set_error(STOMSFEM_EVERSION, "not a version-%u surrogate checkpoint", kCkptVersion);
  if (hc == 2) return set_error(STOMSFEM_EINVAL, "truncated surrogate checkpoint");
  stomsfem_grid g;
  g.nf = r.val<int32_t>();
  g.nc = r.val<int32_t>();
  g.f = r.val<double>();
  stomsfem_field fd;
  fd.kind = r.val<int32_t>();
  fd.nbx = r.val<int32_t>();
  fd.nby = r.val<int32_t>();
  fd.width = r.val<double>();
  fd.scale = r.val<double>();
  fd.contrast_log = r.val<double>();
  fd.gain = r.val<double>();
  const double tau = r.val<double>();
  const int32_t nfam = r.val<int32_t>(), nparams = r.val<int32_t>(), step = r.val<int32_t>();
  if (!r.ok || nfam < 1 || nparams != kParams || step < 0)
    return set_error(STOMSFEM_EINVAL, "inconsistent surrogate checkpoint header");
  const size_t np = (size_t)nfam * kParams, nb = (size_t)nfam * kIn * 2;
  if (buf_bytes < r.pos + sizeof(float) * (3 * np + nb))
    return set_error(STOMSFEM_EINVAL, "truncated surrogate checkpoint");
  const float* W = reinterpret_cast<const float*>(static_cast<const unsigned char*>(host_buf) + r.pos);
  std::vector<float> Wc(W, W + np);  // the buffer need not be 4-byte aligned
  stomsfem_surrogate* h = nullptr;
  int32_t nf2 = 0;
  int rc = stomsfem_surrogate_create(&g, &fd, tau, Wc.data(), &h, &nf2);
  if (rc) return rc;
  if (nf2 != nfam) {
    sg_free(h);
    return set_error(STOMSFEM_EINVAL, "surrogate checkpoint has %d families, the grid/field give %d", nfam, nf2);
  }
  std::vector<float> tmp(np > nb ? np : nb);
  const unsigned char* base = static_cast<const unsigned char*>(host_buf) + r.pos + sizeof(float) * np;
  std::memcpy(tmp.data(), base, sizeof(float) * np);
  rc = check_cuda(cudaMemcpy(h->m, tmp.data(), sizeof(float) * np, cudaMemcpyHostToDevice), "copy m");
  base += sizeof(float) * np;
  if (!rc) {
    std::memcpy(tmp.data(), base, sizeof(float) * np);
    rc = check_cuda(cudaMemcpy(h->v, tmp.data(), sizeof(float) * np, cudaMemcpyHostToDevice), "copy v");
  }
  base += sizeof(float) * np;
  if (!rc) {
    std::memcpy(tmp.data(), base, sizeof(float) * nb);
    rc = check_cuda(cudaMemcpy(h->box, tmp.data(), sizeof(float) * nb, cudaMemcpyHostToDevice), "copy box");
  }
  if (rc) {
    sg_free(h);
    return rc;
  }
  h->step = step;
  if (n_families) *n_families = nfam;
  *out = h;
  return STOMSFEM_OK;
}

template <bool F32>
static int train_launch_t(const TrainArgs& A, int nfam, cudaStream_t st) {
  const size_t smem = sizeof(TrainSmemT<F32>);
  STOMSFEM_TRY_CUDA(
      cudaFuncSetAttribute(surrogate_train_kernel<F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  surrogate_train_kernel<F32><<<nfam, 256, smem, st>>>(A);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  return STOMSFEM_OK;
}
static int train_launch(const TrainArgs& A, int nfam, bool fp32, cudaStream_t st) {
  return fp32 ? train_launch_t<true>(A, nfam, st) : train_launch_t<false>(A, nfam, st);
}

extern "C" int stomsfem_surrogate_train(stomsfem_surrogate* h, const stomsfem_surrogate_cfg* cfg,
                                        const double* xi, const double* a, const double* Ke,
                                        const double* be, int32_t S, float* loss_hist,
                                        stomsfem_stream_t stream) {
  if (!h || !cfg || S <= 0 || !xi || !a || !Ke || !be) return set_error(STOMSFEM_EINVAL, "bad arguments");
  if (cfg->steps <= 0) return set_error(STOMSFEM_EINVAL, "steps must be > 0");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::vector<int> row0(h->nfam + 1, 0);
  for (int f = 0; f < h->nfam; ++f) row0[f + 1] = row0[f] + S * h->fam_ncell[f];
  const size_t N = (size_t)row0[h->nfam];
  float *X = nullptr, *Y = nullptr, *loss = nullptr;
  int* row0_d = nullptr;
  int rc = STOMSFEM_OK;
  auto cleanup = [&]() {
    cudaFree(X);
    cudaFree(Y);
    cudaFree(loss);
    cudaFree(row0_d);
  };
#define TRY(x)                                       \
  if ((rc = check_cuda((x), #x)) != STOMSFEM_OK) {   \
    cleanup();                                       \
    return rc;                                       \
  }
  TRY(cudaMalloc(&X, sizeof(float) * N * kIn));
  TRY(cudaMalloc(&Y, sizeof(float) * N * kOut));
  TRY(cudaMalloc(&loss, sizeof(float) * (size_t)h->nfam * cfg->steps));
  TRY(cudaMalloc(&row0_d, sizeof(int) * (h->nfam + 1)));
  TRY(cudaMemcpyAsync(row0_d, row0.data(), sizeof(int) * (h->nfam + 1), cudaMemcpyHostToDevice, st));
  const int rho = h->grid.nf / h->grid.nc;
  surrogate_prepare_kernel<<<1024, 256, 0, st>>>(S, h->grid.nc, rho, h->grid.nf, h->grid.f, h->K, xi, a, Ke, be,
                                                 h->var_ids_d, h->cell_fam_d, h->cell_pos_d, row0_d,
                                                 h->fam_ncell_d, X, Y);
  TRY(cudaGetLastError());
  surrogate_box_kernel<<<h->nfam, 32, 0, st>>>(row0_d, X, h->box);
  TRY(cudaGetLastError());
  TrainArgs A;
  A.nfam = h->nfam;
  A.fam_row0 = row0_d;
  A.row_lo = A.row_hi = 0;
  A.X = X;
  A.Y = Y;
  A.W = h->W;
  A.m = h->m;
  A.v = h->v;
  A.grad_out = nullptr;
  A.loss_out = loss;
  A.steps = cfg->steps;
  A.step0 = h->step;
  A.lr = (float)cfg->lr;
  A.lr_min = (float)cfg->lr_min;
  A.beta1 = (float)cfg->beta1;
  A.beta2 = (float)cfg->beta2;
  A.eps = (float)cfg->eps;
  A.seed = cfg->seed;
  A.grad_only = 0;
  if ((rc = train_launch(A, h->nfam, cfg->fp32_products != 0, st)) != STOMSFEM_OK) {
    cleanup();
    return rc;
  }
  h->step += cfg->steps;
  if (loss_hist) {
    std::vector<float> lh((size_t)h->nfam * cfg->steps);
    TRY(cudaMemcpyAsync(lh.data(), loss, sizeof(float) * lh.size(), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    for (int s = 0; s < cfg->steps; ++s) {
      double acc = 0.0;
      for (int f = 0; f < h->nfam; ++f) acc += lh[(size_t)f * cfg->steps + s];
      loss_hist[s] = (float)(acc / h->nfam);
    }
  } else {
    TRY(cudaStreamSynchronize(st));
  }
#undef TRY
  cleanup();
  return STOMSFEM_OK;
}

extern "C" int stomsfem_surrogate_grad(const float* weights, const float* X, const float* T, int32_t fp32_products,
                                       float* grad, float* loss, stomsfem_stream_t stream) {
  if (!weights || !X || !T || !grad) return set_error(STOMSFEM_EINVAL, "NULL device pointer");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  TrainArgs A;
  std::memset(&A, 0, sizeof(A));
  A.nfam = 1;
  A.fam_row0 = nullptr;  // the batch's rows are [0, 64)
  A.row_lo = 0;
  A.row_hi = kBatch;
  A.X = X;
  A.Y = T;
  A.W = const_cast<float*>(weights);  // read only in the gradient mode
  A.m = const_cast<float*>(weights);
  A.v = const_cast<float*>(weights);
  A.grad_out = grad;
  A.loss_out = loss;
  A.steps = 1;
  A.grad_only = 1;
  return train_launch(A, 1, fp32_products != 0, st);
}

// Seeded Xavier-uniform initial weights: W[o][i] = lim (2 u - 1), lim =
// sqrt(6 / (fan_in + fan_out)), u the top 53 bits of SplitMix64 of (seed,
// family, parameter index) over 2^53; biases zero.
extern "C" int stomsfem_surrogate_init_weights(int32_t n_families, uint64_t seed, float* w_host) {
  if (n_families < 1 || !w_host) return set_error(STOMSFEM_EINVAL, "need n_families >= 1 and a host buffer");
  const int wo[4] = {oW1, oW2, oW3, oW4}, bo[4] = {oB1, oB2, oB3, oB4};
  const int fin[4] = {kIn, kHid, kHid, kHid}, fout[4] = {kHid, kHid, kHid, kOut};
  for (int f = 0; f < n_families; ++f) {
    float* w = w_host + (size_t)f * kParams;
    for (int l = 0; l < 4; ++l) {
      const double lim = std::sqrt(6.0 / (double)(fin[l] + fout[l]));
      for (int q = 0; q < fin[l] * fout[l]; ++q) {
        const uint64_t key = seed ^ ((uint64_t)f << 48) ^ (uint64_t)(wo[l] + q);
        const double u = (double)(splitmix64(key) >> 11) * (1.0 / 9007199254740992.0);
        w[wo[l] + q] = (float)(lim * (2.0 * u - 1.0));
      }
      for (int q = 0; q < fout[l]; ++q) w[bo[l] + q] = 0.f;
    }
  }
  return STOMSFEM_OK;
}

namespace {

struct InferLayout {
  size_t X, uor, Xf, abar, ahar, Wb, tfam, list, count, err, fb, total;
  size_t Wb2 = 0, K2 = 0, b2 = 0, f2 = 0;  // the ensemble partner's pass
  long long rows_pad, units;
  int ntiles;
};

InferLayout infer_layout(const stomsfem_surrogate* h, int S, std::vector<int>* row0, std::vector<int>* tfam) {
  InferLayout L;
  long long rows = 0;
  int tiles = 0;
  if (row0) row0->assign(h->nfam + 1, 0);
  if (tfam) tfam->clear();
  for (int f = 0; f < h->nfam; ++f) {
    const long long n = (long long)S * h->fam_ncell[f];
    const int t = (int)((n + kTile - 1) / kTile);
    if (row0) (*row0)[f] = (int)rows;
    if (tfam)
      for (int i = 0; i < t; ++i) tfam->push_back(f);
    rows += (long long)t * kTile;
    tiles += t;
  }
  if (row0) (*row0)[h->nfam] = (int)rows;
  L.rows_pad = rows;
  L.ntiles = tiles;
  L.units = (long long)S * h->ncell;
  auto al = [](size_t x) { return (x + 1023) & ~size_t(1023); };
  size_t o = 0;
  L.X = o;    o += al(rows * kInPad * 2);
  L.uor = o;  o += al(rows * 4);
  L.Xf = o;   o += al(L.units * kIn * 4);
  L.abar = o; o += al(L.units * 8);
  L.ahar = o; o += al(L.units * 8);
  L.Wb = o;   o += al((size_t)h->nfam * kWbSize * 2);
  L.tfam = o; o += al((size_t)(h->nfam + 1) * 4);
  L.list = o; o += al(L.units * 4);
  L.count = o; o += 1024;
  L.err = o;  o += 1024;
  if (h->partner) {
    L.Wb2 = o; o += al((size_t)h->nfam * kWbSize * 2);
    L.K2 = o;  o += al(L.units * 10 * 8);
    L.b2 = o;  o += al(L.units * 4 * 8);
    L.f2 = o;  o += al(L.units);
  }
  L.fb = o;
  o += upscale_list_workspace_fp64(&h->grid);
  L.total = o;
  return L;
}

}  // namespace

extern "C" int stomsfem_surrogate_workspace_size(const stomsfem_surrogate* h, int32_t S, size_t* bytes) {
  if (!h || S < 0 || !bytes) return set_error(STOMSFEM_EINVAL, "bad arguments");
  *bytes = infer_layout(h, S, nullptr, nullptr).total;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_surrogate_infer(stomsfem_surrogate* h, const double* xi, const double* a, int32_t S,
                                        double delta, double* Ke, double* be, uint8_t* fell_back,
                                        void* workspace, size_t workspace_bytes, stomsfem_stream_t stream) {
  if (!h || S < 0) return set_error(STOMSFEM_EINVAL, "bad arguments");
  if (S == 0) return STOMSFEM_OK;
  if (!xi || !a || !Ke || !be || !fell_back || !workspace) return set_error(STOMSFEM_EINVAL, "NULL device pointer");
  if (!(delta >= 0.0)) return set_error(STOMSFEM_EINVAL, "delta must be >= 0");
  const InferLayout L = infer_layout(h, S, nullptr, nullptr);
  if (workspace_bytes < L.total)
    return set_error(STOMSFEM_ENOMEM, "surrogate workspace %zu < %zu", workspace_bytes, L.total);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  auto* X = reinterpret_cast<__nv_bfloat16*>(ws + L.X);
  int* uor = reinterpret_cast<int*>(ws + L.uor);
  float* Xf = reinterpret_cast<float*>(ws + L.Xf);
  double* abar = reinterpret_cast<double*>(ws + L.abar);
  double* ahar = reinterpret_cast<double*>(ws + L.ahar);
  auto* Wb = reinterpret_cast<__nv_bfloat16*>(ws + L.Wb);
  int* tf = reinterpret_cast<int*>(ws + L.tfam);
  int32_t* list = reinterpret_cast<int32_t*>(ws + L.list);
  int32_t* count = reinterpret_cast<int32_t*>(ws + L.count);
  int32_t* err = reinterpret_cast<int32_t*>(ws + L.err);
  const int rho = h->grid.nf / h->grid.nc;
  // family row starts (in the list slot, written before the list is) and tile starts
  int* row0_d = reinterpret_cast<int*>(ws + L.list);
  surrogate_tiles_kernel<<<1, 32, 0, st>>>(h->nfam, h->fam_ncell_d, S, row0_d, tf);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  STOMSFEM_TRY_CUDA(cudaMemsetAsync(uor, 0xFF, L.rows_pad * 4, st));
  STOMSFEM_TRY_CUDA(cudaMemsetAsync(count, 0, 8, st));
  STOMSFEM_TRY_CUDA(cudaMemsetAsync(err, 0, 8, st));
  const int sms = device_sm_count() > 0 ? device_sm_count() : 152;
  surrogate_pack_kernel<<<sms * 2, 256, 0, st>>>(h->nfam, h->W, Wb);
  surrogate_infer_prepare_kernel<<<sms * 8, 128, 0, st>>>(S, h->grid.nc, rho, h->grid.nf, h->K, xi, a, h->var_ids_d,
                                                         h->cell_fam_d, h->cell_pos_d, row0_d, h->fam_ncell_d, X, uor,
                                                         Xf, abar, ahar);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  surrogate_zero_pad_kernel<<<h->nfam, 128, 0, st>>>(row0_d, h->fam_ncell_d, S, X);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  InferArgs A;
  A.X = X;
  A.unit_of_row = uor;
  A.tile0 = tf;
  A.nfam = h->nfam;
  A.Wb = Wb;
  A.W = h->W;
  A.box = h->box;
  A.Xf = Xf;
  A.abar = abar;
  A.ahar = ahar;
  A.f = h->grid.f;
  A.H = 1.0 / h->grid.nc;
  A.delta = delta;
  A.margin = 0.01;
  A.Ke = Ke;
  A.be = be;
  A.flag = fell_back;
  A.err = err;
  const size_t smem = 1024 + kTile * 128 * 3 + kHid * 128 * 5 + kOut * 128 * 2;
  STOMSFEM_TRY_CUDA(cudaFuncSetAttribute(surrogate_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  float proj[100];
  zero_row_sum_projector(proj);
  STOMSFEM_TRY_CUDA(cudaMemcpyToSymbolAsync(kZeroRowSumProj, proj, sizeof(proj), 0, cudaMemcpyHostToDevice, st));
  surrogate_infer_kernel<<<L.ntiles, kInferThreads, smem, st>>>(A);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  if (h->partner) {
    // the partner network on the same inputs (its own outputs and flags in
    // scratch), then the disagreement test on the units the rules accepted
    const stomsfem_surrogate* p2 = h->partner;
    auto* Wb2 = reinterpret_cast<__nv_bfloat16*>(ws + L.Wb2);
    surrogate_pack_kernel<<<sms * 2, 256, 0, st>>>(p2->nfam, p2->W, Wb2);
    InferArgs A2 = A;
    A2.Wb = Wb2;
    A2.W = p2->W;
    A2.box = p2->box;
    A2.Ke = reinterpret_cast<double*>(ws + L.K2);
    A2.be = reinterpret_cast<double*>(ws + L.b2);
    A2.flag = ws + L.f2;
    surrogate_infer_kernel<<<L.ntiles, kInferThreads, smem, st>>>(A2);
    STOMSFEM_TRY_CUDA(cudaGetLastError());
    surrogate_ensemble_kernel<<<sms * 4, 256, 0, st>>>(L.units, Ke, A2.Ke, h->ens_tol, fell_back);
    STOMSFEM_TRY_CUDA(cudaGetLastError());
  }
  surrogate_compact_kernel<<<sms * 4, 256, 0, st>>>(L.units, fell_back, err, list, count);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  return upscale_list_fp64(&h->grid, a, S, list, count, Ke, be, ws + L.fb, L.total - L.fb, st);
}

extern "C" int stomsfem_surrogate_set_partner(stomsfem_surrogate* h, const stomsfem_surrogate* partner, double tol) {
  if (!h) return set_error(STOMSFEM_EINVAL, "surrogate is NULL");
  if (!partner) {
    h->partner = nullptr;
    h->ens_tol = 0.0;
    return STOMSFEM_OK;
  }
  if (partner == h) return set_error(STOMSFEM_EINVAL, "a surrogate cannot be its own partner");
  if (!(tol >= 0.0)) return set_error(STOMSFEM_EINVAL, "tol must be >= 0");
  const bool same = partner->grid.nf == h->grid.nf && partner->grid.nc == h->grid.nc &&
                    partner->nfam == h->nfam && partner->fam_cell == h->fam_cell &&
                    partner->k_cell == h->k_cell && partner->var_ids == h->var_ids;
  if (!same) return set_error(STOMSFEM_EINVAL, "the partner must have the same grid, local variables and families");
  h->partner = partner;
  h->ens_tol = tol;
  return STOMSFEM_OK;
}
