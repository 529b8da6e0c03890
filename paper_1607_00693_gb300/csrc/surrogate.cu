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
#include <cstring>
#include <map>
#include <vector>

#include "common.cuh"
#include "stomsfem.h"

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

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// ---------------------------------------------------------------- training

struct TrainSmem {
  __nv_bfloat16 W1[kHid * kIn], W2[kHid * kHid], W3[kHid * kHid], W4[kOut * kHid];  // [out][in]
  __nv_bfloat16 X[kBatch * kIn];
  __nv_bfloat16 Z1[kBatch * kHid], Z2[kBatch * kHid], Z3[kBatch * kHid];  // pre-activations
  __nv_bfloat16 H1[kBatch * kHid], H2[kBatch * kHid], H3[kBatch * kHid];  // GELU(Z)
  __nv_bfloat16 D1[kBatch * kHid], D2[kBatch * kHid];                     // dZ ping-pong
  __nv_bfloat16 DY[kBatch * kOut];
  float T[kBatch * kOut];
  float gb[kHid];  // bias gradient of the layer being processed
  float loss;
  int rows[kBatch];
};

struct TrainArgs {
  int nfam;
  const int* fam_row0;   // [nfam + 1] row ranges of each family in X/Y
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

__global__ void __launch_bounds__(256) surrogate_train_kernel(TrainArgs A) {
  extern __shared__ __align__(16) unsigned char tsm_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(tsm_raw);
  const int fam = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  float* Wm = A.W + (size_t)fam * kParams;
  float* Mm = A.m + (size_t)fam * kParams;
  float* Vm = A.v + (size_t)fam * kParams;
  const int r0 = A.fam_row0[fam], r1 = A.fam_row0[fam + 1];
  const int nrows = r1 - r0;
  if (nrows <= 0) return;
  for (int i = tid; i < kHid * kIn; i += 256) S.W1[i] = __float2bfloat16_rn(Wm[oW1 + i]);
  for (int i = tid; i < kHid * kHid; i += 256) {
    S.W2[i] = __float2bfloat16_rn(Wm[oW2 + i]);
    S.W3[i] = __float2bfloat16_rn(Wm[oW3 + i]);
  }
  for (int i = tid; i < kOut * kHid; i += 256) S.W4[i] = __float2bfloat16_rn(Wm[oW4 + i]);
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
    for (int i = tid; i < kBatch * kIn; i += 256) S.X[i] = __float2bfloat16_rn(A.X[(size_t)S.rows[i / kIn] * kIn + i % kIn]);
    for (int i = tid; i < kBatch * kOut; i += 256) S.T[i] = A.Y[(size_t)S.rows[i / kOut] * kOut + i % kOut];
    __syncthreads();
    // ---- forward: hidden layers [64 x 128]; warp w owns columns [16w, 16w+16)
#define FWD_LAYER(AIN, KIN, WS, BOFF, ZOUT, HOUT)                                              \
  {                                                                                            \
    for (int mt = 0; mt < kBatch / 16; ++mt)                                                   \
      for (int nt = 0; nt < 2; ++nt) {                                                         \
        const int m0 = mt * 16, n0 = warp * 16 + nt * 8;                                       \
        float c[4] = {0, 0, 0, 0};                                                             \
        mma_tile(RowMajor{AIN, KIN}, ColMajor{WS, KIN}, m0, n0, KIN, c, lane);                \
        for (int q = 0; q < 4; ++q) {                                                          \
          const int row = m0 + g + (q >> 1) * 8, col = n0 + 2 * t4 + (q & 1);                \
          const float z = c[q] + Wm[BOFF + col];                                               \
          ZOUT[row * kHid + col] = __float2bfloat16_rn(z);                                     \
          HOUT[row * kHid + col] = __float2bfloat16_rn(gelu(z));                               \
        }                                                                                      \
      }                                                                                        \
    __syncthreads();                                                                           \
  }
    FWD_LAYER(S.X, kIn, S.W1, oB1, S.Z1, S.H1)
    FWD_LAYER(S.H1, kHid, S.W2, oB2, S.Z2, S.H2)
    FWD_LAYER(S.H2, kHid, S.W3, oB3, S.Z3, S.H3)
#undef FWD_LAYER
    // ---- output layer [64 x 16]: 8 tiles, one per warp; dY = 2 (Y - T) / (B * 13)
    {
      const int m0 = (warp >> 1) * 16, n0 = (warp & 1) * 8;
      float c[4] = {0, 0, 0, 0};
      mma_tile(RowMajor{S.H3, kHid}, ColMajor{S.W4, kHid}, m0, n0, kHid, c, lane);
      float ls = 0.f;
      for (int q = 0; q < 4; ++q) {
        const int row = m0 + g + (q >> 1) * 8, col = n0 + 2 * t4 + (q & 1);
        const float y = c[q] + Wm[oB4 + col];
        const float d = (col < kOutUsed) ? (y - S.T[row * kOut + col]) : 0.f;
        ls += d * d;
        S.DY[row * kOut + col] = __float2bfloat16_rn(2.f * d / (kBatch * kOutUsed));
      }
      ls = warp_sum(ls);
      if (lane == 0) atomicAdd(&S.loss, ls / (kBatch * kOutUsed));
    }
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
    // ---- layer 4: dW4 [16 x 128] = dY^T H3 ; db4 ; dZ3 = (dY W4) * gelu'(Z3)
    for (int tt = warp; tt < 16; tt += 8) {
      const int n0 = tt * 8;
      float c[4] = {0, 0, 0, 0};
      mma_tile(ColMajor{S.DY, kOut}, RowMajor{S.H3, kHid}, 0, n0, kBatch, c, lane);
      for (int q = 0; q < 4; ++q) {
        const int o = g + (q >> 1) * 8, i = n0 + 2 * t4 + (q & 1);
        apply(oW4 + o * kHid + i, c[q]);
      }
    }
    if (tid < kOut) {
      float s = 0.f;
      for (int b = 0; b < kBatch; ++b) s += __bfloat162float(S.DY[b * kOut + tid]);
      apply(oB4 + tid, s);
    }
    if (tid < kHid) S.gb[tid] = 0.f;
    __syncthreads();
    // dH3 = dY W4 (W4 [out][in]: B(k = o, n = i) = W4[o][i])
    for (int mt = 0; mt < kBatch / 16; ++mt)
      for (int nt = 0; nt < 2; ++nt) {
        const int m0 = mt * 16, n0 = warp * 16 + nt * 8;
        float c[4] = {0, 0, 0, 0};
        mma_tile(RowMajor{S.DY, kOut}, RowMajor{S.W4, kHid}, m0, n0, kOut, c, lane);
        float cs0 = 0.f, cs1 = 0.f;
        for (int q = 0; q < 4; ++q) {
          const int row = m0 + g + (q >> 1) * 8, col = n0 + 2 * t4 + (q & 1);
          const float dz = c[q] * gelu_grad(__bfloat162float(S.Z3[row * kHid + col]));
          S.D1[row * kHid + col] = __float2bfloat16_rn(dz);
          if (q & 1) cs1 += dz; else cs0 += dz;
        }
        // column sums over the 16 rows of this tile: reduce over g (lanes with equal t4)
        for (int o = 4; o < 32; o <<= 1) {
          cs0 += __shfl_xor_sync(0xffffffffu, cs0, o);
          cs1 += __shfl_xor_sync(0xffffffffu, cs1, o);
        }
        if (g == 0) {
          atomicAdd(&S.gb[n0 + 2 * t4], cs0);
          atomicAdd(&S.gb[n0 + 2 * t4 + 1], cs1);
        }
      }
    __syncthreads();
    // W4 may now change (its old values were used above)
    if (!A.grad_only)
      for (int i = tid; i < kOut * kHid; i += 256) S.W4[i] = __float2bfloat16_rn(Wm[oW4 + i]);
    // ---- hidden layers 3, 2, 1: dW = dZ^T H_in, db, dZ_in = (dZ W) * gelu'(Z_in)
#define BWD_LAYER(DZ, HIN, KIN, WS, WOFF, BOFF, ZIN, DZOUT, HAS_IN)                           \
  {                                                                                            \
    /* dW [128 x KIN]: warp w owns rows [16w, 16w + 16) */                                    \
    for (int nt = 0; nt < KIN / 8; ++nt) {                                                     \
      const int m0 = warp * 16, n0 = nt * 8;                                                   \
      float c[4] = {0, 0, 0, 0};                                                               \
      mma_tile(ColMajor{DZ, kHid}, RowMajor{HIN, KIN}, m0, n0, kBatch, c, lane);              \
      for (int q = 0; q < 4; ++q) {                                                            \
        const int o = m0 + g + (q >> 1) * 8, i = n0 + 2 * t4 + (q & 1);                       \
        apply(WOFF + o * KIN + i, c[q]);                                                       \
      }                                                                                        \
    }                                                                                          \
    if (tid < kHid) apply(BOFF + tid, S.gb[tid]);                                              \
    __syncthreads();                                                                           \
    if (HAS_IN) {                                                                              \
      if (tid < kHid) S.gb[tid] = 0.f;                                                         \
      __syncthreads();                                                                         \
      for (int mt = 0; mt < kBatch / 16; ++mt)                                                 \
        for (int nt = 0; nt < 2; ++nt) {                                                       \
          const int m0 = mt * 16, n0 = warp * 16 + nt * 8;                                     \
          float c[4] = {0, 0, 0, 0};                                                           \
          mma_tile(RowMajor{DZ, kHid}, RowMajor{WS, kHid}, m0, n0, kHid, c, lane);            \
          float cs0 = 0.f, cs1 = 0.f;                                                          \
          for (int q = 0; q < 4; ++q) {                                                        \
            const int row = m0 + g + (q >> 1) * 8, col = n0 + 2 * t4 + (q & 1);              \
            const float dz = c[q] * gelu_grad(__bfloat162float(ZIN[row * kHid + col]));       \
            DZOUT[row * kHid + col] = __float2bfloat16_rn(dz);                                 \
            if (q & 1) cs1 += dz; else cs0 += dz;                                              \
          }                                                                                    \
          for (int o = 4; o < 32; o <<= 1) {                                                   \
            cs0 += __shfl_xor_sync(0xffffffffu, cs0, o);                                       \
            cs1 += __shfl_xor_sync(0xffffffffu, cs1, o);                                       \
          }                                                                                    \
          if (g == 0) {                                                                        \
            atomicAdd(&S.gb[n0 + 2 * t4], cs0);                                                \
            atomicAdd(&S.gb[n0 + 2 * t4 + 1], cs1);                                            \
          }                                                                                    \
        }                                                                                      \
      __syncthreads();                                                                         \
    }                                                                                          \
  }
    BWD_LAYER(S.D1, S.H2, kHid, S.W3, oW3, oB3, S.Z2, S.D2, 1)
    if (!A.grad_only)
      for (int i = tid; i < kHid * kHid; i += 256) S.W3[i] = __float2bfloat16_rn(Wm[oW3 + i]);
    BWD_LAYER(S.D2, S.H1, kHid, S.W2, oW2, oB2, S.Z1, S.D1, 1)
    if (!A.grad_only)
      for (int i = tid; i < kHid * kHid; i += 256) S.W2[i] = __float2bfloat16_rn(Wm[oW2 + i]);
    BWD_LAYER(S.D1, S.X, kIn, S.W1, oW1, oB1, S.Z1, S.D2, 0)
    if (!A.grad_only)
      for (int i = tid; i < kHid * kIn; i += 256) S.W1[i] = __float2bfloat16_rn(Wm[oW1 + i]);
#undef BWD_LAYER
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

static int train_launch(const TrainArgs& A, int nfam, cudaStream_t st) {
  const size_t smem = sizeof(TrainSmem);
  STOMSFEM_TRY_CUDA(cudaFuncSetAttribute(surrogate_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  surrogate_train_kernel<<<nfam, 256, smem, st>>>(A);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  return STOMSFEM_OK;
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
  if ((rc = train_launch(A, h->nfam, st)) != STOMSFEM_OK) {
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

extern "C" int stomsfem_surrogate_grad(const float* weights, const float* X, const float* T, float* grad,
                                       float* loss, stomsfem_stream_t stream) {
  if (!weights || !X || !T || !grad) return set_error(STOMSFEM_EINVAL, "NULL device pointer");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int* row0_d = nullptr;
  STOMSFEM_TRY_CUDA(cudaMalloc(&row0_d, sizeof(int) * 2));
  const int row0[2] = {0, kBatch};
  int rc = check_cuda(cudaMemcpyAsync(row0_d, row0, sizeof(row0), cudaMemcpyHostToDevice, st), "memcpy");
  if (rc == STOMSFEM_OK) {
    TrainArgs A;
    std::memset(&A, 0, sizeof(A));
    A.nfam = 1;
    A.fam_row0 = row0_d;
    A.X = X;
    A.Y = T;
    A.W = const_cast<float*>(weights);
    A.m = const_cast<float*>(weights);
    A.v = const_cast<float*>(weights);
    A.grad_out = grad;
    A.loss_out = loss;
    A.steps = 1;
    A.grad_only = 1;
    rc = train_launch(A, 1, st);
  }
  if (rc == STOMSFEM_OK) rc = check_cuda(cudaStreamSynchronize(st), "sync");
  cudaFree(row0_d);
  return rc;
}
