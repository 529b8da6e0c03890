// Fine-grid Q1 FEM for large grids (the level-1 solves of the two-level
// Monte Carlo estimator, Remark in Sec. 4.1.1, Eq. MCmean2level): the
// standard Q1 system on the (nf-1)^2 interior nodes, zero Dirichlet data,
// load f h^2 per node, for a batch of samples, by conjugate gradients in
// FP64 preconditioned with one geometric multigrid V-cycle in FP32.
//
// Multigrid: levels nf_0 = nf, nf_{l+1} = nf_l / 2 down to nf_L <= 16;
// prolongation P (coarse node (I, J) at fine node (2I, 2J)) bilinear, or,
// when the batch's coefficient contrast exceeds kMgOdContrast, with the
// other fine nodes' weights from the fine stencil (mgf_interp_kernel);
// restriction P^T, Galerkin coarse operators A_{l+1} = P^T A_l P (9-point
// stencils again), damped Jacobi smoothing (omega = 0.8, two sweeps before
// and after the coarse correction: a symmetric V-cycle, so the
// preconditioner is symmetric positive definite and plain CG applies), and
// 60 Jacobi sweeps on the coarsest grid.  Stencils are stored per level and
// sample in FP32, structure of arrays over the full (nf_l+1)^2 node grid,
// in symmetric form: five couplings per node (centre, east, north,
// north-east, north-west), the other four read from the neighbours, so
// every level's operator is exactly symmetric (boundary nodes carry zero
// stencils and stay zero).
//
// CG: x, r, p, Ap in FP64; the matrix-vector product applies the fine
// 9-point stencil in FP64, formed from a once per solve and stored in
// symmetric form (five entries per node, nine FMAs per product); the
// per-sample dot products are block sums with one atomic per block; the
// step lengths are computed on the device.  The host checks convergence
// (max over samples of |r| / |f|) every few iterations.
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace stomsfem {

constexpr int kMgMaxLevels = 12;
constexpr float kMgOmega = 0.8f;
constexpr int kMgCoarseSweeps = 60;
constexpr int kMgThreads = 256;
// Coefficient contrast (max a / min a over the batch) above which the
// transfers between levels use the operator-dependent prolongation; below
// it the bilinear one, which converges as fast there (the same 12 CG
// iterations on the lognormal 1024^2 medium of contrast 100) and moves
// fewer bytes per cycle.
constexpr double kMgOdContrast = 1e3;

struct MgLevel {
  int nf;          // elements per side
  int N;           // (nf + 1)^2 nodes
  float* st;       // [S][5][N]: centre, east, north, north-east, north-west
  float* u;        // [S][N]
  float* u2;       // [S][N] (Jacobi ping-pong)
  float* f;        // [S][N]
  float* r;        // [S][N]
  float* P;        // [S][4][N]: prolongation weights from the next coarser level (per node type)
  float* dv;       // [S][N]: Jacobi divisor (see mgf_divisor_kernel)
};

__device__ __forceinline__ bool interior(int i, int j, int nf) { return i > 0 && j > 0 && i < nf && j < nf; }

// Stencils of every level in symmetric form: st[m][node] for m = 0..4 the
// centre, east, north, north-east and north-west couplings of the node; the
// west, south, south-west and south-east couplings are the east, north,
// north-east and north-west ones of the neighbour there (zero at the
// boundary nodes, whose values stay zero in every multigrid vector).
// Entry k = (dj + 1) * 3 + (di + 1) of the 9-point stencil of node v:
__device__ __forceinline__ int st_arr(int k) {  // array m holding entry k
  return k == 4 ? 0 : (k == 5 || k == 3) ? 1 : (k == 7 || k == 1) ? 2 : (k == 8 || k == 0) ? 3 : 4;
}
__device__ __forceinline__ long st_node(int k, long v, int W) {  // node whose array holds it
  const int di = k % 3 - 1, dj = k / 3 - 1;
  return (dj < 0 || (dj == 0 && di < 0)) ? v + dj * W + di : v;
}
template <int K>
__device__ __forceinline__ float st9(const float* __restrict__ st, size_t N, long v, int W) {
  constexpr int di = K % 3 - 1, dj = K / 3 - 1;
  constexpr int m = K == 4 ? 0 : (K == 5 || K == 3) ? 1 : (K == 7 || K == 1) ? 2 : (K == 8 || K == 0) ? 3 : 4;
  constexpr bool own = !(dj < 0 || (dj == 0 && di < 0));
  return st[(size_t)m * N + (own ? v : v + dj * W + di)];
}

// Level-0 stencil from a, FP32 for the preconditioner (symmetric form
// above); and the FP64 operator of the CG in symmetric form,
// st64[k][node] for k = centre, east, north, north-east, north-west (the
// west, south, south-west and south-east entries of a node are the east,
// north, north-east and north-west entries of its neighbours there; zero
// at the boundary nodes, whose values are zero in every CG vector).
__global__ void mgf_fine_stencil_kernel(int nf, const double* __restrict__ a, float* __restrict__ st,
                                        double* __restrict__ st64) {
  const int s = blockIdx.y;
  const int N = (nf + 1) * (nf + 1);
  const double* as = a + (size_t)s * nf * nf;
  float* ss = st + (size_t)s * 5 * N;
  double* s64 = st64 + (size_t)s * 5 * N;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
    const int i = v % (nf + 1), j = v / (nf + 1);
    float c[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    double d[5] = {0, 0, 0, 0, 0};
    if (interior(i, j, nf)) {
      const double aSW = as[(size_t)(j - 1) * nf + i - 1], aSE = as[(size_t)(j - 1) * nf + i];
      const double aNE = as[(size_t)j * nf + i], aNW = as[(size_t)j * nf + i - 1];
      // products with 1/6 and 1/3, not quotients: an FP64 division is a
      // long instruction sequence on the FP64 pipe
      constexpr double k6 = 1.0 / 6.0, k3 = 1.0 / 3.0;
      d[0] = (4.0 * k6) * (aSW + aSE + aNE + aNW);
      d[1] = -(aSE + aNE) * k6;
      d[2] = -(aNW + aNE) * k6;
      d[3] = -aNE * k3;
      d[4] = -aNW * k3;
      c[4] = (float)((4.0 * k6) * (aSW + aSE + aNE + aNW));
      c[3] = (float)(-(aSW + aNW) * k6);  // west
      c[5] = (float)(-(aSE + aNE) * k6);  // east
      c[1] = (float)(-(aSW + aSE) * k6);  // south
      c[7] = (float)(-(aNW + aNE) * k6);  // north
      c[0] = (float)(-aSW * k3);
      c[2] = (float)(-aSE * k3);
      c[8] = (float)(-aNE * k3);
      c[6] = (float)(-aNW * k3);
    }
    ss[v] = c[4];
    ss[(size_t)N + v] = c[5];
    ss[(size_t)2 * N + v] = c[7];
    ss[(size_t)3 * N + v] = c[8];
    ss[(size_t)4 * N + v] = c[6];
#pragma unroll
    for (int k = 0; k < 5; ++k) s64[(size_t)k * N + v] = d[k];
  }
}

// The 9-point stencil of interior node v (entries k = (dj + 1) * 3 + di + 1).
__device__ __forceinline__ void stencil9(const float* __restrict__ st, size_t N, long v, int W, float a[9]) {
  a[0] = st9<0>(st, N, v, W);
  a[1] = st9<1>(st, N, v, W);
  a[2] = st9<2>(st, N, v, W);
  a[3] = st9<3>(st, N, v, W);
  a[4] = st9<4>(st, N, v, W);
  a[5] = st9<5>(st, N, v, W);
  a[6] = st9<6>(st, N, v, W);
  a[7] = st9<7>(st, N, v, W);
  a[8] = st9<8>(st, N, v, W);
}

// The Jacobi divisor of a node from its nine entries (mgf_divisor_kernel).
__device__ __forceinline__ float jacobi_divisor(const float a[9]) {
  const float l1 = fabsf(a[0]) + fabsf(a[1]) + fabsf(a[2]) + fabsf(a[3]) + fabsf(a[5]) + fabsf(a[6]) +
                   fabsf(a[7]) + fabsf(a[8]);
  return fmaxf(a[4], 0.5f * (a[4] + l1));
}

// Operator-dependent prolongation (the black-box interpolation of Dendy,
// J. Comput. Phys. 48, 1982, for 9-point stencils): a fine node between
// two coarse nodes of a row takes weights from its stencil collapsed onto
// that row (columns summed: w_W = -a_W / a_C, w_E = -a_E / a_C), one between
// two coarse nodes of a column from the stencil collapsed onto the column;
// a cell-centre node solves its own equation with its four edge neighbours
// interpolated so.  Where the stencil sums to zero the weights sum to one;
// next to the Dirichlet boundary the couplings to boundary nodes (zero in
// the symmetric form) drop out.  Across jumps of the coefficient the
// weights follow the operator, which keeps the coarse-grid correction
// effective where bilinear interpolation is not.
// (A collapsed centre that is not positive, which a coarse Galerkin
// operator can in principle give, takes the bilinear weights instead.)
__device__ __forceinline__ void interp_row(const float a[9], float& wW, float& wE) {
  const float c = a[1] + a[4] + a[7];
  wW = c > 0.f ? -(a[0] + a[3] + a[6]) / c : 0.5f;
  wE = c > 0.f ? -(a[2] + a[5] + a[8]) / c : 0.5f;
}
__device__ __forceinline__ void interp_col(const float a[9], float& wS, float& wN) {
  const float c = a[3] + a[4] + a[5];
  wS = c > 0.f ? -(a[0] + a[1] + a[2]) / c : 0.5f;
  wN = c > 0.f ? -(a[6] + a[7] + a[8]) / c : 0.5f;
}

// Weights P[m][node] of every fine node: between coarse nodes of a row
// (x odd, y even) m = 0, 1 for the west and east ones; of a column (x even,
// y odd) m = 0, 1 for the south and north ones; a cell centre (both odd)
// m = 0..3 for its south-west, south-east, north-east and north-west
// corners; zero elsewhere (coarse-grid nodes take their coarse value).
__global__ void mgf_interp_kernel(int nff, const float* __restrict__ stf, float* __restrict__ P) {
  const int s = blockIdx.y;
  const int W = nff + 1;
  const size_t N = (size_t)W * W;
  const float* sf = stf + (size_t)s * 5 * N;
  float* ps = P + (size_t)s * 4 * N;
  for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < (long)N; v += (long)gridDim.x * blockDim.x) {
    const int x = (int)(v % W), y = (int)(v / W);
    float w[4] = {0.f, 0.f, 0.f, 0.f};
    if (interior(x, y, nff) && ((x | y) & 1)) {
      float a[9];
      stencil9(sf, N, v, W, a);
      if ((x & 1) && !(y & 1)) {
        interp_row(a, w[0], w[1]);
      } else if (!(x & 1) && (y & 1)) {
        interp_col(a, w[0], w[1]);
      } else {
        // edge neighbours: south and north between coarse nodes of a row,
        // west and east between coarse nodes of a column
        float sW = 0.f, sE = 0.f, nW = 0.f, nE = 0.f, wS = 0.f, wN = 0.f, eS = 0.f, eN = 0.f, b[9];
        if (y - 1 > 0) { stencil9(sf, N, v - W, W, b); interp_row(b, sW, sE); }
        if (y + 1 < nff) { stencil9(sf, N, v + W, W, b); interp_row(b, nW, nE); }
        if (x - 1 > 0) { stencil9(sf, N, v - 1, W, b); interp_col(b, wS, wN); }
        if (x + 1 < nff) { stencil9(sf, N, v + 1, W, b); interp_col(b, eS, eN); }
        const float c = a[4];
        if (c > 0.f) {
          w[0] = -(a[0] + a[1] * sW + a[3] * wS) / c;  // south-west corner
          w[1] = -(a[2] + a[1] * sE + a[5] * eS) / c;  // south-east
          w[2] = -(a[8] + a[7] * nE + a[5] * eN) / c;  // north-east
          w[3] = -(a[6] + a[7] * nW + a[3] * wN) / c;  // north-west
        } else {
          w[0] = w[1] = w[2] = w[3] = 0.25f;
        }
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) ps[(size_t)m * N + v] = w[m];
  }
}

// Weight of fine node (gx, gy) in the prolongation of coarse node (I, J):
// the stored operator-dependent weights (OD), else bilinear (1, 1/2, 1/4).
template <bool OD>
__device__ __forceinline__ float pweight(const float* __restrict__ ps, size_t N, int W, int gx, int gy, int I, int J) {
  const int dx = gx - 2 * I, dy = gy - 2 * J;
  if (dx < -1 || dx > 1 || dy < -1 || dy > 1) return 0.f;
  if constexpr (!OD) return (dx == 0 ? 1.f : 0.5f) * (dy == 0 ? 1.f : 0.5f);
  const size_t g = (size_t)gy * W + gx;
  const bool ox = gx & 1, oy = gy & 1;
  if (!ox && !oy) return (dx == 0 && dy == 0) ? 1.f : 0.f;
  if (ox && !oy) return dy != 0 ? 0.f : ps[(dx > 0 ? 0 : 1) * N + g];
  if (!ox && oy) return dx != 0 ? 0.f : ps[(dy > 0 ? 0 : 1) * N + g];
  const int m = dy > 0 ? (dx > 0 ? 0 : 1) : (dx < 0 ? 2 : 3);
  return ps[(size_t)m * N + g];
}

// Galerkin coarse stencils A_c = P^T A_f P at the interior coarse nodes.
template <bool OD>
__global__ void mgf_rap_kernel(int nff, const float* __restrict__ stf, const float* __restrict__ P,
                               float* __restrict__ stc) {
  const int s = blockIdx.y;
  const int nfc = nff / 2;
  const int Wf = nff + 1;
  const int Nf = Wf * Wf, Nc = (nfc + 1) * (nfc + 1);
  const float* sf = stf + (size_t)s * 5 * Nf;
  const float* ps = P + (size_t)s * 4 * Nf;
  float* sc = stc + (size_t)s * 5 * Nc;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < Nc; v += gridDim.x * blockDim.x) {
    const int I = v % (nfc + 1), J = v / (nfc + 1);
    float out[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (interior(I, J, nfc)) {
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          const int fx = 2 * I + di, fy = 2 * J + dj;  // fine node in the support of coarse (I, J)
          const float wf = pweight<OD>(ps, Nf, Wf, fx, fy, I, J);
          if (wf == 0.f) continue;
          const int fv = fy * Wf + fx;
          for (int ej = -1; ej <= 1; ++ej)
            for (int ei = -1; ei <= 1; ++ei) {
              const int k = (ej + 1) * 3 + ei + 1;
              const float afv = sf[(size_t)st_arr(k) * Nf + st_node(k, fv, Wf)];
              if (afv == 0.f) continue;
              const int gx = fx + ei, gy = fy + ej;  // neighbour fine node
              if constexpr (!OD) {
                // coarse nodes (I + cI, J + cJ) whose hats cover (gx, gy)
                for (int cJ = -1; cJ <= 1; ++cJ)
                  for (int cI = -1; cI <= 1; ++cI) {
                    const int Ic = I + cI, Jc = J + cJ;
                    if (!interior(Ic, Jc, nfc)) continue;
                    const float pg = pweight<false>(ps, Nf, Wf, gx, gy, Ic, Jc);
                    if (pg != 0.f) out[(cJ + 1) * 3 + cI + 1] += wf * afv * pg;
                  }
                continue;
              }
              // the coarse nodes whose prolongation covers (gx, gy): one,
              // two or four by the node's type, with their weights
              int pI[4], pJ[4], np = 0;
              float pw[4];
              const size_t gv = (size_t)gy * Wf + gx;
              const int I0 = gx >> 1, J0 = gy >> 1;
              if (!(gx & 1) && !(gy & 1)) {
                pI[0] = I0; pJ[0] = J0; pw[0] = 1.f; np = 1;
              } else if (!(gy & 1)) {
                pI[0] = I0; pJ[0] = J0; pw[0] = ps[gv];
                pI[1] = I0 + 1; pJ[1] = J0; pw[1] = ps[(size_t)Nf + gv]; np = 2;
              } else if (!(gx & 1)) {
                pI[0] = I0; pJ[0] = J0; pw[0] = ps[gv];
                pI[1] = I0; pJ[1] = J0 + 1; pw[1] = ps[(size_t)Nf + gv]; np = 2;
              } else {
                pI[0] = I0; pJ[0] = J0; pw[0] = ps[gv];
                pI[1] = I0 + 1; pJ[1] = J0; pw[1] = ps[(size_t)Nf + gv];
                pI[2] = I0 + 1; pJ[2] = J0 + 1; pw[2] = ps[(size_t)2 * Nf + gv];
                pI[3] = I0; pJ[3] = J0 + 1; pw[3] = ps[(size_t)3 * Nf + gv]; np = 4;
              }
              for (int q = 0; q < np; ++q) {
                const int cI = pI[q] - I, cJ = pJ[q] - J;
                if (cI < -1 || cI > 1 || cJ < -1 || cJ > 1 || !interior(pI[q], pJ[q], nfc) || pw[q] == 0.f) continue;
                out[(cJ + 1) * 3 + cI + 1] += wf * afv * pw[q];
              }
            }
        }
    }
    sc[v] = out[4];
    sc[(size_t)Nc + v] = out[5];
    sc[(size_t)2 * Nc + v] = out[7];
    sc[(size_t)3 * Nc + v] = out[8];
    sc[(size_t)4 * Nc + v] = out[6];
  }
}

// (A u)_v at an interior node from the symmetric stencil form.
__device__ __forceinline__ float apply9(const float* __restrict__ st, size_t N, long v, const float* __restrict__ u,
                                        int W) {
  float t = 0.f;
  t = fmaf(st9<0>(st, N, v, W), u[v - W - 1], t);
  t = fmaf(st9<1>(st, N, v, W), u[v - W], t);
  t = fmaf(st9<2>(st, N, v, W), u[v - W + 1], t);
  t = fmaf(st9<3>(st, N, v, W), u[v - 1], t);
  t = fmaf(st9<4>(st, N, v, W), u[v], t);
  t = fmaf(st9<5>(st, N, v, W), u[v + 1], t);
  t = fmaf(st9<6>(st, N, v, W), u[v + W - 1], t);
  t = fmaf(st9<7>(st, N, v, W), u[v + W], t);
  t = fmaf(st9<8>(st, N, v, W), u[v + W + 1], t);
  return t;
}

// Jacobi divisor of each interior node: its diagonal entry, or half the
// sum of the diagonal and the off-diagonal magnitudes where those exceed
// the diagonal.  With omega = 0.8 the damped sweep then converges on every
// level with a symmetric positive definite operator (the l1-Jacobi bound:
// the divisors are at least (a_ii + sum |a_ij|) / 1.6), so the V-cycle stays
// symmetric positive definite whatever the Galerkin coarse operators look
// like; on the fine level, an M-matrix, it is the diagonal itself.
__global__ void mgf_divisor_kernel(int nf, const float* __restrict__ st, float* __restrict__ dv) {
  const int s = blockIdx.y;
  const int W = nf + 1;
  const size_t N = (size_t)W * W;
  const float* ss = st + (size_t)s * 5 * N;
  for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < (long)N; v += (long)gridDim.x * blockDim.x) {
    float d = 1.f;
    if (interior((int)(v % W), (int)(v / W), nf)) {
      float a[9];
      stencil9(ss, N, v, W, a);
      d = jacobi_divisor(a);
    }
    dv[(size_t)s * N + v] = d;
  }
}

// One damped Jacobi sweep: uo = ui + omega (f - A ui) / divisor (zero_in: ui = 0).
// OD (operator-dependent transfers, whose coarse operators need not be
// diagonally dominant): the divisor of mgf_divisor_kernel, read in the
// sweep from zero and formed from the loaded entries in the others; with
// the bilinear transfers the diagonal entry, as the M-matrix levels allow.
template <bool OD>
__global__ void mgf_jacobi_kernel(int nf, const float* __restrict__ st, const float* __restrict__ dv,
                                  const float* __restrict__ f, const float* __restrict__ ui, float* __restrict__ uo,
                                  int zero_in) {
  const int s = blockIdx.y;
  const int W = nf + 1, N = W * W;
  const float* ss = st + (size_t)s * 5 * N;
  const float* fs = f + (size_t)s * N;
  const float* us = ui + (size_t)s * N;
  float* os = uo + (size_t)s * N;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
    const int i = v % W, j = v / W;
    float o = 0.f;
    if (interior(i, j, nf)) {
      if (zero_in) {
        o = 0.f + kMgOmega * (fs[v] - 0.f) / (OD ? dv[(size_t)s * N + v] : ss[v]);
      } else {
        float a[9];
        stencil9(ss, N, v, W, a);
        float t = 0.f;
        t = fmaf(a[0], us[v - W - 1], t);
        t = fmaf(a[1], us[v - W], t);
        t = fmaf(a[2], us[v - W + 1], t);
        t = fmaf(a[3], us[v - 1], t);
        t = fmaf(a[4], us[v], t);
        t = fmaf(a[5], us[v + 1], t);
        t = fmaf(a[6], us[v + W - 1], t);
        t = fmaf(a[7], us[v + W], t);
        t = fmaf(a[8], us[v + W + 1], t);
        o = us[v] + kMgOmega * (fs[v] - t) / (OD ? jacobi_divisor(a) : a[4]);
      }
    }
    os[v] = o;
  }
}

// The coarsest grid (nf <= 16: at most 289 nodes): all kMgCoarseSweeps
// damped Jacobi sweeps from zero in one launch, one CTA per sample, the
// iterates in shared memory; each sweep is mgf_jacobi_kernel's arithmetic.
constexpr int kMgCoarseMaxNodes = 289;
constexpr int kMgCoarseThreads = 320;

__global__ void __launch_bounds__(kMgCoarseThreads) mgf_coarse_kernel(int nf, const float* __restrict__ st,
                                                                      const float* __restrict__ dv,
                                                                      const float* __restrict__ f,
                                                                      float* __restrict__ u) {
  __shared__ float buf[2][kMgCoarseMaxNodes];
  const int s = blockIdx.x;
  const int W = nf + 1, N = W * W;
  const int v = threadIdx.x;
  const bool in = v < N && interior(v % W, v / W, nf);
  float c[9], fv = 0.f;
  const float* ss = st + (size_t)s * 5 * N;
#pragma unroll
  for (int k = 0; k < 9; ++k) c[k] = in ? ss[(size_t)st_arr(k) * N + st_node(k, v, W)] : 0.f;
  if (in) fv = f[(size_t)s * N + v];
  const float dd = in ? dv[(size_t)s * N + v] : 1.f;
  float o = in ? 0.f + kMgOmega * (fv - 0.f) / dd : 0.f;  // the first sweep, from zero
  if (v < N) buf[0][v] = o;
  __syncthreads();
  for (int k = 1; k < kMgCoarseSweeps; ++k) {
    const float* ui = buf[(k - 1) & 1];
    if (in) {
      float t = 0.f;
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
        for (int di = -1; di <= 1; ++di) t = fmaf(c[(dj + 1) * 3 + di + 1], ui[v + dj * W + di], t);
      o = ui[v] + kMgOmega * (fv - t) / dd;
    }
    if (v < N) buf[k & 1][v] = o;
    __syncthreads();
  }
  if (v < N) u[(size_t)s * N + v] = o;
}

// r = f - A u at the interior nodes (0 elsewhere).
__global__ void mgf_residual_kernel(int nf, const float* __restrict__ st, const float* __restrict__ f,
                                    const float* __restrict__ u, float* __restrict__ r) {
  const int s = blockIdx.y;
  const int W = nf + 1, N = W * W;
  const float* ss = st + (size_t)s * 5 * N;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
    const int i = v % W, j = v / W;
    r[(size_t)s * N + v] = interior(i, j, nf) ? f[(size_t)s * N + v] - apply9(ss, N, v, u + (size_t)s * N, W) : 0.f;
  }
}

// f_c = P^T r_f at the interior coarse nodes.
template <bool OD>
__global__ void mgf_restrict_kernel(int nff, const float* __restrict__ P, const float* __restrict__ rf,
                                    float* __restrict__ fc) {
  const int s = blockIdx.y;
  const int nfc = nff / 2, Wf = nff + 1, Wc = nfc + 1;
  const int Nf = Wf * Wf, Nc = Wc * Wc;
  const float* ps = P + (size_t)s * 4 * Nf;
  const float* r = rf + (size_t)s * Nf;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < Nc; v += gridDim.x * blockDim.x) {
    const int I = v % Wc, J = v / Wc;
    float t = 0.f;
    if (interior(I, J, nfc)) {
      if constexpr (OD) {
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            const int gx = 2 * I + dx, gy = 2 * J + dy;
            t = fmaf(pweight<true>(ps, Nf, Wf, gx, gy, I, J), r[(size_t)gy * Wf + gx], t);
          }
      } else {
        const float* q = r + (size_t)(2 * J) * Wf + 2 * I;
        t = q[0] + 0.5f * (q[-1] + q[1] + q[-Wf] + q[Wf]) + 0.25f * (q[-Wf - 1] + q[-Wf + 1] + q[Wf - 1] + q[Wf + 1]);
      }
    }
    fc[(size_t)s * Nc + v] = t;
  }
}

// u_f += P u_c at the interior fine nodes.
template <bool OD>
__global__ void mgf_prolong_kernel(int nff, const float* __restrict__ P, const float* __restrict__ uc,
                                   float* __restrict__ uf) {
  const int s = blockIdx.y;
  const int nfc = nff / 2, Wf = nff + 1, Wc = nfc + 1;
  const int Nf = Wf * Wf, Nc = Wc * Wc;
  const float* ps = P + (size_t)s * 4 * Nf;
  const float* u = uc + (size_t)s * Nc;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < Nf; v += gridDim.x * blockDim.x) {
    const int x = v % Wf, y = v / Wf;
    if (!interior(x, y, nff)) continue;
    const int I0 = x >> 1, J0 = y >> 1;
    float t;
    if constexpr (!OD) {
      const int I1 = (x & 1) ? I0 + 1 : I0, J1 = (y & 1) ? J0 + 1 : J0;
      t = 0.25f * (u[J0 * Wc + I0] + u[J0 * Wc + I1] + u[J1 * Wc + I0] + u[J1 * Wc + I1]);
    } else if (!(x & 1) && !(y & 1)) {
      t = u[J0 * Wc + I0];
    } else if (!(y & 1)) {  // between coarse nodes I0, I0 + 1 of row J0
      t = ps[v] * u[J0 * Wc + I0] + ps[(size_t)Nf + v] * u[J0 * Wc + I0 + 1];
    } else if (!(x & 1)) {  // between coarse nodes J0, J0 + 1 of column I0
      t = ps[v] * u[J0 * Wc + I0] + ps[(size_t)Nf + v] * u[(J0 + 1) * Wc + I0];
    } else {  // cell centre: corners SW, SE, NE, NW
      t = ps[v] * u[J0 * Wc + I0] + ps[(size_t)Nf + v] * u[J0 * Wc + I0 + 1] +
          ps[(size_t)2 * Nf + v] * u[(J0 + 1) * Wc + I0 + 1] + ps[(size_t)3 * Nf + v] * u[(J0 + 1) * Wc + I0];
    }
    uf[(size_t)s * Nf + v] += t;
  }
}

// mm[0] = bit pattern of max a, mm[1] = that of min a over the positive
// entries of a (the patterns of positive doubles order like their values;
// mm[0] starts at zero, mm[1] at the pattern 0x7F7F7F7F7F7F7F7F, a positive
// double of about 1.4e306).
__global__ void mgf_range_kernel(long long n, const double* __restrict__ a, unsigned long long* __restrict__ mm) {
  unsigned long long hi = 0, lo = 0x7F7F7F7F7F7F7F7Full;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = a[i];
    if (v > 0.0) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(v);
      hi = max(hi, b);
      lo = min(lo, b);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(mm, hi);
    atomicMin(mm + 1, lo);
  }
}

// ---------------------------------------------------------------- CG (FP64)

// Block sum of v into acc[s] (one atomic per block).
__device__ __forceinline__ void block_sum_to(double v, double* acc) {
  __shared__ double part[kMgThreads / 32];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) part[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = l < (int)(blockDim.x >> 5) ? part[l] : 0.0;
    t = warp_sum(t);
    if (l == 0) atomicAdd(acc, t);
  }
  __syncthreads();
}

// Ap = A p (the stored FP64 stencil in symmetric form), and pAp[s] += p . Ap.
__global__ void __launch_bounds__(kMgThreads) cg_matvec_kernel(int nf, const double* __restrict__ st64,
                                                               const double* __restrict__ p, double* __restrict__ Ap,
                                                               double* __restrict__ pAp) {
  const int s = blockIdx.y;
  const int W = nf + 1, N = W * W;
  const double* C = st64 + (size_t)s * 5 * N;
  const double *E = C + N, *Nn = C + 2 * (size_t)N, *NE = C + 3 * (size_t)N, *NW = C + 4 * (size_t)N;
  const double* ps = p + (size_t)s * N;
  double acc = 0.0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
    const int i = v % W, j = v / W;
    double t = 0.0;
    if (interior(i, j, nf)) {
      const double* q = ps + v;
      t = C[v] * q[0];
      t = fma(E[v], q[1], t);
      t = fma(E[v - 1], q[-1], t);
      t = fma(Nn[v], q[W], t);
      t = fma(Nn[v - W], q[-W], t);
      t = fma(NE[v], q[W + 1], t);
      t = fma(NE[v - W - 1], q[-W - 1], t);
      t = fma(NW[v], q[W - 1], t);
      t = fma(NW[v - W + 1], q[-W + 1], t);
      acc += q[0] * t;
    }
    Ap[(size_t)s * N + v] = t;
  }
  block_sum_to(acc, pAp + s);
}

// Per sample: alpha = rz / pAp (0 once converged or degenerate).
__global__ void cg_alpha_kernel(int S, const double* rz, const double* pAp, const int32_t* done, double* alpha) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S) alpha[s] = (done[s] || !(pAp[s] > 0.0)) ? 0.0 : rz[s] / pAp[s];
}

// x += alpha p, r -= alpha Ap; rr[s] += r . r; the FP32 copy of r for the
// preconditioner.
__global__ void __launch_bounds__(kMgThreads) cg_update_kernel(int nf, const double* __restrict__ alpha,
                                                               const double* __restrict__ p, const double* __restrict__ Ap,
                                                               double* __restrict__ x, double* __restrict__ r,
                                                               float* __restrict__ r32, double* __restrict__ rr) {
  const int s = blockIdx.y;
  const int N = (nf + 1) * (nf + 1);
  const double al = alpha[s];
  double acc = 0.0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
    const size_t q = (size_t)s * N + v;
    x[q] += al * p[q];
    const double rv = r[q] - al * Ap[q];
    r[q] = rv;
    r32[q] = (float)rv;
    acc += rv * rv;
  }
  block_sum_to(acc, rr + s);
}

// rz[s] += r . z (z the FP32 preconditioned residual).
__global__ void __launch_bounds__(kMgThreads) cg_rz_kernel(int nf, const double* __restrict__ r,
                                                           const float* __restrict__ z, double* __restrict__ rz) {
  const int s = blockIdx.y;
  const int N = (nf + 1) * (nf + 1);
  double acc = 0.0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x)
    acc += r[(size_t)s * N + v] * (double)z[(size_t)s * N + v];
  block_sum_to(acc, rz + s);
}

// p = z + beta p, beta = rz_new / rz_old (p = z on the first step, where p
// is not read: the workspace holds whatever it held before).
__global__ void cg_direction_kernel(int nf, const float* __restrict__ z, const double* __restrict__ rz_new,
                                    const double* __restrict__ rz_old, const int32_t* done, int first,
                                    double* __restrict__ p) {
  const int s = blockIdx.y;
  const int N = (nf + 1) * (nf + 1);
  const double beta = (first || done[s] || !(rz_old[s] != 0.0)) ? 0.0 : rz_new[s] / rz_old[s];
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
    const size_t q = (size_t)s * N + v;
    p[q] = done[s] ? 0.0 : first ? (double)z[q] : (double)z[q] + beta * p[q];
  }
}

// r = b (f h^2 at the interior nodes), x = 0, |b|^2 per sample.
__global__ void __launch_bounds__(kMgThreads) cg_init_kernel(int nf, double fh2, double* __restrict__ x,
                                                             double* __restrict__ r, float* __restrict__ r32,
                                                             double* __restrict__ bb) {
  const int s = blockIdx.y;
  const int W = nf + 1, N = W * W;
  double acc = 0.0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
    const int i = v % W, j = v / W;
    const double b = interior(i, j, nf) ? fh2 : 0.0;
    x[(size_t)s * N + v] = 0.0;
    r[(size_t)s * N + v] = b;
    r32[(size_t)s * N + v] = (float)b;
    acc += b * b;
  }
  block_sum_to(acc, bb + s);
}

}  // namespace stomsfem

using namespace stomsfem;

namespace {

// Level sizes: nf_0 = nf halved while even and above 16.
int mg_levels(int nf, int* nfs) {
  int L = 0;
  nfs[L++] = nf;
  while (nfs[L - 1] > 16 && nfs[L - 1] % 2 == 0 && L < kMgMaxLevels) {
    nfs[L] = nfs[L - 1] / 2;
    ++L;
  }
  return L;
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
size_t range_offset(int S) { return (sizeof(double) * 6 * S + sizeof(int32_t) * S + 7) & ~size_t(7); }
size_t scal_bytes(int S) { return range_offset(S) + 2 * sizeof(unsigned long long); }

// Workspace layout of a batch of S samples.
size_t mg_layout(int nf, int S, MgLevel* lv, int* L, unsigned char* base, double** vec, double** scal) {
  int nfs[kMgMaxLevels];
  *L = mg_levels(nf, nfs);
  size_t o = 0;
  for (int l = 0; l < *L; ++l) {
    const size_t N = (size_t)(nfs[l] + 1) * (nfs[l] + 1);
    lv[l].nf = nfs[l];
    lv[l].N = (int)N;
    lv[l].st = reinterpret_cast<float*>(base + o);
    o += al256(sizeof(float) * 5 * N * S);
    lv[l].u = reinterpret_cast<float*>(base + o);
    o += al256(sizeof(float) * N * S);
    lv[l].u2 = reinterpret_cast<float*>(base + o);
    o += al256(sizeof(float) * N * S);
    lv[l].f = reinterpret_cast<float*>(base + o);
    o += al256(sizeof(float) * N * S);
    lv[l].r = reinterpret_cast<float*>(base + o);
    o += al256(sizeof(float) * N * S);
    lv[l].P = reinterpret_cast<float*>(base + o);  // unused on the coarsest level
    o += l + 1 < *L ? al256(sizeof(float) * 4 * N * S) : 0;
    lv[l].dv = reinterpret_cast<float*>(base + o);
    o += al256(sizeof(float) * N * S);
  }
  const size_t N0 = (size_t)(nf + 1) * (nf + 1);
  for (int k = 0; k < 4; ++k) {  // r, p, Ap (x is the caller's u), then the FP64 stencil [S][5][N0]
    vec[k] = reinterpret_cast<double*>(base + o);
    o += al256(sizeof(double) * N0 * S * (k == 3 ? 5 : 1));
  }
  *scal = reinterpret_cast<double*>(base + o);  // alpha, pAp, rz, rz_old, rr, bb [S] doubles, done [S] int,
                                                // then the coefficient range (2 x 8 bytes, 8-aligned)
  o += al256(scal_bytes(S));
  return o;
}

dim3 grid2(int N, int S) {
  const int sms = device_sm_count() > 0 ? device_sm_count() : 152;
  long long bx = (N + kMgThreads - 1) / kMgThreads;
  const long long cap = ((long long)sms * 8 + S - 1) / S;
  if (bx > cap) bx = cap;
  if (bx < 1) bx = 1;
  return dim3((unsigned)bx, (unsigned)S);
}

// z = V-cycle(r) on level l (f of level l holds the right-hand side; the
// result in u of level l).
template <bool OD>
int vcycle(MgLevel* lv, int L, int l, int S, cudaStream_t st) {
  MgLevel& c = lv[l];
  const dim3 g = grid2(c.N, S);
  if (l == L - 1) {
    if (c.N > kMgCoarseMaxNodes) return set_error(STOMSFEM_EINVAL, "coarsest grid of %d nodes", c.N);
    mgf_coarse_kernel<<<S, kMgCoarseThreads, 0, st>>>(c.nf, c.st, c.dv, c.f, c.u);
    return check_cuda(cudaGetLastError(), "coarse sweeps");
  }
  // pre-smoothing from zero
  mgf_jacobi_kernel<OD><<<g, kMgThreads, 0, st>>>(c.nf, c.st, c.dv, c.f, c.u, c.u2, 1);
  mgf_jacobi_kernel<OD><<<g, kMgThreads, 0, st>>>(c.nf, c.st, c.dv, c.f, c.u2, c.u, 0);
  mgf_residual_kernel<<<g, kMgThreads, 0, st>>>(c.nf, c.st, c.f, c.u, c.r);
  MgLevel& n = lv[l + 1];
  mgf_restrict_kernel<OD><<<grid2(n.N, S), kMgThreads, 0, st>>>(c.nf, c.P, c.r, n.f);
  int rc = vcycle<OD>(lv, L, l + 1, S, st);
  if (rc) return rc;
  mgf_prolong_kernel<OD><<<g, kMgThreads, 0, st>>>(c.nf, c.P, n.u, c.u);
  mgf_jacobi_kernel<OD><<<g, kMgThreads, 0, st>>>(c.nf, c.st, c.dv, c.f, c.u, c.u2, 0);
  mgf_jacobi_kernel<OD><<<g, kMgThreads, 0, st>>>(c.nf, c.st, c.dv, c.f, c.u2, c.u, 0);
  return check_cuda(cudaGetLastError(), "v-cycle");
}

}  // namespace

namespace stomsfem {

size_t fine_mg_workspace_bytes(int nf, int S) {
  MgLevel lv[kMgMaxLevels];
  int L;
  double* vec[4];
  double* scal;
  return mg_layout(nf, S, lv, &L, nullptr, vec, &scal);
}

bool fine_mg_supported(int nf) {
  int nfs[kMgMaxLevels];
  const int L = mg_levels(nf, nfs);
  return L >= 2 && nfs[L - 1] <= 16;
}

// u [S][(nf+1)^2] (boundary 0) solves the Q1 system of each sample to
// |r| <= rtol |b|; returns the largest relative residual in *res and the
// iterations in *iters.  Synchronises the stream.
int fine_mg_solve(int nf, double f, const double* a, int S, double* u, void* workspace, size_t workspace_bytes,
                  double rtol, int max_iters, cudaStream_t st, double* res, int* iters) {
  MgLevel lv[kMgMaxLevels];
  int L;
  double* vec[4];
  double* scal;
  const size_t need = mg_layout(nf, S, lv, &L, static_cast<unsigned char*>(workspace), vec, &scal);
  if (workspace_bytes < need)
    return set_error(STOMSFEM_ENOMEM, "fine FEM workspace %zu < %zu bytes", workspace_bytes, need);
  double *r = vec[0], *p = vec[1], *Ap = vec[2], *st64 = vec[3];
  double *alpha = scal, *pAp = scal + S, *rz = scal + 2 * S, *rz_old = scal + 3 * S, *rr = scal + 4 * S,
         *bb = scal + 5 * S;
  int32_t* done = reinterpret_cast<int32_t*>(scal + 6 * S);
  const int N0 = lv[0].N;
  const dim3 g0 = grid2(N0, S);
  unsigned long long* range = reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned char*>(scal) +
                                                                   range_offset(S));
  STOMSFEM_TRY_CUDA(cudaMemsetAsync(scal, 0, scal_bytes(S), st));
  STOMSFEM_TRY_CUDA(cudaMemsetAsync(range + 1, 0x7F, sizeof(unsigned long long), st));
  const int sms = device_sm_count() > 0 ? device_sm_count() : 152;
  mgf_range_kernel<<<sms * 4, kMgThreads, 0, st>>>((long long)S * nf * nf, a, range);
  const double h = 1.0 / nf;
  cg_init_kernel<<<g0, kMgThreads, 0, st>>>(nf, f * h * h, u, r, lv[0].f, bb);
  std::vector<double> hb(S), hr(S);
  std::vector<int32_t> hd(S, 0);
  unsigned long long hrange[2] = {0, 0};
  STOMSFEM_TRY_CUDA(cudaMemcpyAsync(hb.data(), bb, sizeof(double) * S, cudaMemcpyDeviceToHost, st));
  STOMSFEM_TRY_CUDA(cudaMemcpyAsync(hrange, range, sizeof(hrange), cudaMemcpyDeviceToHost, st));
  STOMSFEM_TRY_CUDA(cudaStreamSynchronize(st));
  double amax, amin;
  std::memcpy(&amax, &hrange[0], sizeof(double));
  std::memcpy(&amin, &hrange[1], sizeof(double));
  const bool od = amax > kMgOdContrast * amin;
  // multigrid set-up: stencils of every level
  mgf_fine_stencil_kernel<<<g0, kMgThreads, 0, st>>>(nf, a, lv[0].st, st64);
  for (int l = 0; l + 1 < L; ++l) {
    if (od) {
      mgf_interp_kernel<<<grid2(lv[l].N, S), kMgThreads, 0, st>>>(lv[l].nf, lv[l].st, lv[l].P);
      mgf_rap_kernel<true><<<grid2(lv[l + 1].N, S), kMgThreads, 0, st>>>(lv[l].nf, lv[l].st, lv[l].P,
                                                                          lv[l + 1].st);
    } else {
      mgf_rap_kernel<false><<<grid2(lv[l + 1].N, S), kMgThreads, 0, st>>>(lv[l].nf, lv[l].st, lv[l].P,
                                                                           lv[l + 1].st);
    }
  }
  for (int l = 0; l < L; ++l)
    mgf_divisor_kernel<<<grid2(lv[l].N, S), kMgThreads, 0, st>>>(lv[l].nf, lv[l].st, lv[l].dv);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  auto cycle = [&]() { return od ? vcycle<true>(lv, L, 0, S, st) : vcycle<false>(lv, L, 0, S, st); };
  // z = M r, rz = r . z, p = z
  int rc = cycle();
  if (rc) return rc;
  cg_rz_kernel<<<g0, kMgThreads, 0, st>>>(nf, r, lv[0].u, rz);
  cg_direction_kernel<<<g0, kMgThreads, 0, st>>>(nf, lv[0].u, rz, rz_old, done, 1, p);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  double worst = 1.0;
  int it = 0;
  for (it = 1; it <= max_iters; ++it) {
    STOMSFEM_TRY_CUDA(cudaMemsetAsync(pAp, 0, sizeof(double) * S, st));
    STOMSFEM_TRY_CUDA(cudaMemsetAsync(rr, 0, sizeof(double) * S, st));
    cg_matvec_kernel<<<g0, kMgThreads, 0, st>>>(nf, st64, p, Ap, pAp);
    cg_alpha_kernel<<<(S + 127) / 128, 128, 0, st>>>(S, rz, pAp, done, alpha);
    cg_update_kernel<<<g0, kMgThreads, 0, st>>>(nf, alpha, p, Ap, u, r, lv[0].f, rr);
    STOMSFEM_TRY_CUDA(cudaGetLastError());
    if (it % 4 == 0 || it == max_iters) {
      STOMSFEM_TRY_CUDA(cudaMemcpyAsync(hr.data(), rr, sizeof(double) * S, cudaMemcpyDeviceToHost, st));
      STOMSFEM_TRY_CUDA(cudaStreamSynchronize(st));
      worst = 0.0;
      bool all = true, finite = true;
      for (int s = 0; s < S; ++s) {
        const double rel = hb[s] > 0.0 ? std::sqrt(hr[s] / hb[s]) : 0.0;
        if (!std::isfinite(rel)) finite = false;
        if (rel <= rtol) hd[s] = 1;
        if (!hd[s]) all = false;
        worst = std::max(worst, rel);
      }
      if (!finite)
        return set_error(STOMSFEM_ENOTSPD, "fine FEM CG: non-finite residual after %d iterations", it);
      if (all) break;
      STOMSFEM_TRY_CUDA(cudaMemcpyAsync(done, hd.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice, st));
    }
    rc = cycle();
    if (rc) return rc;
    STOMSFEM_TRY_CUDA(cudaMemcpyAsync(rz_old, rz, sizeof(double) * S, cudaMemcpyDeviceToDevice, st));
    STOMSFEM_TRY_CUDA(cudaMemsetAsync(rz, 0, sizeof(double) * S, st));
    cg_rz_kernel<<<g0, kMgThreads, 0, st>>>(nf, r, lv[0].u, rz);
    cg_direction_kernel<<<g0, kMgThreads, 0, st>>>(nf, lv[0].u, rz, rz_old, done, 0, p);
    STOMSFEM_TRY_CUDA(cudaGetLastError());
  }
  if (res) *res = worst;
  if (iters) *iters = it > max_iters ? max_iters : it;
  if (!(worst <= rtol))
    return set_error(STOMSFEM_ENOTSPD, "fine FEM CG: relative residual %.3e after %d iterations", worst, max_iters);
  return STOMSFEM_OK;
}

}  // namespace stomsfem
