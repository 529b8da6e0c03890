// Fine-grid Q1 FEM for large grids (the level-1 solves of the two-level
// Monte Carlo estimator, Remark in Sec. 4.1.1, Eq. MCmean2level): the
// standard Q1 system on the (nf-1)^2 interior nodes, zero Dirichlet data,
// load f h^2 per node, for a batch of samples, by conjugate gradients in
// FP64 preconditioned with one geometric multigrid V-cycle in FP32.
//
// Multigrid: levels nf_0 = nf, nf_{l+1} = nf_l / 2 down to nf_L <= 16;
// bilinear prolongation P (coarse node (I, J) at fine node (2I, 2J)),
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
#include <vector>

#include "common.cuh"

namespace stomsfem {

constexpr int kMgMaxLevels = 12;
constexpr float kMgOmega = 0.8f;
constexpr int kMgCoarseSweeps = 60;
constexpr int kMgThreads = 256;

struct MgLevel {
  int nf;          // elements per side
  int N;           // (nf + 1)^2 nodes
  float* st;       // [S][5][N]: centre, east, north, north-east, north-west
  float* u;        // [S][N]
  float* u2;       // [S][N] (Jacobi ping-pong)
  float* f;        // [S][N]
  float* r;        // [S][N]
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

// Bilinear prolongation weight of coarse node c at fine coordinate x (1D).
__device__ __forceinline__ float hat(int x, int c2) {
  const int d = abs(x - c2);
  return d == 0 ? 1.f : (d == 1 ? 0.5f : 0.f);
}

// Galerkin coarse stencils A_c = P^T A_f P at the interior coarse nodes.
__global__ void mgf_rap_kernel(int nff, const float* __restrict__ stf, float* __restrict__ stc) {
  const int s = blockIdx.y;
  const int nfc = nff / 2;
  const int Nf = (nff + 1) * (nff + 1), Nc = (nfc + 1) * (nfc + 1);
  const float* sf = stf + (size_t)s * 5 * Nf;
  float* sc = stc + (size_t)s * 5 * Nc;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < Nc; v += gridDim.x * blockDim.x) {
    const int I = v % (nfc + 1), J = v / (nfc + 1);
    float out[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (interior(I, J, nfc)) {
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          const int fx = 2 * I + di, fy = 2 * J + dj;  // fine node in the support of coarse (I, J)
          const float wf = hat(fx, 2 * I) * hat(fy, 2 * J);
          const int fv = fy * (nff + 1) + fx;
          for (int ej = -1; ej <= 1; ++ej)
            for (int ei = -1; ei <= 1; ++ei) {
              const int k = (ej + 1) * 3 + ei + 1;
              const float afv = sf[(size_t)st_arr(k) * Nf + st_node(k, fv, nff + 1)];
              if (afv == 0.f) continue;
              const int gx = fx + ei, gy = fy + ej;  // neighbour fine node
              // coarse nodes (I + cI, J + cJ) whose hats cover (gx, gy)
              for (int cJ = -1; cJ <= 1; ++cJ)
                for (int cI = -1; cI <= 1; ++cI) {
                  const int Ic = I + cI, Jc = J + cJ;
                  if (!interior(Ic, Jc, nfc)) continue;
                  const float pg = hat(gx, 2 * Ic) * hat(gy, 2 * Jc);
                  if (pg != 0.f) out[(cJ + 1) * 3 + cI + 1] += wf * afv * pg;
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

// One damped Jacobi sweep: uo = ui + omega (f - A ui) / diag (zero_in: ui = 0).
__global__ void mgf_jacobi_kernel(int nf, const float* __restrict__ st, const float* __restrict__ f,
                                  const float* __restrict__ ui, float* __restrict__ uo, int zero_in) {
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
      const float d = ss[v];
      const float au = zero_in ? 0.f : apply9(ss, N, v, us, W);
      o = (zero_in ? 0.f : us[v]) + kMgOmega * (fs[v] - au) / d;
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
  float o = in ? 0.f + kMgOmega * (fv - 0.f) / c[4] : 0.f;  // the first sweep, from zero
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
      o = ui[v] + kMgOmega * (fv - t) / c[4];
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
__global__ void mgf_restrict_kernel(int nff, const float* __restrict__ rf, float* __restrict__ fc) {
  const int s = blockIdx.y;
  const int nfc = nff / 2, Wf = nff + 1, Wc = nfc + 1;
  const int Nf = Wf * Wf, Nc = Wc * Wc;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < Nc; v += gridDim.x * blockDim.x) {
    const int I = v % Wc, J = v / Wc;
    float t = 0.f;
    if (interior(I, J, nfc)) {
      const float* r = rf + (size_t)s * Nf + (size_t)(2 * J) * Wf + 2 * I;
      t = r[0] + 0.5f * (r[-1] + r[1] + r[-Wf] + r[Wf]) + 0.25f * (r[-Wf - 1] + r[-Wf + 1] + r[Wf - 1] + r[Wf + 1]);
    }
    fc[(size_t)s * Nc + v] = t;
  }
}

// u_f += P u_c at the interior fine nodes.
__global__ void mgf_prolong_kernel(int nff, const float* __restrict__ uc, float* __restrict__ uf) {
  const int s = blockIdx.y;
  const int nfc = nff / 2, Wf = nff + 1, Wc = nfc + 1;
  const int Nf = Wf * Wf, Nc = Wc * Wc;
  const float* u = uc + (size_t)s * Nc;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < Nf; v += gridDim.x * blockDim.x) {
    const int x = v % Wf, y = v / Wf;
    if (!interior(x, y, nff)) continue;
    const int I0 = x / 2, J0 = y / 2;
    const int I1 = (x & 1) ? I0 + 1 : I0, J1 = (y & 1) ? J0 + 1 : J0;
    const float t = 0.25f * (u[J0 * Wc + I0] + u[J0 * Wc + I1] + u[J1 * Wc + I0] + u[J1 * Wc + I1]);
    uf[(size_t)s * Nf + v] += t;
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
  }
  const size_t N0 = (size_t)(nf + 1) * (nf + 1);
  for (int k = 0; k < 4; ++k) {  // r, p, Ap (x is the caller's u), then the FP64 stencil [S][5][N0]
    vec[k] = reinterpret_cast<double*>(base + o);
    o += al256(sizeof(double) * N0 * S * (k == 3 ? 5 : 1));
  }
  *scal = reinterpret_cast<double*>(base + o);  // alpha, pAp, rz, rz_old, rr, bb [S] doubles, done [S] int
  o += al256(sizeof(double) * 6 * S + sizeof(int32_t) * S);
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
int vcycle(MgLevel* lv, int L, int l, int S, cudaStream_t st) {
  MgLevel& c = lv[l];
  const dim3 g = grid2(c.N, S);
  if (l == L - 1) {
    if (c.N > kMgCoarseMaxNodes) return set_error(STOMSFEM_EINVAL, "coarsest grid of %d nodes", c.N);
    mgf_coarse_kernel<<<S, kMgCoarseThreads, 0, st>>>(c.nf, c.st, c.f, c.u);
    return check_cuda(cudaGetLastError(), "coarse sweeps");
  }
  // pre-smoothing from zero
  mgf_jacobi_kernel<<<g, kMgThreads, 0, st>>>(c.nf, c.st, c.f, c.u, c.u2, 1);
  mgf_jacobi_kernel<<<g, kMgThreads, 0, st>>>(c.nf, c.st, c.f, c.u2, c.u, 0);
  mgf_residual_kernel<<<g, kMgThreads, 0, st>>>(c.nf, c.st, c.f, c.u, c.r);
  MgLevel& n = lv[l + 1];
  mgf_restrict_kernel<<<grid2(n.N, S), kMgThreads, 0, st>>>(c.nf, c.r, n.f);
  int rc = vcycle(lv, L, l + 1, S, st);
  if (rc) return rc;
  mgf_prolong_kernel<<<g, kMgThreads, 0, st>>>(c.nf, n.u, c.u);
  mgf_jacobi_kernel<<<g, kMgThreads, 0, st>>>(c.nf, c.st, c.f, c.u, c.u2, 0);
  mgf_jacobi_kernel<<<g, kMgThreads, 0, st>>>(c.nf, c.st, c.f, c.u2, c.u, 0);
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
  // multigrid set-up: stencils of every level
  mgf_fine_stencil_kernel<<<g0, kMgThreads, 0, st>>>(nf, a, lv[0].st, st64);
  for (int l = 0; l + 1 < L; ++l)
    mgf_rap_kernel<<<grid2(lv[l + 1].N, S), kMgThreads, 0, st>>>(lv[l].nf, lv[l].st, lv[l + 1].st);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  STOMSFEM_TRY_CUDA(cudaMemsetAsync(scal, 0, sizeof(double) * 6 * S + sizeof(int32_t) * S, st));
  const double h = 1.0 / nf;
  cg_init_kernel<<<g0, kMgThreads, 0, st>>>(nf, f * h * h, u, r, lv[0].f, bb);
  std::vector<double> hb(S), hr(S);
  std::vector<int32_t> hd(S, 0);
  STOMSFEM_TRY_CUDA(cudaMemcpyAsync(hb.data(), bb, sizeof(double) * S, cudaMemcpyDeviceToHost, st));
  STOMSFEM_TRY_CUDA(cudaStreamSynchronize(st));
  // z = M r, rz = r . z, p = z
  int rc = vcycle(lv, L, 0, S, st);
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
    rc = vcycle(lv, L, 0, S, st);
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
