// Reduced-basis (POD) upscaling, Sec. 3.2 of the paper.
//
// Offline (Alg. 3, Eq. KLphi), per coarse cell, FP64:
//   phibar_l = training mean of the multiscale basis phi_l (l = 1..4),
//   abar     = training mean of the coefficient on the cell,
//   C        = covariance of the centred interior snapshots (all four l
//              stacked, one shared basis per cell),
//   KL in the energy inner product <u,v> = u^T Abar v (footnote of Eq.
//   KLphi): Abar = R R^T, B = R^T C R = W Lambda W^T (parallel cyclic Jacobi),
//   zeta_q = R^{-T} w_q, kept while sqrt(lambda_q / lambda_1) >= tol,
//   element tensors T_e = W_e^T K_ref W_e of the extended basis
//   Wfull = [phibar_1..4, zeta_1..r] in packed upper-triangle order.
// Online (Alg. 4, Eqs. localRB and localRBsystem), per (sample, cell):
//   G(omega) = Wfull^T A(omega) Wfull = sum_e a_e T_e  -> one GEMM per cell,
//              [samples x elements] x [elements x packed entries], BF16
//              operands, FP32 accumulation in tensor memory (tcgen05);
//   (V^T A V) c_l = -V^T A phibar_l: r x r FP32 Cholesky in a warp;
//   optional FP64 refinement: residual through the fine 9-point stencil;
//   K_e = a(phibar + V c, phibar + V c), b_e = f int (phibar + V c).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "ckpt.cuh"
#include "common.cuh"
#include "tc_gemm.cuh"

namespace stomsfem {

constexpr int kPodMaxRhoSmall = 8;  // the covariance eigensolver, refinement, affine and per-l bases
constexpr int kPodMaxRho = 32;      // elements per cell side (1024 elements: 16 K steps of 64)
constexpr int kPodMaxN = 49;        // interior nodes of a small cell, (rho - 1)^2
constexpr int kPodSnapMax = 96;     // large cells: snapshot columns (4 x training samples)
constexpr int kPodMaxRank = 27;    // (4 + r)(5 + r)/2 <= 496 packed entries fit 512 TMEM columns
constexpr int kPodK = 64;          // elements per GEMM K step (one 128-byte BF16 row)
constexpr int kPodTileM = 128;
constexpr int kPodAffParts = 17;   // affine parts: the constant one and up to 16 local parameters

__device__ __forceinline__ int pidx(int a, int b, int P0) {
  // packed upper-triangle index of (a, b), a <= b < P0
  return a * P0 - (a * (a - 1)) / 2 + (b - a);
}

__device__ __constant__ double kKref[4][4] = {{4.0 / 6, -1.0 / 6, -2.0 / 6, -1.0 / 6},
                                              {-1.0 / 6, 4.0 / 6, -1.0 / 6, -2.0 / 6},
                                              {-2.0 / 6, -1.0 / 6, 4.0 / 6, -1.0 / 6},
                                              {-1.0 / 6, -2.0 / 6, -1.0 / 6, 4.0 / 6}};

struct PodDims {
  int nf, nc, rho, N2, n, ne, P0, P, Ppad, ncell;
  double f;
  int per_l;  // 1: one basis per basis function l = 1..3 (columns 4 + l * rcl ..), else one shared basis
  int rcl;    // per-l: the column block of each basis (its rank cap)
  int Kp;     // GEMM K: the cell's elements rounded up to kPodK
};

__host__ __device__ inline int pod_kp(int ne) { return (ne + kPodK - 1) / kPodK * kPodK; }

// Number of reduced unknowns a solve lane set spans: r (shared basis) or
// 3 blocks of rcl (per-l bases).
__host__ __device__ inline int pod_vcols(const PodDims& d) { return d.P0 - 4; }

// ------------------------------------------------------------------ offline

// phibar[cell][4][N2], abar[cell][ne]
__global__ void pod_mean_kernel(PodDims d, const double* __restrict__ phi, const double* __restrict__ a,
                                int Ns, double* __restrict__ phibar, double* __restrict__ abar) {
  const int cell = blockIdx.x;
  const int cx = cell % d.nc, cy = cell / d.nc;
  for (int q = threadIdx.x; q < 4 * d.N2; q += blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < Ns; ++t) s += phi[((size_t)t * d.ncell + cell) * 4 * d.N2 + q];
    phibar[(size_t)cell * 4 * d.N2 + q] = s / Ns;
  }
  for (int e = threadIdx.x; e < d.ne; e += blockDim.x) {
    const int ex = e % d.rho, ey = e / d.rho;
    double s = 0.0;
    for (int t = 0; t < Ns; ++t) s += a[((size_t)t * d.nf + cy * d.rho + ey) * d.nf + cx * d.rho + ex];
    abar[(size_t)cell * d.ne + e] = s / Ns;
  }
}

// interior node q (0..n-1) -> cell node index
__device__ __forceinline__ int inner_node(int q, int rho) {
  const int m = rho - 1;
  const int j = q / m + 1, i = q % m + 1;
  return j * (rho + 1) + i;
}

// Covariance of the centred interior snapshots: cov[cell][n][n].
__global__ void pod_cov_kernel(PodDims d, const double* __restrict__ phi, int Ns,
                               const double* __restrict__ phibar, double* __restrict__ cov) {
  const int cell = blockIdx.x;
  const int n = d.n;
  const double* pb = phibar + (size_t)cell * 4 * d.N2;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    if (j < i) continue;
    const int vi = inner_node(i, d.rho), vj = inner_node(j, d.rho);
    double s = 0.0;
    for (int t = 0; t < Ns; ++t) {
      const double* ph = phi + ((size_t)t * d.ncell + cell) * 4 * d.N2;
#pragma unroll
      for (int l = 0; l < 4; ++l) s += (ph[l * d.N2 + vi] - pb[l * d.N2 + vi]) * (ph[l * d.N2 + vj] - pb[l * d.N2 + vj]);
    }
    s /= (4.0 * Ns);
    cov[((size_t)cell * n + i) * n + j] = s;
    cov[((size_t)cell * n + j) * n + i] = s;
  }
}

// Per-l bases: covariance of the centred interior snapshots of phi_l alone,
// cov[cell][l][n][n] for l = 0..2 (blockIdx.y = l).
__global__ void pod_cov_per_l_kernel(PodDims d, const double* __restrict__ phi, int Ns,
                                     const double* __restrict__ phibar, double* __restrict__ cov) {
  const int cell = blockIdx.x, l = blockIdx.y;
  const int n = d.n;
  const double* pb = phibar + (size_t)cell * 4 * d.N2 + (size_t)l * d.N2;
  double* C = cov + ((size_t)cell * 3 + l) * n * n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    if (j < i) continue;
    const int vi = inner_node(i, d.rho), vj = inner_node(j, d.rho);
    double s = 0.0;
    for (int t = 0; t < Ns; ++t) {
      const double* ph = phi + ((size_t)t * d.ncell + cell) * 4 * d.N2 + (size_t)l * d.N2;
      s += (ph[vi] - pb[vi]) * (ph[vj] - pb[vj]);
    }
    s /= (double)Ns;
    C[i * n + j] = s;
    C[j * n + i] = s;
  }
}

// W[cell][N2][P0] = [phibar_1..4, 0 ...] (the per-l eigen blocks then write
// their own columns).
__global__ void pod_w_init_kernel(PodDims d, const double* __restrict__ phibar, double* __restrict__ W) {
  const int cell = blockIdx.x;
  double* Wc = W + (size_t)cell * d.N2 * d.P0;
  for (int idx = threadIdx.x; idx < d.N2 * d.P0; idx += blockDim.x) {
    const int node = idx / d.P0, col = idx % d.P0;
    Wc[idx] = col < 4 ? phibar[(size_t)cell * 4 * d.N2 + col * d.N2 + node] : 0.0;
  }
}

// Parallel cyclic Jacobi on the symmetric ne2 x ne2 matrix B (ne2 even,
// row stride ld, shared memory), eigenvectors accumulated into the columns
// of Z (initialised here to the identity): round-robin pairs (position 0
// fixed, the others rotating), at most 40 sweeps, stopping when the
// off-diagonal mass falls below 1e-30 of the diagonal's.  Every thread of
// the CTA takes part; cs and pairs hold ne2 / 2 entries, offn one.
__device__ void pod_jacobi(double* B, double* Z, int ld, int ne2, double (*cs)[2], int (*pairs)[2],
                           double* offn) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < ne2 * ne2; idx += nt) {
    const int i = idx / ne2, j = idx % ne2;
    Z[i * ld + j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  const int np = ne2 / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (tid == 0) {
      double off = 0.0, dia = 0.0;
      for (int i = 0; i < ne2; ++i)
        for (int j = 0; j < ne2; ++j) (i == j ? dia : off) += B[i * ld + j] * B[i * ld + j];
      *offn = (off <= 1e-30 * dia) ? -1.0 : off;
    }
    __syncthreads();
    if (*offn < 0.0) break;
    for (int rnd = 0; rnd < ne2 - 1; ++rnd) {
      for (int k = tid; k < np; k += nt) {
        int a = (k == 0) ? 0 : 1 + (k - 1 + rnd) % (ne2 - 1);
        int b = 1 + (ne2 - 2 - k + rnd) % (ne2 - 1);
        if (a > b) { const int t = a; a = b; b = t; }
        pairs[k][0] = a;
        pairs[k][1] = b;
        const double app = B[a * ld + a], aqq = B[b * ld + b], apq = B[a * ld + b];
        double c = 1.0, sn = 0.0;
        if (fabs(apq) > 1e-300) {
          const double th = (aqq - app) / (2.0 * apq);
          const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
          sn = t * c;
        }
        cs[k][0] = c;
        cs[k][1] = sn;
      }
      __syncthreads();
      // rows: B[a,:], B[b,:]
      for (int idx = tid; idx < np * ne2; idx += nt) {
        const int k = idx / ne2, j = idx % ne2;
        const int a = pairs[k][0], b = pairs[k][1];
        const double c = cs[k][0], sn = cs[k][1];
        const double x = B[a * ld + j], y = B[b * ld + j];
        B[a * ld + j] = c * x - sn * y;
        B[b * ld + j] = sn * x + c * y;
      }
      __syncthreads();
      // columns: B[:,a], B[:,b] and the vectors Z[:,a], Z[:,b]
      for (int idx = tid; idx < np * ne2; idx += nt) {
        const int k = idx / ne2, i = idx % ne2;
        const int a = pairs[k][0], b = pairs[k][1];
        const double c = cs[k][0], sn = cs[k][1];
        const double x = B[i * ld + a], y = B[i * ld + b];
        B[i * ld + a] = c * x - sn * y;
        B[i * ld + b] = sn * x + c * y;
        const double zx = Z[i * ld + a], zy = Z[i * ld + b];
        Z[i * ld + a] = c * zx - sn * zy;
        Z[i * ld + b] = sn * zx + c * zy;
      }
      __syncthreads();
    }
  }
}

// One CTA per cell (and, per-l, per basis function blockIdx.y): energy
// metric, KL eigenproblem, rank, basis.
//   W [cell][N2][P0]: columns 0..3 = phibar_l, 4..4+r-1 = zeta_q (0 on the
//   boundary), the rest 0.  lam [cell][n] eigenvalues, descending.
__global__ void pod_eig_kernel(PodDims d, const double* __restrict__ cov,
                               const double* __restrict__ phibar, const double* __restrict__ abar,
                               double tol, int max_rank, const int32_t* __restrict__ ranks_in,
                               double* __restrict__ W, double* __restrict__ lam_out,
                               int32_t* __restrict__ ranks_out, int32_t* __restrict__ err) {
  // per-l: problem (cell, l) = rank / eigenvalue slot cell * 3 + l, basis
  // columns from 4 + l * rcl; shared: slot cell, columns from 4
  const int l_blk = d.per_l ? (int)blockIdx.y : 0;
  const int slot_id = d.per_l ? (int)blockIdx.x * 3 + l_blk : (int)blockIdx.x;
  const int col0 = 4 + l_blk * (d.per_l ? d.rcl : 0);
  extern __shared__ double eig_smem[];  // three (kPodMaxN+1)^2 matrices
  typedef double Mat[kPodMaxN + 1];
  Mat* R = reinterpret_cast<Mat*>(eig_smem);
  Mat* B = R + (kPodMaxN + 1);
  Mat* Z = B + (kPodMaxN + 1);
  __shared__ double cs[(kPodMaxN + 1) / 2][2];
  __shared__ int pairs[(kPodMaxN + 1) / 2][2];
  __shared__ int order[kPodMaxN + 1];
  __shared__ double offn;
  __shared__ int s_rank;
  const int cell = blockIdx.x;
  const int n = d.n, rho = d.rho, m = rho - 1;
  const int ne2 = (n + 1) & ~1;  // even size for the round-robin ordering
  const int tid = threadIdx.x, nt = blockDim.x;
  // --- Abar on the interior nodes (dense), into R
  for (int idx = tid; idx < ne2 * ne2; idx += nt) R[idx / ne2][idx % ne2] = 0.0;
  __syncthreads();
  if (tid == 0) {
    for (int ey = 0; ey < rho; ++ey)
      for (int ex = 0; ex < rho; ++ex) {
        const double ae = abar[(size_t)cell * d.ne + ey * rho + ex];
        const int ci[4] = {ex, ex + 1, ex + 1, ex}, cj[4] = {ey, ey, ey + 1, ey + 1};
        for (int r = 0; r < 4; ++r) {
          if (ci[r] <= 0 || ci[r] >= rho || cj[r] <= 0 || cj[r] >= rho) continue;
          const int qr = (cj[r] - 1) * m + ci[r] - 1;
          for (int c = 0; c < 4; ++c) {
            if (ci[c] <= 0 || ci[c] >= rho || cj[c] <= 0 || cj[c] >= rho) continue;
            R[qr][(cj[c] - 1) * m + ci[c] - 1] += ae * kKref[r][c];
          }
        }
      }
  }
  __syncthreads();
  // --- Cholesky Abar = R R^T (lower, in place)
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      const double v = R[k][k];
      if (!(v > 0.0)) atomicOr(err, 1);
      R[k][k] = sqrt(v > 0.0 ? v : 1.0);
    }
    __syncthreads();
    for (int i = k + 1 + tid; i < n; i += nt) R[i][k] /= R[k][k];
    __syncthreads();
    for (int idx = tid; idx < (n - k - 1) * (n - k - 1); idx += nt) {
      const int i = k + 1 + idx / (n - k - 1), j = k + 1 + idx % (n - k - 1);
      if (j <= i) R[i][j] -= R[i][k] * R[j][k];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < ne2 * ne2; idx += nt) {
    const int i = idx / ne2, j = idx % ne2;
    if (j > i || i >= n) R[i][j] = (i == j && i >= n) ? 1.0 : (j > i ? 0.0 : R[i][j]);
  }
  __syncthreads();
  // --- B = R^T C R: Z = C R, then B = R^T Z
  const double* C = cov + (size_t)slot_id * n * n;
  for (int idx = tid; idx < ne2 * ne2; idx += nt) {
    const int i = idx / ne2, j = idx % ne2;
    double s = 0.0;
    if (i < n && j < n)
      for (int k = j; k < n; ++k) s += C[i * n + k] * R[k][j];
    Z[i][j] = s;
  }
  __syncthreads();
  for (int idx = tid; idx < ne2 * ne2; idx += nt) {
    const int i = idx / ne2, j = idx % ne2;
    double s = 0.0;
    for (int k = i; k < n; ++k) s += R[k][i] * Z[k][j];
    B[i][j] = s;
  }
  __syncthreads();
  // --- parallel cyclic Jacobi with round-robin pairs; Z accumulates vectors
  pod_jacobi(&B[0][0], &Z[0][0], kPodMaxN + 1, ne2, cs, pairs, &offn);
  // --- order eigenvalues (descending) among the n real ones
  for (int i = tid; i < n; i += nt) {
    int rank = 0;
    for (int j = 0; j < n; ++j)
      if (B[j][j] > B[i][i] || (B[j][j] == B[i][i] && j < i)) ++rank;
    order[rank] = i;
  }
  __syncthreads();
  if (tid == 0) {
    int r;
    if (ranks_in) {
      r = ranks_in[slot_id];
    } else {
      const double l1 = B[order[0]][order[0]] > 0 ? B[order[0]][order[0]] : 1.0;
      r = 0;
      while (r < n && sqrt(fmax(B[order[r]][order[r]], 0.0) / l1) >= tol) ++r;
    }
    if (r > max_rank) r = max_rank;
    if (r < 1) r = 1;
    if (r > n) r = n;
    s_rank = r;
    ranks_out[slot_id] = r;
  }
  for (int i = tid; i < n; i += nt) lam_out[(size_t)slot_id * n + i] = B[order[i]][order[i]];
  __syncthreads();
  const int r = s_rank;
  // --- zeta_q = R^{-T} w_q (back substitution with the upper factor R^T)
  double* Wc = W + (size_t)cell * d.N2 * d.P0;
  if (!d.per_l) {  // per-l: pod_w_init_kernel wrote phibar and the zeros
    for (int idx = tid; idx < d.N2 * d.P0; idx += nt) {
      const int node = idx / d.P0, col = idx % d.P0;
      Wc[idx] = col < 4 ? phibar[(size_t)cell * 4 * d.N2 + col * d.N2 + node] : 0.0;
    }
    __syncthreads();
  }
  for (int q = tid; q < r; q += nt) {
    const int src = order[q];
    // x = R^{-T} w: solve R^T x = w from the last row up
    for (int i = n - 1; i >= 0; --i) {
      double s = Z[i][src];
      for (int k = i + 1; k < n; ++k) s -= R[k][i] * Wc[(size_t)inner_node(k, rho) * d.P0 + col0 + q];
      Wc[(size_t)inner_node(i, rho) * d.P0 + col0 + q] = s / R[i][i];
    }
  }
}

// ---- large cells (H/h > 8): the KL eigenproblem in snapshot space.
// With X the m = 4 Ns centred interior snapshots (columns t * 4 + l) and
// Abar the training-mean energy matrix, the covariance C = X X^T / m and
// the snapshot matrix M = X^T Abar X / m have the same nonzero eigenvalues
// in the energy inner product (B = R^T C R and M = Y^T Y with Y = R^T X /
// sqrt(m), Abar = R R^T), and M v = lambda v gives the Abar-orthonormal mode
// zeta = X v / sqrt(m lambda) = R^-T (Y v / sqrt(lambda)): the m x m problem
// replaces the n x n one (n = 961 at H/h = 32).

// X[cell][i][j] and Y = Abar X (the training-mean 9-point stencil applied to
// the centred snapshots, zero on the cell boundary), FP64.
__global__ void pod_snap_xy_kernel(PodDims d, const double* __restrict__ phi, int Ns,
                                   const double* __restrict__ phibar, const double* __restrict__ abar,
                                   double* __restrict__ X, double* __restrict__ Y) {
  const int cell = blockIdx.x;
  const int rho = d.rho, NN = rho + 1, m = 4 * Ns;
  const double* pb = phibar + (size_t)cell * 4 * d.N2;
  const double* ab = abar + (size_t)cell * d.ne;
  auto xc = [&](int t, int l, int ix, int iy) -> double {  // centred value, 0 on the boundary
    if (ix <= 0 || iy <= 0 || ix >= rho || iy >= rho) return 0.0;
    const int node = iy * NN + ix;
    return phi[((size_t)t * d.ncell + cell) * 4 * d.N2 + (size_t)l * d.N2 + node] - pb[(size_t)l * d.N2 + node];
  };
  for (int idx = threadIdx.x; idx < d.n * m; idx += blockDim.x) {
    const int i = idx / m, j = idx % m, t = j >> 2, l = j & 3;
    const int ix = i % (rho - 1) + 1, iy = i / (rho - 1) + 1;
    double y = 0.0;
    // the four elements around the node; r = the node's corner in each
    for (int ey = iy - 1; ey <= iy; ++ey)
      for (int ex = ix - 1; ex <= ix; ++ex) {
        const int cx[4] = {ex, ex + 1, ex + 1, ex}, cy[4] = {ey, ey, ey + 1, ey + 1};
        const int r = (ix == ex ? (iy == ey ? 0 : 3) : (iy == ey ? 1 : 2));
        double t4 = 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) t4 += kKref[r][c] * xc(t, l, cx[c], cy[c]);
        y += ab[ey * rho + ex] * t4;
      }
    X[((size_t)cell * d.n + i) * m + j] = xc(t, l, ix, iy);
    Y[((size_t)cell * d.n + i) * m + j] = y;
  }
}

// One CTA per cell: M = X^T Y / m (upper triangle, mirrored: Abar is
// symmetric, so M is up to rounding) in shared memory, its
// eigenpairs (pod_jacobi), rank, eigenvalues (lam [cell][n], descending,
// zero past m), and W = [phibar_1..4, zeta_1..r, 0 ...].
__global__ void pod_snap_eig_kernel(PodDims d, const double* __restrict__ X, const double* __restrict__ Y, int Ns,
                                    const double* __restrict__ phibar, double tol, int max_rank,
                                    const int32_t* __restrict__ ranks_in, double* __restrict__ W,
                                    double* __restrict__ lam_out, int32_t* __restrict__ ranks_out) {
  constexpr int LD = kPodSnapMax + 1;
  extern __shared__ double snap_smem[];
  double* B = snap_smem;       // [m][LD]
  double* Z = B + kPodSnapMax * LD;
  __shared__ double cs[kPodSnapMax / 2][2];
  __shared__ int pairs[kPodSnapMax / 2][2];
  __shared__ int order[kPodSnapMax];
  __shared__ double offn, s_scale[kPodSnapMax];
  __shared__ int s_rank;
  const int cell = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int m = 4 * Ns, n = d.n;
  const double* Xc = X + (size_t)cell * n * m;
  const double* Yc = Y + (size_t)cell * n * m;
  for (int idx = tid; idx < m * m; idx += nt) {
    const int j = idx / m, k = idx % m;
    if (k < j) continue;
    double sxy = 0.0;
    for (int i = 0; i < n; ++i) sxy += Xc[(size_t)i * m + j] * Yc[(size_t)i * m + k];
    const double v = sxy / m;
    B[j * LD + k] = v;
    B[k * LD + j] = v;
  }
  __syncthreads();
  pod_jacobi(B, Z, LD, m, cs, pairs, &offn);
  for (int i = tid; i < m; i += nt) {
    int rank = 0;
    for (int j = 0; j < m; ++j)
      if (B[j * LD + j] > B[i * LD + i] || (B[j * LD + j] == B[i * LD + i] && j < i)) ++rank;
    order[rank] = i;
  }
  __syncthreads();
  if (tid == 0) {
    int r;
    if (ranks_in) {
      r = ranks_in[cell];
    } else {
      const double l1 = B[order[0] * LD + order[0]] > 0 ? B[order[0] * LD + order[0]] : 1.0;
      r = 0;
      while (r < m && sqrt(fmax(B[order[r] * LD + order[r]], 0.0) / l1) >= tol) ++r;
    }
    if (r > max_rank) r = max_rank;
    if (r > m) r = m;
    if (r < 1) r = 1;
    s_rank = r;
    ranks_out[cell] = r;
  }
  for (int i = tid; i < n; i += nt) lam_out[(size_t)cell * n + i] = i < m ? B[order[i] * LD + order[i]] : 0.0;
  __syncthreads();
  const int r = s_rank;
  // 1 / sqrt(m lambda) per kept mode (a non-positive eigenvalue, only
  // reachable through pinned ranks, gives a zero column)
  for (int q = tid; q < r; q += nt) {
    const double lq = B[order[q] * LD + order[q]];
    s_scale[q] = lq > 0.0 ? 1.0 / sqrt((double)m * lq) : 0.0;
  }
  __syncthreads();
  double* Wc = W + (size_t)cell * d.N2 * d.P0;
  const int rho = d.rho, NN = rho + 1;
  for (int idx = tid; idx < d.N2 * d.P0; idx += nt) {
    const int node = idx / d.P0, col = idx % d.P0;
    double v = 0.0;
    if (col < 4) {
      v = phibar[(size_t)cell * 4 * d.N2 + (size_t)col * d.N2 + node];
    } else if (col - 4 < r) {
      const int ix = node % NN, iy = node / NN;
      if (ix > 0 && iy > 0 && ix < rho && iy < rho) {
        const int i = (iy - 1) * (rho - 1) + (ix - 1), src = order[col - 4];
        for (int j = 0; j < m; ++j) v += Xc[(size_t)i * m + j] * Z[j * LD + src];
        v *= s_scale[col - 4];
      }
    }
    Wc[idx] = v;
  }
}

// Large cells: T[cell][j][e] = Wfull_e,alpha^T K_ref Wfull_e,beta (packed pair
// j = (alpha, beta)) in BF16, from FP32 products (the BF16 rounding of T is
// far above their error), 64 elements at a time: the corner values w and
// K_ref w of the block's elements staged in shared memory, each thread
// writing consecutive elements of one pair (coalesced rows).  The load
// terms wl as in pod_tensor_kernel (FP64).
__global__ void pod_tensor_large_kernel(PodDims d, const double* __restrict__ W, __nv_bfloat16* __restrict__ T,
                                        __nv_bfloat16* __restrict__ Tlo, double* __restrict__ wl) {
  extern __shared__ float tl_smem[];
  float* w = tl_smem;                       // [64][4][P0]
  float* kw = tl_smem + kPodK * 4 * d.P0;   // [64][4][P0]
  __shared__ int s_a[512], s_b[512];
  const int cell = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const double* Wc = W + (size_t)cell * d.N2 * d.P0;
  const int rho = d.rho, P0 = d.P0;
  for (int j = tid; j < d.P; j += nt) {
    int a = 0, rem = j;
    while (rem >= P0 - a) { rem -= P0 - a; ++a; }
    s_a[j] = a;
    s_b[j] = a + rem;
  }
  for (int e0 = 0; e0 < d.Kp; e0 += kPodK) {
    __syncthreads();
    for (int idx = tid; idx < kPodK * P0; idx += nt) {
      const int el = idx / P0, al = idx % P0, e = e0 + el;
      float c4[4] = {0.f, 0.f, 0.f, 0.f};
      if (e < d.ne) {
        const int ex = e % rho, ey = e / rho;
        const int nodes[4] = {ey * (rho + 1) + ex, ey * (rho + 1) + ex + 1, (ey + 1) * (rho + 1) + ex + 1,
                              (ey + 1) * (rho + 1) + ex};
#pragma unroll
        for (int r = 0; r < 4; ++r) c4[r] = (float)Wc[(size_t)nodes[r] * P0 + al];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        float k = 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) k = fmaf((float)kKref[r][c], c4[c], k);
        w[(el * 4 + r) * P0 + al] = c4[r];
        kw[(el * 4 + r) * P0 + al] = k;
      }
    }
    __syncthreads();
    for (int idx = tid; idx < d.Ppad * kPodK; idx += nt) {
      const int j = idx / kPodK, el = idx % kPodK;
      float v = 0.f;
      if (j < d.P) {
        const int a = s_a[j], b = s_b[j];
#pragma unroll
        for (int r = 0; r < 4; ++r) v = fmaf(w[(el * 4 + r) * P0 + a], kw[(el * 4 + r) * P0 + b], v);
      }
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      T[((size_t)cell * d.Ppad + j) * d.Kp + e0 + el] = hi;
      Tlo[((size_t)cell * d.Ppad + j) * d.Kp + e0 + el] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
  }
  const double h = 1.0 / d.nf;
  for (int al = tid; al < P0; al += nt) {
    double s = 0.0;
    for (int ey = 0; ey < rho; ++ey)
      for (int ex = 0; ex < rho; ++ex)
        s += Wc[(size_t)(ey * (rho + 1) + ex) * P0 + al] + Wc[(size_t)(ey * (rho + 1) + ex + 1) * P0 + al] +
             Wc[(size_t)((ey + 1) * (rho + 1) + ex + 1) * P0 + al] + Wc[(size_t)((ey + 1) * (rho + 1) + ex) * P0 + al];
    wl[(size_t)cell * P0 + al] = d.f * h * h / 4.0 * s;
  }
}

// T[cell][j][e] (BF16, K-major rows of Kp = 64 elements: small cells) and the load terms
// wl[cell][alpha] = f int Wfull_alpha.
__global__ void pod_tensor_kernel(PodDims d, const double* __restrict__ W, __nv_bfloat16* __restrict__ T,
                                  __nv_bfloat16* __restrict__ Tlo, double* __restrict__ wl) {
  const int cell = blockIdx.x;
  const double* Wc = W + (size_t)cell * d.N2 * d.P0;
  const int rho = d.rho;
  for (int idx = threadIdx.x; idx < d.Ppad * d.Kp; idx += blockDim.x) {
    const int j = idx / d.Kp, e = idx % d.Kp;
    double v = 0.0;
    if (j < d.P && e < d.ne) {
      // invert the packed index
      int a = 0, rem = j;
      while (rem >= d.P0 - a) { rem -= d.P0 - a; ++a; }
      const int b = a + rem;
      const int ex = e % rho, ey = e / rho;
      const int nodes[4] = {ey * (rho + 1) + ex, ey * (rho + 1) + ex + 1, (ey + 1) * (rho + 1) + ex + 1,
                            (ey + 1) * (rho + 1) + ex};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const double wa = Wc[(size_t)nodes[r] * d.P0 + a];
#pragma unroll
        for (int c = 0; c < 4; ++c) v += wa * kKref[r][c] * Wc[(size_t)nodes[c] * d.P0 + b];
      }
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
    T[((size_t)cell * d.Ppad + j) * d.Kp + e] = hi;
    Tlo[((size_t)cell * d.Ppad + j) * d.Kp + e] = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
  }
  const double h = 1.0 / d.nf;
  for (int al = threadIdx.x; al < d.P0; al += blockDim.x) {
    double s = 0.0;
    for (int ey = 0; ey < rho; ++ey)
      for (int ex = 0; ex < rho; ++ex)
        s += Wc[(size_t)(ey * (rho + 1) + ex) * d.P0 + al] + Wc[(size_t)(ey * (rho + 1) + ex + 1) * d.P0 + al] +
             Wc[(size_t)((ey + 1) * (rho + 1) + ex + 1) * d.P0 + al] + Wc[(size_t)((ey + 1) * (rho + 1) + ex) * d.P0 + al];
    wl[(size_t)cell * d.P0 + al] = d.f * h * h / 4.0 * s;
  }
}

// Affine parts of the reduced quantities (Eq. localAF): for the packed
// pair j = (alpha, beta) of W = [phibar_1..4, V],
//   Gaff[cell][0][j] = sum_e Wfull_e,alpha^T K_ref Wfull_e,beta,
//   Gaff[cell][k][j] = sum_e psi_k(x_e) Wfull_e,alpha^T K_ref Wfull_e,beta,
// psi_k the k-th local bump at the element centroids (zero past the
// cell's local parameters).  FP64 sums, stored in FP32.
__global__ void pod_affine_parts_kernel(PodDims d, const double* __restrict__ W, const double* __restrict__ psi,
                                        float* __restrict__ Gaff) {
  const int cell = blockIdx.x;
  const double* Wc = W + (size_t)cell * d.N2 * d.P0;
  const double* pc = psi + (size_t)cell * 16 * kPodK;
  const int rho = d.rho;
  for (int j = threadIdx.x; j < d.Ppad; j += blockDim.x) {
    double acc[kPodAffParts];
#pragma unroll
    for (int k = 0; k < kPodAffParts; ++k) acc[k] = 0.0;
    if (j < d.P) {
      int a = 0, rem = j;
      while (rem >= d.P0 - a) { rem -= d.P0 - a; ++a; }
      const int b = a + rem;
      for (int e = 0; e < d.ne; ++e) {
        const int ex = e % rho, ey = e / rho;
        const int nodes[4] = {ey * (rho + 1) + ex, ey * (rho + 1) + ex + 1, (ey + 1) * (rho + 1) + ex + 1,
                              (ey + 1) * (rho + 1) + ex};
        double t = 0.0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const double wa = Wc[(size_t)nodes[r] * d.P0 + a];
#pragma unroll
          for (int c = 0; c < 4; ++c) t += wa * kKref[r][c] * Wc[(size_t)nodes[c] * d.P0 + b];
        }
        acc[0] += t;
#pragma unroll
        for (int k = 1; k < kPodAffParts; ++k) acc[k] += pc[(size_t)(k - 1) * kPodK + e] * t;
      }
    }
#pragma unroll
    for (int k = 0; k < kPodAffParts; ++k) Gaff[((size_t)cell * kPodAffParts + k) * d.Ppad + j] = (float)acc[k];
  }
}

// ------------------------------------------------------------------ online

// a [S][nf][nf] -> Ab [cell][Spad][Kp] BF16 and its remainder Ablo = BF16(a -
// Ab) (zero padded rows and columns)
__global__ void pod_gather_kernel(PodDims d, const double* __restrict__ a, int S, int Spad,
                                  __nv_bfloat16* __restrict__ Ab, __nv_bfloat16* __restrict__ Ablo) {
  const long long total = (long long)d.ncell * Spad * d.Kp;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(idx % d.Kp);
    const long long t = idx / d.Kp;
    const int s = (int)(t % Spad), cell = (int)(t / Spad);
    float v = 0.f;
    if (s < S && e < d.ne) {
      const int cx = cell % d.nc, cy = cell / d.nc, ex = e % d.rho, ey = e / d.rho;
      v = (float)a[((size_t)s * d.nf + cy * d.rho + ey) * d.nf + cx * d.rho + ex];
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    Ab[idx] = hi;
    Ablo[idx] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

constexpr uint32_t kWaitLimit = 1u << 24;  // about 2 s

// G[cell][s][j] = sum_e Ab[cell][s][e] T[cell][j][e]: one CTA per (128-sample
// tile, cell); the K dimension (the cell's elements, Kp of them) in steps of
// 64: the operands' step staged into 128-byte-swizzled shared memory, 4
// MMAs of K = 16 per N-chunk of <= 256 into one TMEM accumulator, and the
// step's completion awaited (bounded) on an mbarrier before the next step
// overwrites the buffers.  split: both operands as BF16 pairs (hi, lo =
// BF16 of the remainder) and three products per step, Ab T + Ab Tlo + Ablo
// T (the dropped Ablo Tlo is below 2^-16 relative), so G carries about
// 16 bits instead of BF16's 8; one product otherwise.
__global__ void __launch_bounds__(128, 1)
pod_gemm_kernel(PodDims d, int Spad, const __nv_bfloat16* __restrict__ Ab, const __nv_bfloat16* __restrict__ Ablo,
                const __nv_bfloat16* __restrict__ T, const __nv_bfloat16* __restrict__ Tlo, int split,
                float* __restrict__ G, int32_t* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // sA[0..1]: 128 rows x 128 B each; sB[0..1]: Ppad rows x 128 B each
  unsigned char* sA[2] = {smem, smem + kPodTileM * 128};
  unsigned char* sB[2] = {smem + 2 * kPodTileM * 128, smem + 2 * kPodTileM * 128 + (size_t)d.Ppad * 128};
  __shared__ uint64_t mbar;
  __shared__ uint32_t taddr_s;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cell = blockIdx.y;
  const int s0 = blockIdx.x * kPodTileM;
  const int nk = d.Kp / kPodK;
  const int rowv = d.Kp / 8;  // 16-byte chunks per operand row
  const int nparts = split ? 2 : 1;
  uint32_t ncols = 32;
  while ((int)ncols < d.Ppad) ncols <<= 1;
  if (warp == 0) tc::tmem_alloc(&taddr_s, ncols);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  const uint4* gA[2] = {reinterpret_cast<const uint4*>(Ab + ((size_t)cell * Spad + s0) * d.Kp),
                        reinterpret_cast<const uint4*>(Ablo + ((size_t)cell * Spad + s0) * d.Kp)};
  const uint4* gB[2] = {reinterpret_cast<const uint4*>(T + (size_t)cell * d.Ppad * d.Kp),
                        reinterpret_cast<const uint4*>(Tlo + (size_t)cell * d.Ppad * d.Kp)};
  bool ok = true;
  uint32_t taddr = 0;
  for (int kc = 0; kc < nk; ++kc) {
    // stage K step kc: 16-byte asynchronous copies into the swizzled layout
    // (every thread's copies in flight at once), then wait for them
    for (int part = 0; part < nparts; ++part) {
      for (int c = tid; c < kPodTileM * 8; c += 128) {
        const int row = c >> 3, ch = c & 7;
        tc::cp_async16(sA[part] + tc::sw128_offset(row, ch * 8), gA[part] + (size_t)row * rowv + kc * 8 + ch);
      }
      for (int c = tid; c < d.Ppad * 8; c += 128) {
        const int row = c >> 3, ch = c & 7;
        tc::cp_async16(sB[part] + tc::sw128_offset(row, ch * 8), gB[part] + (size_t)row * rowv + kc * 8 + ch);
      }
    }
    tc::cp_async_wait_all();
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    taddr = taddr_s;
    if (tid == 0) {
      // products (A part, B part): (0, 0), then with split (0, 1) and (1, 0)
      const int nprod = split ? 3 : 1;
      for (int pr = 0; pr < nprod; ++pr) {
        const int pa = pr == 2 ? 1 : 0, pb = pr == 1 ? 1 : 0;
        const uint32_t a0 = tc::smem_u32(sA[pa]), b0 = tc::smem_u32(sB[pb]);
        for (int nb = 0; nb < d.Ppad; nb += 256) {
          const int nsz = min(256, d.Ppad - nb);
          const uint32_t idesc = tc::idesc_bf16_f32(kPodTileM, nsz);
#pragma unroll
          for (int kk = 0; kk < kPodK / 16; ++kk) {
            const uint64_t ad = tc::sdesc_sw128(a0 + kk * 32);
            const uint64_t bd = tc::sdesc_sw128(b0 + nb * 128 + kk * 32);
            tc::mma_bf16(taddr + nb, ad, bd, idesc, (kc > 0 || pr > 0 || kk > 0) ? 1u : 0u);
          }
        }
      }
      tc::mma_commit(&mbar);
      s_ok = tc::mbar_wait_bounded(&mbar, kc & 1, kWaitLimit) ? 1 : 0;
    }
    __syncthreads();
    tc::fence_after_sync();
    if (!s_ok) {
      ok = false;
      break;
    }
  }
  if (!ok) {
    if (tid == 0) atomicOr(err, 2);
  } else {
    float* Grow = G + ((size_t)cell * Spad + s0 + warp * 32 + lane) * d.Ppad;
    for (int col = 0; col < d.Ppad; col += 16) {
      float v[16];
      tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + col, v);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        reinterpret_cast<float4*>(Grow + col)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr_s, ncols);
}

// ---- warp r x r Cholesky with 4 right-hand sides (lane q owns row q)
// Broadcasts go through a per-warp shared scratch sw[40] (a 16-byte
// aligned float array): sw[0..31] a column or row, sw[32] a pivot,
// sw[36..39] the pivot row's right-hand sides.

template <int J>
__device__ __forceinline__ void small_chol(float (&Mq)[32], float (&Fq)[4], int lane, int r, bool& bad,
                                           float* sw) {
  if constexpr (J < 32) {
    if (J < r) {
      if (lane == J) {
        sw[32] = Mq[J];
        *reinterpret_cast<float4*>(sw + 36) = make_float4(Fq[0], Fq[1], Fq[2], Fq[3]);
      }
      __syncwarp();
      const float dj = sw[32];
      if (!(dj > 0.f)) bad = true;
      const float dinv = rsqrtf(dj > 0.f ? dj : 1.f);
      const float4 f4 = *reinterpret_cast<const float4*>(sw + 36);
      const float yj[4] = {f4.x * dinv, f4.y * dinv, f4.z * dinv, f4.w * dinv};
      const float lj = (lane > J && lane < r) ? Mq[J] * dinv : 0.f;
      if (lane > J && lane < r) {
        Mq[J] = lj;
#pragma unroll
        for (int l = 0; l < 4; ++l) Fq[l] -= lj * yj[l];
      }
      if (lane == J) {
        Mq[J] = dinv;  // keep the reciprocal pivot
#pragma unroll
        for (int l = 0; l < 4; ++l) Fq[l] = yj[l];
      }
      sw[lane] = lj;  // the pivot column, zero at and above the pivot
      __syncwarp();
#pragma unroll
      for (int p = J + 1; p < 32; ++p) Mq[p] -= lj * sw[p];
      __syncwarp();
    }
    small_chol<J + 1>(Mq, Fq, lane, r, bad, sw);
  }
}

// forward (L y = f) with the stored factor, lane q holds f_q / y_q
template <int J>
__device__ __forceinline__ void small_fwd(const float (&Mq)[32], float (&Fq)[4], int lane, int r, float* sw) {
  if constexpr (J < 32) {
    if (J < r) {
      if (lane == J) {
        sw[32] = Mq[J];
        *reinterpret_cast<float4*>(sw + 36) = make_float4(Fq[0], Fq[1], Fq[2], Fq[3]);
      }
      __syncwarp();
      const float dinv = sw[32];
      const float4 f4 = *reinterpret_cast<const float4*>(sw + 36);
      const float yj[4] = {f4.x * dinv, f4.y * dinv, f4.z * dinv, f4.w * dinv};
      if (lane > J && lane < r) {
#pragma unroll
        for (int l = 0; l < 4; ++l) Fq[l] -= Mq[J] * yj[l];
      }
      if (lane == J) {
#pragma unroll
        for (int l = 0; l < 4; ++l) Fq[l] = yj[l];
      }
      __syncwarp();
    }
    small_fwd<J + 1>(Mq, Fq, lane, r, sw);
  }
}

// backward (L^T x = y), column oriented: lane q holds y_q then x_q.  The
// entry L[p][q] lives in lane p's row at position q; lane J publishes its
// row for the lanes q < J.
template <int J>
__device__ __forceinline__ void small_bwd(const float (&Mq)[32], float (&Fq)[4], int lane, int r, float* sw) {
  if constexpr (J >= 0) {
    if (J < r) {
      if (lane == J) {
#pragma unroll
        for (int q = 0; q < J; ++q) sw[q] = Mq[q];
        sw[32] = Mq[J];
        *reinterpret_cast<float4*>(sw + 36) = make_float4(Fq[0], Fq[1], Fq[2], Fq[3]);
      }
      __syncwarp();
      const float dinv = sw[32];
      const float4 f4 = *reinterpret_cast<const float4*>(sw + 36);
      const float xj[4] = {f4.x * dinv, f4.y * dinv, f4.z * dinv, f4.w * dinv};
      if (lane < J) {
        const float lq = sw[lane];
#pragma unroll
        for (int l = 0; l < 4; ++l) Fq[l] -= lq * xj[l];
      }
      if (lane == J) {
#pragma unroll
        for (int l = 0; l < 4; ++l) Fq[l] = xj[l];
      }
      __syncwarp();
    }
    small_bwd<J - 1>(Mq, Fq, lane, r, sw);
  }
}

struct PodSolveArgs {
  PodDims d;
  int S, Spad, refine;
  const float* G;         // [cell][Spad][Ppad] reduced quantities, or NULL with Gaff
  const float* Gaff;      // affine parts [cell][kPodAffParts][Ppad] (Eq. localAF), or NULL
  const double* xi;       // [S][K] parameters (affine mode)
  const int* aff_var;     // [cell][16] local parameter ids, -1 padded
  int K;
  double gain, scale;
  const double* W;
  const double* wl;
  const int32_t* ranks;
  const double* a;
  double* Ke;
  double* be;
  int32_t* status;
  const int32_t* err;
};

constexpr int kPodSolveWarps = 4;
constexpr int kPodN2Max = (kPodMaxRhoSmall + 1) * (kPodMaxRhoSmall + 1);  // refinement: small cells only

// REFINE: the FP64 stencil refinement of c (refine_iters > 0) is compiled
// into its own kernel, so the unrefined launch carries only its own code;
// PER_L: the handle has one basis per basis function (PodDims::per_l).
template <bool REFINE, bool PER_L>
__global__ void __launch_bounds__(kPodSolveWarps * 32)
pod_solve_kernel(PodSolveArgs A) {
  __shared__ double s_c[kPodSolveWarps][32][4];
  __shared__ double s_u[kPodSolveWarps][kPodN2Max][4];
  __shared__ double s_au[kPodSolveWarps][kPodN2Max][4];
  __shared__ float s_g[kPodSolveWarps][512];
  __shared__ float s_coef[kPodSolveWarps][kPodAffParts];
  __shared__ __align__(16) float s_w[kPodSolveWarps][40];
  __shared__ float s_cf[kPodSolveWarps][32][4];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const PodDims& d = A.d;
  const long long units = (long long)A.S * d.ncell;
  const int P0 = d.P0;
  const int rho = d.rho, NN = rho + 1;
  const double nanv = __longlong_as_double(0x7ff8000000000000ll);
  for (long long u = (long long)blockIdx.x * kPodSolveWarps + wib; u < units;
       u += (long long)gridDim.x * kPodSolveWarps) {
    const int s = (int)(u / d.ncell), cell = (int)(u % d.ncell);
    double* Ke = A.Ke + (size_t)u * 10;
    double* be = A.be + (size_t)u * 4;
    if (A.err[0] != 0) {
      if (lane < 10) Ke[lane] = nanv;
      if (lane < 4) be[lane] = nanv;
      if (lane == 0 && A.status) A.status[u] = STOMSFEM_ETIMEOUT;
      continue;
    }
    // reduced unknowns: the shared basis's r, or the per-l blocks of rcl
    // columns (ranks rl[0..2]; the columns past a block's rank are zero)
    int r, rl0 = 0, rl1 = 0, rl2 = 0;
    if (PER_L) {
      rl0 = A.ranks[cell * 3];
      rl1 = A.ranks[cell * 3 + 1];
      rl2 = A.ranks[cell * 3 + 2];
      r = 3 * d.rcl;
    } else {
      r = A.ranks[cell];
    }
    auto vact = [&](int q) {  // reduced unknown q is a basis vector
      if (!PER_L) return q < r;
      const int b = q / d.rcl;
      return b < 3 && q - b * d.rcl < (b == 0 ? rl0 : (b == 1 ? rl1 : rl2));
    };
    const float* g;
    if (A.Gaff) {
      // Eq. localAF: W^T A(xi) W = gain G_0 + scale sum_k xi_k G_k, the
      // reduced quantities of this unit assembled in shared memory
      if (lane < kPodAffParts) {
        float c = 0.f;
        if (lane == 0) {
          c = (float)A.gain;
        } else if (lane <= 16) {
          const int v = A.aff_var[cell * 16 + lane - 1];
          if (v >= 0) c = (float)(A.scale * A.xi[(size_t)s * A.K + v]);
        }
        s_coef[wib][lane] = c;
      }
      __syncwarp();
      const float* Gc = A.Gaff + (size_t)cell * kPodAffParts * d.Ppad;
      for (int p = lane; p < d.P; p += 32) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < kPodAffParts; ++k) t = fmaf(s_coef[wib][k], Gc[(size_t)k * d.Ppad + p], t);
        s_g[wib][p] = t;
      }
      __syncwarp();
      g = s_g[wib];
    } else {
      g = A.G + ((size_t)cell * A.Spad + s) * d.Ppad;
    }
    // row q of V^T A V and right-hand sides -V^T A phibar_l; per-l bases:
    // the block-diagonal system of the three (V_l^T A V_l) c_l =
    // -V_l^T A phibar_l, identity rows past each block's rank, and no
    // fourth right-hand side (phi_4 = 1 - sum, the partition of unity)
    const bool qa = vact(lane);
    const int qb = PER_L ? lane / d.rcl : 0;
    float Mq[32], Fq[4];
#pragma unroll
    for (int p = 0; p < 32; ++p) {
      float v = 0.f;
      if (lane < r && p < r) {
        if (qa && vact(p) && (!PER_L || p / d.rcl == qb))
          v = g[pidx(4 + min(lane, p), 4 + max(lane, p), P0)];
        else if (p == lane && !qa)
          v = 1.f;
      }
      Mq[p] = v;
    }
#pragma unroll
    for (int l = 0; l < 4; ++l)
      Fq[l] = (lane < r && qa && (!PER_L || l == qb)) ? -g[pidx(l, 4 + lane, P0)] : 0.f;
    bool bad = false;
    small_chol<0>(Mq, Fq, lane, r, bad, s_w[wib]);
    small_bwd<31>(Mq, Fq, lane, r, s_w[wib]);
    const double* Wc = A.W + (size_t)cell * d.N2 * P0;
    const double* wl = A.wl + (size_t)cell * P0;
    using TOut = typename std::conditional<REFINE, double, float>::type;
    TOut Kv[10], bv[4];
    if constexpr (!REFINE) {
      if (PER_L) {
        // S[l][l'] = x_l^T G x_l' with x_l = e_l + c_l (c_l in block l), l,
        // l' < 3; row / column 4 from the zero row sums (phi_4 = 1 - sum and
        // A 1 = 0); b_l = wl^T x_l, b_4 = f H^2 - sum.  FP32, like the solve.
#pragma unroll
        for (int l = 0; l < 4; ++l) s_cf[wib][lane][l] = lane < r ? Fq[l] : 0.f;
        __syncwarp();
        float gx[3];  // (G x_l')[alpha], alpha = lane < P0
#pragma unroll
        for (int lp = 0; lp < 3; ++lp) {
          float t = 0.f;
          if (lane < P0) {
            t = g[pidx(min(lane, lp), max(lane, lp), P0)];
            for (int q = 0; q < r; ++q) t = fmaf(g[pidx(min(lane, 4 + q), max(lane, 4 + q), P0)], s_cf[wib][q][lp], t);
          }
          gx[lp] = t;
        }
        float S3[3][3];
#pragma unroll
        for (int l = 0; l < 3; ++l)
#pragma unroll
          for (int lp = 0; lp < 3; ++lp) {
            const float t = (lane >= 4 && lane < 4 + r) ? s_cf[wib][lane - 4][l] * gx[lp] : 0.f;
            S3[l][lp] = __shfl_sync(0xffffffffu, gx[lp], l) + warp_sum(t);
          }
        float Sf[4][4];
        float tot = 0.f;
#pragma unroll
        for (int l = 0; l < 3; ++l) {
          float rs = 0.f;
#pragma unroll
          for (int lp = 0; lp < 3; ++lp) {
            Sf[l][lp] = 0.5f * (S3[l][lp] + S3[lp][l]);
            rs += Sf[l][lp];
          }
          Sf[l][3] = -rs;
          tot += rs;
        }
        Sf[3][3] = tot;
        int q = 0;
#pragma unroll
        for (int l = 0; l < 4; ++l)
#pragma unroll
          for (int lp = l; lp < 4; ++lp) Kv[q++] = Sf[l][lp];
        const float wv = (lane < r) ? (float)wl[4 + lane] : 0.f;
        const double fH2 = d.f / ((double)d.nc * (double)d.nc);
        double bsum = 0.0;
#pragma unroll
        for (int l = 0; l < 3; ++l) {
          bv[l] = (float)wl[l] + warp_sum(wv * Fq[l]);
          bsum += (double)bv[l];
        }
        bv[3] = (float)(fH2 - bsum);
      } else {
      // K = G_pp + G_pV c ; b = wl_p + wl_V c, in FP32 like the reduced
      // solve itself (the warp-wide FP64 sums cost the narrow FP64 pipe
      // more than the solve); converted to FP64 once, at the store
      int q = 0;
#pragma unroll
      for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int lp = l; lp < 4; ++lp) {
          float t = (lane < r) ? g[pidx(l, 4 + lane, P0)] * Fq[lp] : 0.f;
          t = warp_sum(t);
          Kv[q++] = g[pidx(l, lp, P0)] + t;
        }
      const float wv = (lane < r) ? (float)wl[4 + lane] : 0.f;
#pragma unroll
      for (int l = 0; l < 4; ++l) bv[l] = (float)wl[l] + warp_sum(wv * Fq[l]);
      }
    } else {
      // FP64 refinement of c through the fine stencil of A(omega)
      const int cx = cell % d.nc, cy = cell / d.nc;
      const double* ac = A.a + ((size_t)s * d.nf + cy * rho) * d.nf + cx * rho;
      double cq[4];
#pragma unroll
      for (int l = 0; l < 4; ++l) cq[l] = (lane < r) ? (double)Fq[l] : 0.0;
      for (int it = 0; it <= A.refine; ++it) {
        if (lane < 32) {
#pragma unroll
          for (int l = 0; l < 4; ++l) s_c[wib][lane][l] = cq[l];
        }
        __syncwarp();
        // u_l = phibar_l + V c_l on all cell nodes
        for (int v = lane; v < d.N2; v += 32) {
          const double* wr = Wc + (size_t)v * P0;
          double t[4] = {wr[0], wr[1], wr[2], wr[3]};
          for (int q = 0; q < r; ++q) {
            const double vq = wr[4 + q];
#pragma unroll
            for (int l = 0; l < 4; ++l) t[l] += vq * s_c[wib][q][l];
          }
          if (PER_L) t[3] = 1.0 - t[0] - t[1] - t[2];  // the partition of unity
#pragma unroll
          for (int l = 0; l < 4; ++l) s_u[wib][v][l] = t[l];
        }
        __syncwarp();
        if (it == A.refine) break;
        // (A u_l) at interior nodes by the 9-point stencil
        for (int v = lane; v < d.N2; v += 32) {
          const int i = v % NN, j = v / NN;
          double t[4] = {0, 0, 0, 0};
          if (i > 0 && j > 0 && i < rho && j < rho) {
            const double aSW = ac[(size_t)(j - 1) * d.nf + i - 1], aSE = ac[(size_t)(j - 1) * d.nf + i];
            const double aNE = ac[(size_t)j * d.nf + i], aNW = ac[(size_t)j * d.nf + i - 1];
            const double cC = (2.0 / 3.0) * (aSW + aSE + aNE + aNW);
            const double cW = -(aSW + aNW) / 6.0, cE = -(aSE + aNE) / 6.0;
            const double cS = -(aSW + aSE) / 6.0, cN = -(aNE + aNW) / 6.0;
#pragma unroll
            for (int l = 0; l < 4; ++l) {
              t[l] = cC * s_u[wib][v][l] + cW * s_u[wib][v - 1][l] + cE * s_u[wib][v + 1][l] +
                     cS * s_u[wib][v - NN][l] + cN * s_u[wib][v + NN][l] -
                     aSW / 3.0 * s_u[wib][v - NN - 1][l] - aSE / 3.0 * s_u[wib][v - NN + 1][l] -
                     aNE / 3.0 * s_u[wib][v + NN + 1][l] - aNW / 3.0 * s_u[wib][v + NN - 1][l];
            }
          }
#pragma unroll
          for (int l = 0; l < 4; ++l) s_au[wib][v][l] = t[l];
        }
        __syncwarp();
        // residual R_q = -zeta_q^T (A u) and the correction through the FP32 factor
        float Rq[4] = {0.f, 0.f, 0.f, 0.f};
        if (lane < r) {
          double t[4] = {0, 0, 0, 0};
          for (int v = 0; v < d.N2; ++v) {
            const double vq = Wc[(size_t)v * P0 + 4 + lane];
            if (vq != 0.0) {
#pragma unroll
              for (int l = 0; l < 4; ++l) t[l] += vq * s_au[wib][v][l];
            }
          }
#pragma unroll
          for (int l = 0; l < 4; ++l) Rq[l] = (float)(-t[l]);
          if (PER_L) {  // each block's residual is its own basis function's
#pragma unroll
            for (int l = 0; l < 4; ++l)
              if (l != qb || !qa) Rq[l] = 0.f;
          }
        }
        small_fwd<0>(Mq, Rq, lane, r, s_w[wib]);
        small_bwd<31>(Mq, Rq, lane, r, s_w[wib]);
        if (lane < r) {
#pragma unroll
          for (int l = 0; l < 4; ++l) cq[l] += (double)Rq[l];
        }
        __syncwarp();
      }
      // K_e by the edge/diagonal difference form of the element energy, b_e
      double M[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
      for (int e = lane; e < d.ne; e += 32) {
        const int ex = e % rho, ey = e / rho;
        const int n0 = ey * NN + ex, n1 = n0 + 1, n2 = n0 + NN + 1, n3 = n0 + NN;
        const double ae = ac[(size_t)ey * d.nf + ex];
        double dd[4][6];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const double c0 = s_u[wib][n0][l], c1 = s_u[wib][n1][l], c2 = s_u[wib][n2][l], c3 = s_u[wib][n3][l];
          dd[l][0] = c0 - c1; dd[l][1] = c1 - c2; dd[l][2] = c2 - c3;
          dd[l][3] = c3 - c0; dd[l][4] = c0 - c2; dd[l][5] = c1 - c3;
        }
        int q = 0;
#pragma unroll
        for (int l = 0; l < 4; ++l)
#pragma unroll
          for (int lp = l; lp < 4; ++lp) {
            M[q++] += ae * (dd[l][0] * dd[lp][0] + dd[l][1] * dd[lp][1] + dd[l][2] * dd[lp][2] +
                            dd[l][3] * dd[lp][3] + 2.0 * (dd[l][4] * dd[lp][4] + dd[l][5] * dd[lp][5]));
          }
      }
#pragma unroll
      for (int q = 0; q < 10; ++q) Kv[q] = warp_sum(M[q]) / 6.0;
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const double t = warp_sum((lane < r) ? wl[4 + lane] * s_c[wib][lane][l] : 0.0);
        bv[l] = wl[l] + t;
      }
      if (PER_L) bv[3] = d.f / ((double)d.nc * (double)d.nc) - bv[0] - bv[1] - bv[2];
    }
    const bool fail = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < 10; ++q) Ke[q] = fail ? nanv : Kv[q];
#pragma unroll
      for (int l = 0; l < 4; ++l) be[l] = fail ? nanv : bv[l];
      if (A.status) A.status[u] = fail ? STOMSFEM_ENOTSPD : 0;
    }
    __syncwarp();
  }
}

}  // namespace stomsfem

using namespace stomsfem;

struct stomsfem_pod {
  PodDims d;
  float* Gaff = nullptr;    // affine parts [cell][17][Ppad] (stomsfem_pod_set_affine)
  int32_t* aff_var = nullptr;
  int32_t* zero = nullptr;  // an error word that stays 0 (the affine online stage has no GEMM)
  int K = 0;
  double gain = 0.0, scale = 0.0;
  int max_rank;
  double* W = nullptr;          // [cell][N2][P0]
  double* wl = nullptr;         // [cell][P0]
  double* lam = nullptr;        // [cell][n]
  __nv_bfloat16* T = nullptr;   // [cell][Ppad][Kp]
  __nv_bfloat16* Tlo = nullptr; // [cell][Ppad][Kp]: BF16 of T's remainder
  int split = 1;                // online GEMM with the BF16 remainders (three products)
  int32_t* ranks = nullptr;     // [cell]
  int32_t* err = nullptr;       // [1] device error word
};

static void pod_free(stomsfem_pod* p) {
  if (!p) return;
  cudaFree(p->Gaff);
  cudaFree(p->aff_var);
  cudaFree(p->zero);
  cudaFree(p->W);
  cudaFree(p->wl);
  cudaFree(p->lam);
  cudaFree(p->T);
  cudaFree(p->Tlo);
  cudaFree(p->ranks);
  cudaFree(p->err);
  delete p;
}

// The offline stage, one shared basis per cell (per_l = 0: ranks [ncell])
// or one basis per basis function l = 1..3 (per_l = 1: ranks [ncell][3],
// max_rank per basis).
static int pod_build_impl(const stomsfem_grid* grid, const double* phi_snap, const double* a_train,
                          int32_t S_train, double tol, int32_t max_rank, const int32_t* ranks_in,
                          stomsfem_pod** out, int32_t* ranks_out, stomsfem_stream_t stream, int per_l) {
  if (!grid || !out || grid->nf <= 0 || grid->nc <= 0 || grid->nf % grid->nc)
    return set_error(STOMSFEM_EINVAL, "bad grid / out");
  const int rho = grid->nf / grid->nc;
  if (rho < 2 || rho > kPodMaxRho)
    return set_error(STOMSFEM_EINVAL, "POD needs 2 <= H/h <= %d (got %d)", kPodMaxRho, rho);
  if (S_train < 1 || !phi_snap || !a_train) return set_error(STOMSFEM_EINVAL, "no training data");
  // cells above H/h = 8: the snapshot-space eigenproblem (one shared basis)
  const bool large = rho > kPodMaxRhoSmall;
  if (large && per_l) return set_error(STOMSFEM_EINVAL, "per-l bases need H/h <= %d", kPodMaxRhoSmall);
  if (large && 4 * S_train > kPodSnapMax)
    return set_error(STOMSFEM_EINVAL, "H/h > %d: at most %d training samples (got %d)", kPodMaxRhoSmall,
                     kPodSnapMax / 4, S_train);
  const int rank_cap = per_l ? kPodMaxRank / 3 : kPodMaxRank;
  if (max_rank < 1 || max_rank > rank_cap)
    return set_error(STOMSFEM_EINVAL, "max_rank must be in [1, %d]", rank_cap);
  if (!(tol > 0.0) && !ranks_in) return set_error(STOMSFEM_EINVAL, "tol must be > 0");
  *out = nullptr;
  stomsfem_pod* p = new stomsfem_pod();
  PodDims& d = p->d;
  d.nf = grid->nf;
  d.nc = grid->nc;
  d.rho = rho;
  d.N2 = (rho + 1) * (rho + 1);
  d.n = (rho - 1) * (rho - 1);
  d.ne = rho * rho;
  d.ncell = grid->nc * grid->nc;
  d.f = grid->f;
  d.Kp = pod_kp(d.ne);
  const int rcap = max_rank < d.n ? max_rank : d.n;
  const int nslot = per_l ? 3 : 1;  // eigenproblems per cell
  d.per_l = per_l;
  d.rcl = per_l ? rcap : 0;
  d.P0 = 4 + nslot * rcap;
  d.P = d.P0 * (d.P0 + 1) / 2;
  d.Ppad = (d.P + 15) & ~15;
  p->max_rank = rcap;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int32_t* rin_d = nullptr;
  double *phibar = nullptr, *abar = nullptr, *cov = nullptr;
  auto fail = [&](int rc) {
    cudaFree(rin_d);
    cudaFree(phibar);
    cudaFree(abar);
    cudaFree(cov);
    pod_free(p);
    return rc;
  };
  int rc;
#define TRY(x)                                   \
  if ((rc = check_cuda((x), #x)) != STOMSFEM_OK) \
    return fail(rc);
  TRY(cudaMalloc(&p->W, sizeof(double) * d.ncell * d.N2 * d.P0));
  TRY(cudaMalloc(&p->wl, sizeof(double) * d.ncell * d.P0));
  TRY(cudaMalloc(&p->lam, sizeof(double) * d.ncell * nslot * d.n));
  TRY(cudaMalloc(&p->T, sizeof(__nv_bfloat16) * d.ncell * d.Ppad * d.Kp));
  TRY(cudaMalloc(&p->Tlo, sizeof(__nv_bfloat16) * d.ncell * d.Ppad * d.Kp));
  TRY(cudaMalloc(&p->ranks, sizeof(int32_t) * d.ncell * nslot));
  TRY(cudaMalloc(&p->err, sizeof(int32_t)));
  TRY(cudaMalloc(&phibar, sizeof(double) * d.ncell * 4 * d.N2));
  TRY(cudaMalloc(&abar, sizeof(double) * d.ncell * d.ne));
  // small cells: the covariances; large cells: the snapshots X and Abar X
  TRY(cudaMalloc(&cov, large ? sizeof(double) * 2 * d.ncell * d.n * 4 * S_train
                             : sizeof(double) * d.ncell * nslot * d.n * d.n));
  TRY(cudaMemsetAsync(p->err, 0, sizeof(int32_t), st));
  if (ranks_in) {
    TRY(cudaMalloc(&rin_d, sizeof(int32_t) * d.ncell * nslot));
    TRY(cudaMemcpyAsync(rin_d, ranks_in, sizeof(int32_t) * d.ncell * nslot, cudaMemcpyHostToDevice, st));
  }
  pod_mean_kernel<<<d.ncell, 256, 0, st>>>(d, phi_snap, a_train, S_train, phibar, abar);
  if (large) {
    double* X = cov;
    double* Y = cov + (size_t)d.ncell * d.n * 4 * S_train;
    pod_snap_xy_kernel<<<d.ncell, 256, 0, st>>>(d, phi_snap, S_train, phibar, abar, X, Y);
    const size_t snap_smem = sizeof(double) * 2 * kPodSnapMax * (kPodSnapMax + 1);
    TRY(cudaFuncSetAttribute(pod_snap_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)snap_smem));
    pod_snap_eig_kernel<<<d.ncell, 256, snap_smem, st>>>(d, X, Y, S_train, phibar, tol, rcap, rin_d, p->W, p->lam,
                                                         p->ranks);
    const size_t tl_smem = sizeof(float) * 2 * kPodK * 4 * d.P0;
    TRY(cudaFuncSetAttribute(pod_tensor_large_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tl_smem));
    pod_tensor_large_kernel<<<d.ncell, 256, tl_smem, st>>>(d, p->W, p->T, p->Tlo, p->wl);
  } else if (per_l) {
    pod_cov_per_l_kernel<<<dim3(d.ncell, 3), 256, 0, st>>>(d, phi_snap, S_train, phibar, cov);
    pod_w_init_kernel<<<d.ncell, 256, 0, st>>>(d, phibar, p->W);
  } else {
    pod_cov_kernel<<<d.ncell, 256, 0, st>>>(d, phi_snap, S_train, phibar, cov);
  }
  if (!large) {
    const size_t eig_smem = sizeof(double) * 3 * (kPodMaxN + 1) * (kPodMaxN + 1);
    TRY(cudaFuncSetAttribute(pod_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)eig_smem));
    pod_eig_kernel<<<dim3(d.ncell, nslot), 256, eig_smem, st>>>(d, cov, phibar, abar, tol, rcap, rin_d, p->W,
                                                                 p->lam, p->ranks, p->err);
    pod_tensor_kernel<<<d.ncell, 256, 0, st>>>(d, p->W, p->T, p->Tlo, p->wl);
  }
  TRY(cudaGetLastError());
  int32_t herr = 0;
  TRY(cudaMemcpyAsync(&herr, p->err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  std::vector<int32_t> rk(d.ncell * nslot);
  TRY(cudaMemcpyAsync(rk.data(), p->ranks, sizeof(int32_t) * d.ncell * nslot, cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
#undef TRY
  if (herr != 0) return fail(set_error(STOMSFEM_ENOTSPD, "training-mean energy matrix not positive definite"));
  if (ranks_out) std::memcpy(ranks_out, rk.data(), sizeof(int32_t) * d.ncell * nslot);
  cudaFree(rin_d);
  cudaFree(phibar);
  cudaFree(abar);
  cudaFree(cov);
  *out = p;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_pod_build(const stomsfem_grid* grid, const double* phi_snap,
                                  const double* a_train, int32_t S_train, double tol,
                                  int32_t max_rank, const int32_t* ranks_in, stomsfem_pod** out,
                                  int32_t* ranks_out, stomsfem_stream_t stream) {
  return pod_build_impl(grid, phi_snap, a_train, S_train, tol, max_rank, ranks_in, out, ranks_out, stream, 0);
}

extern "C" int stomsfem_pod_build_per_l(const stomsfem_grid* grid, const double* phi_snap, const double* a_train,
                                        int32_t S_train, double tol, int32_t max_rank_per_l,
                                        const int32_t* ranks_in, stomsfem_pod** out, int32_t* ranks_out,
                                        stomsfem_stream_t stream) {
  return pod_build_impl(grid, phi_snap, a_train, S_train, tol, max_rank_per_l, ranks_in, out, ranks_out, stream, 1);
}

extern "C" int stomsfem_pod_destroy(stomsfem_pod* pod) {
  pod_free(pod);
  return STOMSFEM_OK;
}

extern "C" int stomsfem_pod_eigenvalues(const stomsfem_pod* pod, double* lam_host) {
  if (!pod || !lam_host) return set_error(STOMSFEM_EINVAL, "NULL argument");
  STOMSFEM_TRY_CUDA(cudaMemcpy(lam_host, pod->lam,
                               sizeof(double) * pod->d.ncell * (pod->d.per_l ? 3 : 1) * pod->d.n,
                               cudaMemcpyDeviceToHost));
  return STOMSFEM_OK;
}

static const char kPodMagic[8] = {'S', 'T', 'M', 'F', 'P', 'O', 'D', '1'};
static const char kPodMagicPerL[8] = {'S', 'T', 'M', 'F', 'P', 'O', 'D', 'L'};  // per-l bases

extern "C" int stomsfem_pod_save(const stomsfem_pod* pod, void* host_buf, size_t buf_bytes, size_t* bytes) {
  if (!pod || !bytes) return set_error(STOMSFEM_EINVAL, "NULL pod / bytes");
  const PodDims& d = pod->d;
  const int nslot = d.per_l ? 3 : 1;
  const size_t nW = (size_t)d.ncell * d.N2 * d.P0, nwl = (size_t)d.ncell * d.P0,
               nlam = (size_t)d.ncell * nslot * d.n;
  const size_t nT = (size_t)d.ncell * d.Ppad * d.Kp;
  std::vector<double> W, wl, lam;
  std::vector<__nv_bfloat16> T;
  std::vector<int32_t> rk;
  if (host_buf) {
    W.resize(nW);
    wl.resize(nwl);
    lam.resize(nlam);
    T.resize(nT);
    rk.resize((size_t)d.ncell * nslot);
    STOMSFEM_TRY_CUDA(cudaMemcpy(W.data(), pod->W, sizeof(double) * nW, cudaMemcpyDeviceToHost));
    STOMSFEM_TRY_CUDA(cudaMemcpy(wl.data(), pod->wl, sizeof(double) * nwl, cudaMemcpyDeviceToHost));
    STOMSFEM_TRY_CUDA(cudaMemcpy(lam.data(), pod->lam, sizeof(double) * nlam, cudaMemcpyDeviceToHost));
    STOMSFEM_TRY_CUDA(cudaMemcpy(T.data(), pod->T, sizeof(__nv_bfloat16) * nT, cudaMemcpyDeviceToHost));
    STOMSFEM_TRY_CUDA(cudaMemcpy(rk.data(), pod->ranks, sizeof(int32_t) * d.ncell * nslot, cudaMemcpyDeviceToHost));
  }
  CkptWriter w(host_buf, buf_bytes);
  ckpt_header(w, d.per_l ? kPodMagicPerL : kPodMagic);
  const int32_t dims[11] = {d.nf, d.nc, d.rho, d.N2, d.n, d.ne, d.P0, d.P, d.Ppad, d.ncell, pod->max_rank};
  w.put(dims, sizeof(dims));
  w.val<double>(d.f);
  w.put(host_buf ? (const void*)W.data() : nullptr, sizeof(double) * nW);
  w.put(host_buf ? (const void*)wl.data() : nullptr, sizeof(double) * nwl);
  w.put(host_buf ? (const void*)lam.data() : nullptr, sizeof(double) * nlam);
  w.put(host_buf ? (const void*)T.data() : nullptr, sizeof(__nv_bfloat16) * nT);
  w.put(host_buf ? (const void*)rk.data() : nullptr, sizeof(int32_t) * d.ncell * nslot);
  *bytes = w.pos;
  if (host_buf && !w.fits()) return set_error(STOMSFEM_ENOMEM, "checkpoint buffer %zu < %zu bytes", buf_bytes, w.pos);
  return STOMSFEM_OK;
}

extern "C" int stomsfem_pod_load(const void* host_buf, size_t buf_bytes, stomsfem_pod** out) {
  if (!host_buf || !out) return set_error(STOMSFEM_EINVAL, "NULL buffer / out");
  *out = nullptr;
  CkptReader r(host_buf, buf_bytes);
  int hc = ckpt_check_header(r, kPodMagic);
  int per_l = 0;
  if (hc == 1) {  // the per-l kind?
    r = CkptReader(host_buf, buf_bytes);
    hc = ckpt_check_header(r, kPodMagicPerL);
    per_l = 1;
  }
  if (hc == 1) return set_error(STOMSFEM_EVERSION, "not a version-%u POD checkpoint", kCkptVersion);
  if (hc == 2) return set_error(STOMSFEM_EINVAL, "truncated POD checkpoint");
  const int nslot = per_l ? 3 : 1;
  int32_t dims[11];
  r.get(dims, sizeof(dims));
  PodDims d;
  d.nf = dims[0];
  d.nc = dims[1];
  d.rho = dims[2];
  d.N2 = dims[3];
  d.n = dims[4];
  d.ne = dims[5];
  d.P0 = dims[6];
  d.P = dims[7];
  d.Ppad = dims[8];
  d.ncell = dims[9];
  d.f = r.val<double>();
  const int rcap = dims[10];
  d.per_l = per_l;
  d.rcl = per_l ? rcap : 0;
  d.Kp = pod_kp(d.ne);
  // the stored sizes must be the ones the build derives from the grid
  const bool consistent = r.ok && d.nc > 0 && d.nf % d.nc == 0 && d.rho == d.nf / d.nc && d.rho >= 2 &&
                          d.rho <= kPodMaxRho && (!per_l || d.rho <= kPodMaxRhoSmall) &&
                          d.N2 == (d.rho + 1) * (d.rho + 1) &&
                          d.n == (d.rho - 1) * (d.rho - 1) && d.ne == d.rho * d.rho && d.ncell == d.nc * d.nc &&
                          rcap >= 1 && rcap <= d.n && rcap * nslot <= kPodMaxRank && d.P0 == 4 + nslot * rcap &&
                          d.P == d.P0 * (d.P0 + 1) / 2 &&
                          d.Ppad == ((d.P + 15) & ~15);
  if (!consistent) return set_error(STOMSFEM_EINVAL, "inconsistent POD checkpoint header");
  const size_t nW = (size_t)d.ncell * d.N2 * d.P0, nwl = (size_t)d.ncell * d.P0,
               nlam = (size_t)d.ncell * nslot * d.n;
  const size_t nT = (size_t)d.ncell * d.Ppad * d.Kp;
  const size_t need = r.pos + sizeof(double) * (nW + nwl + nlam) + sizeof(__nv_bfloat16) * nT +
                      sizeof(int32_t) * d.ncell * nslot;
  if (buf_bytes < need) return set_error(STOMSFEM_EINVAL, "truncated POD checkpoint (%zu < %zu)", buf_bytes, need);
  const unsigned char* base = static_cast<const unsigned char*>(host_buf) + r.pos;
  auto* p = new stomsfem_pod();
  p->d = d;
  p->max_rank = rcap;
  int rc;
#define TRY(x)                                     \
  if ((rc = check_cuda((x), #x)) != STOMSFEM_OK) { \
    pod_free(p);                                   \
    return rc;                                     \
  }
  TRY(cudaMalloc(&p->W, sizeof(double) * nW));
  TRY(cudaMalloc(&p->wl, sizeof(double) * nwl));
  TRY(cudaMalloc(&p->lam, sizeof(double) * nlam));
  TRY(cudaMalloc(&p->T, sizeof(__nv_bfloat16) * nT));
  TRY(cudaMalloc(&p->ranks, sizeof(int32_t) * d.ncell * nslot));
  TRY(cudaMalloc(&p->err, sizeof(int32_t)));
  TRY(cudaMemcpy(p->W, base, sizeof(double) * nW, cudaMemcpyHostToDevice));
  base += sizeof(double) * nW;
  TRY(cudaMemcpy(p->wl, base, sizeof(double) * nwl, cudaMemcpyHostToDevice));
  base += sizeof(double) * nwl;
  TRY(cudaMemcpy(p->lam, base, sizeof(double) * nlam, cudaMemcpyHostToDevice));
  base += sizeof(double) * nlam;
  TRY(cudaMemcpy(p->T, base, sizeof(__nv_bfloat16) * nT, cudaMemcpyHostToDevice));
  base += sizeof(__nv_bfloat16) * nT;
  std::vector<int32_t> rk((size_t)d.ncell * nslot);
  std::memcpy(rk.data(), base, sizeof(int32_t) * d.ncell * nslot);
  for (int c = 0; c < d.ncell * nslot; ++c)
    if (rk[c] < 0 || rk[c] > rcap) {
      pod_free(p);
      return set_error(STOMSFEM_EINVAL, "POD checkpoint: rank %d of slot %d outside [0, %d]", rk[c], c, rcap);
    }
  TRY(cudaMemcpy(p->ranks, rk.data(), sizeof(int32_t) * d.ncell * nslot, cudaMemcpyHostToDevice));
  TRY(cudaMemset(p->err, 0, sizeof(int32_t)));
  // T's BF16 remainders are not stored: the build's kernel recomputes them
  // (and the same T and wl) from W
  TRY(cudaMalloc(&p->Tlo, sizeof(__nv_bfloat16) * nT));
  if (d.rho > kPodMaxRhoSmall) {
    const size_t tl_smem = sizeof(float) * 2 * kPodK * 4 * d.P0;
    TRY(cudaFuncSetAttribute(pod_tensor_large_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tl_smem));
    pod_tensor_large_kernel<<<d.ncell, 256, tl_smem>>>(d, p->W, p->T, p->Tlo, p->wl);
  } else {
    pod_tensor_kernel<<<d.ncell, 256>>>(d, p->W, p->T, p->Tlo, p->wl);
  }
  TRY(cudaGetLastError());
  TRY(cudaDeviceSynchronize());
#undef TRY
  *out = p;
  return STOMSFEM_OK;
}

// Workspace: Ab, Ablo ([cell][Spad][Kp] BF16 each), then G [cell][Spad][Ppad]
// FP32.
static size_t pod_ws_layout(const PodDims& d, int S, size_t* off_lo, size_t* off_G) {
  const int Spad = (S + kPodTileM - 1) / kPodTileM * kPodTileM;
  const size_t ab = ((size_t)d.ncell * Spad * d.Kp * 2 + 1023) & ~size_t(1023);
  *off_lo = ab;
  *off_G = 2 * ab;
  return 2 * ab + (size_t)d.ncell * Spad * d.Ppad * 4;
}

extern "C" int stomsfem_pod_workspace_size(const stomsfem_pod* pod, int32_t S, size_t* bytes) {
  if (!pod || S < 0 || !bytes) return set_error(STOMSFEM_EINVAL, "bad arguments");
  size_t ol, og;
  *bytes = pod_ws_layout(pod->d, S, &ol, &og);
  return STOMSFEM_OK;
}

extern "C" int stomsfem_pod_upscale(stomsfem_pod* pod, const double* a, int32_t S,
                                    int32_t refine_iters, double* Ke, double* be,
                                    int32_t* unit_status, void* workspace, size_t workspace_bytes,
                                    stomsfem_stream_t stream) {
  if (!pod) return set_error(STOMSFEM_EINVAL, "pod is NULL");
  if (S < 0 || refine_iters < 0 || refine_iters > 16) return set_error(STOMSFEM_EINVAL, "bad S / refine_iters");
  const PodDims& d = pod->d;
  if (refine_iters > 0 && d.rho > kPodMaxRhoSmall)
    return set_error(STOMSFEM_EINVAL, "the FP64 refinement needs H/h <= %d", kPodMaxRhoSmall);
  if (S == 0) return STOMSFEM_OK;
  if (!a || !Ke || !be || !workspace) return set_error(STOMSFEM_EINVAL, "NULL device pointer");
  size_t ol, og;
  const size_t need = pod_ws_layout(d, S, &ol, &og);
  if (workspace_bytes < need) return set_error(STOMSFEM_ENOMEM, "POD workspace %zu < %zu", workspace_bytes, need);
  const int Spad = (S + kPodTileM - 1) / kPodTileM * kPodTileM;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  auto* Ab = reinterpret_cast<__nv_bfloat16*>(workspace);
  auto* Ablo = reinterpret_cast<__nv_bfloat16*>(static_cast<unsigned char*>(workspace) + ol);
  float* G = reinterpret_cast<float*>(static_cast<unsigned char*>(workspace) + og);
  const int sms = device_sm_count() > 0 ? device_sm_count() : 152;
  pod_gather_kernel<<<sms * 8, 256, 0, st>>>(d, a, S, Spad, Ab, Ablo);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  const int parts = pod->split ? 2 : 1;
  const size_t smem = 1024 + parts * ((size_t)kPodTileM * 128 + (size_t)d.Ppad * 128);
  const size_t smem_req = smem < 120 * 1024 ? 120 * 1024 : smem;  // one CTA per SM (TMEM)
  STOMSFEM_TRY_CUDA(cudaFuncSetAttribute(pod_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_req));
  dim3 grd(Spad / kPodTileM, d.ncell);
  pod_gemm_kernel<<<grd, 128, smem_req, st>>>(d, Spad, Ab, Ablo, pod->T, pod->Tlo, pod->split, G, pod->err);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  PodSolveArgs A;
  A.d = d;
  A.S = S;
  A.Spad = Spad;
  A.refine = refine_iters;
  A.G = G;
  A.Gaff = nullptr;
  A.xi = nullptr;
  A.aff_var = nullptr;
  A.K = 0;
  A.gain = A.scale = 0.0;
  A.W = pod->W;
  A.wl = pod->wl;
  A.ranks = pod->ranks;
  A.a = a;
  A.Ke = Ke;
  A.be = be;
  A.status = unit_status;
  A.err = pod->err;
  const long long units = (long long)S * d.ncell;
  long long blocks = (units + kPodSolveWarps - 1) / kPodSolveWarps;
  if (blocks > (long long)sms * 16) blocks = (long long)sms * 16;
  {
    auto kern = A.refine > 0 ? (d.per_l ? pod_solve_kernel<true, true> : pod_solve_kernel<true, false>)
                             : (d.per_l ? pod_solve_kernel<false, true> : pod_solve_kernel<false, false>);
    kern<<<(unsigned)blocks, kPodSolveWarps * 32, 0, st>>>(A);
  }
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  return STOMSFEM_OK;
}

extern "C" int stomsfem_pod_set_affine(stomsfem_pod* pod, const stomsfem_grid* grid, const stomsfem_field* field,
                                       double tau, stomsfem_stream_t stream) {
  if (!pod || !grid || !field) return set_error(STOMSFEM_EINVAL, "NULL argument");
  const PodDims& d = pod->d;
  if (grid->nf != d.nf || grid->nc != d.nc) return set_error(STOMSFEM_EINVAL, "grid does not match the POD handle");
  if (d.rho > kPodMaxRhoSmall) return set_error(STOMSFEM_EINVAL, "the affine parts need H/h <= %d", kPodMaxRhoSmall);
  if (field->kind != STOMSFEM_FIELD_AFFINE)
    return set_error(STOMSFEM_EINVAL, "the affine reduced basis needs an affine field (kind %d)", STOMSFEM_FIELD_AFFINE);
  if (!(field->width > 0.0) || field->nbx <= 0 || field->nby <= 0) return set_error(STOMSFEM_EINVAL, "bad field");
  const int ncell = d.ncell, rho = d.rho;
  std::vector<int32_t> kc(ncell), ids((size_t)ncell * 16), fam(ncell);
  int32_t nfam = 0;
  int rc = stomsfem_local_vars(grid, field, tau, kc.data(), ids.data(), fam.data(), &nfam);
  if (rc) return rc;
  // local bumps at the element centroids of every cell
  std::vector<double> psi((size_t)ncell * 16 * kPodK, 0.0);
  const double w2 = field->width * field->width;
  for (int cell = 0; cell < ncell; ++cell) {
    const int cx = cell % d.nc, cy = cell / d.nc;
    for (int k = 0; k < kc[cell]; ++k) {
      const int v = ids[(size_t)cell * 16 + k];
      const double px = (v % field->nbx + 0.5) / field->nbx, py = (v / field->nbx + 0.5) / field->nby;
      for (int e = 0; e < d.ne; ++e) {
        const double x = (cx * rho + e % rho + 0.5) / d.nf, y = (cy * rho + e / rho + 0.5) / d.nf;
        psi[((size_t)cell * 16 + k) * kPodK + e] = std::exp(-((x - px) * (x - px) + (y - py) * (y - py)) / w2);
      }
    }
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double* psi_d = nullptr;
  cudaFree(pod->Gaff);
  cudaFree(pod->aff_var);
  cudaFree(pod->zero);
  pod->Gaff = nullptr;
  pod->aff_var = nullptr;
  pod->zero = nullptr;
  auto fail = [&](int code) {
    cudaFree(psi_d);
    cudaFree(pod->Gaff);
    cudaFree(pod->aff_var);
    cudaFree(pod->zero);
    pod->Gaff = nullptr;
    pod->aff_var = nullptr;
    pod->zero = nullptr;
    return code;
  };
#define TRY(x)                                   \
  if ((rc = check_cuda((x), #x)) != STOMSFEM_OK) \
    return fail(rc);
  TRY(cudaMalloc(&psi_d, sizeof(double) * psi.size()));
  TRY(cudaMalloc(&pod->Gaff, sizeof(float) * (size_t)ncell * kPodAffParts * d.Ppad));
  TRY(cudaMalloc(&pod->aff_var, sizeof(int32_t) * ids.size()));
  TRY(cudaMalloc(&pod->zero, sizeof(int32_t)));
  TRY(cudaMemsetAsync(pod->zero, 0, sizeof(int32_t), st));
  TRY(cudaMemcpyAsync(psi_d, psi.data(), sizeof(double) * psi.size(), cudaMemcpyHostToDevice, st));
  TRY(cudaMemcpyAsync(pod->aff_var, ids.data(), sizeof(int32_t) * ids.size(), cudaMemcpyHostToDevice, st));
  pod_affine_parts_kernel<<<ncell, 128, 0, st>>>(d, pod->W, psi_d, pod->Gaff);
  TRY(cudaGetLastError());
  TRY(cudaStreamSynchronize(st));
#undef TRY
  cudaFree(psi_d);
  pod->K = field->nbx * field->nby;
  pod->gain = field->gain;
  pod->scale = field->scale;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_pod_upscale_affine(stomsfem_pod* pod, const double* xi, const double* a, int32_t S,
                                           int32_t refine_iters, double* Ke, double* be, int32_t* unit_status,
                                           stomsfem_stream_t stream) {
  if (!pod) return set_error(STOMSFEM_EINVAL, "pod is NULL");
  if (!pod->Gaff) return set_error(STOMSFEM_EINVAL, "stomsfem_pod_set_affine was not called on this handle");
  if (S < 0 || refine_iters < 0 || refine_iters > 16) return set_error(STOMSFEM_EINVAL, "bad S / refine_iters");
  if (S == 0) return STOMSFEM_OK;
  if (!xi || !Ke || !be) return set_error(STOMSFEM_EINVAL, "NULL device pointer");
  if (refine_iters > 0 && !a) return set_error(STOMSFEM_EINVAL, "refinement needs the coefficient a");
  const PodDims& d = pod->d;
  if (d.Ppad > 512) return set_error(STOMSFEM_EINVAL, "reduced size %d > 512", d.Ppad);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  PodSolveArgs A;
  A.d = d;
  A.S = S;
  A.Spad = 0;
  A.refine = refine_iters;
  A.G = nullptr;
  A.Gaff = pod->Gaff;
  A.xi = xi;
  A.aff_var = pod->aff_var;
  A.K = pod->K;
  A.gain = pod->gain;
  A.scale = pod->scale;
  A.W = pod->W;
  A.wl = pod->wl;
  A.ranks = pod->ranks;
  A.a = a;
  A.Ke = Ke;
  A.be = be;
  A.status = unit_status;
  A.err = pod->zero;
  const int sms = device_sm_count() > 0 ? device_sm_count() : 152;
  const long long units = (long long)S * d.ncell;
  long long blocks = (units + kPodSolveWarps - 1) / kPodSolveWarps;
  if (blocks > (long long)sms * 16) blocks = (long long)sms * 16;
  {
    auto kern = A.refine > 0 ? (d.per_l ? pod_solve_kernel<true, true> : pod_solve_kernel<true, false>)
                             : (d.per_l ? pod_solve_kernel<false, true> : pod_solve_kernel<false, false>);
    kern<<<(unsigned)blocks, kPodSolveWarps * 32, 0, st>>>(A);
  }
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  return STOMSFEM_OK;
}

extern "C" int stomsfem_build_pod(const stomsfem_grid* grid, const double* phi_snap, const double* a_train,
                                  int32_t S_train, double tol, int32_t max_rank, const int32_t* ranks_in,
                                  stomsfem_pod** out, int32_t* ranks_out, stomsfem_stream_t stream) {
  return stomsfem_pod_build(grid, phi_snap, a_train, S_train, tol, max_rank, ranks_in, out, ranks_out, stream);
}

extern "C" int stomsfem_pod_set_gemm_split(stomsfem_pod* pod, int32_t split) {
  if (!pod || split < 0 || split > 1) return set_error(STOMSFEM_EINVAL, "pod NULL or split not 0 / 1");
  pod->split = split;
  return STOMSFEM_OK;
}
