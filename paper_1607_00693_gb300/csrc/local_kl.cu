// Local KL parametrization of the random field (Sec. 2.1.1, Def. of the
// local KL expansion): on the patch P_m of every coarse cell (the cell and
// an oversampling layer of o fine elements, clipped to the domain) the
// covariance is restricted to P_m, its eigenpairs (lambda_k, f_k) with
// int_P f_k^2 = 1 are computed once (offline), and every field sample
// kappa gets its local parameters
//   xi_k = lambda_k^{-1/2} int_P (kappa - kappa_bar) f_k     (online),
// the inputs that the patch's cell problem depends on (Eq. MsFEB2).
//
// Discretisation: kappa piecewise constant on the fine elements (value at
// the centroid), midpoint quadrature with weight h^2 per element, so the
// integral operator on P_m is h^2 C_m (C_m the covariance between the
// patch's element centroids) and f_k = u_k / h with u_k its orthonormal
// eigenvectors.  Covariances: the bump fields' log-coefficient
// s^2 var sum_i psi_i(x) psi_i(y), or the Gaussian sigma^2 exp(-|x-y|^2 /
// beta^2) of the short-correlation example (Sec. 5.3).
//
// Offline: one CTA per cell, FP64, the operator in shared memory and a
// parallel cyclic Jacobi eigensolver (round-robin pairs); the projection
// weights w_k(e) = h u_k(e) / sqrt(lambda_k) are stored per cell, so that
// online xi_k = sum_e w_k(e) (kappa_e - kappa_bar_e).  Online: one warp per
// (sample, cell), lane k accumulates xi_k over the patch's elements (staged
// in shared memory), FP64.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace stomsfem {

constexpr int kKlMaxN = 112;  // patch elements (two n x n FP64 matrices in shared memory)
constexpr int kKlMaxK = 32;   // modes kept per patch (one lane each online)
constexpr int kKlWarps = 4;

struct KlDims {
  int nf, nc, rho, o, ncell, kmax, cov_kind, nbx, nby;
  double h, width, s2var, beta, sigma2;
};

__device__ __forceinline__ void kl_patch(const KlDims& d, int cell, int& x0, int& x1, int& y0, int& y1) {
  const int cx = cell % d.nc, cy = cell / d.nc;
  x0 = max(0, cx * d.rho - d.o);
  x1 = min(d.nf, (cx + 1) * d.rho + d.o);
  y0 = max(0, cy * d.rho - d.o);
  y1 = min(d.nf, (cy + 1) * d.rho + d.o);
}

// Covariance between the centroids of fine elements (ex, ey) and (fx, fy).
__device__ double kl_cov(const KlDims& d, int ex, int ey, int fx, int fy) {
  const double px = (ex + 0.5) * d.h, py = (ey + 0.5) * d.h, qx = (fx + 0.5) * d.h, qy = (fy + 0.5) * d.h;
  if (d.cov_kind == STOMSFEM_KL_GAUSSIAN) {
    const double dx = px - qx, dy = py - qy;
    return d.sigma2 * exp(-(dx * dx + dy * dy) / (d.beta * d.beta));
  }
  double s = 0.0;
  const double iw2 = 1.0 / (d.width * d.width);
  for (int by = 0; by < d.nby; ++by)
    for (int bx = 0; bx < d.nbx; ++bx) {
      const double cx = (bx + 0.5) / d.nbx, cy = (by + 0.5) / d.nby;
      const double ap = (px - cx) * (px - cx) + (py - cy) * (py - cy);
      const double aq = (qx - cx) * (qx - cx) + (qy - cy) * (qy - cy);
      s += exp(-ap * iw2) * exp(-aq * iw2);
    }
  return d.s2var * s;
}

// One CTA per cell: h^2 C on the patch, Jacobi eigenpairs, descending
// order, truncation (K modes: energy > 0 the fewest reaching that share of
// the spectrum, else kmax, capped by the positive eigenvalues), weights.
//   lam [cell][kmax], wts [cell][kmax][kKlMaxN], kcell [cell]
__global__ void __launch_bounds__(256) local_kl_build_kernel(KlDims d, double energy, double* __restrict__ lam,
                                                             double* __restrict__ wts, int32_t* __restrict__ kcell) {
  extern __shared__ double kl_smem[];
  const int cell = blockIdx.x;
  int x0, x1, y0, y1;
  kl_patch(d, cell, x0, x1, y0, y1);
  const int px = x1 - x0, n = px * (y1 - y0);
  const int ne2 = (n + 1) & ~1;  // even size for the round-robin pairs
  double* B = kl_smem;             // [ne2][ne2]
  double* Z = kl_smem + ne2 * ne2;  // eigenvectors
  __shared__ double cs[kKlMaxN / 2][2];
  __shared__ int pairs[kKlMaxN / 2][2];
  __shared__ int order[kKlMaxN];
  __shared__ double offn;
  __shared__ int s_k;
  const int tid = threadIdx.x, nt = blockDim.x;
  const double w = d.h * d.h;
  for (int idx = tid; idx < ne2 * ne2; idx += nt) {
    const int i = idx / ne2, j = idx % ne2;
    double v = 0.0;
    if (i < n && j < n) v = w * kl_cov(d, x0 + i % px, y0 + i / px, x0 + j % px, y0 + j / px);
    B[idx] = v;
    Z[idx] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int np = ne2 / 2;
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (tid == 0) {
      double off = 0.0, dia = 0.0;
      for (int i = 0; i < ne2; ++i)
        for (int j = 0; j < ne2; ++j) (i == j ? dia : off) += B[i * ne2 + j] * B[i * ne2 + j];
      offn = (off <= 1e-30 * dia) ? -1.0 : off;
    }
    __syncthreads();
    if (offn < 0.0) break;
    for (int rnd = 0; rnd < ne2 - 1; ++rnd) {
      for (int k = tid; k < np; k += nt) {
        int a = (k == 0) ? 0 : 1 + (k - 1 + rnd) % (ne2 - 1);
        int b = 1 + (ne2 - 2 - k + rnd) % (ne2 - 1);
        if (a > b) {
          const int t = a;
          a = b;
          b = t;
        }
        pairs[k][0] = a;
        pairs[k][1] = b;
        const double app = B[a * ne2 + a], aqq = B[b * ne2 + b], apq = B[a * ne2 + b];
        double c = 1.0, s = 0.0;
        if (fabs(apq) > 1e-300) {
          const double th = (aqq - app) / (2.0 * apq);
          const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
          s = t * c;
        }
        cs[k][0] = c;
        cs[k][1] = s;
      }
      __syncthreads();
      for (int idx = tid; idx < np * ne2; idx += nt) {  // rows a, b
        const int k = idx / ne2, j = idx % ne2;
        const int a = pairs[k][0], b = pairs[k][1];
        const double c = cs[k][0], s = cs[k][1];
        const double x = B[a * ne2 + j], y = B[b * ne2 + j];
        B[a * ne2 + j] = c * x - s * y;
        B[b * ne2 + j] = s * x + c * y;
      }
      __syncthreads();
      for (int idx = tid; idx < np * ne2; idx += nt) {  // columns a, b and the vectors
        const int k = idx / ne2, i = idx % ne2;
        const int a = pairs[k][0], b = pairs[k][1];
        const double c = cs[k][0], s = cs[k][1];
        const double x = B[i * ne2 + a], y = B[i * ne2 + b];
        B[i * ne2 + a] = c * x - s * y;
        B[i * ne2 + b] = s * x + c * y;
        const double zx = Z[i * ne2 + a], zy = Z[i * ne2 + b];
        Z[i * ne2 + a] = c * zx - s * zy;
        Z[i * ne2 + b] = s * zx + c * zy;
      }
      __syncthreads();
    }
  }
  // descending order of the n real eigenvalues
  for (int i = tid; i < n; i += nt) {
    int rank = 0;
    for (int j = 0; j < n; ++j)
      if (B[j * ne2 + j] > B[i * ne2 + i] || (B[j * ne2 + j] == B[i * ne2 + i] && j < i)) ++rank;
    order[rank] = i;
  }
  __syncthreads();
  if (tid == 0) {
    const double l1 = B[order[0] * ne2 + order[0]];
    int k = 0;
    if (energy > 0.0) {
      double tot = 0.0, cum = 0.0;
      for (int i = 0; i < n; ++i) tot += fmax(B[order[i] * ne2 + order[i]], 0.0);
      while (k < n && cum < energy * tot * (1.0 - 1e-15)) cum += fmax(B[order[k] * ne2 + order[k]], 0.0), ++k;
    } else {
      k = d.kmax;
    }
    // only modes with a positive eigenvalue carry a parameter
    int kpos = 0;
    while (kpos < n && B[order[kpos] * ne2 + order[kpos]] > 1e-12 * l1) ++kpos;
    k = min(min(k, kpos), d.kmax);
    s_k = k < 1 ? 1 : k;
    kcell[cell] = s_k;
  }
  __syncthreads();
  const int K = s_k;
  for (int idx = tid; idx < d.kmax * kKlMaxN; idx += nt) {
    const int k = idx / kKlMaxN, e = idx % kKlMaxN;
    double v = 0.0, lk = 0.0;
    if (k < K) {
      const int src = order[k];
      lk = B[src * ne2 + src];
      if (e < n) v = d.h * Z[e * ne2 + src] / sqrt(lk);
    }
    wts[((size_t)cell * d.kmax + k) * kKlMaxN + e] = v;
    if (e == 0) lam[(size_t)cell * d.kmax + k] = lk;
  }
}

// xi[s][cell][k] = sum_e w_k(e) (kappa_e - kappa_bar_e) over the patch
// (k < the cell's count; 0 past it).  One warp per (sample, cell).
__global__ void __launch_bounds__(kKlWarps * 32) local_kl_project_kernel(KlDims d, int S, const double* __restrict__ kappa,
                                                                          const double* __restrict__ kbar,
                                                                          const double* __restrict__ wts,
                                                                          const int32_t* __restrict__ kcell,
                                                                          double* __restrict__ xi) {
  __shared__ double s_v[kKlWarps][kKlMaxN];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long units = (long long)S * d.ncell;
  for (long long u = (long long)blockIdx.x * kKlWarps + wib; u < units; u += (long long)gridDim.x * kKlWarps) {
    const int s = (int)(u / d.ncell), cell = (int)(u % d.ncell);
    int x0, x1, y0, y1;
    kl_patch(d, cell, x0, x1, y0, y1);
    const int px = x1 - x0, n = px * (y1 - y0);
    const double* ks = kappa + (size_t)s * d.nf * d.nf;
    for (int e = lane; e < n; e += 32) {
      const size_t g = (size_t)(y0 + e / px) * d.nf + (x0 + e % px);
      s_v[wib][e] = ks[g] - (kbar ? kbar[g] : 0.0);
    }
    __syncwarp();
    const int K = kcell[cell];
    if (lane < d.kmax) {
      double t = 0.0;
      if (lane < K) {
        const double* wk = wts + ((size_t)cell * d.kmax + lane) * kKlMaxN;
        for (int e = 0; e < n; ++e) t = fma(wk[e], s_v[wib][e], t);
      }
      xi[(size_t)u * d.kmax + lane] = t;
    }
    __syncwarp();
  }
}

}  // namespace stomsfem

using namespace stomsfem;

struct stomsfem_local_kl {
  KlDims d;
  double* lam = nullptr;   // [ncell][kmax]
  double* wts = nullptr;   // [ncell][kmax][kKlMaxN]
  int32_t* kcell = nullptr;
};

static void kl_free(stomsfem_local_kl* h) {
  if (!h) return;
  cudaFree(h->lam);
  cudaFree(h->wts);
  cudaFree(h->kcell);
  delete h;
}

extern "C" int stomsfem_local_kl_build(const stomsfem_grid* grid, int32_t oversample, int32_t cov_kind,
                                       const stomsfem_field* field, double var, double beta, double sigma,
                                       int32_t kmax, double energy, stomsfem_local_kl** out, int32_t* k_out,
                                       stomsfem_stream_t stream) {
  if (!grid || !out || grid->nf <= 0 || grid->nc <= 0 || grid->nf % grid->nc)
    return set_error(STOMSFEM_EINVAL, "bad grid / out");
  if (oversample < 0) return set_error(STOMSFEM_EINVAL, "oversample < 0");
  if (kmax < 1 || kmax > kKlMaxK) return set_error(STOMSFEM_EINVAL, "kmax must be in [1, %d]", kKlMaxK);
  if (!(energy >= 0.0 && energy <= 1.0)) return set_error(STOMSFEM_EINVAL, "energy must be in [0, 1]");
  const int rho = grid->nf / grid->nc;
  const int side = rho + 2 * oversample < grid->nf ? rho + 2 * oversample : grid->nf;
  if (side * side > kKlMaxN)
    return set_error(STOMSFEM_EINVAL, "patch of %d x %d elements exceeds %d", side, side, kKlMaxN);
  KlDims d;
  d.nf = grid->nf;
  d.nc = grid->nc;
  d.rho = rho;
  d.o = oversample;
  d.ncell = grid->nc * grid->nc;
  d.kmax = kmax;
  d.cov_kind = cov_kind;
  d.h = 1.0 / grid->nf;
  d.nbx = d.nby = 0;
  d.width = 1.0;
  d.s2var = 0.0;
  d.beta = beta;
  d.sigma2 = sigma * sigma;
  if (cov_kind == STOMSFEM_KL_BUMPS) {
    if (!field || field->nbx < 1 || field->nby < 1 || !(field->width > 0.0) || !(var > 0.0))
      return set_error(STOMSFEM_EINVAL, "bump covariance needs a bump field and var > 0");
    d.nbx = field->nbx;
    d.nby = field->nby;
    d.width = field->width;
    d.s2var = field->scale * field->scale * var;
  } else if (cov_kind == STOMSFEM_KL_GAUSSIAN) {
    if (!(beta > 0.0) || !(sigma > 0.0)) return set_error(STOMSFEM_EINVAL, "Gaussian covariance needs beta, sigma > 0");
  } else {
    return set_error(STOMSFEM_EINVAL, "unknown covariance kind %d", cov_kind);
  }
  *out = nullptr;
  auto* h = new stomsfem_local_kl();
  h->d = d;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc;
#define TRY(x)                                     \
  if ((rc = check_cuda((x), #x)) != STOMSFEM_OK) { \
    kl_free(h);                                    \
    return rc;                                     \
  }
  TRY(cudaMalloc(&h->lam, sizeof(double) * d.ncell * kmax));
  TRY(cudaMalloc(&h->wts, sizeof(double) * d.ncell * kmax * kKlMaxN));
  TRY(cudaMalloc(&h->kcell, sizeof(int32_t) * d.ncell));
  const int n = side * side, ne2 = (n + 1) & ~1;
  const size_t smem = sizeof(double) * 2 * ne2 * ne2;
  TRY(cudaFuncSetAttribute(local_kl_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  local_kl_build_kernel<<<d.ncell, 256, smem, st>>>(d, energy, h->lam, h->wts, h->kcell);
  TRY(cudaGetLastError());
  std::vector<int32_t> kc(d.ncell);
  TRY(cudaMemcpyAsync(kc.data(), h->kcell, sizeof(int32_t) * d.ncell, cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
#undef TRY
  if (k_out)
    for (int c = 0; c < d.ncell; ++c) k_out[c] = kc[c];
  *out = h;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_local_kl_destroy(stomsfem_local_kl* h) {
  kl_free(h);
  return STOMSFEM_OK;
}

extern "C" int stomsfem_local_kl_modes(const stomsfem_local_kl* h, double* lam_host, double* w_host) {
  if (!h) return set_error(STOMSFEM_EINVAL, "handle is NULL");
  const KlDims& d = h->d;
  if (lam_host)
    STOMSFEM_TRY_CUDA(cudaMemcpy(lam_host, h->lam, sizeof(double) * d.ncell * d.kmax, cudaMemcpyDeviceToHost));
  if (w_host)
    STOMSFEM_TRY_CUDA(
        cudaMemcpy(w_host, h->wts, sizeof(double) * d.ncell * d.kmax * kKlMaxN, cudaMemcpyDeviceToHost));
  return STOMSFEM_OK;
}

extern "C" int stomsfem_local_kl_project(const stomsfem_local_kl* h, const double* kappa, const double* kappa_bar,
                                         int32_t S, double* xi, stomsfem_stream_t stream) {
  if (!h || S < 0) return set_error(STOMSFEM_EINVAL, "bad handle / S");
  if (S == 0) return STOMSFEM_OK;
  if (!kappa || !xi) return set_error(STOMSFEM_EINVAL, "NULL device pointer");
  const KlDims& d = h->d;
  const long long units = (long long)S * d.ncell;
  const int sms = device_sm_count() > 0 ? device_sm_count() : 152;
  long long blocks = (units + kKlWarps - 1) / kKlWarps;
  if (blocks > (long long)sms * 16) blocks = (long long)sms * 16;
  local_kl_project_kernel<<<(unsigned)blocks, kKlWarps * 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      d, S, kappa, kappa_bar, h->wts, h->kcell, xi);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  return STOMSFEM_OK;
}
