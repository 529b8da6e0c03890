// Random interpolation of the local upscaled quantities (Sec. 3.1,
// Algorithms 1 and 2): per patch family, K_e and b_e of the family's first
// cell at the points of an anisotropic tensor collocation grid in the local
// parameters (offline, through the FP64 upscaler), and the tensor Lagrange
// interpolant of every entry evaluated per (sample, cell) online.  A unit
// whose local parameters leave [-1, 1] is upscaled directly (the remark
// closing Sec. 3.1.1).
#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "ckpt.cuh"
#include "common.cuh"

namespace stomsfem {

constexpr int kRiMaxDim = 16;         // interpolated directions per cell
constexpr int kRiMaxNu = 8;           // degree per direction
constexpr int kRiMaxNodes = kRiMaxNu + 1;
constexpr int kRiMaxSlots = 64;       // sum over directions of (nu + 1)
constexpr int kRiUnits = 256;         // units per CTA (one tile)
constexpr int kRiThreads = 128;       // two units per thread
constexpr int kRiMaxBlock = 16;       // grid points of the inner block (weights kept per unit)
constexpr long long kRiMaxPoints = 2048;  // one family's table in shared memory, 64 B per point

struct RiFam {
  int ndim, npts, ncell, cell0;  // directions, grid points, cells, first entry in fam_cells
  long long pt0;                 // first point in the concatenated tables
  int radix[kRiMaxDim];          // nu + 1 per direction
  int slot0[kRiMaxDim];          // first node slot of each direction
  int din, nb, nslot_out;        // inner directions (the last din), their grid points, outer node slots
};

struct RiPlan {
  int ncell = 0, nfam = 0, K = 0;
  std::vector<int> fam;        // [ncell]
  std::vector<int> var;        // [ncell][16], -1 padded, in table order
  std::vector<int> nu;         // [ncell][16], 0 padded
  std::vector<RiFam> F;        // [nfam]
  std::vector<int> rep;        // [nfam] first cell
  std::vector<int> fam_cells;  // cells grouped by family, ascending within a family
  long long npoints = 0;
};

// Strength of bump i on a cell: the largest |d log a / d xi_i| over the
// closed cell rectangle (d2 = squared distance of the centre to it).
static double ri_influence(const stomsfem_field* fd, double d2) {
  const double psi = std::exp(-d2 / (fd->width * fd->width));
  if (fd->kind == STOMSFEM_FIELD_EXP) return std::fabs(fd->scale) * psi;
  return std::fabs(fd->contrast_log * fd->gain) * 0.25 * psi;
}

// Smallest degree nu whose Chebyshev-coefficient bound of exp(g t),
// 2 (g/2)^(nu+1) / (nu+1)!, is <= eps; capped at nu_max.
static int ri_choose_nu(double g, double eps, int nu_max) {
  int nu = 0;
  double term = g;  // nu = 0: 2 (g/2) / 1!
  while (nu < nu_max && term > eps) {
    ++nu;
    term *= (g / 2.0) / (double)(nu + 1);
  }
  return nu;
}

static int ri_make_plan(const stomsfem_grid* g, const stomsfem_field* fd, double eps, int nu_max, RiPlan& P) {
  if (!g || !fd) return set_error(STOMSFEM_EINVAL, "grid/field is NULL");
  if (g->nf <= 0 || g->nc <= 0 || g->nf % g->nc) return set_error(STOMSFEM_EINVAL, "bad grid");
  if (fd->kind != STOMSFEM_FIELD_EXP && fd->kind != STOMSFEM_FIELD_EXP_SIGMOID)
    return set_error(STOMSFEM_EINVAL, "unknown field kind %d", fd->kind);
  if (fd->nbx <= 0 || fd->nby <= 0 || !(fd->width > 0.0)) return set_error(STOMSFEM_EINVAL, "bad field");
  if (!(eps > 0.0)) return set_error(STOMSFEM_EINVAL, "eps must be > 0");
  if (nu_max < 1 || nu_max > kRiMaxNu) return set_error(STOMSFEM_EINVAL, "nu_max must be in [1, %d]", kRiMaxNu);
  const int nc = g->nc, ncell = nc * nc;
  const double H = 1.0 / nc;
  P.ncell = ncell;
  P.K = fd->nbx * fd->nby;
  P.fam.assign(ncell, -1);
  P.var.assign((size_t)ncell * kRiMaxDim, -1);
  P.nu.assign((size_t)ncell * kRiMaxDim, 0);
  P.F.clear();
  P.rep.clear();
  std::map<std::vector<long long>, int> index;
  std::vector<std::vector<int>> members;
  for (int cell = 0; cell < ncell; ++cell) {
    const int cx = cell % nc, cy = cell / nc;
    const double x0 = cx * H, x1 = (cx + 1) * H, y0 = cy * H, y1 = (cy + 1) * H;
    struct D { int nu; long long oy, ox; int var; };
    std::vector<D> dims;
    for (int by = 0; by < fd->nby; ++by)
      for (int bx = 0; bx < fd->nbx; ++bx) {
        const double px = (bx + 0.5) / fd->nbx, py = (by + 0.5) / fd->nby;
        const double dx = std::max(std::max(x0 - px, 0.0), px - x1);
        const double dy = std::max(std::max(y0 - py, 0.0), py - y1);
        const int nu = ri_choose_nu(ri_influence(fd, dx * dx + dy * dy), eps, nu_max);
        if (nu >= 1)
          dims.push_back({nu, std::llround((py - y0) * g->nf * 1e6), std::llround((px - x0) * g->nf * 1e6),
                          by * fd->nbx + bx});
      }
    std::sort(dims.begin(), dims.end(), [](const D& a, const D& b) {
      if (a.nu != b.nu) return a.nu < b.nu;
      if (a.oy != b.oy) return a.oy < b.oy;
      return a.ox < b.ox;
    });
    if ((int)dims.size() > kRiMaxDim)
      return set_error(STOMSFEM_EINVAL, "cell %d has %zu interpolated directions > %d (raise eps)", cell,
                       dims.size(), kRiMaxDim);
    std::vector<long long> key;
    for (size_t k = 0; k < dims.size(); ++k) {
      key.push_back(dims[k].oy);
      key.push_back(dims[k].ox);
      key.push_back(dims[k].nu);
      P.var[(size_t)cell * kRiMaxDim + k] = dims[k].var;
      P.nu[(size_t)cell * kRiMaxDim + k] = dims[k].nu;
    }
    auto it = index.find(key);
    if (it == index.end()) {
      const int f = (int)P.F.size();
      index.emplace(key, f);
      RiFam F{};
      F.ndim = (int)dims.size();
      long long n = 1;
      int slot = 0;
      for (int k = 0; k < F.ndim; ++k) {
        F.radix[k] = dims[k].nu + 1;
        F.slot0[k] = slot;
        slot += F.radix[k];
        n *= F.radix[k];
      }
      if (slot > kRiMaxSlots)
        return set_error(STOMSFEM_EINVAL, "family of cell %d needs %d node slots > %d (raise eps)", cell, slot,
                         kRiMaxSlots);
      if (n > kRiMaxPoints)
        return set_error(STOMSFEM_EINVAL, "family of cell %d has %lld grid points > %lld (raise eps or lower nu_max)",
                         cell, n, kRiMaxPoints);
      F.npts = (int)n;
      // inner block: the longest run of last directions with <= kRiMaxBlock points
      F.din = 0;
      F.nb = 1;
      while (F.din < F.ndim && F.nb * F.radix[F.ndim - 1 - F.din] <= kRiMaxBlock) {
        F.nb *= F.radix[F.ndim - 1 - F.din];
        ++F.din;
      }
      F.nslot_out = F.ndim - F.din > 0 ? F.slot0[F.ndim - F.din - 1] + F.radix[F.ndim - F.din - 1] : 0;
      P.F.push_back(F);
      P.rep.push_back(cell);
      members.emplace_back();
      P.fam[cell] = f;
    } else {
      P.fam[cell] = it->second;
    }
    members[P.fam[cell]].push_back(cell);
  }
  P.nfam = (int)P.F.size();
  P.fam_cells.clear();
  long long pt = 0;
  for (int f = 0; f < P.nfam; ++f) {
    P.F[f].cell0 = (int)P.fam_cells.size();
    P.F[f].ncell = (int)members[f].size();
    P.F[f].pt0 = pt;
    pt += P.F[f].npts;
    P.fam_cells.insert(P.fam_cells.end(), members[f].begin(), members[f].end());
  }
  P.npoints = pt;
  return STOMSFEM_OK;
}

// n nodes on [-1, 1], ascending: Chebyshev points of the first kind, or the
// zeros of the Legendre polynomial P_n (Newton on the three-term recurrence
// from the asymptotic first guess cos(pi (j + 3/4) / (n + 1/2))).
static void ri_nodes(int kind, int n, double* x) {
  const double pi = 3.14159265358979323846;
  for (int j = 0; j < n; ++j) {
    if (kind == STOMSFEM_RI_CHEBYSHEV) {
      x[j] = -std::cos((2 * j + 1) * pi / (2.0 * n));
      continue;
    }
    double t = -std::cos(pi * (j + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;  // P_0, P_1
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_n(t), p0 = P_{n-1}(t); P_n' = n (t P_n - P_{n-1}) / (t^2 - 1)
      const double dp = n * (t * p1 - p0) / (t * t - 1.0);
      const double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[j] = (n == 1) ? 0.0 : t;
  }
}

// Barycentric weights 1 / prod_{k != j} (x_j - x_k), scaled to max |w| = 1.
static void ri_bary(const double* x, int n, double* w) {
  double mx = 0.0;
  for (int j = 0; j < n; ++j) {
    double p = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) p *= x[j] - x[k];
    w[j] = 1.0 / p;
    mx = std::max(mx, std::fabs(w[j]));
  }
  for (int j = 0; j < n; ++j) w[j] /= mx;
}

// ---- device

// Ke/be of the listed units (one per collocation point) into the tables.
__global__ void ri_gather_kernel(int n, const int32_t* __restrict__ list, const double* __restrict__ Ke,
                                 const double* __restrict__ be, double* __restrict__ tab64,
                                 float* __restrict__ tab32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * 16; i += gridDim.x * blockDim.x) {
    const int j = i / 16, q = i % 16;
    const long long u = list[j];
    double v = 0.0;
    if (q < 10) v = Ke[u * 10 + q];
    else if (q < 14) v = be[u * 4 + (q - 10)];
    if (q < 14) tab64[(size_t)j * 14 + q] = v;
    tab32[(size_t)j * 16 + q] = (float)v;
  }
}

// First tile of every family for S samples (tiles of kRiUnits units).
__global__ void ri_tiles_kernel(int nfam, const RiFam* __restrict__ fam, int S, int* __restrict__ tile0) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int t = 0;
  for (int f = 0; f < nfam; ++f) {
    tile0[f] = t;
    t += (int)(((long long)S * fam[f].ncell + kRiUnits - 1) / kRiUnits);
  }
  tile0[nfam] = t;
}

struct RiEvalArgs {
  const double* xi;
  int K, S, ncell, nfam;
  int max_pts, max_nb, max_slot;  // shared-memory layout of the launch
  const RiFam* fam;
  const int* tile0;      // [nfam + 1]
  const float* x;        // [nfam][kRiMaxSlots] nodes
  const float* w;        // [nfam][kRiMaxSlots] barycentric weights
  const int* cell_var;   // [ncell][16]
  const int* fam_cells;  // [ncell]
  const float4* tab;     // [points][4] (14 entries + 2 zeros per point)
  double* Ke;
  double* be;
  uint8_t* flag;
  int32_t* list;         // units to upscale directly (NULL: no coefficient given)
  int32_t* count;
};

// 1-d Lagrange values of one direction at t in the second (true)
// barycentric form; a node hit exactly gives the unit vector.
template <int N>
__device__ __forceinline__ void ri_values(const float* sx, const float* sw, float t, float (&l)[N]) {
  int hit = -1;
  float sum = 0.f;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const float d = t - sx[j];
    if (d == 0.f) hit = j;
    l[j] = __fdividef(sw[j], d);
    sum += l[j];
  }
  const float inv = 1.f / sum;
#pragma unroll
  for (int j = 0; j < N; ++j) l[j] = (hit >= 0) ? (j == hit ? 1.f : 0.f) : l[j] * inv;
}

// Direction of radix n at t: an inner direction multiplies the unit's
// block weights sW[0..len) into sW[0..n len) (this direction slowest), an
// outer one stores its values at its node slots of sL.
__device__ __forceinline__ void ri_direction(bool inner, int n, const float* sx, const float* sw, float t,
                                             float* sW, float* sL, int slot0, int q, int len) {
  switch (n) {
#define RI_DIR(N)                                                                            \
  case N: {                                                                                  \
    float l[N];                                                                              \
    ri_values<N>(sx, sw, t, l);                                                              \
    if (inner) {                                                                             \
      _Pragma("unroll") for (int j = N - 1; j >= 1; --j) for (int i = 0; i < len; ++i)       \
          sW[(j * len + i) * kRiUnits + q] = l[j] * sW[i * kRiUnits + q];                     \
      for (int i = 0; i < len; ++i) sW[i * kRiUnits + q] *= l[0];                            \
    } else {                                                                                 \
      _Pragma("unroll") for (int j = 0; j < N; ++j) sL[(slot0 + j) * kRiUnits + q] = l[j];   \
    }                                                                                        \
    break;                                                                                   \
  }
    RI_DIR(2) RI_DIR(3) RI_DIR(4) RI_DIR(5) RI_DIR(6) RI_DIR(7) RI_DIR(8) RI_DIR(9)
#undef RI_DIR
    default:
      break;
  }
}

// Sum over the family's grid for the thread's two units: outer index o
// (the product of the outer directions' 1-d values, at the node slots
// sO[o][k] of sL) times the NB inner points (block weights held in
// registers), table rows broadcast from shared memory.
template <int NB>
__device__ __forceinline__ void ri_accumulate(const float4* __restrict__ sV, const float* __restrict__ sW,
                                              const float* __restrict__ sL, const uint8_t* __restrict__ sO,
                                              const RiFam& F, int tid,
                                              float (&acc0)[14], float (&acc1)[14]) {
  float w0[NB], w1[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    w0[b] = sW[b * kRiUnits + tid];
    w1[b] = sW[b * kRiUnits + tid + kRiThreads];
  }
#pragma unroll
  for (int q = 0; q < 14; ++q) acc0[q] = acc1[q] = 0.f;
  const int dout = F.ndim - F.din;
  const int nout = F.npts / NB;
  const float4* v = sV;
  const uint8_t* so = sO;
  for (int o = 0; o < nout; ++o) {
    float b0 = 1.f, b1 = 1.f;
    for (int k = 0; k < dout; ++k) {
      const int sl = so[k] * kRiUnits + tid;
      b0 *= sL[sl];
      b1 *= sL[sl + kRiThreads];
    }
    so += dout;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const float wa = b0 * w0[b], wb = b1 * w1[b];
      const float4 v0 = v[4 * b], v1 = v[4 * b + 1], v2 = v[4 * b + 2], v3 = v[4 * b + 3];
      const float e[14] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y, v2.z, v2.w, v3.x, v3.y};
#pragma unroll
      for (int q = 0; q < 14; ++q) {
        acc0[q] = fmaf(wa, e[q], acc0[q]);
        acc1[q] = fmaf(wb, e[q], acc1[q]);
      }
    }
    v += 4 * NB;
  }
}

// One tile of 256 units of one family; thread t takes units t and t + 128.
// Shared memory: the family's table [npts][16]; per unit (column q) the
// inner block weights sW[b][q] (b < nb: products over the last din
// directions) and the outer directions' 1-d values sL[slot][q]; the outer
// node slots per outer index sO[o][k] (uniform over the tile).
__global__ void __launch_bounds__(kRiThreads) ri_eval_kernel(RiEvalArgs A) {
  extern __shared__ float4 sV[];
  __shared__ RiFam F;
  __shared__ float sx[kRiMaxSlots], sw[kRiMaxSlots];
  float* sW = reinterpret_cast<float*>(sV + (size_t)A.max_pts * 4);
  float* sL = sW + (size_t)A.max_nb * kRiUnits;
  uint8_t* sO = reinterpret_cast<uint8_t*>(sL + (size_t)A.max_slot * kRiUnits);
  const int tid = threadIdx.x;
  const int tile = blockIdx.x;
  int lo = 0, hi = A.nfam;  // tile0[lo] <= tile < tile0[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (A.tile0[mid] <= tile) lo = mid;
    else hi = mid;
  }
  const int f = lo;
  if (tid == 0) F = A.fam[f];
  if (tid < kRiMaxSlots) {
    sx[tid] = A.x[f * kRiMaxSlots + tid];
    sw[tid] = A.w[f * kRiMaxSlots + tid];
  }
  __syncthreads();
  {
    const float4* src = A.tab + F.pt0 * 4;
    for (int i = tid; i < F.npts * 4; i += kRiThreads) sV[i] = src[i];
  }
  const int D = F.ndim, dout = F.ndim - F.din;
  // node slots of the outer directions per outer index (last outer direction fastest)
  for (int o = tid; o < F.npts / F.nb; o += kRiThreads) {
    int rem = o;
    for (int k = dout - 1; k >= 0; --k) {
      sO[o * dout + k] = (uint8_t)(F.slot0[k] + rem % F.radix[k]);
      rem /= F.radix[k];
    }
  }
  long long u[2];
  bool run[2], out[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int q = tid + h * kRiThreads;
    const long long r = (long long)(tile - A.tile0[f]) * kRiUnits + q;
    run[h] = r < (long long)A.S * F.ncell;
    out[h] = false;
    u[h] = 0;
    if (!run[h]) continue;
    const int s = (int)(r / F.ncell), pos = (int)(r % F.ncell);
    const int cell = A.fam_cells[F.cell0 + pos];
    u[h] = (long long)s * A.ncell + cell;
    const double* xs = A.xi + (size_t)s * A.K;
    const int* vars = A.cell_var + cell * kRiMaxDim;
    // inner block weights by Kronecker products, last direction first;
    // then the outer directions' 1-d values
    sW[q] = 1.f;
    int len = 1;
    for (int k = D - 1; k >= 0; --k) {
      const double t = xs[vars[k]];
      if (!(fabs(t) <= 1.0)) out[h] = true;
      const int n = F.radix[k];
      ri_direction(k >= dout, n, sx + F.slot0[k], sw + F.slot0[k], (float)t, sW, sL, F.slot0[k], q, len);
      if (k >= dout) len *= n;
    }
  }
  __syncthreads();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (!run[h] || !out[h]) continue;
    if (A.list) {
      A.flag[u[h]] = 1;
      A.list[atomicAdd(A.count, 1)] = (int32_t)u[h];
    } else {
      const double nanv = __longlong_as_double(0x7ff8000000000000ll);
      A.flag[u[h]] = 2;
      for (int q = 0; q < 10; ++q) A.Ke[u[h] * 10 + q] = nanv;
      for (int l = 0; l < 4; ++l) A.be[u[h] * 4 + l] = nanv;
    }
  }
  if (!run[0]) return;  // the second unit of a thread runs only with the first
  float acc0[14], acc1[14];
  switch (F.nb) {
#define RI_NB(N) \
  case N:        \
    ri_accumulate<N>(sV, sW, sL, sO, F, tid, acc0, acc1); \
    break;
    RI_NB(1) RI_NB(2) RI_NB(3) RI_NB(4) RI_NB(5) RI_NB(6) RI_NB(7) RI_NB(8)
    RI_NB(9) RI_NB(10) RI_NB(12) RI_NB(14) RI_NB(15) RI_NB(16)
#undef RI_NB
    default:
      for (int q = 0; q < 14; ++q) acc0[q] = acc1[q] = __int_as_float(0x7fc00000);  // unreachable sizes
  }
  if (!out[0]) {
    A.flag[u[0]] = 0;
#pragma unroll
    for (int q = 0; q < 10; ++q) A.Ke[u[0] * 10 + q] = (double)acc0[q];
#pragma unroll
    for (int l = 0; l < 4; ++l) A.be[u[0] * 4 + l] = (double)acc0[10 + l];
  }
  if (run[1] && !out[1]) {
    A.flag[u[1]] = 0;
#pragma unroll
    for (int q = 0; q < 10; ++q) A.Ke[u[1] * 10 + q] = (double)acc1[q];
#pragma unroll
    for (int l = 0; l < 4; ++l) A.be[u[1] * 4 + l] = (double)acc1[10 + l];
  }
}

}  // namespace stomsfem

using namespace stomsfem;

struct stomsfem_ri {
  stomsfem_grid grid;
  stomsfem_field field;
  double eps;
  int nu_max, kind;
  RiPlan P;
  RiFam* fam_d = nullptr;
  float *x_d = nullptr, *w_d = nullptr, *tab32 = nullptr;
  double* tab64 = nullptr;
  int *cell_var_d = nullptr, *fam_cells_d = nullptr;
};

static void ri_free(stomsfem_ri* h) {
  if (!h) return;
  cudaFree(h->fam_d);
  cudaFree(h->x_d);
  cudaFree(h->w_d);
  cudaFree(h->tab32);
  cudaFree(h->tab64);
  cudaFree(h->cell_var_d);
  cudaFree(h->fam_cells_d);
  delete h;
}

extern "C" int stomsfem_ri_plan(const stomsfem_grid* grid, const stomsfem_field* field, double eps,
                                int32_t nu_max, int32_t* family, int32_t* var_ids, int32_t* nu,
                                int32_t* n_families, int64_t* n_points) {
  RiPlan P;
  const int rc = ri_make_plan(grid, field, eps, nu_max, P);
  if (rc) return rc;
  for (int c = 0; c < P.ncell; ++c) {
    if (family) family[c] = P.fam[c];
    for (int k = 0; k < kRiMaxDim; ++k) {
      if (var_ids) var_ids[c * kRiMaxDim + k] = P.var[(size_t)c * kRiMaxDim + k];
      if (nu) nu[c * kRiMaxDim + k] = P.nu[(size_t)c * kRiMaxDim + k];
    }
  }
  if (n_families) *n_families = P.nfam;
  if (n_points) *n_points = P.npoints;
  return STOMSFEM_OK;
}

// A handle with its plan, node tables and (unfilled) interpolation tables
// on the device; xd receives the FP64 nodes per family and slot.
static int ri_setup(const stomsfem_grid* grid, const stomsfem_field* field, double eps, int32_t nu_max,
                    int32_t nodes, stomsfem_ri** out, std::vector<double>& xd) {
  *out = nullptr;
  if (nodes != STOMSFEM_RI_CHEBYSHEV && nodes != STOMSFEM_RI_LEGENDRE)
    return set_error(STOMSFEM_EINVAL, "unknown node family %d", nodes);
  auto* h = new stomsfem_ri();
  int rc = ri_make_plan(grid, field, eps, nu_max, h->P);
  if (rc) {
    delete h;
    return rc;
  }
  h->grid = *grid;
  h->field = *field;
  h->eps = eps;
  h->nu_max = nu_max;
  h->kind = nodes;
  RiPlan& P = h->P;
  // nodes and barycentric weights per family and direction
  std::vector<float> xs((size_t)P.nfam * kRiMaxSlots, 0.f), ws((size_t)P.nfam * kRiMaxSlots, 0.f);
  xd.assign((size_t)P.nfam * kRiMaxSlots, 0.0);
  for (int f = 0; f < P.nfam; ++f)
    for (int k = 0; k < P.F[f].ndim; ++k) {
      const int n = P.F[f].radix[k], s0 = P.F[f].slot0[k];
      double x[kRiMaxNodes], w[kRiMaxNodes];
      ri_nodes(nodes, n, x);
      ri_bary(x, n, w);
      for (int j = 0; j < n; ++j) {
        xd[(size_t)f * kRiMaxSlots + s0 + j] = x[j];
        xs[(size_t)f * kRiMaxSlots + s0 + j] = (float)x[j];
        ws[(size_t)f * kRiMaxSlots + s0 + j] = (float)w[j];
      }
    }
#define TRY(x)                                     \
  if ((rc = check_cuda((x), #x)) != STOMSFEM_OK) { \
    ri_free(h);                                    \
    return rc;                                     \
  }
  TRY(cudaMalloc(&h->fam_d, sizeof(RiFam) * P.nfam));
  TRY(cudaMalloc(&h->x_d, sizeof(float) * xs.size()));
  TRY(cudaMalloc(&h->w_d, sizeof(float) * ws.size()));
  TRY(cudaMalloc(&h->tab32, sizeof(float) * 16 * P.npoints));
  TRY(cudaMalloc(&h->tab64, sizeof(double) * 14 * P.npoints));
  TRY(cudaMalloc(&h->cell_var_d, sizeof(int) * P.var.size()));
  TRY(cudaMalloc(&h->fam_cells_d, sizeof(int) * P.fam_cells.size()));
  TRY(cudaMemcpy(h->fam_d, P.F.data(), sizeof(RiFam) * P.nfam, cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(h->x_d, xs.data(), sizeof(float) * xs.size(), cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(h->w_d, ws.data(), sizeof(float) * ws.size(), cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(h->cell_var_d, P.var.data(), sizeof(int) * P.var.size(), cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(h->fam_cells_d, P.fam_cells.data(), sizeof(int) * P.fam_cells.size(), cudaMemcpyHostToDevice));
#undef TRY
  *out = h;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_ri_build(const stomsfem_grid* grid, const stomsfem_field* field, double eps,
                                 int32_t nu_max, int32_t nodes, stomsfem_ri** out, int32_t* n_families,
                                 stomsfem_stream_t stream) {
  if (!out) return set_error(STOMSFEM_EINVAL, "out is NULL");
  std::vector<double> xd;
  stomsfem_ri* h = nullptr;
  int rc = ri_setup(grid, field, eps, nu_max, nodes, out, xd);
  if (rc) return rc;
  h = *out;
  *out = nullptr;
  RiPlan& P = h->P;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int ncell = P.ncell, nf = grid->nf, K = P.K;
  double *xi_c = nullptr, *a_c = nullptr, *Ke_c = nullptr, *be_c = nullptr;
  int32_t* list_c = nullptr;
  void* fbws = nullptr;
  auto fail = [&](int code) {
    cudaFree(xi_c);
    cudaFree(a_c);
    cudaFree(Ke_c);
    cudaFree(be_c);
    cudaFree(list_c);
    cudaFree(fbws);
    ri_free(h);
    return code;
  };
#define TRY(x)                                     \
  if ((rc = check_cuda((x), #x)) != STOMSFEM_OK) \
    return fail(rc);
  // collocation: every grid point of a family is one sample of the
  // coefficient (local parameters at the point's nodes, the others 0);
  // the family's first cell of that sample is upscaled in FP64
  const size_t per_pt = (size_t)nf * nf * 8 + (size_t)ncell * 112 + (size_t)K * 8 + 4;
  long long chunk = (256ll << 20) / (long long)per_pt;
  chunk = std::max(1ll, std::min(chunk, std::min(4096ll, P.npoints)));
  const size_t fb_bytes = upscale_list_workspace_fp64(grid);
  TRY(cudaMalloc(&xi_c, sizeof(double) * chunk * K));
  TRY(cudaMalloc(&a_c, sizeof(double) * chunk * nf * nf));
  TRY(cudaMalloc(&Ke_c, sizeof(double) * chunk * ncell * 10));
  TRY(cudaMalloc(&be_c, sizeof(double) * chunk * ncell * 4));
  TRY(cudaMalloc(&list_c, sizeof(int32_t) * (chunk + 1)));
  TRY(cudaMalloc(&fbws, fb_bytes));
  std::vector<double> xi_h((size_t)chunk * K);
  std::vector<int32_t> list_h((size_t)chunk + 1);
  int f = 0;
  for (long long t0 = 0; t0 < P.npoints; t0 += chunk) {
    const int n = (int)std::min(chunk, P.npoints - t0);
    std::fill(xi_h.begin(), xi_h.end(), 0.0);
    for (int j = 0; j < n; ++j) {
      const long long t = t0 + j;
      while (t >= P.F[f].pt0 + P.F[f].npts) ++f;
      const RiFam& F = P.F[f];
      const int cell = P.rep[f];
      long long p = t - F.pt0;
      for (int k = F.ndim - 1; k >= 0; --k) {
        const int d = (int)(p % F.radix[k]);
        p /= F.radix[k];
        xi_h[(size_t)j * K + P.var[(size_t)cell * kRiMaxDim + k]] = xd[(size_t)f * kRiMaxSlots + F.slot0[k] + d];
      }
      list_h[j] = j * ncell + cell;
    }
    list_h[chunk] = n;  // count
    TRY(cudaMemcpyAsync(xi_c, xi_h.data(), sizeof(double) * n * K, cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(list_c, list_h.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(list_c + chunk, &list_h[chunk], sizeof(int32_t), cudaMemcpyHostToDevice, st));
    rc = stomsfem_sample_coef(grid, field, xi_c, n, a_c, stream);
    if (rc) return fail(rc);
    rc = upscale_list_fp64(grid, a_c, n, list_c, list_c + chunk, Ke_c, be_c, fbws, fb_bytes, st);
    if (rc) return fail(rc);
    ri_gather_kernel<<<(n * 16 + 255) / 256, 256, 0, st>>>(n, list_c, Ke_c, be_c, h->tab64 + t0 * 14,
                                                            h->tab32 + t0 * 16);
    TRY(cudaGetLastError());
    TRY(cudaStreamSynchronize(st));  // host buffers are refilled for the next chunk
  }
  cudaFree(xi_c);
  cudaFree(a_c);
  cudaFree(Ke_c);
  cudaFree(be_c);
  cudaFree(list_c);
  cudaFree(fbws);
#undef TRY
  if (n_families) *n_families = P.nfam;
  *out = h;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_ri_destroy(stomsfem_ri* ri) {
  ri_free(ri);
  return STOMSFEM_OK;
}

extern "C" int stomsfem_ri_values(const stomsfem_ri* ri, double* V_host, int64_t n_points) {
  if (!ri || !V_host) return set_error(STOMSFEM_EINVAL, "bad arguments");
  if (n_points != ri->P.npoints)
    return set_error(STOMSFEM_EINVAL, "n_points %lld != %lld", (long long)n_points, ri->P.npoints);
  STOMSFEM_TRY_CUDA(cudaMemcpy(V_host, ri->tab64, sizeof(double) * 14 * n_points, cudaMemcpyDeviceToHost));
  return STOMSFEM_OK;
}

static size_t ri_fb_bytes(const stomsfem_ri* ri) {
  return upscale_list_workspace_fp64(&ri->grid);
}

extern "C" int stomsfem_ri_workspace_size(const stomsfem_ri* ri, int32_t S, size_t* bytes) {
  if (!ri || S < 0 || !bytes) return set_error(STOMSFEM_EINVAL, "bad arguments");
  size_t o = 256 * (((size_t)(ri->P.nfam + 1) * 4 + 255) / 256);  // tile starts
  o += 256;                                                        // count
  o += 256 * (((size_t)S * ri->P.ncell * 4 + 255) / 256);         // direct-upscale list
  o += ri_fb_bytes(ri);
  *bytes = o;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_ri_upscale(stomsfem_ri* ri, const double* xi, const double* a, int32_t S, double* Ke,
                                   double* be, uint8_t* fell_back, void* workspace, size_t workspace_bytes,
                                   stomsfem_stream_t stream) {
  if (!ri || S < 0) return set_error(STOMSFEM_EINVAL, "bad arguments");
  if (S == 0) return STOMSFEM_OK;
  if (!xi || !Ke || !be || !fell_back || !workspace) return set_error(STOMSFEM_EINVAL, "NULL device pointer");
  size_t need = 0;
  stomsfem_ri_workspace_size(ri, S, &need);
  if (workspace_bytes < need) return set_error(STOMSFEM_ENOMEM, "RI workspace %zu < %zu", workspace_bytes, need);
  const RiPlan& P = ri->P;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  int* tile0 = reinterpret_cast<int*>(ws);
  size_t o = 256 * (((size_t)(P.nfam + 1) * 4 + 255) / 256);
  int32_t* count = reinterpret_cast<int32_t*>(ws + o);
  o += 256;
  int32_t* list = reinterpret_cast<int32_t*>(ws + o);
  o += 256 * (((size_t)S * P.ncell * 4 + 255) / 256);
  long long tiles = 0;
  for (int f = 0; f < P.nfam; ++f) tiles += ((long long)S * P.F[f].ncell + kRiUnits - 1) / kRiUnits;
  if (tiles > 0x7fffffffll) return set_error(STOMSFEM_EINVAL, "S too large for one call");
  int maxpts = 0, maxnb = 1, maxslot = 0;
  size_t maxouter = 0;
  for (int f = 0; f < P.nfam; ++f) {
    maxpts = std::max(maxpts, P.F[f].npts);
    maxnb = std::max(maxnb, P.F[f].nb);
    maxslot = std::max(maxslot, P.F[f].nslot_out);
    maxouter = std::max(maxouter, (size_t)(P.F[f].npts / P.F[f].nb) * (P.F[f].ndim - P.F[f].din));
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  STOMSFEM_TRY_CUDA(cudaMemsetAsync(count, 0, 4, st));
  ri_tiles_kernel<<<1, 32, 0, st>>>(P.nfam, ri->fam_d, S, tile0);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  RiEvalArgs A;
  A.xi = xi;
  A.K = P.K;
  A.S = S;
  A.ncell = P.ncell;
  A.nfam = P.nfam;
  A.max_pts = maxpts;
  A.max_nb = maxnb;
  A.max_slot = maxslot;
  A.fam = ri->fam_d;
  A.tile0 = tile0;
  A.x = ri->x_d;
  A.w = ri->w_d;
  A.cell_var = ri->cell_var_d;
  A.fam_cells = ri->fam_cells_d;
  A.tab = reinterpret_cast<const float4*>(ri->tab32);
  A.Ke = Ke;
  A.be = be;
  A.flag = fell_back;
  A.list = a ? list : nullptr;
  A.count = count;
  const size_t smem = (size_t)maxpts * 64 + (size_t)(maxnb + maxslot) * kRiUnits * 4 + ((maxouter + 15) & ~(size_t)15);
  if (smem > 227 * 1024) return set_error(STOMSFEM_EINVAL, "RI tables need %zu B of shared memory", smem);
  STOMSFEM_TRY_CUDA(cudaFuncSetAttribute(ri_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ri_eval_kernel<<<(unsigned)tiles, kRiThreads, smem, st>>>(A);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  if (!a) return STOMSFEM_OK;
  return upscale_list_fp64(&ri->grid, a, S, list, count, Ke, be, ws + o, workspace_bytes - o, st);
}

static const char kRiMagic[8] = {'S', 'T', 'M', 'F', 'R', 'I', 'T', '1'};

extern "C" int stomsfem_ri_save(const stomsfem_ri* ri, void* host_buf, size_t buf_bytes, size_t* bytes) {
  if (!ri || !bytes) return set_error(STOMSFEM_EINVAL, "NULL ri / bytes");
  const size_t nv = (size_t)ri->P.npoints * 14;
  std::vector<double> V;
  if (host_buf) {
    V.resize(nv);
    STOMSFEM_TRY_CUDA(cudaMemcpy(V.data(), ri->tab64, sizeof(double) * nv, cudaMemcpyDeviceToHost));
  }
  CkptWriter w(host_buf, buf_bytes);
  ckpt_header(w, kRiMagic);
  w.val<int32_t>(ri->grid.nf);
  w.val<int32_t>(ri->grid.nc);
  w.val<double>(ri->grid.f);
  w.val<int32_t>(ri->field.kind);
  w.val<int32_t>(ri->field.nbx);
  w.val<int32_t>(ri->field.nby);
  w.val<double>(ri->field.width);
  w.val<double>(ri->field.scale);
  w.val<double>(ri->field.contrast_log);
  w.val<double>(ri->field.gain);
  w.val<double>(ri->eps);
  w.val<int32_t>(ri->nu_max);
  w.val<int32_t>(ri->kind);
  w.val<int64_t>(ri->P.npoints);
  w.put(host_buf ? (const void*)V.data() : nullptr, sizeof(double) * nv);
  *bytes = w.pos;
  if (host_buf && !w.fits()) return set_error(STOMSFEM_ENOMEM, "checkpoint buffer %zu < %zu bytes", buf_bytes, w.pos);
  return STOMSFEM_OK;
}

extern "C" int stomsfem_ri_load(const void* host_buf, size_t buf_bytes, stomsfem_ri** out, int32_t* n_families) {
  if (!host_buf || !out) return set_error(STOMSFEM_EINVAL, "NULL buffer / out");
  *out = nullptr;
  CkptReader r(host_buf, buf_bytes);
  const int hc = ckpt_check_header(r, kRiMagic);
  if (hc == 1) return set_error(STOMSFEM_EVERSION, "not a version-%u interpolation checkpoint", kCkptVersion);
  if (hc == 2) return set_error(STOMSFEM_EINVAL, "truncated interpolation checkpoint");
  stomsfem_grid grid;
  grid.nf = r.val<int32_t>();
  grid.nc = r.val<int32_t>();
  grid.f = r.val<double>();
  stomsfem_field field;
  field.kind = r.val<int32_t>();
  field.nbx = r.val<int32_t>();
  field.nby = r.val<int32_t>();
  field.width = r.val<double>();
  field.scale = r.val<double>();
  field.contrast_log = r.val<double>();
  field.gain = r.val<double>();
  const double eps = r.val<double>();
  const int32_t nu_max = r.val<int32_t>(), kind = r.val<int32_t>();
  const int64_t npts = r.val<int64_t>();
  if (!r.ok) return set_error(STOMSFEM_EINVAL, "truncated interpolation checkpoint");
  if (kind != STOMSFEM_RI_CHEBYSHEV && kind != STOMSFEM_RI_LEGENDRE)
    return set_error(STOMSFEM_EINVAL, "interpolation checkpoint with node family %d", kind);
  {
    // the families are re-derived on the host: their grid must be the stored one
    RiPlan P0;
    const int rp = ri_make_plan(&grid, &field, eps, nu_max, P0);
    if (rp) return set_error(STOMSFEM_EINVAL, "inconsistent interpolation checkpoint header");
    if (P0.npoints != npts)
      return set_error(STOMSFEM_EINVAL, "interpolation checkpoint holds %lld grid points, its plan %lld",
                       (long long)npts, P0.npoints);
  }
  const size_t nv = (size_t)npts * 14;
  if (buf_bytes < r.pos + sizeof(double) * nv) return set_error(STOMSFEM_EINVAL, "truncated interpolation checkpoint");
  std::vector<double> xd;
  stomsfem_ri* h = nullptr;
  int rc = ri_setup(&grid, &field, eps, nu_max, kind, &h, xd);
  if (rc) return rc;
  std::vector<double> V(nv);
  r.get(V.data(), sizeof(double) * nv);
  std::vector<float> V32((size_t)npts * 16, 0.f);
  for (int64_t p = 0; p < npts; ++p)
    for (int q = 0; q < 14; ++q) V32[(size_t)p * 16 + q] = (float)V[(size_t)p * 14 + q];
  rc = check_cuda(cudaMemcpy(h->tab64, V.data(), sizeof(double) * nv, cudaMemcpyHostToDevice), "cudaMemcpy");
  if (rc == STOMSFEM_OK)
    rc = check_cuda(cudaMemcpy(h->tab32, V32.data(), sizeof(float) * V32.size(), cudaMemcpyHostToDevice), "cudaMemcpy");
  if (rc) {
    ri_free(h);
    return rc;
  }
  if (n_families) *n_families = h->P.nfam;
  *out = h;
  return STOMSFEM_OK;
}
