// Coarse assembly and solve (Eq. upscaleSUF) and Monte Carlo moments
// (Eq. MCestimate); the same with mixed boundary data (Sec. 5.2, Eqs.
// xsquarewave / ysquarewave).  One warp per sample: the coarse matrix over the
// (nc-1)^2 interior coarse nodes is again a 9-point-stencil SPD matrix,
// assembled row by row from the K_e of the four cells around each node
// and factorised in FP64 with the blocked banded Cholesky of the cell
// problems (column blocks of 16, rows generated one block ahead).
#include "band_block.cuh"
#include "common.cuh"

namespace stomsfem {

__device__ __forceinline__ int kidx(int l, int lp) {
  // packed upper-triangle index of the symmetric 4x4 entry (l, lp)
  if (l > lp) { const int t = l; l = lp; lp = t; }
  return l * 4 - (l * (l - 1)) / 2 + (lp - l);
}

// Row generator of the coarse system for the blocked solver: a row's five
// band entries and its load, summed from the K_e and b_e of the four cells
// around the node (loads issued one block ahead by prefetch, which stores
// the six sums in the row's raw slot).
struct CoarseBlkGen {
  const double* Ke;  // this sample [nc*nc][10]
  const double* be;  // [nc*nc][4]
  int nc, mx;        // mx = nc - 1 interior nodes per row
  static constexpr int kRaw = 8;
  struct Raw {
    double e[5], rhs;
  };
  __device__ __forceinline__ double K(int cx, int cy, int l, int lp) const {
    return __ldg(Ke + (size_t)(cy * nc + cx) * 10 + kidx(l, lp));
  }
  __device__ __forceinline__ void load(int r, Raw& w) const {
    const int J = r / mx + 1, I = r - (J - 1) * mx + 1;
    // cells around node (I, J): SW (I-1,J-1) node=NE(2); SE (I,J-1) node=NW(3);
    // NE (I,J) node=SW(0); NW (I-1,J) node=SE(1)
    w.e[0] = K(I - 1, J - 1, 2, 2) + K(I, J - 1, 3, 3) + K(I, J, 0, 0) + K(I - 1, J, 1, 1);
    w.e[1] = I > 1 ? K(I - 1, J - 1, 2, 3) + K(I - 1, J, 1, 0) : 0.0;           // west
    w.e[2] = (I < mx && J > 1) ? K(I, J - 1, 3, 1) : 0.0;                       // south-east
    w.e[3] = J > 1 ? K(I - 1, J - 1, 2, 1) + K(I, J - 1, 3, 0) : 0.0;           // south
    w.e[4] = (I > 1 && J > 1) ? K(I - 1, J - 1, 2, 0) : 0.0;                   // south-west
    w.rhs = __ldg(be + (size_t)((J - 1) * nc + I - 1) * 4 + 2) + __ldg(be + (size_t)((J - 1) * nc + I) * 4 + 3) +
            __ldg(be + (size_t)(J * nc + I) * 4 + 0) + __ldg(be + (size_t)(J * nc + I - 1) * 4 + 1);
  }
  __device__ __forceinline__ void prefetch(int r, double* dst) const {
    Raw w;
    load(r, w);
#pragma unroll
    for (int k = 0; k < 5; ++k) dst[k] = w.e[k];
    dst[5] = w.rhs;
  }
  __device__ __forceinline__ void from_smem(const double* src, Raw& w) const {
#pragma unroll
    for (int k = 0; k < 5; ++k) w.e[k] = src[k];
    w.rhs = src[5];
  }
  template <typename T, int NR = 1>
  __device__ __forceinline__ void make(int, const Raw& w, T e[5], T* rh) const {
#pragma unroll
    for (int k = 0; k < 5; ++k) e[k] = (T)w.e[k];
    rh[0] = (T)w.rhs;
  }
};

constexpr int kCoarseBlkWarps = 2;

// Row generator of the standard Q1 FEM on the fine grid (the u_h of the
// two-level estimator, Eq. MCmean2level): the element matrices are
// a_e K_ref, so a row's five band entries come from the four elements
// around the node (SW, SE, NE, NW of the node), and its load is f h^2.
struct FineFemGen {
  const double* a;  // this sample [nf][nf]
  int nf, mx;       // mx = nf - 1 interior nodes per row
  double fh2;       // f h^2
  static constexpr int kRaw = 4;
  struct Raw {
    double sw, se, ne, nw;
  };
  __device__ __forceinline__ void load(int r, Raw& w) const {
    const int J = r / mx + 1, I = r - (J - 1) * mx + 1;
    w.sw = __ldg(a + (size_t)(J - 1) * nf + I - 1);
    w.se = __ldg(a + (size_t)(J - 1) * nf + I);
    w.ne = __ldg(a + (size_t)J * nf + I);
    w.nw = __ldg(a + (size_t)J * nf + I - 1);
  }
  __device__ __forceinline__ void prefetch(int r, double* dst) const {
    Raw w;
    load(r, w);
    dst[0] = w.sw;
    dst[1] = w.se;
    dst[2] = w.ne;
    dst[3] = w.nw;
  }
  __device__ __forceinline__ void from_smem(const double* src, Raw& w) const {
    w.sw = src[0];
    w.se = src[1];
    w.ne = src[2];
    w.nw = src[3];
  }
  // K_ref = [4 -1 -2 -1; -1 4 -1 -2; -2 -1 4 -1; -1 -2 -1 4] / 6 (SW, SE, NE, NW)
  template <typename T, int NR = 1>
  __device__ __forceinline__ void make(int r, const Raw& w, T e[5], T* rh) const {
    const int J = r / mx + 1, I = r - (J - 1) * mx + 1;
    const double s6 = 1.0 / 6.0;
    e[0] = (T)(4.0 * s6 * (w.sw + w.se + w.ne + w.nw));
    e[1] = (T)(I > 1 ? -s6 * (w.sw + w.nw) : 0.0);                 // west
    e[2] = (T)((I < mx && J > 1) ? -2.0 * s6 * w.se : 0.0);        // south-east
    e[3] = (T)(J > 1 ? -s6 * (w.sw + w.se) : 0.0);                 // south
    e[4] = (T)((I > 1 && J > 1) ? -2.0 * s6 * w.sw : 0.0);         // south-west
    rh[0] = (T)fh2;
  }
};

template <int RPL>
__global__ void __launch_bounds__(kCoarseBlkWarps * 32)
fine_fem_kernel(int nf, int S, double f, const double* __restrict__ a, double* __restrict__ u, unsigned char* ws,
                size_t slot_bytes, size_t l_bytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int mx = nf - 1, n = mx * mx, b = nf;
  const BlkSmem<double> sm = make_blk<double>(smem + wib * blk_smem_bytes<double>(16, b), 16, b);
  const int gw = blockIdx.x * kCoarseBlkWarps + wib, nw = gridDim.x * kCoarseBlkWarps;
  unsigned char* slot = ws + (size_t)gw * slot_bytes;
  double* Lg = reinterpret_cast<double*>(slot);
  double* x = reinterpret_cast<double*>(slot + l_bytes);
  const int NN = nf + 1;
  const double h = 1.0 / nf;
  for (int s = gw; s < S; s += nw) {
    const FineFemGen gen{a + (size_t)s * nf * nf, nf, mx, f * h * h};
    int fail = -1;
    if (n > 0) {
      fail = blk_factor<32, double, 1, RPL>(gen, n, b, b, sm, Lg, x, lane);
      blk_backward<32, double, 1>(n, b, b, sm, Lg, x, lane);
    }
    __syncwarp();
    double* us = u + (size_t)s * NN * NN;
    const double nanv = __longlong_as_double(0x7ff8000000000000ll);
    for (int q = lane; q < NN * NN; q += 32) {
      const int I = q % NN, J = q / NN;
      double v = 0.0;
      if (I > 0 && J > 0 && I < nf && J < nf) v = fail < 0 ? x[(J - 1) * mx + (I - 1)] : nanv;
      us[q] = v;
    }
    __syncwarp();
  }
}

// d[s][coarse node] = u_fine at that node (minus u_coarse when given).
__global__ void restrict_kernel(int nf, int nc, int S, const double* __restrict__ uf, const double* __restrict__ uc,
                                double* __restrict__ d) {
  const int NC = nc + 1, NF = nf + 1, rho = nf / nc;
  const long long total = (long long)S * NC * NC;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / (NC * NC)), q = (int)(i % (NC * NC));
    const int I = q % NC, J = q / NC;
    double v = uf[(size_t)s * NF * NF + (size_t)(J * rho) * NF + I * rho];
    if (uc) v -= uc[i];
    d[i] = v;
  }
}

template <int RPL>
__global__ void __launch_bounds__(kCoarseBlkWarps * 32)
coarse_blk_kernel(int nc, int S, const double* __restrict__ Ke, const double* __restrict__ be,
                  double* __restrict__ u, unsigned char* ws, size_t slot_bytes, size_t l_bytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int mx = nc - 1, n = mx * mx, b = nc;
  const BlkSmem<double> sm =
      make_blk<double>(smem + wib * blk_smem_bytes<double>(16, b, CoarseBlkGen::kRaw), 16, b, CoarseBlkGen::kRaw);
  const int gw = blockIdx.x * kCoarseBlkWarps + wib, nw = gridDim.x * kCoarseBlkWarps;
  unsigned char* slot = ws + (size_t)gw * slot_bytes;
  double* Lg = reinterpret_cast<double*>(slot);
  double* x = reinterpret_cast<double*>(slot + l_bytes);
  const int NN = nc + 1;
  for (int s = gw; s < S; s += nw) {
    const CoarseBlkGen gen{Ke + (size_t)s * nc * nc * 10, be + (size_t)s * nc * nc * 4, nc, mx};
    int fail = -1;
    if (n > 0) {
      fail = blk_factor<32, double, 1, RPL>(gen, n, b, b, sm, Lg, x, lane);
      blk_backward<32, double, 1>(n, b, b, sm, Lg, x, lane);
    }
    __syncwarp();
    double* us = u + (size_t)s * NN * NN;
    const double nanv = __longlong_as_double(0x7ff8000000000000ll);
    for (int q = lane; q < NN * NN; q += 32) {
      const int I = q % NN, J = q / NN;
      double v = 0.0;
      if (I > 0 && J > 0 && I < nc && J < nc) v = fail < 0 ? x[(J - 1) * mx + (I - 1)] : nanv;
      us[q] = v;
    }
    __syncwarp();
  }
}

// Mixed boundary data (the anisotropy study of Sec. 5.2, Eqs. xsquarewave
// and ysquarewave): every coarse node is an unknown (mx = nc + 1 nodes per
// row, half bandwidth mx + 1).  A node with dm != 0 has the row u = g; a
// free node's row sums the cells around it that exist (zero flux needs no
// other term on the boundary), and each coupling to a prescribed neighbour
// moves, times its g, to the right-hand side (symmetric elimination, so the
// matrix stays SPD for the blocked Cholesky).
struct CoarseBcGen {
  const double* Ke;   // this sample [nc*nc][10]
  const double* be;   // [nc*nc][4]
  const uint8_t* dm;  // [(nc+1)^2] nonzero: prescribed value
  const double* gv;   // [(nc+1)^2] the prescribed values
  int nc, mx;         // mx = nc + 1 nodes per row
  static constexpr int kRaw = 8;
  using Raw = CoarseBlkGen::Raw;
  __device__ __forceinline__ double K(int cx, int cy, int l, int lp) const {
    return __ldg(Ke + (size_t)(cy * nc + cx) * 10 + kidx(l, lp));
  }
  __device__ __forceinline__ double B(int cx, int cy, int l) const {
    return __ldg(be + (size_t)(cy * nc + cx) * 4 + l);
  }
  __device__ __forceinline__ void load(int r, Raw& w) const {
#pragma unroll
    for (int k = 0; k < 5; ++k) w.e[k] = 0.0;
    if (__ldg(dm + r)) {
      w.e[0] = 1.0;
      w.rhs = __ldg(gv + r);
      return;
    }
    const int J = r / mx, I = r - J * mx;
    const bool hw = I > 0, he = I < nc, hs = J > 0, hn = J < nc;
    // couplings to the eight neighbours, from the cells around (I, J):
    // SW cell (I-1, J-1) has the node as corner 2, SE cell (I, J-1) as 3,
    // NE cell (I, J) as 0, NW cell (I-1, J) as 1
    double cW = 0, cE = 0, cS = 0, cN = 0, cSW = 0, cSE = 0, cNE = 0, cNW = 0, d = 0, f = 0;
    if (hw && hs) {
      d += K(I - 1, J - 1, 2, 2);
      cSW += K(I - 1, J - 1, 2, 0);
      cS += K(I - 1, J - 1, 2, 1);
      cW += K(I - 1, J - 1, 2, 3);
      f += B(I - 1, J - 1, 2);
    }
    if (he && hs) {
      d += K(I, J - 1, 3, 3);
      cS += K(I, J - 1, 3, 0);
      cSE += K(I, J - 1, 3, 1);
      cE += K(I, J - 1, 3, 2);
      f += B(I, J - 1, 3);
    }
    if (he && hn) {
      d += K(I, J, 0, 0);
      cE += K(I, J, 0, 1);
      cNE += K(I, J, 0, 2);
      cN += K(I, J, 0, 3);
      f += B(I, J, 0);
    }
    if (hw && hn) {
      d += K(I - 1, J, 1, 1);
      cW += K(I - 1, J, 1, 0);
      cN += K(I - 1, J, 1, 2);
      cNW += K(I - 1, J, 1, 3);
      f += B(I - 1, J, 1);
    }
    // a neighbour that exists is either prescribed (to the right-hand side)
    // or free; the free ones below the diagonal are the band entries
    auto nb = [&](bool exists, int q, double c, double* band) {
      if (!exists) return;
      if (__ldg(dm + q))
        f -= c * __ldg(gv + q);
      else if (band)
        *band = c;
    };
    nb(hw, r - 1, cW, &w.e[1]);
    nb(he && hs, r - mx + 1, cSE, &w.e[2]);
    nb(hs, r - mx, cS, &w.e[3]);
    nb(hw && hs, r - mx - 1, cSW, &w.e[4]);
    nb(he, r + 1, cE, nullptr);
    nb(hn, r + mx, cN, nullptr);
    nb(he && hn, r + mx + 1, cNE, nullptr);
    nb(hw && hn, r + mx - 1, cNW, nullptr);
    w.e[0] = d;
    w.rhs = f;
  }
  __device__ __forceinline__ void prefetch(int r, double* dst) const {
    Raw w;
    load(r, w);
#pragma unroll
    for (int k = 0; k < 5; ++k) dst[k] = w.e[k];
    dst[5] = w.rhs;
  }
  __device__ __forceinline__ void from_smem(const double* src, Raw& w) const {
#pragma unroll
    for (int k = 0; k < 5; ++k) w.e[k] = src[k];
    w.rhs = src[5];
  }
  template <typename T, int NR = 1>
  __device__ __forceinline__ void make(int, const Raw& w, T e[5], T* rh) const {
#pragma unroll
    for (int k = 0; k < 5; ++k) e[k] = (T)w.e[k];
    rh[0] = (T)w.rhs;
  }
};

// One warp per sample, as coarse_blk_kernel, over all (nc+1)^2 nodes.
template <int RPL>
__global__ void __launch_bounds__(kCoarseBlkWarps * 32)
coarse_bc_kernel(int nc, int S, const double* __restrict__ Ke, const double* __restrict__ be,
                 const uint8_t* __restrict__ dm, const double* __restrict__ gv, double* __restrict__ u,
                 unsigned char* ws, size_t slot_bytes, size_t l_bytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int mx = nc + 1, n = mx * mx, b = mx + 1;
  const BlkSmem<double> sm =
      make_blk<double>(smem + wib * blk_smem_bytes<double>(16, b, CoarseBcGen::kRaw), 16, b, CoarseBcGen::kRaw);
  const int gw = blockIdx.x * kCoarseBlkWarps + wib, nw = gridDim.x * kCoarseBlkWarps;
  unsigned char* slot = ws + (size_t)gw * slot_bytes;
  double* Lg = reinterpret_cast<double*>(slot);
  double* x = reinterpret_cast<double*>(slot + l_bytes);
  for (int s = gw; s < S; s += nw) {
    const CoarseBcGen gen{Ke + (size_t)s * nc * nc * 10, be + (size_t)s * nc * nc * 4, dm, gv, nc, mx};
    const int fail = blk_factor<32, double, 1, RPL>(gen, n, b, b, sm, Lg, x, lane);
    blk_backward<32, double, 1>(n, b, b, sm, Lg, x, lane);
    __syncwarp();
    double* us = u + (size_t)s * n;
    const double nanv = __longlong_as_double(0x7ff8000000000000ll);
    for (int q = lane; q < n; q += 32) us[q] = fail < 0 ? x[q] : nanv;
    __syncwarp();
  }
}

// Merge this batch's moments into the running ones (pairwise update of
// Chan, Golub and LeVeque): batch mean/M2 two-pass, then combine.
__global__ void moments_kernel(int nn, int S, const double* __restrict__ u, double* mean, double* m2,
                               const double* count) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nn) return;
  double mb = 0.0;
  for (int s = 0; s < S; ++s) mb += u[(size_t)s * nn + q];
  mb /= S;
  double M2b = 0.0;
  for (int s = 0; s < S; ++s) {
    const double d = u[(size_t)s * nn + q] - mb;
    M2b += d * d;
  }
  const double na = count[0], nb = (double)S, nt = na + nb;
  const double delta = mb - mean[q];
  mean[q] = mean[q] + delta * (nb / nt);
  m2[q] = m2[q] + M2b + delta * delta * (na * nb / nt);
}

__global__ void count_kernel(double* count, int S) { count[0] += (double)S; }

// Merge a second set of running moments (mean_b, m2_b, count_b: another
// rank's, or another stream's) into (mean, m2, count): the same pairwise
// update; one block, the counts read before any is written.
__global__ void moments_merge_kernel(int nn, double* mean, double* m2, double* count, const double* __restrict__ mean_b,
                                     const double* __restrict__ m2_b, const double* __restrict__ count_b) {
  const double na = count[0], nb = count_b[0], nt = na + nb;
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {
    if (nb == 0.0) break;
    const double delta = mean_b[q] - mean[q];
    mean[q] = mean[q] + delta * (nb / nt);
    m2[q] = m2[q] + m2_b[q] + delta * delta * (na * nb / nt);
  }
  __syncthreads();
  if (threadIdx.x == 0) count[0] = nt;
}

// ---- Petrov-Galerkin coarse system (Eq. stiffness_local_petrov): row J
// (test node) collects S_e[I_loc][J_loc] over the cells around J, a
// non-symmetric band of half width bw = nc.  Banded LU without pivoting,
// one warp per sample: the rows k..k+bw live in a shared-memory ring (row
// i keeps columns i-bw..i+bw, pitch 2 bw + 2); step k eliminates column k from the bw rows
// below (lane t owns rows k+1+t, k+33+t; with mixed boundary data the
// columns of rows past k+32 are shared by all lanes), writes the finished
// U row and its
// right-hand side to the sample's scratch, and brings in row k+bw+1, whose
// 16 contributions (4 cells x 4 trial corners) were loaded one step ahead.
// Back substitution reads the U rows back with a ring of the last bw
// unknowns.  A zero or non-finite pivot gives the sample NaN values.
constexpr int kCoarsePgWarps = 2;

struct PgRowPrefetch {
  double v;  // contribution of this lane (0 if none)
  int off;   // column offset within the row (-1: none)
  double b;  // load contribution (lanes 0..3)
};

// Lane l < 16 takes cell c = l / 4 around node J and trial corner t = l % 4.
__device__ __forceinline__ PgRowPrefetch pg_row_load(int nc, const double* __restrict__ Ks,
                                                     const double* __restrict__ bs, int J, int n, int lane) {
  PgRowPrefetch p{0.0, -1, 0.0};
  if (J >= n || lane >= 16) return p;
  const int mi = nc - 1;
  const int i = J % mi + 1, j = J / mi + 1;  // coarse node of row J
  const int c = lane >> 2, t = lane & 3;
  // cells with node (i, j) as corner r: NE of (i-1, j-1), NW of (i, j-1),
  // SW of (i, j), SE of (i-1, j)
  const int cx = i - 1 + (c == 1 || c == 2), cy = j - 1 + (c >= 2), r = (c + 2) & 3;
  const int tx = cx + (t == 1 || t == 2), ty = cy + (t >= 2);
  const size_t cell = (size_t)cy * nc + cx;
  if (tx > 0 && tx < nc && ty > 0 && ty < nc) {
    const int I = (ty - 1) * mi + (tx - 1);
    p.v = Ks[cell * 16 + t * 4 + r];
    p.off = I - J + nc;
  }
  if (t == 0) p.b = bs[cell * 4 + r];
  return p;
}

// Row J of the system with mixed boundary data (every node a row, nc + 1
// per row, half bandwidth nc + 2), in two parts so that the loads of the
// next row overlap a whole elimination step: pg_row_fetch_bc issues every
// load with control flow on indices only (no branch waits for a loaded
// value), pg_row_resolve_bc combines the values where the row is consumed.
// A prescribed node's row is u_J = g_J (lane 0); in a free row the lanes
// take the cells and trial corners as pg_row_load, cells outside the domain
// give nothing (zero flux), and a prescribed trial node moves its
// contribution times g to the load.
struct PgRowRawBc {
  double v, b, gJ, gI;  // S_e entry, cell load, prescribed values of row and trial node
  int off;              // column offset of the trial node, -1: no cell
  int t0;               // this lane adds the cell's load
  uint8_t dJ, dI;       // row / trial node prescribed
};

__device__ __forceinline__ PgRowRawBc pg_row_fetch_bc(int nc, const double* __restrict__ Ks,
                                                      const double* __restrict__ bs, const uint8_t* __restrict__ dm,
                                                      const double* __restrict__ gv, int J, int n, int lane) {
  PgRowRawBc q{0.0, 0.0, 0.0, 0.0, -1, 0, 0, 0};
  if (J >= n || lane >= 16) return q;
  const int NN = nc + 1, bw = nc + 2;
  q.dJ = dm[J];
  q.gJ = gv[J];
  const int i = J % NN, j = J / NN;
  const int c = lane >> 2, t = lane & 3;
  const int cx = i - 1 + (c == 1 || c == 2), cy = j - 1 + (c >= 2), r = (c + 2) & 3;
  if (cx < 0 || cx >= nc || cy < 0 || cy >= nc) return q;
  const int tx = cx + (t == 1 || t == 2), ty = cy + (t >= 2);
  const size_t cell = (size_t)cy * nc + cx;
  const int I = ty * NN + tx;
  q.v = Ks[cell * 16 + t * 4 + r];
  q.dI = dm[I];
  q.gI = gv[I];
  q.off = I - J + bw;
  q.t0 = t == 0;
  if (t == 0) q.b = bs[cell * 4 + r];
  return q;
}

__device__ __forceinline__ PgRowPrefetch pg_row_resolve_bc(const PgRowRawBc& q, int bw, int lane) {
  PgRowPrefetch p{0.0, -1, 0.0};
  if (q.dJ) {
    if (lane == 0) {
      p.v = 1.0;
      p.off = bw;
      p.b = q.gJ;
    }
    return p;
  }
  if (q.off < 0) return p;
  if (q.dI) {
    p.b = -q.v * q.gI;
  } else {
    p.v = q.v;
    p.off = q.off;
  }
  if (q.t0) p.b += q.b;
  return p;
}

// BC: the system over every node with mixed boundary data (pg_row_fetch_bc),
// else the interior nodes with zero Dirichlet data.
template <bool BC>
__global__ void __launch_bounds__(kCoarsePgWarps * 32)
coarse_pg_kernel(int nc, int S, const double* __restrict__ Kpg, const double* __restrict__ bpg,
                 const uint8_t* __restrict__ dm, const double* __restrict__ gv, double* __restrict__ u,
                 unsigned char* __restrict__ ws, size_t slot_bytes) {
  extern __shared__ __align__(16) unsigned char smem_pg[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // row pitch PW = W + 1 (even): consecutive lanes, one row apart, then
  // differ by an odd number of doubles and meet different banks
  const int bw = BC ? nc + 2 : nc, W = 2 * bw + 1, PW = W + 1, R = bw + 1;
  const int mi = BC ? nc + 1 : nc - 1, n = mi * mi, NN = nc + 1;
  // row loads in flight during a step (raw values with mixed boundary
  // data), and the contributions they give where the row is consumed
  auto row_load = [&](const double* Ks, const double* bs, int J) {
    if constexpr (BC)
      return pg_row_fetch_bc(nc, Ks, bs, dm, gv, J, n, lane);
    else
      return pg_row_load(nc, Ks, bs, J, n, lane);
  };
  auto resolve = [&](const auto& q) {
    if constexpr (BC)
      return pg_row_resolve_bc(q, bw, lane);
    else
      return q;
  };
  // lanes whose load term is added: one per cell, or (BC) every lane with
  // a term (prescribed trial nodes move theirs to the load)
  auto adds_b = [&](const PgRowPrefetch& p) { return lane < 16 && (BC ? p.b != 0.0 : (lane & 3) == 0); };
  double* Rw = reinterpret_cast<double*>(smem_pg) + (size_t)wib * (R * PW + 3 * R);
  double* yr = Rw + (size_t)R * PW;  // right-hand sides of the window rows
  double* xr = yr + R;              // ring of the last bw unknowns
  double* lm = xr + R;              // multipliers of the rows beyond 32
  double* Ug = reinterpret_cast<double*>(ws + (size_t)(blockIdx.x * kCoarsePgWarps + wib) * slot_bytes);
  const long long gw = (long long)blockIdx.x * kCoarsePgWarps + wib;
  const long long nw = (long long)gridDim.x * kCoarsePgWarps;
  for (long long sl = gw; sl < S; sl += nw) {
    const double* Ks = Kpg + (size_t)sl * nc * nc * 16;
    const double* bs = bpg + (size_t)sl * nc * nc * 4;
    double* us = u + (size_t)sl * NN * NN;
    // window: rows 0..bw (zeroed, then their contributions)
    for (int q = lane; q < R * PW; q += 32) Rw[q] = 0.0;
    for (int q = lane; q < R; q += 32) yr[q] = 0.0;
    __syncwarp();
    for (int J = 0; J < R && J < n; ++J) {
      const PgRowPrefetch p = resolve(row_load(Ks, bs, J));
      if (p.off >= 0) atomicAdd(&Rw[(size_t)(J % R) * PW + p.off], p.v);
      if (adds_b(p)) atomicAdd(&yr[J % R], p.b);
      __syncwarp();
    }
    auto next = row_load(Ks, bs, R);
    bool bad = false;
    for (int k = 0; k < n; ++k) {
      const auto cur_raw = next;
      next = row_load(Ks, bs, k + R + 1);  // in flight during this step
      double* P = Rw + (size_t)(k % R) * PW;
      const double piv = P[bw];
      if (!(fabs(piv) > 0.0) || !(fabs(piv) < 1e300)) bad = true;
      const double inv = 1.0 / piv;
      const double yk = yr[k % R];
      // lane t takes row k+1+t whole (and row k+33+t); with mixed boundary
      // data the band is nc + 2, just past 32 at nc = 32, so there rows
      // k+33..k+bw give lane t-32 only their multipliers and all lanes then
      // share their columns (a second row per lane would double the step's
      // serial update)
      for (int t = lane; t < bw; t += 32) {
        const int i = k + 1 + t;
        double l = 0.0;
        if (i < n) {
          double* Ri = Rw + (size_t)(i % R) * PW;
          l = Ri[bw - 1 - t] * inv;
          Ri[bw - 1 - t] = 0.0;
          if (l != 0.0) {
            if (!BC || t < 32)
              for (int jj = 1; jj <= bw; ++jj) Ri[bw - 1 - t + jj] -= l * P[bw + jj];
            yr[i % R] -= l * yk;
          }
        }
        if (BC && t >= 32) lm[t - 32] = l;
      }
      if (BC && bw > 32) {
        __syncwarp();
        for (int t = 32; t < bw; ++t) {
          const double l = lm[t - 32];
          if (l != 0.0) {
            double* Ri = Rw + (size_t)((k + 1 + t) % R) * PW;
            for (int c = lane; c < bw; c += 32) Ri[bw + c - t] -= l * P[bw + 1 + c];
          }
        }
      }
      // finished U row k (columns k..k+bw) and its right-hand side
      for (int q = lane; q <= bw; q += 32) Ug[(size_t)k * (bw + 2) + q] = P[bw + q];
      if (lane == 0) Ug[(size_t)k * (bw + 2) + bw + 1] = yk;
      __syncwarp();
      // slot of row k takes row k + R
      for (int q = lane; q < W; q += 32) P[q] = 0.0;
      if (lane == 0) yr[k % R] = 0.0;
      __syncwarp();
      if (k + R < n) {
        const PgRowPrefetch cur = resolve(cur_raw);
        if (cur.off >= 0) atomicAdd(&P[cur.off], cur.v);
        if (adds_b(cur)) atomicAdd(&yr[k % R], cur.b);
      }
      __syncwarp();
    }
    bad = __any_sync(0xffffffffu, bad);
    // back substitution, x ring of R entries
    for (int k = n - 1; k >= 0; --k) {
      const double* Uk = Ug + (size_t)k * (bw + 2);
      double part = 0.0;
      for (int jj = 1 + lane; jj <= bw; jj += 32)
        if (k + jj < n) part += Uk[jj] * xr[(k + jj) % R];
      part = warp_sum(part);
      const double xk = (Uk[bw + 1] - part) / Uk[0];
      __syncwarp();
      if (lane == 0) xr[k % R] = xk;
      __syncwarp();
      if (lane == 0) {
        const int q = BC ? k : (k / mi + 1) * NN + (k % mi + 1);
        us[q] = bad ? __longlong_as_double(0x7ff8000000000000ll) : xk;
      }
    }
    if constexpr (!BC) {
      for (int q = lane; q < NN * NN; q += 32) {
        const int i = q % NN, j = q / NN;
        if (i == 0 || j == 0 || i == nc || j == nc) us[q] = 0.0;
      }
    }
    __syncwarp();
  }
}

// Sizes of the Petrov-Galerkin solve: half bandwidth bw (nc, or nc + 2 with
// mixed boundary data, whose rows are all (nc+1)^2 nodes).
static size_t coarse_pg_slot_bytes(int nc, bool bc = false) {
  const int mi = bc ? nc + 1 : nc - 1, n = mi * mi > 0 ? mi * mi : 1, bw = bc ? nc + 2 : nc;
  return ((size_t)n * (bw + 2) * 8 + 255) & ~size_t(255);
}
static size_t coarse_pg_smem(int nc, bool bc = false) {
  const int bw = bc ? nc + 2 : nc;
  return (size_t)kCoarsePgWarps * ((size_t)(bw + 1) * (2 * bw + 2) + 3 * (bw + 1)) * 8;
}

// Galerkin solve with mixed boundary data: factor blocks of the (nc+1)^2
// node system (half bandwidth nc + 2), then the solution.
static size_t coarse_bc_l_bytes(int nc) {
  const int n = (nc + 1) * (nc + 1);
  return (blk_factor_elems(n, nc + 2) * 8 + 255) & ~size_t(255);
}
static size_t coarse_bc_slot_bytes(int nc) {
  const int n = (nc + 1) * (nc + 1);
  return coarse_bc_l_bytes(nc) + (((size_t)n * 8 + 255) & ~size_t(255));
}

// Slot of one sample: the factor blocks, then the solution.
static size_t coarse_l_bytes(int nc) {
  const int mi = nc - 1, n = mi * mi > 0 ? mi * mi : 1;
  return (blk_factor_elems(n, nc) * 8 + 255) & ~size_t(255);
}
static size_t coarse_slot_bytes(int nc) {
  const int mi = nc - 1, n = mi * mi > 0 ? mi * mi : 1;
  return coarse_l_bytes(nc) + (((size_t)n * 8 + 255) & ~size_t(255));
}

}  // namespace stomsfem

using namespace stomsfem;

extern "C" int stomsfem_coarse_workspace_size(const stomsfem_grid* grid, int32_t S, size_t* bytes) {
  if (!grid || grid->nc <= 0 || S < 0 || !bytes) return set_error(STOMSFEM_EINVAL, "bad arguments");
  const int sms = device_sm_count();
  long long slots = (long long)(sms > 0 ? sms : 152) * 8;
  if (slots > S) slots = S;
  if (slots < kCoarseBlkWarps) slots = kCoarseBlkWarps;
  *bytes = coarse_slot_bytes(grid->nc) * (size_t)slots;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_coarse_solve(const stomsfem_grid* grid, const double* Ke, const double* be,
                                     int32_t S, double* u, double* mean, double* m2, double* count,
                                     void* workspace, size_t workspace_bytes,
                                     stomsfem_stream_t stream) {
  if (!grid || grid->nc <= 0) return set_error(STOMSFEM_EINVAL, "bad grid");
  if (grid->nc > 64) return set_error(STOMSFEM_EINVAL, "nc %d > 64 (coarse bandwidth limit)", grid->nc);
  if (S < 0) return set_error(STOMSFEM_EINVAL, "S < 0");
  if (S == 0) return STOMSFEM_OK;
  if (!Ke || !be || !u || !workspace) return set_error(STOMSFEM_EINVAL, "NULL device pointer");
  const bool mom = mean || m2 || count;
  if (mom && !(mean && m2 && count))
    return set_error(STOMSFEM_EINVAL, "mean, m2 and count must be given together");
  const size_t sb = coarse_slot_bytes(grid->nc);
  long long slots = (long long)(workspace_bytes / sb);
  if (slots < kCoarseBlkWarps)
    return set_error(STOMSFEM_ENOMEM, "coarse workspace %zu < %d slots of %zu", workspace_bytes,
                     kCoarseBlkWarps, sb);
  long long blocks = slots / kCoarseBlkWarps;
  const long long need = ((long long)S + kCoarseBlkWarps - 1) / kCoarseBlkWarps;
  if (blocks > need) blocks = need;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int nc = grid->nc;
  const size_t smem = blk_smem_bytes<double>(16, nc, CoarseBlkGen::kRaw) * kCoarseBlkWarps;
  const int rpl = (16 + nc + 31) / 32;
  auto kern = rpl <= 1 ? coarse_blk_kernel<1> : rpl == 2 ? coarse_blk_kernel<2> : coarse_blk_kernel<3>;
  STOMSFEM_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<(unsigned)blocks, kCoarseBlkWarps * 32, smem, st>>>(nc, S, Ke, be, u,
                                                              static_cast<unsigned char*>(workspace), sb,
                                                              coarse_l_bytes(nc));
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  if (mom) {
    const int nn = (grid->nc + 1) * (grid->nc + 1);
    moments_kernel<<<(nn + 127) / 128, 128, 0, st>>>(nn, S, u, mean, m2, count);
    STOMSFEM_TRY_CUDA(cudaGetLastError());
    count_kernel<<<1, 1, 0, st>>>(count, S);
    STOMSFEM_TRY_CUDA(cudaGetLastError());
  }
  return STOMSFEM_OK;
}

extern "C" int stomsfem_coarse_pg_workspace_size(const stomsfem_grid* grid, int32_t S, size_t* bytes) {
  if (!grid || grid->nc <= 0 || S < 0 || !bytes) return set_error(STOMSFEM_EINVAL, "bad arguments");
  const int sms = device_sm_count();
  long long slots = (long long)(sms > 0 ? sms : 152) * 4;
  if (slots > S) slots = S;
  if (slots < kCoarsePgWarps) slots = kCoarsePgWarps;
  *bytes = coarse_pg_slot_bytes(grid->nc) * (size_t)slots;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_coarse_solve_pg(const stomsfem_grid* grid, const double* Kpg, const double* bpg,
                                        int32_t S, double* u, double* mean, double* m2, double* count,
                                        void* workspace, size_t workspace_bytes, stomsfem_stream_t stream) {
  if (!grid || grid->nc <= 0) return set_error(STOMSFEM_EINVAL, "bad grid");
  if (grid->nc < 2) return set_error(STOMSFEM_EINVAL, "nc must be >= 2");
  if (grid->nc > 64) return set_error(STOMSFEM_EINVAL, "nc %d > 64 (coarse bandwidth limit)", grid->nc);
  if (S < 0) return set_error(STOMSFEM_EINVAL, "S < 0");
  if (S == 0) return STOMSFEM_OK;
  if (!Kpg || !bpg || !u || !workspace) return set_error(STOMSFEM_EINVAL, "NULL device pointer");
  const bool mom = mean || m2 || count;
  if (mom && !(mean && m2 && count))
    return set_error(STOMSFEM_EINVAL, "mean, m2 and count must be given together");
  const size_t sb = coarse_pg_slot_bytes(grid->nc);
  long long slots = (long long)(workspace_bytes / sb);
  if (slots < kCoarsePgWarps)
    return set_error(STOMSFEM_ENOMEM, "coarse workspace %zu < %d slots of %zu", workspace_bytes, kCoarsePgWarps,
                     sb);
  long long blocks = slots / kCoarsePgWarps;
  const long long need = ((long long)S + kCoarsePgWarps - 1) / kCoarsePgWarps;
  if (blocks > need) blocks = need;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t smem = coarse_pg_smem(grid->nc);
  STOMSFEM_TRY_CUDA(
      cudaFuncSetAttribute(coarse_pg_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  coarse_pg_kernel<false><<<(unsigned)blocks, kCoarsePgWarps * 32, smem, st>>>(
      grid->nc, S, Kpg, bpg, nullptr, nullptr, u, static_cast<unsigned char*>(workspace), sb);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  if (mom) {
    const int nn = (grid->nc + 1) * (grid->nc + 1);
    moments_kernel<<<(nn + 127) / 128, 128, 0, st>>>(nn, S, u, mean, m2, count);
    STOMSFEM_TRY_CUDA(cudaGetLastError());
    count_kernel<<<1, 1, 0, st>>>(count, S);
    STOMSFEM_TRY_CUDA(cudaGetLastError());
  }
  return STOMSFEM_OK;
}

// Largest coarse grid of the solves with mixed boundary data: their half
// bandwidth nc + 2 stays within the 64 of the other coarse solves.
constexpr int kCoarseBcMaxNc = 62;

extern "C" int stomsfem_coarse_bc_workspace_size(const stomsfem_grid* grid, int32_t pg, int32_t S, size_t* bytes) {
  if (!grid || grid->nc <= 0 || S < 0 || !bytes || (pg != 0 && pg != 1))
    return set_error(STOMSFEM_EINVAL, "bad arguments");
  const int sms = device_sm_count();
  const int warps = pg ? kCoarsePgWarps : kCoarseBlkWarps;
  long long slots = (long long)(sms > 0 ? sms : 152) * (pg ? 4 : 8);
  if (slots > S) slots = S;
  if (slots < warps) slots = warps;
  *bytes = (pg ? coarse_pg_slot_bytes(grid->nc, true) : coarse_bc_slot_bytes(grid->nc)) * (size_t)slots;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_coarse_solve_bc(const stomsfem_grid* grid, int32_t pg, const double* K, const double* b,
                                        const uint8_t* dirichlet, const double* g, int32_t S, double* u,
                                        double* mean, double* m2, double* count, void* workspace,
                                        size_t workspace_bytes, stomsfem_stream_t stream) {
  if (!grid || grid->nc <= 0) return set_error(STOMSFEM_EINVAL, "bad grid");
  if (grid->nc > kCoarseBcMaxNc)
    return set_error(STOMSFEM_EINVAL, "nc %d > %d (bandwidth limit with mixed boundary data)", grid->nc,
                     kCoarseBcMaxNc);
  if (pg != 0 && pg != 1) return set_error(STOMSFEM_EINVAL, "pg must be 0 or 1");
  if (S < 0) return set_error(STOMSFEM_EINVAL, "S < 0");
  if (S == 0) return STOMSFEM_OK;
  if (!K || !b || !dirichlet || !g || !u || !workspace) return set_error(STOMSFEM_EINVAL, "NULL device pointer");
  const bool mom = mean || m2 || count;
  if (mom && !(mean && m2 && count))
    return set_error(STOMSFEM_EINVAL, "mean, m2 and count must be given together");
  const int nc = grid->nc;
  const int warps = pg ? kCoarsePgWarps : kCoarseBlkWarps;
  const size_t sb = pg ? coarse_pg_slot_bytes(nc, true) : coarse_bc_slot_bytes(nc);
  long long slots = (long long)(workspace_bytes / sb);
  if (slots < warps)
    return set_error(STOMSFEM_ENOMEM, "coarse workspace %zu < %d slots of %zu", workspace_bytes, warps, sb);
  long long blocks = slots / warps;
  const long long need = ((long long)S + warps - 1) / warps;
  if (blocks > need) blocks = need;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  if (pg) {
    const size_t smem = coarse_pg_smem(nc, true);
    STOMSFEM_TRY_CUDA(
        cudaFuncSetAttribute(coarse_pg_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    coarse_pg_kernel<true><<<(unsigned)blocks, kCoarsePgWarps * 32, smem, st>>>(nc, S, K, b, dirichlet, g, u, ws, sb);
  } else {
    const int bnd = nc + 2;
    const size_t smem = blk_smem_bytes<double>(16, bnd, CoarseBcGen::kRaw) * kCoarseBlkWarps;
    const int rpl = (16 + bnd + 31) / 32;
    auto kern = rpl <= 1 ? coarse_bc_kernel<1> : rpl == 2 ? coarse_bc_kernel<2> : coarse_bc_kernel<3>;
    STOMSFEM_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)blocks, kCoarseBlkWarps * 32, smem, st>>>(nc, S, K, b, dirichlet, g, u, ws, sb,
                                                                coarse_bc_l_bytes(nc));
  }
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  if (mom) {
    const int nn = (nc + 1) * (nc + 1);
    moments_kernel<<<(nn + 127) / 128, 128, 0, st>>>(nn, S, u, mean, m2, count);
    STOMSFEM_TRY_CUDA(cudaGetLastError());
    count_kernel<<<1, 1, 0, st>>>(count, S);
    STOMSFEM_TRY_CUDA(cudaGetLastError());
  }
  return STOMSFEM_OK;
}

// Fine grids up to 64 elements per side: the blocked banded Cholesky (one
// warp per sample); larger grids: multigrid-preconditioned CG (fine_mg.cu).
constexpr int kFineDirectMax = 64;

extern "C" int stomsfem_fine_fem_workspace_size(const stomsfem_grid* grid, int32_t S, size_t* bytes) {
  if (!grid || grid->nf <= 0 || S < 0 || !bytes) return set_error(STOMSFEM_EINVAL, "bad arguments");
  if (grid->nf > kFineDirectMax) {
    if (!fine_mg_supported(grid->nf))
      return set_error(STOMSFEM_EINVAL, "nf %d: above %d the element count must halve down to 16 or less",
                       grid->nf, kFineDirectMax);
    *bytes = fine_mg_workspace_bytes(grid->nf, S > 0 ? S : 1);
    return STOMSFEM_OK;
  }
  const int sms = device_sm_count();
  long long slots = (long long)(sms > 0 ? sms : 152) * 8;
  if (slots > S) slots = S;
  if (slots < kCoarseBlkWarps) slots = kCoarseBlkWarps;
  *bytes = coarse_slot_bytes(grid->nf) * (size_t)slots;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_fine_fem(const stomsfem_grid* grid, const double* a, int32_t S, double* u, void* workspace,
                                 size_t workspace_bytes, stomsfem_stream_t stream) {
  if (!grid || grid->nf <= 0) return set_error(STOMSFEM_EINVAL, "bad grid");
  if (S < 0) return set_error(STOMSFEM_EINVAL, "S < 0");
  if (S == 0) return STOMSFEM_OK;
  if (!a || !u || !workspace) return set_error(STOMSFEM_EINVAL, "NULL device pointer");
  const int nf = grid->nf;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (nf > kFineDirectMax) {
    if (!fine_mg_supported(nf))
      return set_error(STOMSFEM_EINVAL, "nf %d: above %d the element count must halve down to 16 or less", nf,
                       kFineDirectMax);
    double res = 0.0;
    int iters = 0;
    return fine_mg_solve(nf, grid->f, a, S, u, workspace, workspace_bytes, 1e-13, 400, st, &res, &iters);
  }
  const size_t sb = coarse_slot_bytes(nf);
  long long slots = (long long)(workspace_bytes / sb);
  if (slots < kCoarseBlkWarps)
    return set_error(STOMSFEM_ENOMEM, "fine FEM workspace %zu < %d slots of %zu", workspace_bytes, kCoarseBlkWarps, sb);
  long long blocks = slots / kCoarseBlkWarps;
  const long long need = ((long long)S + kCoarseBlkWarps - 1) / kCoarseBlkWarps;
  if (blocks > need) blocks = need;
  const size_t smem = blk_smem_bytes<double>(16, nf) * kCoarseBlkWarps;
  const int rpl = (16 + nf + 31) / 32;
  auto kern = rpl <= 1 ? fine_fem_kernel<1> : rpl == 2 ? fine_fem_kernel<2> : fine_fem_kernel<3>;
  STOMSFEM_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<(unsigned)blocks, kCoarseBlkWarps * 32, smem, st>>>(nf, S, grid->f, a, u, static_cast<unsigned char*>(workspace),
                                                             sb, coarse_l_bytes(nf));
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  return STOMSFEM_OK;
}

extern "C" int stomsfem_restrict_to_coarse(const stomsfem_grid* grid, const double* u_fine, const double* u_coarse,
                                           int32_t S, double* d, stomsfem_stream_t stream) {
  if (!grid || grid->nf <= 0 || grid->nc <= 0 || grid->nf % grid->nc) return set_error(STOMSFEM_EINVAL, "bad grid");
  if (S < 0) return set_error(STOMSFEM_EINVAL, "S < 0");
  if (S == 0) return STOMSFEM_OK;
  if (!u_fine || !d) return set_error(STOMSFEM_EINVAL, "NULL device pointer");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const long long total = (long long)S * (grid->nc + 1) * (grid->nc + 1);
  const int sms = device_sm_count() > 0 ? device_sm_count() : 152;
  long long blocks = (total + 255) / 256;
  if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
  restrict_kernel<<<(unsigned)blocks, 256, 0, st>>>(grid->nf, grid->nc, S, u_fine, u_coarse, d);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  return STOMSFEM_OK;
}

extern "C" int stomsfem_mc_moments(int32_t n, int32_t S, const double* u, double* mean, double* m2, double* count,
                                   stomsfem_stream_t stream) {
  if (n <= 0 || S < 0) return set_error(STOMSFEM_EINVAL, "bad n / S");
  if (S == 0) return STOMSFEM_OK;
  if (!u || !mean || !m2 || !count) return set_error(STOMSFEM_EINVAL, "NULL device pointer");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  moments_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, S, u, mean, m2, count);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  count_kernel<<<1, 1, 0, st>>>(count, S);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  return STOMSFEM_OK;
}

extern "C" int stomsfem_mc_merge(int32_t n, double* mean, double* m2, double* count, const double* mean_b,
                                 const double* m2_b, const double* count_b, stomsfem_stream_t stream) {
  if (n <= 0) return set_error(STOMSFEM_EINVAL, "bad n");
  if (!mean || !m2 || !count || !mean_b || !m2_b || !count_b)
    return set_error(STOMSFEM_EINVAL, "NULL device pointer");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  moments_merge_kernel<<<1, 1024, 0, st>>>(n, mean, m2, count, mean_b, m2_b, count_b);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  return STOMSFEM_OK;
}
