// Simultaneous local upscaling: one warp per (sample, coarse cell) unit.
//
// Per unit (Eq. MsFEB, Remark on oversampling, Eq. stiffness_local):
//   1. patch = cell enlarged by o fine elements per side, clipped to [0,1]^2;
//   2. cell problems: psi_l = p_l + psi0_l with p_l the bilinear nodal
//      function of the patch rectangle and psi0_l vanishing on the patch
//      boundary, A_II psi0_l = -(A p_l)_I for l = SW, SE, NE (the NW one is
//      1 - the others: the four p_l sum to 1 and A 1 = 0); the 9-point Q1
//      matrix rows are generated from a on the fly as the banded Cholesky
//      blocked banded Cholesky needs them (band_block.cuh);
//   3. optional FP64 iterative refinement of the FP32 solution;
//   4. M_jk = a_cell(psi_j, psi_k), m_j = int_cell f psi_j over the cell's
//      fine elements; oversampling recombination phi = D psi with
//      D = C^{-1}, C_jk = psi_j(cell corner k); K_e = D M D^T, b_e = D m.
//   5. Petrov-Galerkin form (Eq. stiffness_local_petrov): N_jk =
//      a_cell(psi_j, q_k) with q_k the cell's bilinear nodal functions
//      (test functions), S_pg = D N (16 entries, row = trial), b = f H^2/4.
//
// Shared by the Galerkin (upscale.cu) and Petrov-Galerkin (upscale_pg.cu)
// translation units, which instantiate the kernel with PG = false / true.
#pragma once
#include <cstdio>
#include <type_traits>

#include "band_block.cuh"
#include "band_tc.cuh"
#include "common.cuh"

namespace stomsfem {

// Warps per block: 4, except 2 for two FP64 units per warp (whose 36 KB of
// shared memory per warp then fit three blocks on an SM).
__host__ __device__ constexpr int upscale_warps(bool fp64, int G) { return fp64 && G == 16 ? 2 : 4; }
constexpr int kMaxBand = 64;       // half bandwidth limit (mx + 1)

struct UnitGeom {
  int x0, y0, Nx, Ny, mx, my, n, b;
  int cx0, cy0;  // cell origin in patch-local node coordinates
};

__device__ inline UnitGeom unit_geom(int nf, int rho, int cx, int cy, int o) {
  UnitGeom g;
  const int x0 = max(0, cx * rho - o), x1 = min(nf, (cx + 1) * rho + o);
  const int y0 = max(0, cy * rho - o), y1 = min(nf, (cy + 1) * rho + o);
  g.x0 = x0;
  g.y0 = y0;
  g.Nx = x1 - x0;
  g.Ny = y1 - y0;
  g.mx = g.Nx - 1;
  g.my = g.Ny - 1;
  g.n = g.mx * g.my;
  g.b = g.mx + 1;
  g.cx0 = cx * rho - x0;
  g.cy0 = cy * rho - y0;
  return g;
}

// Row generator of the patch system: matrix rows from a, right-hand sides
// -(A p_l) at interior nodes in closed form (differences of a only, so the
// small right-hand sides keep their relative accuracy in FP32).
struct PatchGen {
  const double* a;  // this sample's coefficient [nf][nf]
  int nf, x0, y0, Nx, Ny, mx;
  float iNxf, iNyf, rmx;  // 1/Nx, 1/Ny, 1/mx, set by finish()
  double iNxd, iNyd;

  __device__ __forceinline__ void finish() {
    rmx = __frcp_rn((float)mx);
    iNxd = 1.0 / (double)Nx;
    iNyd = 1.0 / (double)Ny;
    iNxf = 1.0f / (float)Nx;
    iNyf = 1.0f / (float)Ny;
  }

  __device__ __forceinline__ double ael(int ex, int ey) const {
    return __ldg(a + (size_t)(y0 + ey) * nf + (x0 + ex));
  }
  __device__ __forceinline__ void node(int r, int& i, int& j) const {
    // j - 1 = floor(r / mx) from a float reciprocal: (r + 1/2) / mx stays at
    // least 1/(2 mx) away from an integer, far above the rounding error
    const int q = __float2int_rz(((float)r + 0.5f) * rmx);
    j = q + 1;
    i = r - q * mx + 1;
  }
  template <typename T>
  __device__ __forceinline__ T coef(int r, int d) const {
    if (d != 0 && d != 1 && d != mx - 1 && d != mx && d != mx + 1) return T(0);
    int i, j;
    node(r, i, j);
    const T aSW = (T)ael(i - 1, j - 1), aSE = (T)ael(i, j - 1);
    const T aNE = (T)ael(i, j), aNW = (T)ael(i - 1, j);
    T v = T(0);
    if (d == 0) v += (T(2) / T(3)) * (aSW + aSE + aNE + aNW);
    if (d == 1 && i > 1) v -= (aSW + aNW) / T(6);                    // west
    if (d == mx && j > 1) v -= (aSW + aSE) / T(6);                   // south
    if (d == mx + 1 && i > 1 && j > 1) v -= aSW / T(3);              // south-west
    if (d == mx - 1 && i < mx && j > 1) v -= aSE / T(3);             // south-east
    return v;
  }
  // (A X), (A Y), (A XY) at interior node (i, j) for the patch coordinates
  // X = i/Nx, Y = j/Ny; then -(A p_l) for p_SW = 1-X-Y+XY, p_SE = X-XY, p_NE = XY.
  template <typename T>
  __device__ __forceinline__ void ap(int i, int j, T& AX, T& AY, T& AXY) const {
    const T aSW = (T)ael(i - 1, j - 1), aSE = (T)ael(i, j - 1);
    const T aNE = (T)ael(i, j), aNW = (T)ael(i - 1, j);
    AX = ((aSW + aNW) - (aSE + aNE)) / (T(2) * (T)Nx);
    AY = ((aSW + aSE) - (aNW + aNE)) / (T(2) * (T)Ny);
    const T Xc = (T)i / (T)Nx, Yc = (T)j / (T)Ny;
    AXY = Xc * AY + Yc * AX + ((aSE + aNW) - (aNE + aSW)) / (T(3) * (T)Nx * (T)Ny);
  }
  template <typename T>
  __device__ __forceinline__ T rhs(int r, int l) const {
    int i, j;
    node(r, i, j);
    T AX, AY, AXY;
    ap<T>(i, j, AX, AY, AXY);
    if (l == 0) return AX + AY - AXY;
    if (l == 1) return AXY - AX;
    return -AXY;
  }
  // Raw values of row r: the coefficient on the four elements around the node.
  struct Raw {
    double sw, se, ne, nw;
  };
  __device__ __forceinline__ void load(int r, Raw& w) const {
    int i, j;
    node(r, i, j);
    w.sw = ael(i - 1, j - 1);
    w.se = ael(i, j - 1);
    w.ne = ael(i, j);
    w.nw = ael(i - 1, j);
  }
  __device__ __forceinline__ void prefetch(int r, double* dst) const {
    int i, j;
    node(r, i, j);
    const double* p0 = a + (size_t)(y0 + j - 1) * nf + (x0 + i - 1);  // SW element
    cp_async8(dst + 0, p0);
    cp_async8(dst + 1, p0 + 1);
    cp_async8(dst + 2, p0 + nf + 1);
    cp_async8(dst + 3, p0 + nf);
  }
  __device__ __forceinline__ void from_smem(const double* src, Raw& w) const {
    w.sw = src[0];
    w.se = src[1];
    w.ne = src[2];
    w.nw = src[3];
  }
  // Whole row r: band entries at offsets 0, 1 (west), mx-1 (south-east),
  // mx (south), mx+1 (south-west) and the three right-hand sides; NR = 4
  // adds a fourth right-hand side of ones (the load functional of interior
  // nodes, up to the factor h^2).
  template <typename T, int NR = 3>
  __device__ __forceinline__ void make(int r, const Raw& w, T e[5], T* rh) const {
    int i, j;
    node(r, i, j);
    const T aSW = (T)w.sw, aSE = (T)w.se;
    const T aNE = (T)w.ne, aNW = (T)w.nw;
    // divisions replaced by products with reciprocals (one rounding each)
    const T r3 = T(1) / T(3), r6 = T(1) / T(6);
    T iNx, iNy;
    if constexpr (sizeof(T) == 4) {
      iNx = iNxf;
      iNy = iNyf;
    } else {
      iNx = iNxd;
      iNy = iNyd;
    }
    e[0] = (T(2) * r3) * ((aSW + aSE) + (aNE + aNW));
    e[1] = i > 1 ? -(aSW + aNW) * r6 : T(0);
    e[2] = (i < mx && j > 1) ? -aSE * r3 : T(0);
    e[3] = j > 1 ? -(aSW + aSE) * r6 : T(0);
    e[4] = (i > 1 && j > 1) ? -aSW * r3 : T(0);
    const T AX = T(0.5) * ((aSW + aNW) - (aSE + aNE)) * iNx;
    const T AY = T(0.5) * ((aSW + aSE) - (aNW + aNE)) * iNy;
    const T Xc = (T)i * iNx, Yc = (T)j * iNy;
    const T AXY = Xc * AY + Yc * AX + ((aSE + aNW) - (aNE + aSW)) * r3 * iNx * iNy;
    rh[0] = AX + AY - AXY;
    rh[1] = AXY - AX;
    rh[2] = -AXY;
    if constexpr (NR == 4) rh[3] = T(1);
  }
};

// Right-hand side of a refinement step: the FP64 residual
// -(A (p_l + psi0_l)) at interior nodes, psi0 = 0 on the patch boundary.
struct ResidualGen {
  PatchGen pg;
  const double* psi0;  // [n][3]
  __device__ __forceinline__ double psi(int i, int j, int l) const {
    if (i <= 0 || j <= 0 || i > pg.mx || j > pg.Ny - 1) return 0.0;
    return psi0[((size_t)(j - 1) * pg.mx + (i - 1)) * 3 + l];
  }
  // All three right-hand sides of row r: the stencil coefficients and the
  // closed-form -(A p_l) once per node, divisions replaced by products with
  // reciprocals (each residual term then carries a rounding or two of FP64,
  // far below what the refinement resolves).
  __device__ __forceinline__ void rhs3(int r, double out[3]) const {
    int i, j;
    pg.node(r, i, j);
    const double aSW = pg.ael(i - 1, j - 1), aSE = pg.ael(i, j - 1);
    const double aNE = pg.ael(i, j), aNW = pg.ael(i - 1, j);
    constexpr double r3 = 1.0 / 3.0, r6 = 1.0 / 6.0;
    const double AX = 0.5 * ((aSW + aNW) - (aSE + aNE)) * pg.iNxd;
    const double AY = 0.5 * ((aSW + aSE) - (aNW + aNE)) * pg.iNyd;
    const double AXY = ((double)i * pg.iNxd) * AY + ((double)j * pg.iNyd) * AX +
                       ((aSE + aNW) - (aNE + aSW)) * r3 * pg.iNxd * pg.iNyd;
    const double r0[3] = {AX + AY - AXY, AXY - AX, -AXY};
    // A psi0 with the full 9-point stencil
    const double cC = (2.0 / 3.0) * ((aSW + aSE) + (aNE + aNW));
    const double cW = (aSW + aNW) * r6, cE = (aSE + aNE) * r6, cS = (aSW + aSE) * r6, cN = (aNE + aNW) * r6;
    const double dSW = aSW * r3, dSE = aSE * r3, dNE = aNE * r3, dNW = aNW * r3;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      double t = cC * psi(i, j, l);
      t -= cW * psi(i - 1, j, l);
      t -= cE * psi(i + 1, j, l);
      t -= cS * psi(i, j - 1, l);
      t -= cN * psi(i, j + 1, l);
      t -= dSW * psi(i - 1, j - 1, l);
      t -= dSE * psi(i + 1, j - 1, l);
      t -= dNE * psi(i + 1, j + 1, l);
      t -= dNW * psi(i - 1, j + 1, l);
      out[l] = r0[l] - t;
    }
  }
};

// Oscillatory boundary data (the MsFEM option of the short-correlation
// example, Sec. 5.3): on every patch edge the nodal functions interpolate
// their corner values linearly in the edge's harmonic coordinate
// t_k = sum_{e<k} 1/a_e / sum_e 1/a_e (a_e the patch element next to segment
// e: the reduced problem (a u')' = 0 along the edge) instead of in arc
// length.  The unknowns stay psi0_l (zero on the boundary), with the lifting
// p_l = bilinear + d_l, d_l nonzero on the boundary only: on an edge whose
// corner values are c0 (k = 0) and c1 (k = N), d_l(k) = (c1 - c0) delta(k),
// delta(k) = t_k - k / N.  Each unit tabulates delta for its four edges
// once, in shared memory (osc_fill_tables); d_l at a boundary node and its
// share -(A d_l) of the right-hand side at the interior nodes next to the
// boundary read the tables.

// Shared-memory bytes of one unit's tables: 4 edges x (bmax + 1) nodes.
__host__ __device__ inline size_t osc_tab_bytes(int bmax) { return al16(sizeof(double) * 4 * (size_t)(bmax + 1)); }

// Row generator with the oscillatory data: the rows of PatchGen plus the
// ring term in the right-hand sides.
struct PatchGenOsc : PatchGen {
  const double* tab;  // [4][ts] delta of the edges bottom, top, left, right
  int ts;             // table stride (bmax + 1)
  template <typename T, int NR = 3>
  __device__ __forceinline__ void make(int r, const Raw& w, T e[5], T* rh) const;
};

// delta at node k of edge E (0 bottom, 1 top, 2 left, 3 right); the table
// holds 0 at both corners.
__device__ __forceinline__ double osc_delta(const PatchGenOsc& pg, int E, int k) { return pg.tab[E * pg.ts + k]; }

// Lanes 0..3 of a unit's group fill the tables of edges 0..3 (the other
// lanes wait at the caller's __syncwarp): 1/a_e along the edge, then the
// running sums; FP64.
__device__ inline void osc_fill_tables(const PatchGen& pg, double* tab, int ts, int gl) {
  if (gl >= 4) return;
  const int E = gl;
  const int N = E < 2 ? pg.Nx : pg.Ny;
  const size_t row0 = (size_t)(pg.y0 + (E == 1 ? pg.Ny - 1 : 0)) * pg.nf;
  const double* p = pg.a + row0 + pg.x0 + (E == 3 ? pg.Nx - 1 : 0);
  const size_t step = E < 2 ? 1 : (size_t)pg.nf;
  double* t = tab + E * ts;
  double tot = 0.0;
  for (int e = 0; e < N; ++e) {
    const double v = 1.0 / __ldg(p + (size_t)e * step);
    t[e + 1] = v;
    tot += v;
  }
  const double it = 1.0 / tot, iN = 1.0 / (double)N;
  double acc = 0.0;
  t[0] = 0.0;
  for (int k = 1; k < N; ++k) {
    acc += t[k];
    t[k] = acc * it - (double)k * iN;
  }
  t[N] = 0.0;
}

// Adds d_l (l = SW, SE, NE) at patch node (i, j) when it lies on the
// boundary: bottom d_SW = -delta, d_SE = +delta; top d_NE = +delta; left
// d_SW = -delta; right d_SE = -delta, d_NE = +delta.
template <typename T>
__device__ inline void osc_boundary(const PatchGenOsc& pg, int i, int j, T out[3]) {
  if (j == 0 && i > 0 && i < pg.Nx) {
    const double d = osc_delta(pg, 0, i);
    out[0] -= (T)d;
    out[1] += (T)d;
  } else if (j == pg.Ny && i > 0 && i < pg.Nx) {
    out[2] += (T)osc_delta(pg, 1, i);
  } else if (i == 0 && j > 0 && j < pg.Ny) {
    out[0] -= (T)osc_delta(pg, 2, j);
  } else if (i == pg.Nx && j > 0 && j < pg.Ny) {
    const double d = osc_delta(pg, 3, j);
    out[1] -= (T)d;
    out[2] += (T)d;
  }
}

// Adds -(A d_l) at interior node (i, j) next to the boundary: the stencil
// couplings to its boundary neighbours (a_SW/3, (a_SW + a_NW)/6, a_NW/3 to
// the west nodes j-1, j, j+1, and likewise on the other sides) times d_l.
template <typename T>
__device__ inline void osc_ring(const PatchGenOsc& pg, int i, int j, double aSW, double aSE, double aNE, double aNW,
                                T rh[3]) {
  constexpr double r3 = 1.0 / 3.0, r6 = 1.0 / 6.0;
  double r0 = 0.0, r1 = 0.0, r2 = 0.0;
  if (j == 1) {  // bottom edge nodes i-1, i, i+1
    const double t = aSW * r3 * osc_delta(pg, 0, i - 1) + (aSW + aSE) * r6 * osc_delta(pg, 0, i) +
                     aSE * r3 * osc_delta(pg, 0, i + 1);
    r0 -= t;
    r1 += t;
  }
  if (j == pg.Ny - 1)  // top edge
    r2 += aNW * r3 * osc_delta(pg, 1, i - 1) + (aNW + aNE) * r6 * osc_delta(pg, 1, i) +
          aNE * r3 * osc_delta(pg, 1, i + 1);
  if (i == 1)  // left edge nodes j-1, j, j+1
    r0 -= aSW * r3 * osc_delta(pg, 2, j - 1) + (aSW + aNW) * r6 * osc_delta(pg, 2, j) +
          aNW * r3 * osc_delta(pg, 2, j + 1);
  if (i == pg.mx) {  // right edge
    const double t = aSE * r3 * osc_delta(pg, 3, j - 1) + (aSE + aNE) * r6 * osc_delta(pg, 3, j) +
                     aNE * r3 * osc_delta(pg, 3, j + 1);
    r1 -= t;
    r2 += t;
  }
  rh[0] += (T)r0;
  rh[1] += (T)r1;
  rh[2] += (T)r2;
}

template <typename T, int NR>
__device__ __forceinline__ void PatchGenOsc::make(int r, const Raw& w, T e[5], T* rh) const {
  PatchGen::make<T, NR>(r, w, e, rh);
  int i, j;
  node(r, i, j);
  if (i == 1 || j == 1 || i == mx || j == Ny - 1) osc_ring<T>(*this, i, j, w.sw, w.se, w.ne, w.nw, rh);
}

// psi_l at patch node (i, j) for l = 0..2 (bilinear part + correction),
// given its patch coordinates X = i / Nx, Y = j / Ny.
template <typename T, typename TS>
__device__ __forceinline__ void psi_at_xy(const UnitGeom& g, const TS* psi0, int i, int j, T X, T Y, T out[3],
                                          bool with_psi = true) {
  out[0] = (T(1) - X) * (T(1) - Y);
  out[1] = X * (T(1) - Y);
  out[2] = X * Y;
  if (with_psi && i > 0 && j > 0 && i < g.Nx && j < g.Ny) {
    const TS* p = psi0 + ((size_t)(j - 1) * g.mx + (i - 1)) * 3;
    out[0] += (T)p[0];
    out[1] += (T)p[1];
    out[2] += (T)p[2];
  }
}

// The same, computing X and Y.
template <typename T, typename TS>
__device__ __forceinline__ void psi_at(const UnitGeom& g, const TS* psi0, int i, int j, T out[3],
                                       bool with_psi = true) {
  psi_at_xy<T, TS>(g, psi0, i, j, (T)i / (T)g.Nx, (T)j / (T)g.Ny, out, with_psi);
}

// 4x4 inverse by Gauss-Jordan elimination without row exchanges, all
// indices static so the matrix stays in registers.  C_jk = psi_j(corner k)
// is strongly diagonally dominant (the patch basis at the cell corners is
// close to the patch's own bilinear nodal values), so no pivoting is needed;
// a vanishing pivot reports failure.
template <typename T>
__device__ __forceinline__ bool inv4(T C[4][4], T D[4][4]) {
  T M[4][8];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) M[r][c] = c < 4 ? C[r][c] : (c - 4 == r ? T(1) : T(0));
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    ok = ok && (M[c][c] != T(0));
    const T dinv = T(1) / M[c][c];
#pragma unroll
    for (int k = 0; k < 8; ++k) M[c][k] *= dinv;
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (r != c) {
        const T f = M[r][c];
#pragma unroll
        for (int k = 0; k < 8; ++k) M[r][k] -= f * M[c][k];
      }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) D[r][c] = M[r][c + 4];
  return ok;
}

struct UpscaleArgs {
  const double* a;
  const int8_t* oversample;
  int nf, nc, rho, max_o, S;
  double f;
  int refine;
  double* Ke;
  double* be;
  double* phi;
  int32_t* status;
  unsigned char* ws;
  size_t slot_bytes, l_bytes;
  int bmax, nmax;
  long long units;
  const int32_t* unit_list;   // optional: process only these units (device list)
  const int32_t* unit_count;  // device length of unit_list
  double fq, fH2;             // f h^2 / 4 and f H^2 (load scaling)
  const int32_t* cell_list;   // optional: process only these cells (device list)
  const int32_t* cell_count;  // device length of cell_list
  int blocks_per_sm_cap;      // host-side launch shape: at most this many resident CTAs per SM (0: occupancy)
  int order;                  // 0: cells fastest; 1: samples fastest, cells in list order
};

// Launch choices a plan's autotuner may set (stomsfem_plan_tune); the
// defaults are what stomsfem_upscale uses.
struct UpscaleTuning {
  int blocks_per_sm = 0;  // 0: as many as fit
  int split_fp32 = 1;     // FP32 form: separate forward-only launch for the cells without oversampling
  int engine = 0;         // FP32 forms: factorisation engine (kEngine*; 0 = the default for the patch size)
  int order = 0;          // STOMSFEM_ORDER_*: unit order of the persistent launches
};

// Upscale launch modes: 0 every unit (back-substitution route), 1 the
// cells without oversampling by the forward-only route, 2 the other cells.
// Splitting the two routes over two launches keeps one route's code hot per
// kernel; with both in one kernel the instruction working set of an SM
// doubled and cost more than the forward-only route saved.
enum { kModeAll = 0, kModeFwd = 1, kModeRest = 2 };

// Cell lists of the launches (one warp, ballot compaction): list0 the
// cells without oversampling, list1 the others (cells with an oversampling
// outside [0, max_o] included: the kernel flags them), listall every cell;
// counts = {|list0|, |list1|, |listall|}.  sorted = 0: ascending cell index
// (listall unused); sorted = 1: by patch size, largest first (decreasing
// oversampling, the flagged cells last), ascending cell index within one
// size, so that a launch that walks its list with the samples fastest
// takes the longest units first.
static __global__ void upscale_cell_lists_kernel(const int8_t* __restrict__ oversample, int ncell, int max_o,
                                          int sorted, int32_t* __restrict__ list0, int32_t* __restrict__ list1,
                                          int32_t* __restrict__ listall, int32_t* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  int n0 = 0, n1 = 0, na = 0;
  // pass k: sorted, k = max_o .. 0 the cells of oversampling k, then k = -1
  // the flagged ones; unsorted, one pass (k = -2) over all cells
  for (int k = sorted ? max_o : -2; k >= (sorted ? -1 : -2); --k) {
    for (int c0 = 0; c0 < ncell; c0 += 32) {
      const int c = c0 + lane;
      const bool valid = c < ncell;
      const int v = valid ? (int)oversample[c] : 0;
      const bool take = valid && (k == -2 || (k >= 0 ? v == k : (v < 0 || v > max_o)));
      const bool z = take && v == 0;
      const unsigned m0 = __ballot_sync(0xffffffffu, z), m1 = __ballot_sync(0xffffffffu, take && !z);
      const unsigned ma = __ballot_sync(0xffffffffu, take);
      if (z) list0[n0 + __popc(m0 & below)] = c;
      if (take && !z) list1[n1 + __popc(m1 & below)] = c;
      if (sorted && take) listall[na + __popc(ma & below)] = c;
      n0 += __popc(m0);
      n1 += __popc(m1);
      na += __popc(ma);
    }
  }
  if (lane == 0) {
    counts[0] = n0;
    counts[1] = n1;
    counts[2] = na;
  }
}

__device__ __forceinline__ double qnan() { return __longlong_as_double(0x7ff8000000000000ll); }

// Sum over the G lanes of a group (every lane of the group receives it).
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}

// Shared-memory view of one unit for the substitutions (and, without TC,
// the factorisation).
template <typename TK, int TC>
__device__ inline BlkSmem<TK> unit_blk(unsigned char* base, const TcSmem& tsm, int NB, int bmax) {
  if constexpr (TC > 0)
    return tc_blk_view(tsm);
  else
    return make_blk<TK>(base, NB, bmax);
}

// TK: factor/solve type; TA: type of the K_e/b_e accumulation and of the
// recombination; RPL: panel rows per lane (ceil((G/2 + bmax) / G)); G: lanes
// per unit.  G = 32: one unit per warp (any unit order, including a device
// list).  G = 16: a warp takes one cell of two consecutive samples, whose
// patches have the same shape, so its two halves run the same loop bounds
// in lockstep (an odd last sample is mirrored by the idle half, which
// writes nothing).
// OSC: the oscillatory boundary data of the cell problems (PatchGenOsc).
// TC > 0 (FP32 factor, G = 32): the factorisation of band_tc.cuh (window
// in mma accumulator registers, trailing update on the tensor cores with
// operands split into TC TF32 parts, column blocks of 8), b <= 40; the
// substitutions read its 8-column blocks.
template <typename TK, typename TA, int RPL, int G, int MODE, bool PG, bool OSC = false, int TC = 0>
__global__ void __launch_bounds__(upscale_warps(sizeof(TK) == 8, G) * 32,
                                  sizeof(TK) == 4 ? (G == 16 ? 3 : 4) : (G == 16 ? 3 : 2))
upscale_kernel(UpscaleArgs A) {
  // the oscillatory data run every cell by back substitution (one launch)
  static_assert(!OSC || MODE == kModeAll, "oscillatory data: back-substitution route only");
  static_assert(TC == 0 || (G == 32 && sizeof(TK) == 4), "tensor-core factorisation: FP32 factor, one unit per warp");
  constexpr int NB = TC > 0 ? kTcNB : G / 2;
  constexpr int GPW = 32 / G;  // units per warp
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int gl = lane % G, grp = lane / G;
  const int wib = threadIdx.x >> 5;
  // per-unit shared memory (the oscillatory tables follow all of it)
  const size_t unit_smem = TC > 0 ? kTcSmemWarp : blk_smem_bytes<TK>(NB, A.bmax);
  const TcSmem tsm = make_tc(smem + wib * kTcSmemWarp);
  const BlkSmem<TK> sm = unit_blk<TK, TC>(smem + (wib * GPW + grp) * unit_smem, tsm, NB, A.bmax);
  constexpr int WPB = upscale_warps(sizeof(TK) == 8, G);
  const long long gw = (long long)blockIdx.x * WPB + wib;
  const long long nw = (long long)gridDim.x * WPB;
  unsigned char* slot = A.ws + (size_t)(gw * GPW + grp) * A.slot_bytes;
  // solutions are kept in FP64 except in the all-FP32 form
  using TS = typename std::conditional<std::is_same<TA, float>::value, float, double>::type;
  TK* Lg = reinterpret_cast<TK*>(slot);
  TS* psi0 = reinterpret_cast<TS*>(slot + A.l_bytes);
  double* corr = reinterpret_cast<double*>(slot + A.l_bytes) + (size_t)A.nmax * 3;
  const int ncell = A.nc * A.nc;
  const int CN = (A.rho + 1) * (A.rho + 1);

  // cells of this launch (MODE 1, 2: a device list, or all cells when none)
  const int nlc = A.cell_list ? A.cell_count[0] : ncell;
  // work items: (sample, cell) for G = 32, (pair of samples, cell) for G = 16;
  // with a unit list, one entry (G = 32) or two consecutive entries (G = 16:
  // the list holds cells without oversampling only, all of one patch shape,
  // so the two halves of a warp run in lockstep)
  const long long npair = G == 32 ? (long long)A.S : (long long)((A.S + 1) / 2);
  const long long nlist = A.unit_list ? (long long)A.unit_count[0] : 0;
  const long long nwork = A.unit_list ? (G == 32 ? nlist : (nlist + 1) / 2) : npair * nlc;
  for (long long w = gw; w < nwork; w += nw) {
    long long u;
    bool dup = false;  // this half mirrors the other half's unit
    const int ci = A.order ? (int)(w / npair) : (int)(w % nlc);
    const long long pw = A.order ? w % npair : w / nlc;
    const int cell_w = A.cell_list ? A.cell_list[ci] : ci;
    if (G == 32) {
      u = A.unit_list ? (long long)A.unit_list[w] : pw * ncell + cell_w;
    } else if (A.unit_list) {
      long long li = 2 * w + grp;
      if (li >= nlist) {
        li = nlist - 1;
        dup = true;
      }
      u = (long long)A.unit_list[li];
    } else {
      int sp = 2 * (int)pw + grp;
      if (sp >= A.S) {
        sp = A.S - 1;
        dup = true;
      }
      u = (long long)sp * ncell + cell_w;
    }
    const int s = (int)(u / ncell);
    const int cell = (int)(u % ncell);
    const int cx = cell % A.nc, cy = cell / A.nc;
    const int o = A.oversample ? (int)A.oversample[cell] : 0;
    constexpr int KN = PG ? 16 : 10;  // entries of K_e per unit
    double* Ke = A.Ke + (size_t)u * KN;
    double* be = A.be + (size_t)u * 4;
    if (o < 0 || o > A.max_o) {
      if (!dup) {
        if (gl < KN) Ke[gl] = qnan();
        if (gl < 4) be[gl] = qnan();
        if (gl == 0 && A.status) A.status[u] = -1;
      }
      continue;
    }
    const UnitGeom g = unit_geom(A.nf, A.rho, cx, cy, o);
    using Gen = typename std::conditional<OSC, PatchGenOsc, PatchGen>::type;
    Gen pg;
    pg.a = A.a + (size_t)s * A.nf * A.nf;
    pg.nf = A.nf;
    pg.x0 = g.x0;
    pg.y0 = g.y0;
    pg.Nx = g.Nx;
    pg.Ny = g.Ny;
    pg.mx = g.mx;
    pg.finish();
    if constexpr (OSC) {
      pg.tab = reinterpret_cast<const double*>(smem + (size_t)WPB * GPW * unit_smem +
                                               (size_t)(wib * GPW + grp) * osc_tab_bytes(A.bmax));
      pg.ts = A.bmax + 1;
      osc_fill_tables(pg, const_cast<double*>(pg.tab), pg.ts, gl);
      __syncwarp();
    }
    // psi_l at a patch node, with the boundary data's d_l on the boundary
    auto psi_node = [&](int i, int j, TA X, TA Y, TA out[3], bool with_psi) {
      psi_at_xy<TA, TS>(g, psi0, i, j, X, Y, out, with_psi);
      if constexpr (OSC)
        if (i == 0 || j == 0 || i == g.Nx || j == g.Ny) osc_boundary<TA>(pg, i, j, out);
    };
    // A patch that is the cell itself (no oversampling) in the FP32 form,
    // without phi output, takes the forward-only route: K_e(l, m) =
    // p_l^T A p_m - y_l . y_m with y = L^-1 R_l the forward solutions (the
    // Galerkin identity of the cell problem, Eq. stiffness_local with
    // phi_l = p_l + psi_l), and the corner sums of psi_l from z . y_l with
    // z = L^-1 1; no factor is stored and there is no back substitution.
    // The choice depends only on the cell, so both halves of a warp agree.
    // The host sends only such cells to MODE 1 launches.
    constexpr bool fwd_only = MODE == kModeFwd;
    double yy[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    // a failed factorisation still runs every step (the halves of a warp
    // stay in lockstep); its unit gets NaN results and a status below
    int fail = -1;
    if constexpr (fwd_only) {
      if (g.n > 0) {
        if constexpr (TC > 0)
          fail = tc_factor<4, true, Gen, TS, TC>(pg, g.n, g.b, A.bmax, tsm, reinterpret_cast<float*>(Lg), psi0, gl,
                                                 yy);
        else
          fail = blk_factor<G, TK, 4, RPL, Gen, TS, true>(pg, g.n, g.b, A.bmax, sm, Lg, psi0, gl, yy);
      }
    } else if (g.n > 0) {
      // without refinement only psi on the cell's nodes is read: the rows
      // below the cell's first node row (the bottom oversampling layer) need
      // neither stored factor blocks nor back substitution
      const int need_from = A.refine == 0 ? max(0, g.cy0 - 1) * g.mx : 0;
      if constexpr (TC > 0)
        fail = tc_factor<3, false, Gen, TS, TC>(pg, g.n, g.b, A.bmax, tsm, reinterpret_cast<float*>(Lg), psi0, gl);
      else
        fail = blk_factor<G, TK, 3, RPL>(pg, g.n, g.b, A.bmax, sm, Lg, psi0, gl, nullptr, need_from);
      // the factor-and-refine form (FP32 factor, FP64 solutions) calls the
      // substitutions out of line: one copy of each for all its passes
      constexpr bool outlined = sizeof(TK) == 4 && std::is_same<TA, double>::value;
      if constexpr (outlined)
        blk_backward_outlined<G, TK, 3, TS, NB>(g.n, g.b, A.bmax, sm, Lg, psi0, gl, need_from);
      else
        blk_backward<G, TK, 3, TS, NB>(g.n, g.b, A.bmax, sm, Lg, psi0, gl, need_from);
      // FP64 iterative refinement with the factor: corr = residual, solve, add
      for (int it = 0; it < A.refine; ++it) {
        __syncwarp();
        const ResidualGen rg{pg, reinterpret_cast<const double*>(psi0)};
        for (int r = gl; r < g.n; r += G) {
          rg.rhs3(r, corr + (size_t)3 * r);
          if constexpr (OSC) {
            int i, j;
            pg.node(r, i, j);
            if (i == 1 || j == 1 || i == g.mx || j == g.Ny - 1)
              osc_ring<double>(pg, i, j, pg.ael(i - 1, j - 1), pg.ael(i, j - 1), pg.ael(i, j), pg.ael(i - 1, j),
                               corr + (size_t)3 * r);
          }
        }
        __syncwarp();
        if constexpr (outlined) {
          blk_forward_stored_outlined<G, TK, 3, RPL, NB>(g.n, g.b, A.bmax, sm, Lg, corr, gl);
          blk_backward_outlined<G, TK, 3, double, NB>(g.n, g.b, A.bmax, sm, Lg, corr, gl, 0);
        } else {
          blk_forward_stored<G, TK, 3, RPL, NB>(g.n, g.b, A.bmax, sm, Lg, corr, gl);
          blk_backward<G, TK, 3, double, NB>(g.n, g.b, A.bmax, sm, Lg, corr, gl);
        }
        __syncwarp();
        for (int k = gl; k < g.n * 3; k += G) psi0[k] += (TS)corr[k];
      }
    }
    __syncwarp();
    // M_jk = a_cell(psi_j, psi_k) (j, k < 3) by the edge/diagonal difference
    // form of the Q1 element energy, 6 u^T K_ref v = sum_edges du dv +
    // 2 sum_diagonals du dv; m_j = sum over element corners of psi_j.
    TA M[6] = {0, 0, 0, 0, 0, 0};
    TA m[3] = {0, 0, 0};
    const bool patch_is_cell = (g.cx0 == 0 && g.cy0 == 0 && g.Nx == A.rho && g.Ny == A.rho);
    // Petrov-Galerkin: N_jk = a_cell(psi_j, q_k), j, k < 3 (needed only with
    // oversampling or the oscillatory data: otherwise a(phi_l, q_k) =
    // a(phi_l, phi_k), since phi_k - q_k vanishes on the cell boundary and
    // phi_l is discrete-harmonic)
    TA N[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const bool pg_sum = PG && (OSC || !patch_is_cell);
    const TA irho = TA(1) / (TA)A.rho;
    TA iNx, iNy;
    if constexpr (sizeof(TA) == 4) {
      iNx = pg.iNxf;
      iNy = pg.iNyf;
    } else {
      iNx = (TA)pg.iNxd;
      iNy = (TA)pg.iNyd;
    }
    for (int e = gl; e < A.rho * A.rho; e += G) {
      const int ex = e % A.rho, ey = e / A.rho;
      const int i0 = g.cx0 + ex, j0 = g.cy0 + ey;
      TA c0[3], c1[3], c2[3], c3[3];
      // patch coordinates of the element's corners: the product with 1/Nx
      // (1/Ny) and one residual correction q + (i - q N) / N, which rounds
      // like the quotient i / N
      auto quot = [](TA num, TA den, TA inv) {
        const TA q = num * inv;
        return fma(fma(-q, den, num), inv, q);
      };
      const TA Nxf = (TA)g.Nx, Nyf = (TA)g.Ny;
      const TA X0 = quot((TA)i0, Nxf, iNx), X1 = quot((TA)(i0 + 1), Nxf, iNx);
      const TA Y0 = quot((TA)j0, Nyf, iNy), Y1 = quot((TA)(j0 + 1), Nyf, iNy);
      psi_node(i0, j0, X0, Y0, c0, !fwd_only);
      psi_node(i0 + 1, j0, X1, Y0, c1, !fwd_only);
      psi_node(i0 + 1, j0 + 1, X1, Y1, c2, !fwd_only);
      psi_node(i0, j0 + 1, X0, Y1, c3, !fwd_only);
      const TA ae = (TA)pg.ael(i0, j0);
      TA dd[3][6];
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        dd[l][0] = c0[l] - c1[l];
        dd[l][1] = c1[l] - c2[l];
        dd[l][2] = c2[l] - c3[l];
        dd[l][3] = c3[l] - c0[l];
        dd[l][4] = c0[l] - c2[l];
        dd[l][5] = c1[l] - c3[l];
        m[l] += (c0[l] + c1[l]) + (c2[l] + c3[l]);
      }
      int q = 0;
#pragma unroll
      for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int lp = l; lp < 3; ++lp) {
          const TA v = dd[l][0] * dd[lp][0] + dd[l][1] * dd[lp][1] + dd[l][2] * dd[lp][2] +
                       dd[l][3] * dd[lp][3] + TA(2) * (dd[l][4] * dd[lp][4] + dd[l][5] * dd[lp][5]);
          M[q++] += ae * v;
        }
      if constexpr (PG) {
        if (pg_sum) {
          // the cell's bilinears at the element corners (cell coordinates)
          const TA x0 = (TA)ex * irho, x1 = (TA)(ex + 1) * irho;
          const TA y0 = (TA)ey * irho, y1 = (TA)(ey + 1) * irho;
          const TA qc[3][4] = {{(1 - x0) * (1 - y0), (1 - x1) * (1 - y0), (1 - x1) * (1 - y1), (1 - x0) * (1 - y1)},
                               {x0 * (1 - y0), x1 * (1 - y0), x1 * (1 - y1), x0 * (1 - y1)},
                               {x0 * y0, x1 * y0, x1 * y1, x0 * y1}};
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const TA e0 = qc[k][0] - qc[k][1], e1 = qc[k][1] - qc[k][2], e2 = qc[k][2] - qc[k][3];
            const TA e3 = qc[k][3] - qc[k][0], e4 = qc[k][0] - qc[k][2], e5 = qc[k][1] - qc[k][3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              const TA v = dd[j][0] * e0 + dd[j][1] * e1 + dd[j][2] * e2 + dd[j][3] * e3 +
                           TA(2) * (dd[j][4] * e4 + dd[j][5] * e5);
              N[j * 3 + k] += ae * v;
            }
          }
        }
      }
    }
    if constexpr (PG) {
      if (pg_sum) {
#pragma unroll
        for (int q = 0; q < 9; ++q) N[q] = group_sum<G>(N[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) M[q] = group_sum<G>(M[q]);
#pragma unroll
    for (int l = 0; l < 3; ++l) m[l] = group_sum<G>(m[l]);
    if constexpr (fwd_only) {
      // M holds 6 p_l^T A p_m and m the corner sums of p_l: subtract the
      // forward-solution products; every interior node is a corner of four
      // elements, so the corner sums of psi_l are 4 z . y_l
#pragma unroll
      for (int q = 0; q < 9; ++q) yy[q] = group_sum<G>(yy[q]);
#pragma unroll
      for (int q = 0; q < 6; ++q) M[q] = (TA)((double)M[q] - 6.0 * yy[q]);
#pragma unroll
      for (int l = 0; l < 3; ++l) m[l] = (TA)((double)m[l] + 4.0 * yy[6 + l]);
    }

    // recombination D = C^{-1}, C_jk = psi_j(cell corner k); identity when
    // the patch is the cell (its corners carry the bilinear data exactly)
    TA D[4][4];
    bool ok = true;
    if (patch_is_cell) {
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) D[r][c] = (r == c) ? TA(1) : TA(0);
    } else {
      const int ci[4] = {g.cx0, g.cx0 + A.rho, g.cx0 + A.rho, g.cx0};
      const int cj[4] = {g.cy0, g.cy0, g.cy0 + A.rho, g.cy0 + A.rho};
      TA C[4][4];
      for (int k = 0; k < 4; ++k) {
        TA v[3];
        psi_node(ci[k], cj[k], (TA)ci[k] / (TA)g.Nx, (TA)cj[k] / (TA)g.Ny, v, true);
        C[0][k] = v[0];
        C[1][k] = v[1];
        C[2][k] = v[2];
        C[3][k] = TA(1) - v[0] - v[1] - v[2];
      }
      ok = inv4<TA>(C, D);
    }
    if (gl == 0 && !dup && fail >= 0) {
      for (int q = 0; q < KN; ++q) Ke[q] = qnan();
      for (int q = 0; q < 4; ++q) be[q] = qnan();
      if (A.status) A.status[u] = fail + 1;
    }
    if (gl == 0 && !dup && fail < 0) {
      // one lane per unit: FP64 here runs at the narrow pipe's single-lane
      // cost, so divisions become products with constants and the identity
      // recombination of an unoversampled patch is skipped
      double MM[4][4];
      MM[0][0] = M[0]; MM[0][1] = MM[1][0] = M[1]; MM[0][2] = MM[2][0] = M[2];
      MM[1][1] = M[3]; MM[1][2] = MM[2][1] = M[4]; MM[2][2] = M[5];
      for (int r = 0; r < 3; ++r) MM[r][3] = MM[3][r] = -(MM[r][0] + MM[r][1] + MM[r][2]);
      MM[3][3] = -(MM[0][3] + MM[1][3] + MM[2][3]);
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) MM[r][c] *= 1.0 / 6.0;
      double mv[4] = {A.fq * (double)m[0], A.fq * (double)m[1], A.fq * (double)m[2], 0.0};
      mv[3] = A.fH2 - (mv[0] + mv[1] + mv[2]);
      if constexpr (PG) {
        // S_pg = D N4, N4 the 4x4 completion of N (the q_k sum to 1 and so
        // do the psi_j, and a(1, .) = 0), scaled by 1/6; without
        // oversampling S_pg = the Galerkin matrix
        double S4[4][4];
        if (patch_is_cell && !OSC) {
          for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) S4[r][c] = MM[r][c];
        } else {
          double N4[4][4];
          for (int j = 0; j < 3; ++j) {
            for (int k = 0; k < 3; ++k) N4[j][k] = (double)N[j * 3 + k] * (1.0 / 6.0);
            N4[j][3] = -(N4[j][0] + N4[j][1] + N4[j][2]);
          }
          for (int k = 0; k < 4; ++k) N4[3][k] = -(N4[0][k] + N4[1][k] + N4[2][k]);
          for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) {
              double t = 0.0;
              for (int k = 0; k < 4; ++k) t += (double)D[r][k] * N4[k][c];
              S4[r][c] = ok ? t : qnan();
            }
        }
        for (int r = 0; r < 4; ++r)
          for (int c = 0; c < 4; ++c) Ke[r * 4 + c] = S4[r][c];
        for (int r = 0; r < 4; ++r) be[r] = 0.25 * A.fH2;
        if (A.status) A.status[u] = ok ? 0 : STOMSFEM_ENOTSPD;
      } else if (patch_is_cell) {
        int q = 0;
        for (int r = 0; r < 4; ++r)
          for (int c = r; c < 4; ++c) Ke[q++] = MM[r][c];
        for (int r = 0; r < 4; ++r) be[r] = mv[r];
        if (A.status) A.status[u] = 0;
      } else {
      double T4[4][4];
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
          double t = 0.0;
          for (int k = 0; k < 4; ++k) t += (double)D[r][k] * MM[k][c];
          T4[r][c] = t;
        }
      int q = 0;
      for (int r = 0; r < 4; ++r)
        for (int c = r; c < 4; ++c) {
          double t = 0.0;
          for (int k = 0; k < 4; ++k) t += T4[r][k] * (double)D[c][k];
          Ke[q++] = ok ? t : qnan();
        }
      for (int r = 0; r < 4; ++r) {
        double t = 0.0;
        for (int k = 0; k < 4; ++k) t += (double)D[r][k] * mv[k];
        be[r] = ok ? t : qnan();
      }
      if (A.status) A.status[u] = ok ? 0 : STOMSFEM_ENOTSPD;
      }
    }
    if (A.phi && !dup && fail < 0) {
      double* ph = A.phi + (size_t)u * 4 * CN;
      for (int q = gl; q < CN; q += G) {
        const int i = g.cx0 + q % (A.rho + 1), j = g.cy0 + q / (A.rho + 1);
        double v[3];
        psi_at<double, TS>(g, psi0, i, j, v);
        if constexpr (OSC)
          if (i == 0 || j == 0 || i == g.Nx || j == g.Ny) osc_boundary<double>(pg, i, j, v);
        const double v4[4] = {v[0], v[1], v[2], 1.0 - v[0] - v[1] - v[2]};
        for (int l = 0; l < 4; ++l) {
          double t = 0.0;
          for (int k = 0; k < 4; ++k) t += (double)D[l][k] * v4[k];
          ph[(size_t)l * CN + q] = t;
        }
      }
    }
    __syncwarp();
  }
}

static size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

static void slot_layout(int nmax, int bmax, int precision, size_t* slot, size_t* l_bytes) {
  const size_t tk = precision == STOMSFEM_FP64 ? 8 : 4;
  *l_bytes = round256(blk_factor_elems(nmax, bmax) * tk);
  *slot = *l_bytes + round256((size_t)nmax * 3 * 8 * 2);
}

static int validate_grid(const stomsfem_grid* g) {
  if (!g) return set_error(STOMSFEM_EINVAL, "grid is NULL");
  if (g->nf <= 0 || g->nc <= 0 || g->nf % g->nc != 0)
    return set_error(STOMSFEM_EINVAL, "grid: need nf > 0, nc > 0, nf %% nc == 0 (nf=%d nc=%d)",
                     g->nf, g->nc);
  return STOMSFEM_OK;
}

static void patch_limits(const stomsfem_grid* g, int max_o, int* nmax, int* bmax) {
  const int rho = g->nf / g->nc;
  const int side = rho + 2 * max_o < g->nf ? rho + 2 * max_o : g->nf;
  const int m = side - 1;
  *nmax = m * m > 1 ? m * m : 1;
  *bmax = m + 1;
}

template <typename TK, typename TA, int RPL, int G, int MODE, bool PG, bool OSC = false, int TC = 0>
static int launch_upscale(const UpscaleArgs& A, long long max_blocks, cudaStream_t st) {
  auto kern = upscale_kernel<TK, TA, RPL, G, MODE, PG, OSC, TC>;
  constexpr int WPB = upscale_warps(sizeof(TK) == 8, G);
  // (oscillatory data: each unit's edge tables after all the windows)
  const size_t unit_smem = TC > 0 ? kTcSmemWarp : blk_smem_bytes<TK>(G / 2, A.bmax);
  const size_t smem = (unit_smem + (OSC ? osc_tab_bytes(A.bmax) : 0)) * WPB * (32 / G);
  STOMSFEM_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  STOMSFEM_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WPB * 32, smem));
  if (per_sm < 1) return set_error(STOMSFEM_EINVAL, "upscale kernel does not fit on an SM (smem %zu)", smem);
  if (A.blocks_per_sm_cap > 0 && per_sm > A.blocks_per_sm_cap) per_sm = A.blocks_per_sm_cap;
  long long blocks = (long long)per_sm * device_sm_count();
  if (blocks > max_blocks) blocks = max_blocks;
  if (blocks < 1) blocks = 1;
  kern<<<(unsigned)blocks, WPB * 32, smem, st>>>(A);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  return STOMSFEM_OK;
}

template <typename TK, typename TA, int G, int MODE = kModeAll, bool PG = false, bool OSC = false>
static int launch_rpl(const UpscaleArgs& A, long long max_blocks, cudaStream_t st) {
  const int rpl = (G / 2 + A.bmax + G - 1) / G;  // <= 3 (G = 32) or 5 (G = 16) for bmax <= 64
  if (rpl <= 1) return launch_upscale<TK, TA, 1, G, MODE, PG, OSC>(A, max_blocks, st);
  if (rpl == 2) return launch_upscale<TK, TA, 2, G, MODE, PG, OSC>(A, max_blocks, st);
  if (rpl == 3) return launch_upscale<TK, TA, 3, G, MODE, PG, OSC>(A, max_blocks, st);
  if constexpr (G == 16) {
    if (rpl == 4) return launch_upscale<TK, TA, 4, G, MODE, PG, OSC>(A, max_blocks, st);
    return launch_upscale<TK, TA, 5, G, MODE, PG, OSC>(A, max_blocks, st);
  }
  return set_error(STOMSFEM_EINVAL, "bandwidth %d too large", A.bmax);
}

// Bytes at the end of the workspace for the two cell lists of the split
// FP32 launch.
static size_t cell_list_bytes(const stomsfem_grid* g) { return round256(sizeof(int32_t) * (3 * (size_t)g->nc * g->nc + 4)); }

// Lanes per unit of each form: two units per warp.
constexpr int group_lanes(int) { return 16; }

// Factorisation engines of the FP32 forms: the two-units-per-warp FMA
// factorisation of band_block.cuh in column blocks of 8 (any bandwidth),
// the same with one unit per warp in column blocks of 16 (WIDE), or the
// tensor-core factorisation of band_tc.cuh with operands in three TF32
// parts (exact) or two parts (about 2^-21 per product), for patches with a
// half bandwidth in [4, 40].
enum {
  kEngineAuto = STOMSFEM_ENGINE_AUTO,
  kEngineBlocked = STOMSFEM_ENGINE_BLOCKED,
  kEngineTc3 = STOMSFEM_ENGINE_TC3,
  kEngineTc2 = STOMSFEM_ENGINE_TC2,
  kEngineWide = STOMSFEM_ENGINE_WIDE
};

// The engine AUTO resolves to.
constexpr int kEngineDefault = kEngineBlocked;

static bool upscale_tc_eligible(int precision, int rho, int bmax) {
  return precision != STOMSFEM_FP64 && rho >= 4 && bmax <= kTcBMax;
}
// Whether `engine` (not AUTO) may run these patches in this form.
static bool upscale_engine_eligible(int engine, int precision, int rho, int bmax) {
  if (engine == kEngineBlocked) return true;
  if (precision == STOMSFEM_FP64) return false;
  if (engine == kEngineWide) return true;
  return (engine == kEngineTc3 || engine == kEngineTc2) && upscale_tc_eligible(precision, rho, bmax);
}
static int upscale_engine(int requested, int precision, int rho, int bmax) {
  if (precision == STOMSFEM_FP64) return kEngineBlocked;
  const int e = requested == kEngineAuto ? kEngineDefault : requested;
  return upscale_engine_eligible(e, precision, rho, bmax) ? e : kEngineBlocked;
}
// Lanes per unit of the resolved engine.
static int upscale_engine_lanes(int engine) { return engine == kEngineBlocked ? 16 : 32; }
static bool upscale_uses_tc(int precision, int rho, int bmax) {
  return upscale_engine_lanes(upscale_engine(kEngineAuto, precision, rho, bmax)) == 32;
}

// The WIDE engine's launches (upscale_wide.cu; the Galerkin form without
// the oscillatory data).  fp64_acc: TA = double (the FP32 + refinement form).
int launch_wide(bool fp64_acc, int mode, const UpscaleArgs& A, long long max_blocks, cudaStream_t st);

// Launch of an FP32-factor form with the chosen engine.
template <typename TA, int MODE, bool PG, bool OSC>
static int launch_fp32(int engine, const UpscaleArgs& A, long long max_blocks, cudaStream_t st) {
  if (engine == kEngineTc3) return launch_upscale<float, TA, 2, 32, MODE, PG, OSC, 3>(A, max_blocks, st);
  if constexpr (!PG && !OSC) {
    if (engine == kEngineTc2) return launch_upscale<float, TA, 2, 32, MODE, PG, OSC, 2>(A, max_blocks, st);
    if (engine == kEngineWide) return launch_wide(std::is_same<TA, double>::value, MODE, A, max_blocks, st);
  }
  if (engine != kEngineBlocked) return set_error(STOMSFEM_EINVAL, "engine %d not offered for this form", engine);
  return launch_rpl<float, TA, 16, MODE, PG, OSC>(A, max_blocks, st);
}

// The host side of stomsfem_upscale / stomsfem_upscale_pg (PG: Ke holds
// 16 entries per unit; OSC: the oscillatory boundary data of the cell
// problems, stomsfem_upscale_bc).
template <bool PG, bool OSC = false>
int upscale_run(const stomsfem_grid* grid, const double* a, const int8_t* oversample, int32_t max_oversample,
                int32_t S, int32_t precision, int32_t refine_iters, double* Ke, double* be, double* phi,
                int32_t* unit_status, void* workspace, size_t workspace_bytes, stomsfem_stream_t stream,
                const UpscaleTuning& tune = UpscaleTuning()) {
  int rc = validate_grid(grid);
  if (rc) return rc;
  if (S < 0) return set_error(STOMSFEM_EINVAL, "S < 0");
  if (precision < 0 || precision > 2) return set_error(STOMSFEM_EINVAL, "bad precision %d", precision);
  if (max_oversample < 0) return set_error(STOMSFEM_EINVAL, "bad max_oversample");
  if (refine_iters < 0 || refine_iters > 8)
    return set_error(STOMSFEM_EINVAL, "refine_iters must be in [0, 8]");
  if (S == 0) return STOMSFEM_OK;
  if (!a || !Ke || !be || !workspace)
    return set_error(STOMSFEM_EINVAL, "a, Ke, be and workspace must be device pointers");
  const int mo = oversample ? max_oversample : 0;
  int nmax, bmax;
  patch_limits(grid, mo, &nmax, &bmax);
  if (bmax > kMaxBand)
    return set_error(STOMSFEM_EINVAL, "patch bandwidth %d exceeds %d (rho + 2*max_o too large)",
                     bmax, kMaxBand);
  size_t sb, lb;
  slot_layout(nmax, bmax, precision, &sb, &lb);
  const long long units = (long long)S * grid->nc * grid->nc;
  const long long slots = (long long)(workspace_bytes / sb);
  const int engine = upscale_engine(tune.engine, precision, grid->nf / grid->nc, bmax);
  const int G = upscale_engine_lanes(engine);
  const int WPB = upscale_warps(precision == STOMSFEM_FP64, G);
  const int slots_per_block = WPB * (32 / G);
  if (slots < slots_per_block)
    return set_error(STOMSFEM_ENOMEM, "workspace %zu bytes < %d slots of %zu bytes", workspace_bytes,
                     slots_per_block, sb);
  long long max_blocks = slots / slots_per_block;
  const long long items = G == 32 ? units : (long long)((S + 1) / 2) * grid->nc * grid->nc;
  const long long need = (items + WPB - 1) / WPB;
  if (max_blocks > need) max_blocks = need;

  UpscaleArgs A;
  A.a = a;
  A.oversample = oversample;
  A.nf = grid->nf;
  A.nc = grid->nc;
  A.rho = grid->nf / grid->nc;
  A.max_o = mo;
  A.S = S;
  A.f = grid->f;
  A.fq = grid->f / (4.0 * (double)grid->nf * (double)grid->nf);
  A.fH2 = grid->f / ((double)grid->nc * (double)grid->nc);
  A.refine = precision == STOMSFEM_FP32_REFINED ? refine_iters : 0;
  A.Ke = Ke;
  A.be = be;
  A.phi = phi;
  A.status = unit_status;
  A.ws = static_cast<unsigned char*>(workspace);
  A.slot_bytes = sb;
  A.l_bytes = lb;
  A.bmax = bmax;
  A.nmax = nmax;
  A.units = units;
  A.unit_list = nullptr;
  A.unit_count = nullptr;
  A.cell_list = nullptr;
  A.cell_count = nullptr;
  A.blocks_per_sm_cap = tune.blocks_per_sm;
  A.order = tune.order;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // cell lists at the end of the workspace (the split launch, or the order
  // by patch size), when the slots of one block still fit before them
  const int ncell = grid->nc * grid->nc;
  const size_t lbytes = cell_list_bytes(grid);
  const long long slots2 = workspace_bytes > lbytes ? (long long)((workspace_bytes - lbytes) / sb) : 0;
  const bool lists_fit = oversample && slots2 >= slots_per_block;
  unsigned char* lbase = static_cast<unsigned char*>(workspace) + ((workspace_bytes - lbytes) & ~size_t(255));
  int32_t* list0 = reinterpret_cast<int32_t*>(lbase);
  int32_t* list1 = list0 + ncell;
  int32_t* listall = list1 + ncell;
  int32_t* counts = listall + ncell;
  const bool sorted = tune.order == 1 && lists_fit;
  const long long mb = lists_fit && max_blocks > slots2 / slots_per_block ? slots2 / slots_per_block : max_blocks;
  // the oscillatory data: every cell by back substitution in one launch
  // (the forward-only route never forms psi0, which the Petrov-Galerkin
  // sums then need, and one launch mode keeps the compile short)
  if constexpr (!OSC) {
    if (precision == STOMSFEM_FP32 && !phi && tune.split_fp32) {
      // FP32 without phi output: cells without oversampling take the
      // forward-only route in a launch of their own, the others follow
      if (!oversample) return launch_fp32<float, kModeFwd, PG, OSC>(engine, A, max_blocks, st);
      if (lists_fit) {
        upscale_cell_lists_kernel<<<1, 32, 0, st>>>(oversample, ncell, mo, sorted ? 1 : 0, list0, list1, listall,
                                                    counts);
        STOMSFEM_TRY_CUDA(cudaGetLastError());
        A.cell_list = list0;
        A.cell_count = counts;
        rc = launch_fp32<float, kModeFwd, PG, OSC>(engine, A, mb, st);
        if (rc) return rc;
        A.cell_list = list1;
        A.cell_count = counts + 1;
        return launch_fp32<float, kModeRest, PG, OSC>(engine, A, mb, st);
      }
    }
  }
  if (sorted) {
    // one launch over every cell, largest patches first
    upscale_cell_lists_kernel<<<1, 32, 0, st>>>(oversample, ncell, mo, 1, list0, list1, listall, counts);
    STOMSFEM_TRY_CUDA(cudaGetLastError());
    A.cell_list = listall;
    A.cell_count = counts + 2;
    max_blocks = mb;
  }
  if (precision == STOMSFEM_FP64)
    return launch_rpl<double, double, group_lanes(STOMSFEM_FP64), kModeAll, PG, OSC>(A, max_blocks, st);
  if (precision == STOMSFEM_FP32_REFINED) return launch_fp32<double, kModeAll, PG, OSC>(engine, A, max_blocks, st);
  return launch_fp32<float, kModeAll, PG, OSC>(engine, A, max_blocks, st);
}


}  // namespace stomsfem
