/*
 * Plain FP64 CPU oracle for the StoMsFEM local-upscaling hot path
 * (Hou, Li, Zhang: "Exploring the locally low dimensional structure in
 * solving random elliptic PDEs").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls,
 * links or includes this file; only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Everything here is the textbook definition written out, slow and
 * obviously correct, in IEEE double:
 *   - coefficient sampling    a(x, xi) = exp(s * sum_i xi_i psi_i(x))
 *                             (nonlinear transform, Sec. 2.1.3) or the
 *                             bounded-exponent variant exp(L*sigmoid(g*z));
 *   - fine Q1 finite elements (the fine mesh T_h of Sec. 2.2);
 *   - the MsFEM cell problem  -div(a grad phi) = 0 in the patch,
 *                             phi = bilinear nodal function on the patch
 *                             boundary (Eq. MsFEB), solved on T_h, or the
 *                             oscillatory boundary data (harmonic
 *                             coordinate along each edge, Sec. 5.3);
 *   - oversampling            (Remark on oversampling, Sec. 2.2): solve on
 *                             the enlarged patch, recombine the patch
 *                             solutions so the basis is nodal at the cell
 *                             corners, restrict to the cell;
 *   - upscaled stiffness/load (Eq. stiffness_local): S_ll' = int a grad
 *                             phi_l . grad phi_l', b_l = int f phi_l;
 *   - coarse assembly + solve (Eq. upscaleSUF) with zero Dirichlet data;
 *   - fine-grid FEM           (the standard FEM the paper compares with).
 *
 * Linear systems use this file's own banded Cholesky.  Each of the four
 * cell problems is solved separately (no partition-of-unity shortcut) so
 * that sum_l phi_l == 1 remains a genuine check.
 *
 * Conventions: fine grid nf x nf elements on the unit square, h = 1/nf;
 * node (i, j) at (i h, j h), i = x index; arrays are y-major
 * (index j*(nf+1)+i for nodes, ey*nf+ex for elements).  Element corner
 * order SW, SE, NE, NW.  Coarse cell (cx, cy) covers fine elements
 * [cx*rho, (cx+1)*rho) x [cy*rho, (cy+1)*rho), rho = nf/nc.  K_e is
 * packed as the upper triangle row-major: (0,0) (0,1) (0,2) (0,3) (1,1)
 * (1,2) (1,3) (2,2) (2,3) (3,3).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Q1 element stiffness on a square for unit coefficient (independent of
 * the element size in 2D), corners SW, SE, NE, NW. */
static const double KREF[4][4] = {
    {4.0 / 6.0, -1.0 / 6.0, -2.0 / 6.0, -1.0 / 6.0},
    {-1.0 / 6.0, 4.0 / 6.0, -1.0 / 6.0, -2.0 / 6.0},
    {-2.0 / 6.0, -1.0 / 6.0, 4.0 / 6.0, -1.0 / 6.0},
    {-1.0 / 6.0, -2.0 / 6.0, -1.0 / 6.0, 4.0 / 6.0}};

/* corner c of an element (ex, ey): x/y offsets */
static const int CDX[4] = {0, 1, 1, 0};
static const int CDY[4] = {0, 0, 1, 1};

/* ---------------------------------------------------------------- */
/* Coefficient sampling: a(x, xi) at fine-element centroids.          */
/* kind 0: a = exp(scale * z);  kind 1: a = exp(L / (1 + exp(-g z)));  */
/* kind 2 (affine, Eq. RBaffine): a = g + scale * z                   */
/* with z(x) = sum_i xi_i exp(-|x - c_i|^2 / w^2), c_i the lattice     */
/* cell centres ((bx+1/2)/nbx, (by+1/2)/nby), i = by*nbx + bx.         */
/* ---------------------------------------------------------------- */
int orc_sample_coef(int nf, int kind, int nbx, int nby, double width,
                    double scale, double contrast_log, double gain,
                    const double* xi, int S, double* a, int nthreads) {
  if (nf <= 0 || nbx <= 0 || nby <= 0 || S < 0 || width <= 0.0) return -1;
  const int K = nbx * nby;
  const double h = 1.0 / nf;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static) collapse(2)
#endif
  for (int s = 0; s < S; ++s) {
    for (int ey = 0; ey < nf; ++ey) {
      const double y = (ey + 0.5) * h;
      for (int ex = 0; ex < nf; ++ex) {
        const double x = (ex + 0.5) * h;
        double z = 0.0;
        for (int by = 0; by < nby; ++by) {
          const double cy = (by + 0.5) / nby;
          for (int bx = 0; bx < nbx; ++bx) {
            const double cx = (bx + 0.5) / nbx;
            const double r2 = (x - cx) * (x - cx) + (y - cy) * (y - cy);
            z += xi[(size_t)s * K + by * nbx + bx] * exp(-r2 / (width * width));
          }
        }
        double v;
        if (kind == 0)
          v = exp(scale * z);
        else if (kind == 2)
          v = gain + scale * z;
        else
          v = exp(contrast_log / (1.0 + exp(-gain * z)));
        a[((size_t)s * nf + ey) * nf + ex] = v;
      }
    }
  }
  return 0;
}

/* The same coefficient for one sample, only on the element window
 * [ex0, ex1) x [ey0, ey1); the rest of a[nf*nf] is left untouched. */
int orc_sample_coef_window(int nf, int kind, int nbx, int nby, double width, double scale,
                           double contrast_log, double gain, const double* xi, int ex0,
                           int ex1, int ey0, int ey1, double* a) {
  if (nf <= 0 || nbx <= 0 || nby <= 0 || width <= 0.0) return -1;
  if (ex0 < 0 || ey0 < 0 || ex1 > nf || ey1 > nf) return -1;
  const double h = 1.0 / nf;
  for (int ey = ey0; ey < ey1; ++ey) {
    const double y = (ey + 0.5) * h;
    for (int ex = ex0; ex < ex1; ++ex) {
      const double x = (ex + 0.5) * h;
      double z = 0.0;
      for (int by = 0; by < nby; ++by) {
        const double cy = (by + 0.5) / nby;
        for (int bx = 0; bx < nbx; ++bx) {
          const double cx = (bx + 0.5) / nbx;
          const double r2 = (x - cx) * (x - cx) + (y - cy) * (y - cy);
          z += xi[by * nbx + bx] * exp(-r2 / (width * width));
        }
      }
      a[(size_t)ey * nf + ex] =
          kind == 0 ? exp(scale * z) : kind == 2 ? gain + scale * z : exp(contrast_log / (1.0 + exp(-gain * z)));
    }
  }
  return 0;
}

/* ---------------------------------------------------------------- */
/* Banded symmetric positive definite matrices.                       */
/* Storage: band[k*(bw+1) + d] = A[k][k-d], d = 0..bw (lower band).   */
/* ---------------------------------------------------------------- */
static inline double* band_at(double* band, int bw, int r, int c) {
  /* r >= c, r - c <= bw */
  return &band[(size_t)r * (bw + 1) + (r - c)];
}

/* In-place Cholesky A = L L^T, L stored in the same band. Returns 0 or
 * the (1-based) index of the first non-positive pivot. */
static int band_cholesky(double* band, int n, int bw) {
  for (int j = 0; j < n; ++j) {
    /* L[j][j] = sqrt(A[j][j] - sum_{p<j} L[j][p]^2) */
    double s = *band_at(band, bw, j, j);
    const int p0 = j - bw < 0 ? 0 : j - bw;
    for (int p = p0; p < j; ++p) {
      const double l = *band_at(band, bw, j, p);
      s -= l * l;
    }
    if (!(s > 0.0)) return j + 1;
    const double ljj = sqrt(s);
    *band_at(band, bw, j, j) = ljj;
    /* L[i][j] = (A[i][j] - sum_{p<j} L[i][p] L[j][p]) / L[j][j] */
    const int i1 = j + bw < n - 1 ? j + bw : n - 1;
    for (int i = j + 1; i <= i1; ++i) {
      double t = *band_at(band, bw, i, j);
      const int q0 = i - bw > p0 ? i - bw : p0;
      for (int p = q0; p < j; ++p)
        t -= *band_at(band, bw, i, p) * *band_at(band, bw, j, p);
      *band_at(band, bw, i, j) = t / ljj;
    }
  }
  return 0;
}

/* Solve L L^T x = b in place (b overwritten with x). */
static void band_solve(double* band, int n, int bw, double* b) {
  for (int i = 0; i < n; ++i) { /* L y = b */
    double t = b[i];
    const int p0 = i - bw < 0 ? 0 : i - bw;
    for (int p = p0; p < i; ++p) t -= *band_at(band, bw, i, p) * b[p];
    b[i] = t / *band_at(band, bw, i, i);
  }
  for (int i = n - 1; i >= 0; --i) { /* L^T x = y */
    double t = b[i];
    const int q1 = i + bw < n - 1 ? i + bw : n - 1;
    for (int q = i + 1; q <= q1; ++q) t -= *band_at(band, bw, q, i) * b[q];
    b[i] = t / *band_at(band, bw, i, i);
  }
}

/* 4x4 inverse by Gauss-Jordan elimination with partial pivoting. */
static int inv4(const double Ain[4][4], double Ainv[4][4]) {
  double M[4][8];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 8; ++c) M[r][c] = c < 4 ? Ain[r][c] : (c - 4 == r ? 1.0 : 0.0);
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int r = c + 1; r < 4; ++r)
      if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
    if (M[piv][c] == 0.0) return -1;
    if (piv != c)
      for (int k = 0; k < 8; ++k) {
        double t = M[c][k]; M[c][k] = M[piv][k]; M[piv][k] = t;
      }
    const double d = M[c][c];
    for (int k = 0; k < 8; ++k) M[c][k] /= d;
    for (int r = 0; r < 4; ++r)
      if (r != c) {
        const double f = M[r][c];
        for (int k = 0; k < 8; ++k) M[r][k] -= f * M[c][k];
      }
  }
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) Ainv[r][c] = M[r][c + 4];
  return 0;
}

/* ---------------------------------------------------------------- */
/* One MsFEM unit: cell (cx, cy) of one sample, oversampling layer o. */
/*   a      : [nf*nf] coefficient of this sample                       */
/*   Ke[10] : packed upscaled stiffness, be[4] : upscaled load         */
/*   phi    : optional [4][(rho+1)^2] basis on the cell nodes          */
/*   psi    : optional [4][(Nx+1)(Ny+1)] patch solutions (before the   */
/*            oversampling recombination); dims via patch_dims         */
/* Returns 0, or -k for a failed Cholesky at pivot k.                  */
/* ---------------------------------------------------------------- */
void orc_patch_bounds(int nf, int nc, int cx, int cy, int o, int* x0, int* x1,
                      int* y0, int* y1) {
  const int rho = nf / nc;
  *x0 = cx * rho - o < 0 ? 0 : cx * rho - o;
  *x1 = (cx + 1) * rho + o > nf ? nf : (cx + 1) * rho + o;
  *y0 = cy * rho - o < 0 ? 0 : cy * rho - o;
  *y1 = (cy + 1) * rho + o > nf ? nf : (cy + 1) * rho + o;
}

/* Oscillatory boundary data of one patch edge: the harmonic coordinate
 * t_k = sum_{e<k} 1/a_e / sum_e 1/a_e at the edge's nodes k = 0..N, a_e the
 * coefficient of the patch element next to edge segment e, i.e. the
 * solution of the reduced problem (a u')' = 0 along the edge with u = 0, 1
 * at its ends.  a0 points at the first such element, step is the distance
 * between consecutive ones. */
static void edge_harmonic(const double* a0, long step, int N, double* t) {
  double tot = 0.0;
  for (int e = 0; e < N; ++e) tot += 1.0 / a0[(size_t)e * step];
  double acc = 0.0;
  t[0] = 0.0;
  for (int e = 0; e < N; ++e) {
    acc += 1.0 / a0[(size_t)e * step];
    t[e + 1] = acc / tot;
  }
  t[N] = 1.0;
}

/* One unit with boundary data bc: 0 the bilinear nodal functions of the
 * patch (Eq. MsFEB), 1 the oscillatory boundary condition (the MsFEM option
 * of the short-correlation example, Sec. 5.3): on every patch edge the
 * nodal function interpolates its two corner values linearly in the edge's
 * harmonic coordinate (edge_harmonic) instead of in arc length. */
static int cell_solve(int nf, int nc, double f, const double* a, int cx, int cy, int o, int bc,
                      double* Ke, double* be, double* phi, double* psi);

int orc_cell(int nf, int nc, double f, const double* a, int cx, int cy, int o,
             double* Ke, double* be, double* phi, double* psi) {
  return cell_solve(nf, nc, f, a, cx, cy, o, 0, Ke, be, phi, psi);
}

int orc_cell_bc(int nf, int nc, double f, const double* a, int cx, int cy, int o, int bc,
                double* Ke, double* be, double* phi, double* psi) {
  if (bc != 0 && bc != 1) return -1000;
  return cell_solve(nf, nc, f, a, cx, cy, o, bc, Ke, be, phi, psi);
}

static int cell_solve(int nf, int nc, double f, const double* a, int cx, int cy, int o, int bc,
                      double* Ke, double* be, double* phi, double* psi) {
  if (nf <= 0 || nc <= 0 || nf % nc != 0 || o < 0) return -1000;
  const int rho = nf / nc;
  int x0, x1, y0, y1;
  orc_patch_bounds(nf, nc, cx, cy, o, &x0, &x1, &y0, &y1);
  const int Nx = x1 - x0, Ny = y1 - y0;     /* patch elements per side */
  const int mx = Nx - 1, my = Ny - 1;       /* interior nodes per side */
  const int n = mx * my;
  const int bw = mx + 1;                    /* 9-point stencil bandwidth */
  const int PN = (Nx + 1) * (Ny + 1);       /* patch nodes */

  double* band = (double*)calloc((size_t)(n > 0 ? n : 1) * (bw + 1), sizeof(double));
  double* rhs = (double*)calloc((size_t)4 * (n > 0 ? n : 1), sizeof(double));
  double* pv = (double*)malloc(sizeof(double) * 4 * PN); /* psi_l on patch nodes */
  if (!band || !rhs || !pv) { free(band); free(rhs); free(pv); return -1001; }

  /* Boundary data: the bilinear nodal functions of the patch rectangle,
   * p_SW = (1-X)(1-Y), p_SE = X(1-Y), p_NE = X Y, p_NW = (1-X) Y, with
   * X, Y in [0, 1] the patch's own normalised coordinates (Eq. MsFEB). */
  for (int j = 0; j <= Ny; ++j)
    for (int i = 0; i <= Nx; ++i) {
      const double X = (double)i / Nx, Y = (double)j / Ny;
      const int k = j * (Nx + 1) + i;
      pv[0 * PN + k] = (1.0 - X) * (1.0 - Y);
      pv[1 * PN + k] = X * (1.0 - Y);
      pv[2 * PN + k] = X * Y;
      pv[3 * PN + k] = (1.0 - X) * Y;
    }
  if (bc == 1) {
    /* oscillatory data on the four edges; interior values are unknowns
     * (the assembly reads pv at boundary nodes only) */
    double* tb = (double*)malloc(sizeof(double) * (size_t)(2 * (Nx + 1) + 2 * (Ny + 1)));
    if (!tb) { free(band); free(rhs); free(pv); return -1001; }
    double* tt = tb + (Nx + 1);
    double* tl = tt + (Nx + 1);
    double* tr = tl + (Ny + 1);
    edge_harmonic(a + (size_t)y0 * nf + x0, 1, Nx, tb);                 /* bottom: row y0 */
    edge_harmonic(a + (size_t)(y1 - 1) * nf + x0, 1, Nx, tt);           /* top: row y1-1 */
    edge_harmonic(a + (size_t)y0 * nf + x0, nf, Ny, tl);                /* left: column x0 */
    edge_harmonic(a + (size_t)y0 * nf + (x1 - 1), nf, Ny, tr);          /* right: column x1-1 */
    for (int k = 0; k < 4 * PN; ++k) pv[k] = 0.0;
    for (int i = 0; i <= Nx; ++i) {
      const int kb = i, kt = Ny * (Nx + 1) + i;
      pv[0 * PN + kb] = 1.0 - tb[i]; /* SW..SE along the bottom */
      pv[1 * PN + kb] = tb[i];
      pv[3 * PN + kt] = 1.0 - tt[i]; /* NW..NE along the top */
      pv[2 * PN + kt] = tt[i];
    }
    for (int j = 0; j <= Ny; ++j) {
      const int kl = j * (Nx + 1), kr = j * (Nx + 1) + Nx;
      pv[0 * PN + kl] = 1.0 - tl[j]; /* SW..NW along the left */
      pv[3 * PN + kl] = tl[j];
      pv[1 * PN + kr] = 1.0 - tr[j]; /* SE..NE along the right */
      pv[2 * PN + kr] = tr[j];
    }
    free(tb);
  }

  /* Element-by-element assembly of A_II and of -A_IB p_l. */
  for (int ey = 0; ey < Ny; ++ey)
    for (int ex = 0; ex < Nx; ++ex) {
      const double ae = a[(size_t)(y0 + ey) * nf + (x0 + ex)];
      for (int r = 0; r < 4; ++r) {
        const int ri = ex + CDX[r], rj = ey + CDY[r];
        const int r_int = ri > 0 && ri < Nx && rj > 0 && rj < Ny;
        if (!r_int) continue;
        const int rk = (rj - 1) * mx + (ri - 1);
        for (int c = 0; c < 4; ++c) {
          const int ci = ex + CDX[c], cj = ey + CDY[c];
          const double v = ae * KREF[r][c];
          const int c_int = ci > 0 && ci < Nx && cj > 0 && cj < Ny;
          if (c_int) {
            const int ck = (cj - 1) * mx + (ci - 1);
            if (ck <= rk) *band_at(band, bw, rk, ck) += v;
          } else {
            const int pk = cj * (Nx + 1) + ci;
            for (int l = 0; l < 4; ++l) rhs[l * n + rk] -= v * pv[l * PN + pk];
          }
        }
      }
    }

  int rc = 0;
  if (n > 0) {
    rc = band_cholesky(band, n, bw);
    if (rc != 0) { free(band); free(rhs); free(pv); return -rc; }
    for (int l = 0; l < 4; ++l) band_solve(band, n, bw, rhs + (size_t)l * n);
    for (int j = 1; j < Ny; ++j)
      for (int i = 1; i < Nx; ++i)
        for (int l = 0; l < 4; ++l)
          pv[l * PN + j * (Nx + 1) + i] = rhs[l * n + (j - 1) * mx + (i - 1)];
  }
  if (psi) memcpy(psi, pv, sizeof(double) * 4 * PN);

  /* Oversampling recombination: C[j][k] = psi_j(corner k of the cell);
   * phi_i = sum_j Cinv[i][j]... with phi_i(corner k) = delta_ik, i.e.
   * phi = D psi with D C = I, D = C^{-1}. */
  const int ccx[4] = {cx * rho, (cx + 1) * rho, (cx + 1) * rho, cx * rho};
  const int ccy[4] = {cy * rho, cy * rho, (cy + 1) * rho, (cy + 1) * rho};
  double C[4][4], D[4][4];
  for (int j = 0; j < 4; ++j)
    for (int k = 0; k < 4; ++k)
      C[j][k] = pv[j * PN + (ccy[k] - y0) * (Nx + 1) + (ccx[k] - x0)];
  if (inv4(C, D) != 0) { free(band); free(rhs); free(pv); return -1002; }

  /* phi on the cell nodes */
  const int CN = (rho + 1) * (rho + 1);
  double* ph = (double*)malloc(sizeof(double) * 4 * CN);
  if (!ph) { free(band); free(rhs); free(pv); return -1001; }
  for (int j = 0; j <= rho; ++j)
    for (int i = 0; i <= rho; ++i) {
      const int pk = (cy * rho + j - y0) * (Nx + 1) + (cx * rho + i - x0);
      for (int l = 0; l < 4; ++l) {
        double v = 0.0;
        for (int q = 0; q < 4; ++q) v += D[l][q] * pv[q * PN + pk];
        ph[l * CN + j * (rho + 1) + i] = v;
      }
    }

  /* Eq. stiffness_local on the fine grid of the cell: exact integration of
   * a piecewise-constant a against Q1 functions. */
  double S[4][4] = {{0}};
  double b[4] = {0};
  const double h = 1.0 / nf;
  for (int ey = 0; ey < rho; ++ey)
    for (int ex = 0; ex < rho; ++ex) {
      const double ae = a[(size_t)(cy * rho + ey) * nf + (cx * rho + ex)];
      double loc[4][4];
      for (int l = 0; l < 4; ++l)
        for (int c = 0; c < 4; ++c)
          loc[l][c] = ph[l * CN + (ey + CDY[c]) * (rho + 1) + (ex + CDX[c])];
      for (int l = 0; l < 4; ++l)
        for (int lp = 0; lp < 4; ++lp) {
          double e = 0.0;
          for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) e += loc[l][r] * KREF[r][c] * loc[lp][c];
          S[l][lp] += ae * e;
        }
      for (int l = 0; l < 4; ++l)
        for (int c = 0; c < 4; ++c) b[l] += f * h * h / 4.0 * loc[l][c];
    }
  int q = 0;
  for (int l = 0; l < 4; ++l)
    for (int lp = l; lp < 4; ++lp) Ke[q++] = S[l][lp];
  for (int l = 0; l < 4; ++l) be[l] = b[l];
  if (phi) memcpy(phi, ph, sizeof(double) * 4 * CN);
  free(ph); free(band); free(rhs); free(pv);
  return 0;
}

/* All units of S samples.  oversample: [nc*nc] layer widths or NULL (0).
 * Ke [S][nc*nc][10], be [S][nc*nc][4], phi optional
 * [S][nc*nc][4][(rho+1)^2].  status [S*nc*nc] (0 ok). */
int orc_upscale_bc(int nf, int nc, double f, const double* a, const int8_t* oversample, int bc,
                   int S, double* Ke, double* be, double* phi, int32_t* status, int nthreads);

int orc_upscale(int nf, int nc, double f, const double* a, const int8_t* oversample,
                int S, double* Ke, double* be, double* phi, int32_t* status,
                int nthreads) {
  return orc_upscale_bc(nf, nc, f, a, oversample, 0, S, Ke, be, phi, status, nthreads);
}

/* orc_upscale with the boundary data bc of cell_solve. */
int orc_upscale_bc(int nf, int nc, double f, const double* a, const int8_t* oversample, int bc,
                   int S, double* Ke, double* be, double* phi, int32_t* status, int nthreads) {
  if (nf <= 0 || nc <= 0 || nf % nc != 0 || S < 0 || (bc != 0 && bc != 1)) return -1;
  const int rho = nf / nc;
  const int CN = (rho + 1) * (rho + 1);
  const long units = (long)S * nc * nc;
  int bad = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
#endif
  for (long u = 0; u < units; ++u) {
    const int s = (int)(u / (nc * nc));
    const int cell = (int)(u % (nc * nc));
    const int cx = cell % nc, cy = cell / nc;
    const int o = oversample ? oversample[cell] : 0;
    const int rc = cell_solve(nf, nc, f, a + (size_t)s * nf * nf, cx, cy, o, bc,
                              Ke + (size_t)u * 10, be + (size_t)u * 4,
                              phi ? phi + (size_t)u * 4 * CN : NULL, NULL);
    if (status) status[u] = rc;
    if (rc != 0) bad = 1;
  }
  return bad ? -2 : 0;
}

/* Eq. upscaleSUF: assemble the coarse system from the packed K_e and b_e
 * over the (nc+1)^2 coarse nodes, keep the interior nodes (zero Dirichlet
 * on the boundary), solve.  u [S][(nc+1)^2], boundary entries 0. */
int orc_coarse_solve(int nc, const double* Ke, const double* be, int S, double* u) {
  if (nc <= 0 || S < 0) return -1;
  const int NN = nc + 1;
  const int mi = nc - 1, n = mi * mi, bw = mi + 1;
  for (int s = 0; s < S; ++s) {
    double* band = (double*)calloc((size_t)(n > 0 ? n : 1) * (bw + 1), sizeof(double));
    double* rhs = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    if (!band || !rhs) { free(band); free(rhs); return -3; }
    for (int cy = 0; cy < nc; ++cy)
      for (int cx = 0; cx < nc; ++cx) {
        const double* K = Ke + ((size_t)s * nc * nc + cy * nc + cx) * 10;
        const double* B = be + ((size_t)s * nc * nc + cy * nc + cx) * 4;
        double M[4][4];
        int q = 0;
        for (int l = 0; l < 4; ++l)
          for (int lp = l; lp < 4; ++lp) { M[l][lp] = K[q]; M[lp][l] = K[q]; ++q; }
        for (int r = 0; r < 4; ++r) {
          const int ri = cx + CDX[r], rj = cy + CDY[r];
          if (ri <= 0 || ri >= nc || rj <= 0 || rj >= nc) continue;
          const int rk = (rj - 1) * mi + (ri - 1);
          rhs[rk] += B[r];
          for (int c = 0; c < 4; ++c) {
            const int ci = cx + CDX[c], cj = cy + CDY[c];
            if (ci <= 0 || ci >= nc || cj <= 0 || cj >= nc) continue;
            const int ck = (cj - 1) * mi + (ci - 1);
            if (ck <= rk) *band_at(band, bw, rk, ck) += M[r][c];
          }
        }
      }
    int rc = 0;
    if (n > 0) {
      rc = band_cholesky(band, n, bw);
      if (rc == 0) band_solve(band, n, bw, rhs);
    }
    double* us = u + (size_t)s * NN * NN;
    for (int k = 0; k < NN * NN; ++k) us[k] = 0.0;
    if (rc == 0)
      for (int j = 1; j < nc; ++j)
        for (int i = 1; i < nc; ++i) us[j * NN + i] = rhs[(j - 1) * mi + (i - 1)];
    free(band); free(rhs);
    if (rc != 0) return -4;
  }
  return 0;
}

/* Standard Q1 FEM on the fine grid, zero Dirichlet data, load f:
 * u [(nf+1)^2], boundary entries 0. */
int orc_fine_fem(int nf, double f, const double* a, double* u) {
  if (nf <= 0) return -1;
  const int NN = nf + 1, mi = nf - 1, n = mi * mi, bw = mi + 1;
  const double h = 1.0 / nf;
  double* band = (double*)calloc((size_t)(n > 0 ? n : 1) * (bw + 1), sizeof(double));
  double* rhs = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (!band || !rhs) { free(band); free(rhs); return -3; }
  for (int ey = 0; ey < nf; ++ey)
    for (int ex = 0; ex < nf; ++ex) {
      const double ae = a[(size_t)ey * nf + ex];
      for (int r = 0; r < 4; ++r) {
        const int ri = ex + CDX[r], rj = ey + CDY[r];
        if (ri <= 0 || ri >= nf || rj <= 0 || rj >= nf) continue;
        const int rk = (rj - 1) * mi + (ri - 1);
        rhs[rk] += f * h * h / 4.0;
        for (int c = 0; c < 4; ++c) {
          const int ci = ex + CDX[c], cj = ey + CDY[c];
          if (ci <= 0 || ci >= nf || cj <= 0 || cj >= nf) continue;
          const int ck = (cj - 1) * mi + (ci - 1);
          if (ck <= rk) *band_at(band, bw, rk, ck) += ae * KREF[r][c];
        }
      }
    }
  int rc = 0;
  if (n > 0) {
    rc = band_cholesky(band, n, bw);
    if (rc == 0) band_solve(band, n, bw, rhs);
  }
  for (int k = 0; k < NN * NN; ++k) u[k] = 0.0;
  if (rc == 0)
    for (int j = 1; j < nf; ++j)
      for (int i = 1; i < nf; ++i) u[j * NN + i] = rhs[(j - 1) * mi + (i - 1)];
  free(band); free(rhs);
  return rc == 0 ? 0 : -4;
}

/* Solve a dense-in-band SPD system given as a full n x n row-major matrix
 * through this file's banded Cholesky (bw = half bandwidth).  Exposed so
 * that the factorisation itself can be checked against a library solve. */
int orc_band_solve_dense(int n, int bw, const double* A, double* b) {
  double* band = (double*)calloc((size_t)(n > 0 ? n : 1) * (bw + 1), sizeof(double));
  if (!band) return -3;
  for (int r = 0; r < n; ++r)
    for (int c = r - bw < 0 ? 0 : r - bw; c <= r; ++c)
      *band_at(band, bw, r, c) = A[(size_t)r * n + c];
  int rc = band_cholesky(band, n, bw);
  if (rc == 0) band_solve(band, n, bw, b);
  free(band);
  return rc == 0 ? 0 : -4;
}

/* ---------------------------------------------------------------- */
/* Petrov-Galerkin MsFEM (Eq. stiffness_local_petrov): trial functions */
/* the multiscale basis phi_l (with the oversampling recombination),  */
/* test functions the bilinear nodal functions q_l' of the coarse      */
/* cell:  S_ll' = int_cell a grad phi_l . grad q_l',                   */
/*        b_l   = int_cell f q_l = f H^2 / 4.                          */
/* Kpg[16] row-major (row l = trial, column l' = test).  q_l' is       */
/* bilinear on every fine element of the cell, so its nodal values     */
/* give the integral exactly: sum_e a_e phi_e^T K_ref q_e.             */
/* ---------------------------------------------------------------- */
int orc_cell_pg_bc(int nf, int nc, double f, const double* a, int cx, int cy, int o, int bc,
                   double* Kpg, double* bpg);

int orc_cell_pg(int nf, int nc, double f, const double* a, int cx, int cy, int o,
                double* Kpg, double* bpg) {
  return orc_cell_pg_bc(nf, nc, f, a, cx, cy, o, 0, Kpg, bpg);
}

/* orc_cell_pg with the trial basis from the boundary data bc of
 * cell_solve (the test functions stay the cell's bilinears). */
int orc_cell_pg_bc(int nf, int nc, double f, const double* a, int cx, int cy, int o, int bc,
                   double* Kpg, double* bpg) {
  if (nf <= 0 || nc <= 0 || nf % nc != 0 || o < 0 || (bc != 0 && bc != 1)) return -1000;
  const int rho = nf / nc;
  const int CN = (rho + 1) * (rho + 1);
  double Ke[10], be[4];
  double* ph = (double*)malloc(sizeof(double) * 4 * CN);
  if (!ph) return -1001;
  const int rc = cell_solve(nf, nc, f, a, cx, cy, o, bc, Ke, be, ph, NULL);
  if (rc != 0) { free(ph); return rc; }
  double S[4][4] = {{0}};
  for (int ey = 0; ey < rho; ++ey)
    for (int ex = 0; ex < rho; ++ex) {
      const double ae = a[(size_t)(cy * rho + ey) * nf + (cx * rho + ex)];
      double loc[4][4], ql[4][4];
      for (int c = 0; c < 4; ++c) {
        const double X = (double)(ex + CDX[c]) / rho, Y = (double)(ey + CDY[c]) / rho;
        ql[0][c] = (1.0 - X) * (1.0 - Y);
        ql[1][c] = X * (1.0 - Y);
        ql[2][c] = X * Y;
        ql[3][c] = (1.0 - X) * Y;
        for (int l = 0; l < 4; ++l) loc[l][c] = ph[l * CN + (ey + CDY[c]) * (rho + 1) + (ex + CDX[c])];
      }
      for (int l = 0; l < 4; ++l)
        for (int lp = 0; lp < 4; ++lp) {
          double e = 0.0;
          for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) e += loc[l][r] * KREF[r][c] * ql[lp][c];
          S[l][lp] += ae * e;
        }
    }
  for (int l = 0; l < 4; ++l)
    for (int lp = 0; lp < 4; ++lp) Kpg[l * 4 + lp] = S[l][lp];
  const double H = 1.0 / nc;
  for (int l = 0; l < 4; ++l) bpg[l] = f * H * H / 4.0;
  free(ph);
  return 0;
}

/* All units of S samples in the Petrov-Galerkin form: Kpg [S][nc*nc][16],
 * bpg [S][nc*nc][4], status [S*nc*nc]. */
int orc_upscale_pg_bc(int nf, int nc, double f, const double* a, const int8_t* oversample, int bc, int S,
                      double* Kpg, double* bpg, int32_t* status, int nthreads);

int orc_upscale_pg(int nf, int nc, double f, const double* a, const int8_t* oversample, int S,
                   double* Kpg, double* bpg, int32_t* status, int nthreads) {
  return orc_upscale_pg_bc(nf, nc, f, a, oversample, 0, S, Kpg, bpg, status, nthreads);
}

/* orc_upscale_pg with the boundary data bc of cell_solve. */
int orc_upscale_pg_bc(int nf, int nc, double f, const double* a, const int8_t* oversample, int bc, int S,
                      double* Kpg, double* bpg, int32_t* status, int nthreads) {
  if (nf <= 0 || nc <= 0 || nf % nc != 0 || S < 0 || (bc != 0 && bc != 1)) return -1;
  const long units = (long)S * nc * nc;
  int bad = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
#endif
  for (long u = 0; u < units; ++u) {
    const int s = (int)(u / (nc * nc));
    const int cell = (int)(u % (nc * nc));
    const int o = oversample ? oversample[cell] : 0;
    const int rc = orc_cell_pg_bc(nf, nc, f, a + (size_t)s * nf * nf, cell % nc, cell / nc, o, bc,
                                  Kpg + (size_t)u * 16, bpg + (size_t)u * 4);
    if (status) status[u] = rc;
    if (rc != 0) bad = 1;
  }
  return bad ? -2 : 0;
}

/* Banded LU without pivoting of a general matrix with half bandwidth bw
 * (row i keeps columns i-bw..i+bw at band[i*(2bw+1) + (j-i+bw)]),
 * forward elimination of rhs alongside, back substitution into rhs.
 * Returns 0, or k+1 for a zero pivot at step k. */
static int band_lu_solve(double* band, int n, int bw, double* rhs) {
  const int W = 2 * bw + 1;
#define AT(i, j) band[(size_t)(i) * W + ((j) - (i) + bw)]
  for (int k = 0; k < n; ++k) {
    const double piv = AT(k, k);
    if (!(piv != 0.0) || piv != piv) return k + 1;
    const int last = k + bw < n - 1 ? k + bw : n - 1;
    for (int i = k + 1; i <= last; ++i) {
      const double l = AT(i, k) / piv;
      AT(i, k) = 0.0;
      for (int j = k + 1; j <= last; ++j) AT(i, j) -= l * AT(k, j);
      rhs[i] -= l * rhs[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = rhs[k];
    const int last = k + bw < n - 1 ? k + bw : n - 1;
    for (int j = k + 1; j <= last; ++j) s -= AT(k, j) * rhs[j];
    rhs[k] = s / AT(k, k);
  }
#undef AT
  return 0;
}

/* Petrov-Galerkin coarse system: find U with sum_I U_I a(phi_I, q_J) =
 * (f, q_J) for every interior coarse node J, i.e. row J of the matrix
 * collects S_e[I_loc][J_loc] over the cells around J (the transpose of the
 * Galerkin-style assembly).  u [S][(nc+1)^2], boundary entries 0. */
int orc_coarse_solve_pg(int nc, const double* Kpg, const double* bpg, int S, double* u) {
  if (nc <= 0 || S < 0) return -1;
  const int NN = nc + 1;
  const int mi = nc - 1, n = mi * mi, bw = mi + 1, W = 2 * bw + 1;
  for (int s = 0; s < S; ++s) {
    double* band = (double*)calloc((size_t)(n > 0 ? n : 1) * W, sizeof(double));
    double* rhs = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    if (!band || !rhs) { free(band); free(rhs); return -3; }
    for (int cy = 0; cy < nc; ++cy)
      for (int cx = 0; cx < nc; ++cx) {
        const double* K = Kpg + ((size_t)s * nc * nc + cy * nc + cx) * 16;
        const double* B = bpg + ((size_t)s * nc * nc + cy * nc + cx) * 4;
        for (int r = 0; r < 4; ++r) { /* test node J */
          const int ri = cx + CDX[r], rj = cy + CDY[r];
          if (ri <= 0 || ri >= nc || rj <= 0 || rj >= nc) continue;
          const int J = (rj - 1) * mi + (ri - 1);
          rhs[J] += B[r];
          for (int c = 0; c < 4; ++c) { /* trial node I */
            const int ci = cx + CDX[c], cj = cy + CDY[c];
            if (ci <= 0 || ci >= nc || cj <= 0 || cj >= nc) continue;
            const int I = (cj - 1) * mi + (ci - 1);
            band[(size_t)J * W + (I - J + bw)] += K[c * 4 + r];
          }
        }
      }
    int rc = n > 0 ? band_lu_solve(band, n, bw, rhs) : 0;
    double* us = u + (size_t)s * NN * NN;
    for (int k = 0; k < NN * NN; ++k) us[k] = 0.0;
    if (rc == 0)
      for (int j = 1; j < nc; ++j)
        for (int i = 1; i < nc; ++i) us[j * NN + i] = rhs[(j - 1) * mi + (i - 1)];
    free(band); free(rhs);
    if (rc != 0) return -4;
  }
  return 0;
}

/* Mixed boundary data for the coarse system: the boundary conditions of
 * the anisotropy study of the high-contrast example (Sec. 5.2, Eqs.
 * xsquarewave and ysquarewave), i.e. prescribed values on chosen coarse
 * nodes (lines inside the domain included) and zero flux on the rest of
 * the boundary.  Every coarse node is an unknown.  The system over all
 * (nc+1)^2 nodes is assembled from every cell, with no boundary row
 * dropped (the natural condition needs nothing more): pg = 0 Galerkin from
 * the packed K_e [S][nc*nc][10], pg = 1 Petrov-Galerkin from K [S][nc*nc][16]
 * (row = test node J collects S_e[I_loc][J_loc]).  Then the row of every
 * node k with dmask[k] != 0 is replaced by u_k = g[k], and the band is
 * solved by the LU above.  A zero pivot (for instance no Dirichlet node at
 * all, whose pure Neumann matrix is singular) returns -4 and leaves that
 * sample's u NaN.  u [S][(nc+1)^2]. */
int orc_coarse_solve_bc(int nc, int pg, const double* K, const double* b, const uint8_t* dmask,
                        const double* g, int S, double* u) {
  if (nc <= 0 || S < 0 || (pg != 0 && pg != 1)) return -1;
  const int NN = nc + 1, n = NN * NN, bw = NN + 1, W = 2 * bw + 1;
  const int KN = pg ? 16 : 10;
  int ret = 0;
  for (int s = 0; s < S; ++s) {
    double* band = (double*)calloc((size_t)n * W, sizeof(double));
    double* rhs = (double*)calloc((size_t)n, sizeof(double));
    if (!band || !rhs) { free(band); free(rhs); return -3; }
    for (int cy = 0; cy < nc; ++cy)
      for (int cx = 0; cx < nc; ++cx) {
        const double* Kc = K + ((size_t)s * nc * nc + cy * nc + cx) * KN;
        const double* B = b + ((size_t)s * nc * nc + cy * nc + cx) * 4;
        double M[4][4]; /* M[row node][column node] of this cell's contribution */
        if (pg) {
          for (int t = 0; t < 4; ++t)
            for (int c = 0; c < 4; ++c) M[t][c] = Kc[c * 4 + t];
        } else {
          int q = 0;
          for (int l = 0; l < 4; ++l)
            for (int lp = l; lp < 4; ++lp) { M[l][lp] = Kc[q]; M[lp][l] = Kc[q]; ++q; }
        }
        for (int r = 0; r < 4; ++r) {
          const int rk = (cy + CDY[r]) * NN + (cx + CDX[r]);
          rhs[rk] += B[r];
          for (int c = 0; c < 4; ++c) {
            const int ck = (cy + CDY[c]) * NN + (cx + CDX[c]);
            band[(size_t)rk * W + (ck - rk + bw)] += M[r][c];
          }
        }
      }
    for (int k = 0; k < n; ++k)
      if (dmask[k]) {
        for (int d = 0; d < W; ++d) band[(size_t)k * W + d] = 0.0;
        band[(size_t)k * W + bw] = 1.0;
        rhs[k] = g[k];
      }
    const int rc = band_lu_solve(band, n, bw, rhs);
    double* us = u + (size_t)s * n;
    for (int k = 0; k < n; ++k) us[k] = rc == 0 ? rhs[k] : NAN;
    free(band); free(rhs);
    if (rc != 0) ret = -4;
  }
  return ret;
}
