// Blocked warp-level banded SPD solver for 9-point-stencil matrices (one
// warp per system).
//
// Right-looking banded Cholesky in column blocks of NB = 16.  For block K
// (rows/columns [K, K+nb)) the warp
//   1. factorises the tall panel [K, K+np) x [K, K+nb), np = nb + b: each
//      lane holds up to RPL panel rows in registers; the block-row
//      multipliers of each column step are broadcast through a
//      double-buffered shared vector (128-bit loads, one warp sync per
//      step); the NR right-hand sides ride along, which is the forward
//      substitution;
//   2. applies the rank-nb update to the trailing b x b window with 4 x 4
//      register tiles (128-bit shared loads of the transposed panel);
//   3. retires the block's rows and writes the next rows from values the
//      row generator loaded one block earlier (so the global-load latency
//      hides behind the panel and the trailing update).
// The matrix lives only as a window of RW >= NB + b band rows in shared
// memory (RW a power of two; row r at slot r & (RW-1), entry A[r][r-d] at
// column d).  Factor blocks go to global scratch as (NB + bmax) x NB
// row-major tiles; the substitutions stream them back through two shared
// staging buffers with asynchronous copies (next block in flight while the
// current one is used).
//
// Row generator interface:
//   typename Gen::Raw                  raw per-row values,
//   gen.load(r, Raw&)                  issue the global loads of row r,
//   gen.prefetch(r, double* dst4)      asynchronous copy of row r's values,
//   gen.from_smem(const double* src4, Raw&)
//   gen.make<T>(r, const Raw&, T e[5], T rhs[NR])
//                                      band entries A[r][r], A[r][r-1],
//                                      A[r][r-mx+1], A[r][r-mx], A[r][r-mx-1]
//                                      (0 where absent) and the rhs,
//   gen.mx                             offset of the south neighbour.
#pragma once
#include "common.cuh"

namespace stomsfem {

constexpr int kNB = 16;

template <typename T>
struct BlkSmem {
  T* wnd;  // [RW][PW] band rows; the 16 ring rows of the block just
           // factorised hold the trailing panel for the update,
           // p-major: pt[p*RP + (i - nb)] = L[K+i][K+p]
  T* tb;   // 2 x [NB + bmax][NB] factor block staging (aliases wnd)
  T* rhs;  // [RW][4]
  T* lb;   // 2 x [NB] broadcast of the block-row multipliers; [NB][4]
           // block solution in the stored forward substitution
  double* raw;  // [NB][4] coefficient values of the next rows (async prefetch)
  int RW, PW, RP;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline int blk_ring_rows(int bmax) {
  int r = 16;
  while (r < kNB + bmax) r <<= 1;
  return r;
}

// Row pitch: b + 1 band entries, and at least RP = bmax rounded up to 4 so
// that NB rows hold the transposed trailing panel.
__host__ __device__ inline int blk_pitch(int bmax) {
  const int rp = (bmax + 3) & ~3;
  return bmax + 1 > rp ? bmax + 1 : rp;
}

__host__ __device__ inline int blk_wnd_elems(int bmax) {
  const int a = blk_ring_rows(bmax) * blk_pitch(bmax), b = 2 * (kNB + bmax) * kNB;
  return a > b ? a : b;
}

template <typename T>
__host__ __device__ inline size_t blk_smem_bytes(int bmax) {
  const int RW = blk_ring_rows(bmax);
  return al16(sizeof(T) * blk_wnd_elems(bmax)) + al16(sizeof(T) * RW * 4) + al16(sizeof(T) * 4 * kNB) +
         al16(sizeof(double) * kNB * 4);
}

template <typename T>
__device__ inline BlkSmem<T> make_blk(unsigned char* base, int bmax) {
  BlkSmem<T> s;
  s.RW = blk_ring_rows(bmax);
  s.PW = blk_pitch(bmax);
  s.RP = (bmax + 3) & ~3;
  size_t o = 0;
  s.wnd = reinterpret_cast<T*>(base + o);
  s.tb = s.wnd;
  o += al16(sizeof(T) * blk_wnd_elems(bmax));
  s.rhs = reinterpret_cast<T*>(base + o);
  o += al16(sizeof(T) * s.RW * 4);
  s.lb = reinterpret_cast<T*>(base + o);
  o += al16(sizeof(T) * 4 * kNB);
  s.raw = reinterpret_cast<double*>(base + o);
  return s;
}

__host__ __device__ inline size_t blk_factor_elems(int n, int bmax) {
  return (size_t)((n + kNB - 1) / kNB) * (kNB + bmax) * kNB;
}

// The pivot and its reciprocal.  FP32: the hardware reciprocal square root
// (relative error a few ulp), which perturbs the factor at the level of FP32
// rounding; FP64: correctly rounded.
__device__ __forceinline__ void pivot_of(float a, float& d, float& dinv) {
  dinv = rsqrtf(a);
  d = a * dinv;
}
__device__ __forceinline__ void pivot_of(double a, double& d, double& dinv) {
  d = sqrt(a);
  dinv = 1.0 / d;
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Zero n16 consecutive 16-byte chunks of shared memory.
__device__ __forceinline__ void blk_zero16(void* dst, int n16, int lane) {
  float4* d = reinterpret_cast<float4*>(dst);
  for (int v = lane; v < n16; v += 32) d[v] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Rows [r0, r1) of the window (at most 32 rows; row r0 + l uses lane l's raw
// values): the generator's entries and rhs.  The rows' ring slots are zero
// on entry (the whole window is cleared when a factorisation starts, and each
// block's slots again once the block is retired).
template <typename T, int NR, class Gen>
__device__ __forceinline__ void blk_fill_raw(const Gen& gen, const BlkSmem<T>& s, int r0, int r1, int b, int lane,
                                             const typename Gen::Raw& raw) {
  const int msk = s.RW - 1;
  const int mx = gen.mx;
  const int r = r0 + lane;
  if (r < r1) {
    T e[5], rh[NR];
    gen.template make<T>(r, raw, e, rh);
    T* row = s.wnd + (r & msk) * s.PW;
    if (mx >= 3 && mx + 1 <= b) {
      // offsets 0, 1, mx-1, mx, mx+1 are distinct: plain stores
      row[0] = e[0];
      if (r >= 1) row[1] = e[1];
      if (r >= mx - 1) row[mx - 1] = e[2];
      if (r >= mx) row[mx] = e[3];
      if (r >= mx + 1) row[mx + 1] = e[4];
    } else {
      row[0] += e[0];
      if (r >= 1 && 1 <= b) row[1] += e[1];
      if (mx - 1 >= 0 && r >= mx - 1 && mx - 1 <= b) row[mx - 1] += e[2];
      if (r >= mx && mx <= b) row[mx] += e[3];
      if (r >= mx + 1 && mx + 1 <= b) row[mx + 1] += e[4];
    }
#pragma unroll
    for (int c = 0; c < NR; ++c) s.rhs[(r & msk) * 4 + c] = rh[c];
  }
}

// One column step j = J of the panel factorisation, then the next; the
// recursion keeps every register-array index a compile-time constant.
template <int J, typename T, int NR, int RPL>
__device__ __forceinline__ void panel_col(T (&pr)[RPL][kNB], T (&rh)[RPL][NR], T* lb, int lane,
                                          int nb, int np, int K, int& fail) {
  if constexpr (J < kNB) {
    if (J < nb && fail < 0) {
      const T dj = __shfl_sync(0xffffffffu, pr[0][J], J);
      if (!(dj > T(0))) fail = K + J;
      T d, dinv;
      pivot_of(dj > T(0) ? dj : T(1), d, dinv);
      T yj[NR];
#pragma unroll
      for (int c = 0; c < NR; ++c) yj[c] = __shfl_sync(0xffffffffu, rh[0][c], J) * dinv;
      T lq[RPL];
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const int i = lane + 32 * q;
        const bool below = (i > J) && (i < np);
        const T l = below ? pr[q][J] * dinv : T(0);
        if (below) {
          pr[q][J] = l;
#pragma unroll
          for (int c = 0; c < NR; ++c) rh[q][c] -= l * yj[c];
        }
        if (q == 0 && i == J) {
          pr[0][J] = dinv;  // the factor blocks keep 1 / L_jj
#pragma unroll
          for (int c = 0; c < NR; ++c) rh[0][c] = yj[c];
        }
        lq[q] = l;
      }
      if (J + 1 < kNB) {
        T* lbj = lb + (J & 1) * kNB;  // alternate buffers: one sync per step
        if (lane < kNB) lbj[lane] = lq[0];
        __syncwarp();
        T Lv[kNB];
#pragma unroll
        for (int v = 0; v < kNB / 4; ++v) {
          if (4 * v + 3 > J) {
            if constexpr (sizeof(T) == 4) {
              const float4 f = reinterpret_cast<const float4*>(lbj)[v];
              Lv[4 * v] = f.x; Lv[4 * v + 1] = f.y; Lv[4 * v + 2] = f.z; Lv[4 * v + 3] = f.w;
            } else {
              const double2 f0 = reinterpret_cast<const double2*>(lbj)[2 * v];
              const double2 f1 = reinterpret_cast<const double2*>(lbj)[2 * v + 1];
              Lv[4 * v] = f0.x; Lv[4 * v + 1] = f0.y; Lv[4 * v + 2] = f1.x; Lv[4 * v + 3] = f1.y;
            }
          } else {
            Lv[4 * v] = Lv[4 * v + 1] = Lv[4 * v + 2] = Lv[4 * v + 3] = T(0);
          }
        }
#pragma unroll
        for (int p = J + 1; p < kNB; ++p) {
#pragma unroll
          for (int q = 0; q < RPL; ++q) pr[q][p] -= lq[q] * Lv[p];
        }
      }
    }
    panel_col<J + 1, T, NR, RPL>(pr, rh, lb, lane, nb, np, K, fail);
  }
}

// Columns J and J + 1 of a full panel (nb = NB) in one step: the 2 x 2
// diagonal block is factorised from three shuffled entries, both columns of
// multipliers are formed per row, and one broadcast of the two columns
// feeds the rank-2 update of the remaining columns.
template <int J, typename T, int NR, int RPL>
__device__ __forceinline__ void panel_pair(T (&pr)[RPL][kNB], T (&rh)[RPL][NR], T* lb, int lane, int K,
                                           int& fail) {
  if constexpr (J + 1 < kNB) {
    constexpr int J1 = J + 1;
    const T a00 = __shfl_sync(0xffffffffu, pr[0][J], J);
    const T a10 = __shfl_sync(0xffffffffu, pr[0][J], J1);
    const T a11 = __shfl_sync(0xffffffffu, pr[0][J1], J1);
    if (!(a00 > T(0)) && fail < 0) fail = K + J;
    T d0, i0;
    pivot_of(a00 > T(0) ? a00 : T(1), d0, i0);
    const T l10 = a10 * i0;
    const T s11 = a11 - l10 * l10;
    if (!(s11 > T(0)) && fail < 0) fail = K + J1;
    T d1, i1;
    pivot_of(s11 > T(0) ? s11 : T(1), d1, i1);
    T y0[NR], y1[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      y0[c] = __shfl_sync(0xffffffffu, rh[0][c], J) * i0;
      y1[c] = (__shfl_sync(0xffffffffu, rh[0][c], J1) - l10 * y0[c]) * i1;
    }
    T l0q[RPL], l1q[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      // rows at or above J hold no multiplier; rows past the panel are zero
      const bool b0 = q > 0 || lane > J, b1 = q > 0 || lane > J1;
      const T l0 = b0 ? pr[q][J] * i0 : T(0);
      const T l1 = b1 ? (pr[q][J1] - l0 * l10) * i1 : T(0);
#pragma unroll
      for (int c = 0; c < NR; ++c) rh[q][c] -= l0 * y0[c] + l1 * y1[c];
      pr[q][J] = l0;
      pr[q][J1] = l1;
      if (q == 0) {
        if (lane == J) {
          pr[0][J] = i0;  // the factor blocks keep 1 / L_jj
#pragma unroll
          for (int c = 0; c < NR; ++c) rh[0][c] = y0[c];
        }
        if (lane == J1) {
          pr[0][J1] = i1;
#pragma unroll
          for (int c = 0; c < NR; ++c) rh[0][c] = y1[c];
        }
      }
      l0q[q] = l0;
      l1q[q] = l1;
    }
    if (J1 + 1 < kNB) {
      T* lbj = lb + ((J >> 1) & 1) * (2 * kNB);  // alternate buffers: one sync per step
      if (lane < kNB) {
        lbj[lane] = l0q[0];
        lbj[kNB + lane] = l1q[0];
      }
      __syncwarp();
      T L0[kNB], L1[kNB];
#pragma unroll
      for (int v = 0; v < kNB / 4; ++v) {
        if (4 * v + 3 > J1) {
          if constexpr (sizeof(T) == 4) {
            const float4 f = reinterpret_cast<const float4*>(lbj)[v];
            const float4 g = reinterpret_cast<const float4*>(lbj + kNB)[v];
            L0[4 * v] = f.x; L0[4 * v + 1] = f.y; L0[4 * v + 2] = f.z; L0[4 * v + 3] = f.w;
            L1[4 * v] = g.x; L1[4 * v + 1] = g.y; L1[4 * v + 2] = g.z; L1[4 * v + 3] = g.w;
          } else {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const double2 f = reinterpret_cast<const double2*>(lbj)[2 * v + h];
              const double2 g = reinterpret_cast<const double2*>(lbj + kNB)[2 * v + h];
              L0[4 * v + 2 * h] = f.x; L0[4 * v + 2 * h + 1] = f.y;
              L1[4 * v + 2 * h] = g.x; L1[4 * v + 2 * h + 1] = g.y;
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) L0[4 * v + k] = L1[4 * v + k] = T(0);
        }
      }
#pragma unroll
      for (int p = J1 + 1; p < kNB; ++p) {
#pragma unroll
        for (int q = 0; q < RPL; ++q) pr[q][p] -= l0q[q] * L0[p] + l1q[q] * L1[p];
      }
    }
    panel_pair<J + 2, T, NR, RPL>(pr, rh, lb, lane, K, fail);
  }
}

// Factorise (and forward-substitute NR rhs).  Lg: blocks of (NB+bmax) x NB;
// yg[k*NR + c] receives the forward solution.  Returns -1 or the first
// failing pivot index (warp-uniform).
template <typename T, int NR, int RPL, class Gen, typename TS>
__device__ int blk_factor(const Gen& gen, int n, int b, int bmax, const BlkSmem<T>& s,
                          T* __restrict__ Lg, TS* __restrict__ yg, int lane) {
  const int LBS = (kNB + bmax) * kNB;
  const int msk = s.RW - 1;
  const int blk16 = kNB * s.PW * (int)sizeof(T) / 16;  // 16-byte chunks of NB ring rows
  blk_zero16(s.wnd, s.RW / kNB * blk16, lane);
  __syncwarp();
  // first window: rows [0, min(n, NB + b)), generated directly
  int filled = min(n, kNB + b);
  for (int r0 = 0; r0 < filled; r0 += 32) {
    typename Gen::Raw raw;
    if (r0 + lane < filled) gen.load(r0 + lane, raw);
    blk_fill_raw<T, NR>(gen, s, r0, min(filled, r0 + 32), b, lane, raw);
    __syncwarp();
  }
  // rows of the next fill: their coefficient values are copied one block
  // ahead into shared memory by asynchronous copies
  if (filled + lane < min(n, filled + kNB)) gen.prefetch(filled + lane, s.raw + 4 * lane);
  cp_async_commit();
  for (int K = 0, kb = 0; K < n; K += kNB, ++kb) {
    const int nb = min(kNB, n - K);
    const int np = min(nb + b, n - K);
    const int need = min(n, K + kNB + b);
    if (filled < need) {
      cp_async_wait<0>();
      __syncwarp();
      typename Gen::Raw pf;
      if (lane < kNB) gen.from_smem(s.raw + 4 * lane, pf);
      blk_fill_raw<T, NR>(gen, s, filled, need, b, lane, pf);
      filled = need;
      __syncwarp();
      if (filled + lane < min(n, filled + kNB)) gen.prefetch(filled + lane, s.raw + 4 * lane);
      cp_async_commit();
    }
    __syncwarp();
    // ---- 1. panel factorisation in registers
    T pr[RPL][kNB];
    T rh[RPL][NR];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int i = lane + 32 * q;
      const T* row = s.wnd + ((K + i) & msk) * s.PW;
      const bool in = i < np;
#pragma unroll
      for (int p = 0; p < kNB; ++p) {
        const int d = i - p;
        pr[q][p] = (in && p < nb && d >= 0 && d <= b) ? row[d] : T(0);
      }
#pragma unroll
      for (int c = 0; c < NR; ++c) rh[q][c] = in ? s.rhs[((K + i) & msk) * 4 + c] : T(0);
    }
    int fail = -1;
    if (nb == kNB)
      panel_pair<0, T, NR, RPL>(pr, rh, s.lb, lane, K, fail);
    else
      panel_col<0, T, NR, RPL>(pr, rh, s.lb, lane, nb, np, K, fail);
    if (fail >= 0) return fail;
    // ---- write the factor block, forward solution, trailing rhs and panel;
    // rows K..K+NB-1 are retired, and their ring slots (contiguous: RW is a
    // multiple of NB) hold no live row until the next fill
    T* Lb = Lg + (size_t)kb * LBS;
    T* pt = s.wnd + (K & msk) * s.PW;
    __syncwarp();
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int i = lane + 32 * q;
      if (i < np) {
        T* dst = Lb + i * kNB;
        if constexpr (sizeof(T) == 4) {
#pragma unroll
          for (int v = 0; v < kNB / 4; ++v)
            reinterpret_cast<float4*>(dst)[v] =
                make_float4(4 * v <= i ? pr[q][4 * v] : 0.f, 4 * v + 1 <= i ? pr[q][4 * v + 1] : 0.f,
                            4 * v + 2 <= i ? pr[q][4 * v + 2] : 0.f,
                            4 * v + 3 <= i ? pr[q][4 * v + 3] : 0.f);
        } else {
#pragma unroll
          for (int v = 0; v < kNB / 2; ++v)
            reinterpret_cast<double2*>(dst)[v] = make_double2(
                2 * v <= i ? pr[q][2 * v] : 0.0, 2 * v + 1 <= i ? pr[q][2 * v + 1] : 0.0);
        }
        if (i < nb) {
#pragma unroll
          for (int c = 0; c < NR; ++c) yg[(size_t)(K + i) * NR + c] = (TS)rh[q][c];
        } else {
          const int slot = (K + i) & msk;
#pragma unroll
          for (int c = 0; c < NR; ++c) s.rhs[slot * 4 + c] = rh[q][c];
#pragma unroll
          for (int p = 0; p < kNB; ++p) pt[p * s.RP + (i - nb)] = pr[q][p];
        }
      }
    }
    __syncwarp();
    // ---- 2. trailing update A22 -= L21 L21^T with 4x4 register tiles
    const int nt = np - nb;
    if (nt > 0) {
      const int T4 = (nt + 3) >> 2;
      const int ntiles = T4 * (T4 + 1) / 2;
      for (int t = lane; t < ntiles; t += 32) {
        int ti = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
        if ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
        if (ti * (ti + 1) / 2 > t) --ti;
        const int tj = t - ti * (ti + 1) / 2;
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][c] = T(0);
        // L[K+nb+ia][K+p] vanishes for nb + ia - p > b: rows of this tile
        // need p >= nb + 4 ti - b only
        const int p0 = max(0, nb + 4 * ti - b);
        const T* col = pt + p0 * s.RP;
#pragma unroll 4
        for (int p = p0; p < nb; ++p, col += s.RP) {
          T va[4], vc[4];
          if constexpr (sizeof(T) == 4) {
            const float4 A4 = *reinterpret_cast<const float4*>(col + 4 * ti);
            const float4 C4 = *reinterpret_cast<const float4*>(col + 4 * tj);
            va[0] = A4.x; va[1] = A4.y; va[2] = A4.z; va[3] = A4.w;
            vc[0] = C4.x; vc[1] = C4.y; vc[2] = C4.z; vc[3] = C4.w;
          } else {
            const double2 A0 = *reinterpret_cast<const double2*>(col + 4 * ti);
            const double2 A1 = *reinterpret_cast<const double2*>(col + 4 * ti + 2);
            const double2 C0 = *reinterpret_cast<const double2*>(col + 4 * tj);
            const double2 C1 = *reinterpret_cast<const double2*>(col + 4 * tj + 2);
            va[0] = A0.x; va[1] = A0.y; va[2] = A1.x; va[3] = A1.y;
            vc[0] = C0.x; vc[1] = C0.y; vc[2] = C1.x; vc[3] = C1.y;
          }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] += va[a] * vc[c];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int ia = 4 * ti + a;
          if (ia < nt) {
            T* wr = s.wnd + ((K + nb + ia) & msk) * s.PW + ia - 4 * tj;
#pragma unroll
            for (int c = 0; c < 4; ++c)
              if (4 * tj + c <= ia) wr[-c] -= acc[a][c];
          }
        }
      }
    }
    __syncwarp();
    // the retired rows' slots (which held the trailing panel) are cleared for
    // the rows that will occupy them
    blk_zero16(pt, blk16, lane);
    __syncwarp();
  }
  return -1;
}

// The four values of a 16-byte-aligned ring row of a shared [RW][4] array.
__device__ __forceinline__ void ld_row4(const float* p, float (&x)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
__device__ __forceinline__ void ld_row4(const double* p, double (&x)[4]) {
  const double2 v0 = reinterpret_cast<const double2*>(p)[0], v1 = reinterpret_cast<const double2*>(p)[1];
  x[0] = v0.x; x[1] = v0.y; x[2] = v1.x; x[3] = v1.y;
}

// Asynchronous copy of factor block kb into a staging buffer (one commit group).
template <typename T>
__device__ __forceinline__ void blk_stage(const T* __restrict__ Lg, int kb, int n, int b, int bmax, T* dst,
                                          int lane) {
  const int K = kb * kNB;
  const int nb = min(kNB, n - K);
  const int np = min(nb + b, n - K);
  const T* src = Lg + (size_t)kb * (kNB + bmax) * kNB;
  const int nv = np * kNB * (int)sizeof(T) / 16;
  for (int v = lane; v < nv; v += 32)
    cp_async16(reinterpret_cast<unsigned char*>(dst) + 16 * v, reinterpret_cast<const unsigned char*>(src) + 16 * v);
  cp_async_commit();
}

// Back substitution L^T x = y, in place on xg ([n][NR], y in, x out).
template <typename T, int NR, typename TS>
__device__ void blk_backward(int n, int b, int bmax, const BlkSmem<T>& s, const T* __restrict__ Lg,
                             TS* __restrict__ xg, int lane) {
  const int nbk = (n + kNB - 1) / kNB;
  const int msk = s.RW - 1;
  const int stg = (kNB + bmax) * kNB;
  T* xr = s.rhs;  // ring of solution rows
  blk_stage<T>(Lg, nbk - 1, n, b, bmax, s.tb + ((nbk - 1) & 1) * stg, lane);
  for (int kb = nbk - 1; kb >= 0; --kb) {
    const int K = kb * kNB;
    const int nb = min(kNB, n - K);
    const int np = min(nb + b, n - K);
    if (kb > 0) {
      blk_stage<T>(Lg, kb - 1, n, b, bmax, s.tb + ((kb - 1) & 1) * stg, lane);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    const T* tb = s.tb + (kb & 1) * stg;
    // the block's forward solution, loaded before the sums so that its
    // latency overlaps them
    T yin[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) yin[c] = lane < nb ? (T)xg[(size_t)(K + lane) * NR + c] : T(0);
    // column p = lane & 15: yv = y_p - sum over the rows below the block of
    // L[i][p] x_i, the rows split between the two half-warps
    T yv[NR];
    {
      T acc[NR];
#pragma unroll
      for (int c = 0; c < NR; ++c) acc[c] = T(0);
      const int p = lane & (kNB - 1);
#pragma unroll 4
      for (int i = nb + (lane >> 4); i < np; i += 2) {
        const T l = tb[i * kNB + p];
        T xi[4];
        ld_row4(xr + ((K + i) & msk) * 4, xi);
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] += l * xi[c];
      }
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 16);
        yv[c] = lane < nb ? yin[c] - acc[c] : T(0);
      }
    }
    // in-block triangular solve, column oriented: x_p = yv_p / L_pp, then
    // rows q < p subtract L[p][q] x_p; full blocks take the columns in pairs
    // (p, p-1), which shortens the dependent chain of shuffles
    if (nb == kNB) {
#pragma unroll
      for (int p = kNB - 1; p >= 1; p -= 2) {
        const T i1 = tb[p * kNB + p], i0 = tb[(p - 1) * kNB + p - 1], lpq = tb[p * kNB + p - 1];
        T x1[NR], x0[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) {
          x1[c] = __shfl_sync(0xffffffffu, yv[c], p) * i1;
          x0[c] = (__shfl_sync(0xffffffffu, yv[c], p - 1) - lpq * x1[c]) * i0;
        }
        if (lane < p - 1) {
          const T l1 = tb[p * kNB + lane], l0 = tb[(p - 1) * kNB + lane];
#pragma unroll
          for (int c = 0; c < NR; ++c) yv[c] -= l1 * x1[c] + l0 * x0[c];
        }
        if (lane == p) {
#pragma unroll
          for (int c = 0; c < NR; ++c) yv[c] = x1[c];
        }
        if (lane == p - 1) {
#pragma unroll
          for (int c = 0; c < NR; ++c) yv[c] = x0[c];
        }
      }
    } else {
#pragma unroll
      for (int p = kNB - 1; p >= 0; --p) {
        if (p < nb) {
          const T iLpp = tb[p * kNB + p];
          T xp[NR];
#pragma unroll
          for (int c = 0; c < NR; ++c) xp[c] = __shfl_sync(0xffffffffu, yv[c], p) * iLpp;
          if (lane < p) {
            const T l = tb[p * kNB + lane];
#pragma unroll
            for (int c = 0; c < NR; ++c) yv[c] -= l * xp[c];
          }
          if (lane == p) {
#pragma unroll
            for (int c = 0; c < NR; ++c) yv[c] = xp[c];
          }
        }
      }
    }
    if (lane < nb) {
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        xr[((K + lane) & msk) * 4 + c] = yv[c];
        xg[(size_t)(K + lane) * NR + c] = (TS)yv[c];
      }
    }
    __syncwarp();
  }
}

// Forward substitution with the stored factor: rg [n][NR] double holds the
// right-hand side on entry and the forward solution y on exit.
template <typename T, int NR, int RPL>
__device__ void blk_forward_stored(int n, int b, int bmax, const BlkSmem<T>& s,
                                   const T* __restrict__ Lg, double* __restrict__ rg, int lane) {
  const int msk = s.RW - 1;
  const int stg = (kNB + bmax) * kNB;
  const int nbk = (n + kNB - 1) / kNB;
  T* rr = s.rhs;  // ring of pending right-hand-side rows
  int filled = 0;
  blk_stage<T>(Lg, 0, n, b, bmax, s.tb, lane);
  for (int K = 0, kb = 0; K < n; K += kNB, ++kb) {
    const int nb = min(kNB, n - K);
    const int np = min(nb + b, n - K);
    const int need = min(n, K + kNB + b);
    for (int r = filled + lane; r < need; r += 32) {
#pragma unroll
      for (int c = 0; c < NR; ++c) rr[(r & msk) * 4 + c] = (T)rg[(size_t)r * NR + c];
    }
    filled = max(filled, need);
    if (kb + 1 < nbk) {
      blk_stage<T>(Lg, kb + 1, n, b, bmax, s.tb + ((kb + 1) & 1) * stg, lane);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    const T* tb = s.tb + (kb & 1) * stg;
    T yv[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) yv[c] = (lane < nb) ? rr[((K + lane) & msk) * 4 + c] : T(0);
#pragma unroll
    for (int p = 0; p < kNB; ++p) {
      if (p < nb) {
        const T iLpp = tb[p * kNB + p];
        T yp[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) yp[c] = __shfl_sync(0xffffffffu, yv[c], p) * iLpp;
        if (lane > p && lane < nb) {
          const T l = tb[lane * kNB + p];
#pragma unroll
          for (int c = 0; c < NR; ++c) yv[c] -= l * yp[c];
        }
        if (lane == p) {
#pragma unroll
          for (int c = 0; c < NR; ++c) yv[c] = yp[c];
        }
      }
    }
    T* yb = s.lb;  // block solution broadcast
    if (lane < nb) {
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        rg[(size_t)(K + lane) * NR + c] = (double)yv[c];
        yb[lane * NR + c] = yv[c];
      }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int i = lane + 32 * q;
      if (i >= nb && i < np) {
        T acc[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = T(0);
        for (int p = 0; p < nb; ++p) {
          const T l = tb[i * kNB + p];
#pragma unroll
          for (int c = 0; c < NR; ++c) acc[c] += l * yb[p * NR + c];
        }
        const int slot = (K + i) & msk;
#pragma unroll
        for (int c = 0; c < NR; ++c) rr[slot * 4 + c] -= acc[c];
      }
    }
    __syncwarp();
  }
}

}  // namespace stomsfem
