// Blocked banded SPD solver for 9-point-stencil matrices, one system per
// group of G lanes (G = 32: one system per warp; G = 16: two systems of the
// same shape per warp, which run in lockstep so that every warp-wide sync
// and every loop bound is shared by both halves).
//
// Right-looking banded Cholesky in column blocks of NB = G/2.  For block K
// (rows/columns [K, K+nb)) the group
//   1. factorises the tall panel [K, K+np) x [K, K+nb), np = nb + b: each
//      lane holds up to RPL panel rows in registers; full blocks take the
//      columns in pairs (the 2 x 2 diagonal block from three shuffled
//      entries, both columns of multipliers broadcast through a
//      double-buffered shared vector, one warp sync per pair); the NR
//      right-hand sides ride along, which is the forward substitution;
//   2. applies the rank-nb update to the trailing b x b window with 4 x 4
//      register tiles (128-bit shared loads of the transposed panel, which
//      is kept in the ring slots of the rows just retired; each tile row
//      read, updated and written back as one 128-bit access);
//   3. clears the retired slots and writes the next rows from values the
//      row generator copied into shared memory one block earlier.
// The matrix lives only as a window of RW >= NB + b band rows in shared
// memory (RW a multiple of NB; row r at slot r mod RW, entry A[r][r-d] at
// wnd[kWndOff + slot * PW + d]).  With PW = 3 (mod 8) and the offset of 3,
// the four entries A[r][c..c+3] of any column group c = 0 (mod 4) of the
// trailing window, and the four entries d = i-4g-3 .. i-4g of panel row i,
// sit in one aligned 16-byte group: element (r, d) lies at r (PW + 1) - (r
// - d) + const, and PW + 1 = 4 (mod 8), so rows whose slots differ by one
// start an odd number of groups apart, which also keeps eight lanes on
// eight different groups in the panel loads.  Factor blocks go to global scratch as (NB + bmax) x NB
// row-major tiles; the substitutions stream them back through two shared
// staging buffers with asynchronous copies (next block in flight while the
// current one is used).
//
// A failing pivot does not end the factorisation early (the two systems of
// a warp must stay in lockstep): it is replaced by 1, the first failing
// index is returned, and the caller discards the results.
//
// Row generator interface:
//   typename Gen::Raw                  raw per-row values,
//   gen.load(r, Raw&)                  issue the global loads of row r,
//   gen.prefetch(r, double* dst)       copy of row r's values (at most RAWD
//                                      doubles; asynchronous where possible),
//   gen.from_smem(const double* src, Raw&)
//   gen.make<T>(r, const Raw&, T e[5], T rhs[NR])
//                                      band entries A[r][r], A[r][r-1],
//                                      A[r][r-mx+1], A[r][r-mx], A[r][r-mx-1]
//                                      (0 where absent) and the rhs,
//   gen.mx                             offset of the south neighbour.
#pragma once
#include "common.cuh"

namespace stomsfem {

constexpr int kMaxNB = 16;

template <typename T>
struct BlkSmem {
  T* wnd;  // [RW][PW] band rows; the NB ring rows of the block just
           // factorised hold the trailing panel for the update,
           // p-major: pt[p*RP + (i - nb)] = L[K+i][K+p]
  T* tb;   // 2 x [NB + bmax][NB] factor block staging (aliases wnd)
  T* rhs;  // [RW][4]
  T* lb;   // 2 x 2 x [NB] broadcast of the block-row multipliers; [NB][4]
           // block solution in the stored forward substitution
  double* raw;  // [NB][RAWD] generator values of the next rows (prefetched)
  int RW, PW, RP, RAWD;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline int blk_ring_rows(int NB, int bmax) { return (NB + bmax + NB - 1) / NB * NB; }

// Row pitch: b + 1 band entries, and at least RP = bmax rounded up to 4 so
// that NB rows hold the transposed trailing panel (which starts 4 elements
// into the retired rows' span, 16-byte aligned); rounded up to 3 (mod 8),
// the layout of the aligned groups above.
__host__ __device__ inline int blk_pitch(int bmax) {
  const int rp = (bmax + 3) & ~3;
  const int pw = bmax + 1 > rp ? bmax + 1 : rp;
  return pw + ((3 - pw) & 7);
}

// Offset of slot 0's entry d = 0 in the window (elements).
constexpr int kWndOff = 3;

__host__ __device__ inline int blk_wnd_elems(int NB, int bmax) {
  const int a = kWndOff + blk_ring_rows(NB, bmax) * blk_pitch(bmax), b = 2 * (NB + bmax) * NB;
  return a > b ? a : b;
}

// Shared memory of one system, padded to 64 bytes past a multiple of 128
// (at most 112 bytes of padding): the two systems of a warp then sit 16
// banks apart, so that the same access pattern in both halves meets
// different banks.
template <typename T>
__host__ __device__ inline size_t blk_smem_bytes(int NB, int bmax, int rawd = 4) {
  const int RW = blk_ring_rows(NB, bmax);
  const size_t b = al16(sizeof(T) * blk_wnd_elems(NB, bmax)) + al16(sizeof(T) * RW * 4) +
                   al16(sizeof(T) * 4 * NB) + al16(sizeof(double) * NB * rawd);
  return b + ((64 - (b & 127)) & 127);
}

template <typename T>
__device__ inline BlkSmem<T> make_blk(unsigned char* base, int NB, int bmax, int rawd = 4) {
  BlkSmem<T> s;
  s.RAWD = rawd;
  s.RW = blk_ring_rows(NB, bmax);
  s.PW = blk_pitch(bmax);
  s.RP = (bmax + 3) & ~3;
  size_t o = 0;
  s.wnd = reinterpret_cast<T*>(base + o);
  s.tb = s.wnd;
  o += al16(sizeof(T) * blk_wnd_elems(NB, bmax));
  s.rhs = reinterpret_cast<T*>(base + o);
  o += al16(sizeof(T) * s.RW * 4);
  s.lb = reinterpret_cast<T*>(base + o);
  o += al16(sizeof(T) * 4 * NB);
  s.raw = reinterpret_cast<double*>(base + o);
  return s;
}

// Factor scratch (elements) of one system; an upper bound for every NB <= 16.
__host__ __device__ inline size_t blk_factor_elems(int n, int bmax) {
  return (size_t)((n + kMaxNB - 1) / kMaxNB) * (kMaxNB + bmax) * kMaxNB;
}

// x mod RW for 0 <= x < 2 RW.
__device__ __forceinline__ int ring(int x, int RW) { return x >= RW ? x - RW : x; }

// Reciprocal of the pivot, 1 / sqrt(a) (the factor keeps only this).
// FP32: the hardware reciprocal square root (a few ulp).  FP64: the FP32
// estimate refined by two Newton steps y <- y + y (1 - a y^2) / 2, whose
// relative error squares each step (2^-23 -> 2^-45 -> below 2^-53 before the
// final roundings): about ten FP64 operations instead of a correctly rounded
// square root and division, on a part whose FP64 pipe is narrow.  Outside
// the FP32 range the library routines are used.
__device__ __forceinline__ float pivot_rsqrt(float a) { return rsqrtf(a); }
__device__ __forceinline__ double pivot_rsqrt(double a) {
  if (!(a > 1e-30 && a < 1e30)) return 1.0 / sqrt(a);
  double y = (double)rsqrtf((float)a);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double e = fma(-a * y, y, 1.0);
    y = fma(0.5 * y, e, y);
  }
  return y;
}

template <int G, typename T>
__device__ __forceinline__ T gshfl(T v, int src) {
  return __shfl_sync(0xffffffffu, v, src, G);
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

// The four values of a 16-byte-aligned ring row of a shared [RW][4] array.
__device__ __forceinline__ void ld_row4(const float* p, float (&x)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
__device__ __forceinline__ void ld_row4(const double* p, double (&x)[4]) {
  const double2 v0 = reinterpret_cast<const double2*>(p)[0], v1 = reinterpret_cast<const double2*>(p)[1];
  x[0] = v0.x; x[1] = v0.y; x[2] = v1.x; x[3] = v1.y;
}
// Store NR <= 4 values as one 16-byte-aligned ring row (padding with zeros).
template <int NR, typename T>
__device__ __forceinline__ void st_row4(T* p, const T (&x)[NR]) {
  T v[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) v[c] = c < NR ? x[c] : T(0);
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
}

// Zero n16 consecutive 16-byte chunks of shared memory (lanes gl of G).
template <int G>
__device__ __forceinline__ void blk_zero16(void* dst, int n16, int gl) {
  float4* d = reinterpret_cast<float4*>(dst);
  for (int v = gl; v < n16; v += G) d[v] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Zero n elements from p (any element alignment): the elements before the
// first 16-byte boundary and after the last one singly, the rest in
// 16-byte chunks (lanes gl of G).
template <int G, typename T>
__device__ __forceinline__ void blk_zero_span(T* p, int n, int gl) {
  constexpr int E = 16 / (int)sizeof(T);  // elements per chunk
  const int head = min(n, (int)(((16u - ((uint32_t)__cvta_generic_to_shared(p) & 15u)) & 15u) / sizeof(T)));
  const int body = (n - head) / E;
  const int tail0 = head + body * E;
  if (gl < head) p[gl] = T(0);
  blk_zero16<G>(p + head, body, gl);
  if (gl < n - tail0) p[tail0 + gl] = T(0);
}

// Four consecutive elements at a 16-byte-aligned shared address.
__device__ __forceinline__ void ld_grp4(const float* p, float (&v)[4]) {
  const float4 f = *reinterpret_cast<const float4*>(p);
  v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
}
__device__ __forceinline__ void ld_grp4(const double* p, double (&v)[4]) {
  const double2 f0 = reinterpret_cast<const double2*>(p)[0], f1 = reinterpret_cast<const double2*>(p)[1];
  v[0] = f0.x; v[1] = f0.y; v[2] = f1.x; v[3] = f1.y;
}
__device__ __forceinline__ void st_grp4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st_grp4(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// Rows [r0, r1) of the window (at most G rows, in ring slots slot0,
// slot0 + 1, ... mod RW; row r0 + l uses lane l's raw values): the
// generator's entries and rhs.  The slots are zero on entry (the whole
// window is cleared when a factorisation starts, and each block's slots
// again once the block is retired).
template <int G, typename T, int NR, class Gen>
__device__ __forceinline__ void blk_fill_raw(const Gen& gen, const BlkSmem<T>& s, int r0, int r1, int slot0, int b,
                                             int gl, const typename Gen::Raw& raw) {
  const int mx = gen.mx;
  const int r = r0 + gl;
  if (r < r1) {
    T e[5], rh[NR];
    gen.template make<T, NR>(r, raw, e, rh);
    const int slot = ring(slot0 + gl, s.RW);
    T* row = s.wnd + kWndOff + slot * s.PW;
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
    st_row4<NR>(s.rhs + slot * 4, rh);
  }
}

// Load NB consecutive values of a shared buffer into registers (16-byte
// loads); groups wholly below index `from` are set to zero instead.
template <int NB, typename T>
__device__ __forceinline__ void ld_vec(const T* src, T (&v)[NB], int from) {
#pragma unroll
  for (int g = 0; g < NB / 4; ++g) {
    if (4 * g + 3 >= from) {
      if constexpr (sizeof(T) == 4) {
        const float4 f = reinterpret_cast<const float4*>(src)[g];
        v[4 * g] = f.x; v[4 * g + 1] = f.y; v[4 * g + 2] = f.z; v[4 * g + 3] = f.w;
      } else {
        const double2 f0 = reinterpret_cast<const double2*>(src)[2 * g];
        const double2 f1 = reinterpret_cast<const double2*>(src)[2 * g + 1];
        v[4 * g] = f0.x; v[4 * g + 1] = f0.y; v[4 * g + 2] = f1.x; v[4 * g + 3] = f1.y;
      }
    } else {
      v[4 * g] = v[4 * g + 1] = v[4 * g + 2] = v[4 * g + 3] = T(0);
    }
  }
}

// One column step j = J of the panel factorisation (partial last block),
// then the next; the recursion keeps every register-array index a
// compile-time constant.
template <int J, int G, typename T, int NR, int RPL, int NB = G / 2>
__device__ __forceinline__ void panel_col(T (&pr)[RPL][NB], T (&rh)[RPL][NR], T* lb, int gl, int nb, int np,
                                          int K, int& fail) {
  if constexpr (J < NB) {
    if (J < nb) {
      const T dj = gshfl<G>(pr[0][J], J);
      if (!(dj > T(0)) && fail < 0) fail = K + J;
      const T dinv = pivot_rsqrt(dj > T(0) ? dj : T(1));
      T yj[NR];
#pragma unroll
      for (int c = 0; c < NR; ++c) yj[c] = gshfl<G>(rh[0][c], J) * dinv;
      T lq[RPL];
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const int i = gl + G * q;
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
      if (J + 1 < NB) {
        T* lbj = lb + (J & 1) * NB;  // alternate buffers: one sync per step
        if (gl < NB) lbj[gl] = lq[0];
        __syncwarp();
        T Lv[NB];
        ld_vec<NB>(lbj, Lv, J + 1);
#pragma unroll
        for (int p = J + 1; p < NB; ++p) {
#pragma unroll
          for (int q = 0; q < RPL; ++q) pr[q][p] -= lq[q] * Lv[p];
        }
      }
    }
    panel_col<J + 1, G, T, NR, RPL, NB>(pr, rh, lb, gl, nb, np, K, fail);
  }
}

// Columns J and J + 1 of a full panel (nb = NB) in one step: the 2 x 2
// diagonal block is factorised from three shuffled entries, both columns of
// multipliers are formed per row, and one broadcast of the two columns
// feeds the rank-2 update of the remaining columns.
template <int J, int G, typename T, int NR, int RPL, int NB = G / 2>
__device__ __forceinline__ void panel_pair(T (&pr)[RPL][NB], T (&rh)[RPL][NR], T* lb, int gl, int K,
                                           int& fail) {
  if constexpr (J + 1 < NB) {
    constexpr int J1 = J + 1;
    const T a00 = gshfl<G>(pr[0][J], J);
    const T a10 = gshfl<G>(pr[0][J], J1);
    const T a11 = gshfl<G>(pr[0][J1], J1);
    if (!(a00 > T(0)) && fail < 0) fail = K + J;
    const T i0 = pivot_rsqrt(a00 > T(0) ? a00 : T(1));
    const T l10 = a10 * i0;
    const T s11 = a11 - l10 * l10;
    if (!(s11 > T(0)) && fail < 0) fail = K + J1;
    const T i1 = pivot_rsqrt(s11 > T(0) ? s11 : T(1));
    T y0[NR], y1[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      y0[c] = gshfl<G>(rh[0][c], J) * i0;
      y1[c] = (gshfl<G>(rh[0][c], J1) - l10 * y0[c]) * i1;
    }
    T l0q[RPL], l1q[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      // rows at or above J hold no multiplier; rows past the panel are zero
      const bool b0 = q > 0 || gl > J, b1 = q > 0 || gl > J1;
      const T l0 = b0 ? pr[q][J] * i0 : T(0);
      const T l1 = b1 ? (pr[q][J1] - l0 * l10) * i1 : T(0);
#pragma unroll
      for (int c = 0; c < NR; ++c) rh[q][c] -= l0 * y0[c] + l1 * y1[c];
      pr[q][J] = l0;
      pr[q][J1] = l1;
      if (q == 0) {
        if (gl == J) {
          pr[0][J] = i0;  // the factor blocks keep 1 / L_jj
#pragma unroll
          for (int c = 0; c < NR; ++c) rh[0][c] = y0[c];
        }
        if (gl == J1) {
          pr[0][J1] = i1;
#pragma unroll
          for (int c = 0; c < NR; ++c) rh[0][c] = y1[c];
        }
      }
      l0q[q] = l0;
      l1q[q] = l1;
    }
    if (J1 + 1 < NB) {
      T* lbj = lb + ((J >> 1) & 1) * (2 * NB);  // alternate buffers: one sync per step
      if (gl < NB) {
        lbj[gl] = l0q[0];
        lbj[NB + gl] = l1q[0];
      }
      __syncwarp();
      T L0[NB], L1[NB];
      ld_vec<NB>(lbj, L0, J1 + 1);
      ld_vec<NB>(lbj + NB, L1, J1 + 1);
#pragma unroll
      for (int p = J1 + 1; p < NB; ++p) {
#pragma unroll
        for (int q = 0; q < RPL; ++q) pr[q][p] -= l0q[q] * L0[p] + l1q[q] * L1[p];
      }
    }
    panel_pair<J + 2, G, T, NR, RPL, NB>(pr, rh, lb, gl, K, fail);
  }
}

// Factorise (and forward-substitute NR rhs).  Lg: blocks of (NB+bmax) x NB;
// yg[k*NR + c] receives the forward solution.  Returns -1 or the first
// failing pivot index (the factorisation runs to the end either way).
// store_from: the factor blocks wholly below this row are not stored (a
// back substitution that stops there never reads them).
// FWD_ONLY (NR = 4): neither the factor nor y is stored; each lane adds,
// over the rows it finishes, y0 y0, y0 y1, y0 y2, y1 y1, y1 y2, y2 y2 and
// y3 y0, y3 y1, y3 y2 into yy[0..8] (FP64), for the caller to sum over the
// group.
template <int G, typename T, int NR, int RPL, class Gen, typename TS, bool FWD_ONLY = false>
__device__ int blk_factor(const Gen& gen, int n, int b, int bmax, const BlkSmem<T>& s, T* __restrict__ Lg,
                          TS* __restrict__ yg, int gl, double* yy = nullptr, int store_from = 0) {
  constexpr int NB = G / 2;
  const int LBS = (NB + bmax) * NB;
  const int RW = s.RW;
  blk_zero16<G>(s.wnd, (int)(al16(sizeof(T) * (size_t)(kWndOff + RW * s.PW)) / 16), gl);
  __syncwarp();
  int fail = -1;
  // first window: rows [0, min(n, NB + b)) in slots 0.. (no wrap), generated directly
  int filled = min(n, NB + b);
  for (int r0 = 0; r0 < filled; r0 += G) {
    typename Gen::Raw raw;
    if (r0 + gl < filled) gen.load(r0 + gl, raw);
    blk_fill_raw<G, T, NR>(gen, s, r0, min(filled, r0 + G), r0, b, gl, raw);
  }
  __syncwarp();
  int fslot = ring(filled, RW);  // slot of row `filled` (filled <= RW)
  // rows of the next fill: their coefficient values are copied one block
  // ahead into shared memory by asynchronous copies
  if (gl < NB && filled + gl < min(n, filled + NB)) gen.prefetch(filled + gl, s.raw + s.RAWD * gl);
  cp_async_commit();
  int kslot = 0;  // slot of row K
  for (int K = 0, kb = 0; K < n; K += NB, ++kb, kslot = ring(kslot + NB, RW)) {
    const int nb = min(NB, n - K);
    const int np = min(nb + b, n - K);
    const int need = min(n, K + NB + b);
    if (filled < need) {
      cp_async_wait<0>();
      __syncwarp();
      typename Gen::Raw pf;
      if (gl < NB) gen.from_smem(s.raw + s.RAWD * gl, pf);
      blk_fill_raw<G, T, NR>(gen, s, filled, need, fslot, b, gl, pf);
      fslot = ring(fslot + (need - filled), RW);
      filled = need;
      __syncwarp();
      if (gl < NB && filled + gl < min(n, filled + NB)) gen.prefetch(filled + gl, s.raw + s.RAWD * gl);
      cp_async_commit();
    }
    __syncwarp();
    // ---- 1. panel factorisation in registers
    T pr[RPL][NB];
    T rh[RPL][NR];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int i = gl + G * q;
      const bool in = i < np;
      const int slot = ring(kslot + (in ? i : 0), RW);
      const T* row = s.wnd + kWndOff + slot * s.PW;
      // entries d = i - p, p < NB, as NB / 4 aligned groups: group g4 holds
      // d = i - 4 g4 - 3 .. i - 4 g4 (p = 4 g4 + 3 .. 4 g4); entries outside
      // [0, b] (the neighbouring rows' ends and the gaps) are masked
#pragma unroll
      for (int g4 = 0; g4 < NB / 4; ++g4) {
        const int d0 = i - 4 * g4 - 3;
        T v[4] = {T(0), T(0), T(0), T(0)};
        if (in && d0 + 3 >= 0 && d0 <= b) ld_grp4(row + d0, v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int p = 4 * g4 + 3 - k, d = d0 + k;
          pr[q][p] = (p < nb && d >= 0 && d <= b) ? v[k] : T(0);
        }
      }
      T x4[4];
      ld_row4(s.rhs + slot * 4, x4);
#pragma unroll
      for (int c = 0; c < NR; ++c) rh[q][c] = in ? x4[c] : T(0);
    }
    if (nb == NB)
      panel_pair<0, G, T, NR, RPL>(pr, rh, s.lb, gl, K, fail);
    else
      panel_col<0, G, T, NR, RPL>(pr, rh, s.lb, gl, nb, np, K, fail);
    // ---- write the factor block, forward solution, trailing rhs and panel;
    // rows K..K+NB-1 are retired, and their ring slots (contiguous: RW is a
    // multiple of NB) hold no live row until the next fill
    T* Lb = Lg + (size_t)kb * LBS;
    // the transposed trailing panel: 16-byte aligned inside the retired
    // rows' span [kWndOff + kslot PW, kWndOff + (kslot + NB) PW)
    T* pt = s.wnd + kslot * s.PW + 4;
    const bool store_blk = K + NB > store_from;
    __syncwarp();
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int i = gl + G * q;
      if (i < np) {
        T* dst = Lb + i * NB;
        if constexpr (FWD_ONLY) {
          (void)dst;
        } else if (!store_blk) {
          (void)dst;
        } else if constexpr (sizeof(T) == 4) {
#pragma unroll
          for (int v = 0; v < NB / 4; ++v)
            reinterpret_cast<float4*>(dst)[v] =
                make_float4(4 * v <= i ? pr[q][4 * v] : 0.f, 4 * v + 1 <= i ? pr[q][4 * v + 1] : 0.f,
                            4 * v + 2 <= i ? pr[q][4 * v + 2] : 0.f,
                            4 * v + 3 <= i ? pr[q][4 * v + 3] : 0.f);
        } else {
#pragma unroll
          for (int v = 0; v < NB / 2; ++v)
            reinterpret_cast<double2*>(dst)[v] = make_double2(
                2 * v <= i ? pr[q][2 * v] : 0.0, 2 * v + 1 <= i ? pr[q][2 * v + 1] : 0.0);
        }
        if (i < nb) {
          if constexpr (FWD_ONLY) {
            static_assert(NR == 4, "forward-only factorisation carries 4 right-hand sides");
            const double y0 = rh[q][0], y1 = rh[q][1], y2 = rh[q][2], y3 = rh[q][3];
            yy[0] = fma(y0, y0, yy[0]);
            yy[1] = fma(y0, y1, yy[1]);
            yy[2] = fma(y0, y2, yy[2]);
            yy[3] = fma(y1, y1, yy[3]);
            yy[4] = fma(y1, y2, yy[4]);
            yy[5] = fma(y2, y2, yy[5]);
            yy[6] = fma(y3, y0, yy[6]);
            yy[7] = fma(y3, y1, yy[7]);
            yy[8] = fma(y3, y2, yy[8]);
          } else {
#pragma unroll
            for (int c = 0; c < NR; ++c) yg[(size_t)(K + i) * NR + c] = (TS)rh[q][c];
          }
        } else {
          st_row4<NR>(s.rhs + ring(kslot + i, RW) * 4, rh[q]);
#pragma unroll
          for (int p = 0; p < NB; ++p) pt[p * s.RP + (i - nb)] = pr[q][p];
        }
      }
    }
    __syncwarp();
    // ---- 2. trailing update A22 -= L21 L21^T with 4x4 register tiles
    const int nt = np - nb;
    if (nt > 0) {
      const int T4 = (nt + 3) >> 2;
      const int ntiles = T4 * (T4 + 1) / 2;
      const int tslot = ring(kslot + nb, RW);  // slot of row K + nb
      for (int t = gl; t < ntiles; t += G) {
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
        // row ia's columns 4 tj + 3 .. 4 tj are its entries d = ia - 4 tj - 3
        // .. ia - 4 tj: one aligned group (element k is column 4 tj + 3 - k);
        // on a diagonal tile the entries above the diagonal (d < 0: the
        // previous row's end and the gap) are written back unchanged
        const bool diag = ti == tj;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int ia = 4 * ti + a;
          if (ia < nt) {
            T* wr = s.wnd + kWndOff + ring(tslot + ia, RW) * s.PW + (ia - 4 * tj - 3);
            T v[4];
            ld_grp4(wr, v);
#pragma unroll
            for (int k = 0; k < 4; ++k)
              if (!diag || 3 - k <= a) v[k] -= acc[a][3 - k];
            st_grp4(wr, v);
          }
        }
      }
    }
    __syncwarp();
    // the retired rows' slots (which held the trailing panel) are cleared for
    // the rows that will occupy them
    blk_zero_span<G>(s.wnd + kWndOff + kslot * s.PW, NB * s.PW, gl);
    __syncwarp();
  }
  return fail;
}

// Asynchronous copy of factor block kb into a staging buffer (one commit group).
template <int G, typename T, int NB = G / 2>
__device__ __forceinline__ void blk_stage(const T* __restrict__ Lg, int kb, int n, int b, int bmax, T* dst, int gl) {
  const int K = kb * NB;
  const int nb = min(NB, n - K);
  const int np = min(nb + b, n - K);
  const T* src = Lg + (size_t)kb * (NB + bmax) * NB;
  const int nv = np * NB * (int)sizeof(T) / 16;
  for (int v = gl; v < nv; v += G)
    cp_async16(reinterpret_cast<unsigned char*>(dst) + 16 * v, reinterpret_cast<const unsigned char*>(src) + 16 * v);
  cp_async_commit();
}

// Back substitution L^T x = y, in place on xg ([n][NR], y in, x out).
// Factor blocks of NB columns (NB <= G; G / NB lane groups share the rows
// below each block).  stop_from: the substitution ends with the block that
// holds this row (the rows below it keep y).
template <int G, typename T, int NR, typename TS, int NB = G / 2>
__device__ void blk_backward(int n, int b, int bmax, const BlkSmem<T>& s, const T* __restrict__ Lg,
                             TS* __restrict__ xg, int gl, int stop_from = 0) {
  static_assert(G % NB == 0 && NB % 2 == 0, "lane groups of whole blocks");
  const int nbk = (n + NB - 1) / NB;
  const int kb_stop = min(stop_from / NB, nbk - 1);
  const int RW = s.RW;
  const int stg = (NB + bmax) * NB;
  T* xr = s.rhs;  // ring of solution rows
  blk_stage<G, T, NB>(Lg, nbk - 1, n, b, bmax, s.tb + ((nbk - 1) & 1) * stg, gl);
  int kslot = ((nbk - 1) * NB) % RW;  // slot of row K
  for (int kb = nbk - 1; kb >= kb_stop; --kb, kslot = kslot >= NB ? kslot - NB : kslot - NB + RW) {
    const int K = kb * NB;
    const int nb = min(NB, n - K);
    const int np = min(nb + b, n - K);
    if (kb > kb_stop) {
      blk_stage<G, T, NB>(Lg, kb - 1, n, b, bmax, s.tb + ((kb - 1) & 1) * stg, gl);
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
    for (int c = 0; c < NR; ++c) yin[c] = gl < nb ? (T)xg[(size_t)(K + gl) * NR + c] : T(0);
    // column p = gl mod NB: yv = y_p - sum over the rows below the block of
    // L[i][p] x_i, the rows split between the G / NB lane groups
    T yv[NR];
    {
      T acc[NR];
#pragma unroll
      for (int c = 0; c < NR; ++c) acc[c] = T(0);
      const int p = gl & (NB - 1);
#pragma unroll 4
      for (int i = nb + gl / NB; i < np; i += G / NB) {
        const T l = tb[i * NB + p];
        T xi[4];
        ld_row4(xr + ring(kslot + i, RW) * 4, xi);
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] += l * xi[c];
      }
#pragma unroll
      for (int c = 0; c < NR; ++c) {
#pragma unroll
        for (int o = NB; o < G; o <<= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o, G);
        yv[c] = gl < nb ? yin[c] - acc[c] : T(0);
      }
    }
    // in-block triangular solve, column oriented: x_p = yv_p / L_pp, then
    // rows q < p subtract L[p][q] x_p; full blocks take the columns in pairs
    // (p, p-1), which shortens the dependent chain of shuffles
    if (nb == NB) {
#pragma unroll
      for (int p = NB - 1; p >= 1; p -= 2) {
        const T i1 = tb[p * NB + p], i0 = tb[(p - 1) * NB + p - 1], lpq = tb[p * NB + p - 1];
        T x1[NR], x0[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) {
          x1[c] = gshfl<G>(yv[c], p) * i1;
          x0[c] = (gshfl<G>(yv[c], p - 1) - lpq * x1[c]) * i0;
        }
        if (gl < p - 1) {
          const T l1 = tb[p * NB + gl], l0 = tb[(p - 1) * NB + gl];
#pragma unroll
          for (int c = 0; c < NR; ++c) yv[c] -= l1 * x1[c] + l0 * x0[c];
        }
        if (gl == p) {
#pragma unroll
          for (int c = 0; c < NR; ++c) yv[c] = x1[c];
        }
        if (gl == p - 1) {
#pragma unroll
          for (int c = 0; c < NR; ++c) yv[c] = x0[c];
        }
      }
    } else {
#pragma unroll
      for (int p = NB - 1; p >= 0; --p) {
        if (p < nb) {
          const T iLpp = tb[p * NB + p];
          T xp[NR];
#pragma unroll
          for (int c = 0; c < NR; ++c) xp[c] = gshfl<G>(yv[c], p) * iLpp;
          if (gl < p) {
            const T l = tb[p * NB + gl];
#pragma unroll
            for (int c = 0; c < NR; ++c) yv[c] -= l * xp[c];
          }
          if (gl == p) {
#pragma unroll
            for (int c = 0; c < NR; ++c) yv[c] = xp[c];
          }
        }
      }
    }
    if (gl < nb) {
      st_row4<NR>(xr + ring(kslot + gl, RW) * 4, yv);
#pragma unroll
      for (int c = 0; c < NR; ++c) xg[(size_t)(K + gl) * NR + c] = (TS)yv[c];
    }
    __syncwarp();
  }
}

// Forward substitution with the stored factor: rg [n][NR] double holds the
// right-hand side on entry and the forward solution y on exit.
template <int G, typename T, int NR, int RPL, int NB = G / 2>
__device__ void blk_forward_stored(int n, int b, int bmax, const BlkSmem<T>& s, const T* __restrict__ Lg,
                                   double* __restrict__ rg, int gl) {
  const int RW = s.RW;
  const int stg = (NB + bmax) * NB;
  const int nbk = (n + NB - 1) / NB;
  T* rr = s.rhs;  // ring of pending right-hand-side rows
  int filled = 0;
  blk_stage<G, T, NB>(Lg, 0, n, b, bmax, s.tb, gl);
  int kslot = 0;
  for (int K = 0, kb = 0; K < n; K += NB, ++kb, kslot = ring(kslot + NB, RW)) {
    const int nb = min(NB, n - K);
    const int np = min(nb + b, n - K);
    const int need = min(n, K + NB + b);
    // rows [filled, need) lie within NB + b of row K: slot = kslot + (r - K)
    for (int r = filled + gl; r < need; r += G) {
      T v[NR];
#pragma unroll
      for (int c = 0; c < NR; ++c) v[c] = (T)rg[(size_t)r * NR + c];
      st_row4<NR>(rr + ring(kslot + (r - K), RW) * 4, v);
    }
    filled = max(filled, need);
    if (kb + 1 < nbk) {
      blk_stage<G, T, NB>(Lg, kb + 1, n, b, bmax, s.tb + ((kb + 1) & 1) * stg, gl);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    const T* tb = s.tb + (kb & 1) * stg;
    T yv[NR];
    {
      T x4[4];
      ld_row4(rr + ring(kslot + (gl < nb ? gl : 0), RW) * 4, x4);
#pragma unroll
      for (int c = 0; c < NR; ++c) yv[c] = (gl < nb) ? x4[c] : T(0);
    }
#pragma unroll
    for (int p = 0; p < NB; ++p) {
      if (p < nb) {
        const T iLpp = tb[p * NB + p];
        T yp[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) yp[c] = gshfl<G>(yv[c], p) * iLpp;
        if (gl > p && gl < nb) {
          const T l = tb[gl * NB + p];
#pragma unroll
          for (int c = 0; c < NR; ++c) yv[c] -= l * yp[c];
        }
        if (gl == p) {
#pragma unroll
          for (int c = 0; c < NR; ++c) yv[c] = yp[c];
        }
      }
    }
    T* yb = s.lb;  // block solution broadcast
    if (gl < nb) {
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        rg[(size_t)(K + gl) * NR + c] = (double)yv[c];
        yb[gl * NR + c] = yv[c];
      }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int i = gl + G * q;
      if (i >= nb && i < np) {
        T acc[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = T(0);
        for (int p = 0; p < nb; ++p) {
          const T l = tb[i * NB + p];
#pragma unroll
          for (int c = 0; c < NR; ++c) acc[c] += l * yb[p * NR + c];
        }
        T* row = rr + ring(kslot + i, RW) * 4;
        T x4[4];
        ld_row4(row, x4);
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = x4[c] - acc[c];
        st_row4<NR>(row, acc);
      }
    }
    __syncwarp();
  }
}

// Out-of-line copies of the substitutions, for a kernel that runs them
// several times (the factor-and-refine form: its first back substitution
// and each refinement sweep's forward and backward solves share one copy
// each instead of three inlined passes, whose code outgrew the instruction
// cache).
template <int G, typename T, int NR, typename TS, int NB = G / 2>
__device__ __noinline__ void blk_backward_outlined(int n, int b, int bmax, const BlkSmem<T> s,
                                                   const T* __restrict__ Lg, TS* __restrict__ xg, int gl,
                                                   int stop_from) {
  blk_backward<G, T, NR, TS, NB>(n, b, bmax, s, Lg, xg, gl, stop_from);
}
template <int G, typename T, int NR, int RPL, int NB = G / 2>
__device__ __noinline__ void blk_forward_stored_outlined(int n, int b, int bmax, const BlkSmem<T> s,
                                                         const T* __restrict__ Lg, double* __restrict__ rg,
                                                         int gl) {
  blk_forward_stored<G, T, NR, RPL, NB>(n, b, bmax, s, Lg, rg, gl);
}

}  // namespace stomsfem
