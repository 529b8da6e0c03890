// Warp-level banded SPD solver for 9-point-stencil systems.
//
// One warp owns one system A x = rhs (n unknowns, half bandwidth b, NR
// right-hand sides).  The right-looking banded Cholesky keeps only the
// active (b+1) x (b+1) window of the matrix in shared memory as a ring of
// rows: row r lives in slot r % R and its column c in slot c % R, R = b+1.
// After pivot k is eliminated, row k's slot is refilled with row k+b+1,
// which no earlier pivot has touched, straight from the row generator.
// Finalised factor columns L[k..k+b][k] stream to global scratch (one
// coalesced store per column) for the back substitution; the forward
// substitution runs inside the factorisation sweep, so the right-hand
// sides also live in a ring.
//
// Lane t-1 (and t-33, ...) owns row k+t of the window during step k; the
// multipliers of the pivot column are broadcast through shared memory.
#pragma once
#include "common.cuh"

namespace stomsfem {

template <typename T, int NR>
struct BandRing {
  T* w;    // [R][P] window
  T* rhs;  // [R][NR]
  T* lv;   // [R] multipliers of the current pivot column (index t = 1..b)
  int R, P;
};

// Shared-memory bytes of one ring (16-byte aligned pieces).  A ring built
// for half bandwidth bmax serves any system with b <= bmax (R = bmax + 1 >=
// b + 1 keeps the window rows and a row's columns in distinct slots).
template <typename T, int NR>
__host__ __device__ inline size_t ring_bytes(int b) {
  const int R = b + 1, P = R | 1;
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  return al(sizeof(T) * R * P) + al(sizeof(T) * R * NR) + al(sizeof(T) * (R + 1));
}

template <typename T, int NR>
__device__ inline BandRing<T, NR> make_ring(unsigned char* base, int b) {
  BandRing<T, NR> g;
  g.R = b + 1;
  g.P = g.R | 1;
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  g.w = reinterpret_cast<T*>(base);
  g.rhs = reinterpret_cast<T*>(base + al(sizeof(T) * g.R * g.P));
  g.lv = reinterpret_cast<T*>(base + al(sizeof(T) * g.R * g.P) + al(sizeof(T) * g.R * NR));
  return g;
}

// Warp-cooperative fill of row r (slot r % R): entries A[r][r-d], d = 0..b,
// and the NR right-hand-side values.
template <typename T, int NR, class Gen>
__device__ __forceinline__ void ring_fill_row(const Gen& gen, const BandRing<T, NR>& g, int r, int b,
                                              int lane) {
  const int rs = r % g.R;
  T* row = g.w + rs * g.P;
  for (int d = lane; d <= b; d += 32) {
    const int slot = (rs - d + g.R) % g.R;
    row[slot] = (r - d >= 0) ? gen.template coef<T>(r, d) : T(0);
  }
  if (lane < NR) g.rhs[rs * NR + lane] = gen.template rhs<T>(r, lane);
}

// Factorise and forward-substitute.  L column k goes to Lg[k*(b+1) + t]
// (t = 0 is the diagonal); the forward solution y_k to yg[k*NR + j].
// Returns -1 on success, else the first pivot index whose value was not
// positive (warp-uniform).
template <typename T, int NR, class Gen>
__device__ int band_factor_forward(const Gen& gen, int n, int b, const BandRing<T, NR>& g,
                                   T* __restrict__ Lg, double* __restrict__ yg, int lane) {
  const int R = g.R, P = g.P;
  const int r0 = (b < n - 1) ? b : n - 1;
  for (int r = 0; r <= r0; ++r) ring_fill_row<T, NR>(gen, g, r, b, lane);
  __syncwarp();
  int kr = 0;
  for (int k = 0; k < n; ++k) {
    const T akk = g.w[kr * P + kr];
    if (!(akk > T(0))) return k;
    const T d = sqrt(akk);
    const T dinv = T(1) / d;
    for (int t = lane + 1; t <= b; t += 32) {
      T l = T(0);
      if (k + t < n) {
        int rs = kr + t;
        if (rs >= R) rs -= R;
        l = g.w[rs * P + kr] * dinv;
      }
      g.lv[t] = l;
      Lg[(size_t)k * (b + 1) + t] = l;
    }
    if (lane == 0) Lg[(size_t)k * (b + 1)] = d;
    T y[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) y[j] = g.rhs[kr * NR + j] * dinv;
    if (lane < NR) {
#pragma unroll
      for (int j = 0; j < NR; ++j)
        if (j == lane) yg[(size_t)k * NR + j] = (double)y[j];
    }
    __syncwarp();
    for (int t = lane + 1; t <= b; t += 32) {
      if (k + t >= n) break;
      int rs = kr + t;
      if (rs >= R) rs -= R;
      const T lt = g.lv[t];
#pragma unroll
      for (int j = 0; j < NR; ++j) g.rhs[rs * NR + j] -= lt * y[j];
      T* row = g.w + rs * P;
      int c = kr;
      for (int s = 1; s <= t; ++s) {
        c = wrap_inc(c, R);
        row[c] -= lt * g.lv[s];
      }
    }
    __syncwarp();
    if (k + b + 1 < n) {
      ring_fill_row<T, NR>(gen, g, k + b + 1, b, lane);
      __syncwarp();
    }
    kr = wrap_inc(kr, R);
  }
  return -1;
}

// Forward substitution with a stored factor: the right-hand side rows come
// from the generator as they enter the ring (only g.rhs is used).
template <typename T, int NR, class Gen>
__device__ void band_forward_stored(const Gen& gen, int n, int b, const BandRing<T, NR>& g,
                                    const T* __restrict__ Lg, double* __restrict__ yg, int lane) {
  const int R = g.R;
  const int r0 = (b < n - 1) ? b : n - 1;
  for (int r = lane; r <= r0; r += 32) {
#pragma unroll
    for (int j = 0; j < NR; ++j) g.rhs[(r % R) * NR + j] = gen.template rhs<T>(r, j);
  }
  __syncwarp();
  int kr = 0;
  for (int k = 0; k < n; ++k) {
    const T dinv = T(1) / Lg[(size_t)k * (b + 1)];
    T y[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) y[j] = g.rhs[kr * NR + j] * dinv;
    if (lane < NR) {
#pragma unroll
      for (int j = 0; j < NR; ++j)
        if (j == lane) yg[(size_t)k * NR + j] = (double)y[j];
    }
    __syncwarp();
    for (int t = lane + 1; t <= b; t += 32) {
      if (k + t >= n) break;
      int rs = kr + t;
      if (rs >= R) rs -= R;
      const T lt = Lg[(size_t)k * (b + 1) + t];
#pragma unroll
      for (int j = 0; j < NR; ++j) g.rhs[rs * NR + j] -= lt * y[j];
    }
    __syncwarp();
    if (k + b + 1 < n) {
      const int rs = (k + b + 1) % R;
      if (lane < NR) {
#pragma unroll
        for (int j = 0; j < NR; ++j)
          if (j == lane) g.rhs[rs * NR + j] = gen.template rhs<T>(k + b + 1, j);
      }
      __syncwarp();
    }
    kr = wrap_inc(kr, R);
  }
}

// Back substitution L^T x = y in place on xg (y in, x out), using
// xr[R][NR] (shared) as the ring of the last b solution rows.
template <typename T, int NR>
__device__ void band_backward(int n, int b, int R, const T* __restrict__ Lg,
                              double* __restrict__ xg, T* xr, int lane) {
  for (int k = n - 1; k >= 0; --k) {
    T part[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) part[j] = T(0);
    const int kr = k % R;
    for (int t = lane + 1; t <= b; t += 32) {
      if (k + t >= n) break;
      int rs = kr + t;
      if (rs >= R) rs -= R;
      const T l = Lg[(size_t)k * (b + 1) + t];
#pragma unroll
      for (int j = 0; j < NR; ++j) part[j] += l * xr[rs * NR + j];
    }
#pragma unroll
    for (int j = 0; j < NR; ++j) part[j] = warp_sum(part[j]);
    const T dk = Lg[(size_t)k * (b + 1)];
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        const T x = ((T)xg[(size_t)k * NR + j] - part[j]) / dk;
        xr[kr * NR + j] = x;
        xg[(size_t)k * NR + j] = (double)x;
      }
    }
    __syncwarp();
  }
}

}  // namespace stomsfem
