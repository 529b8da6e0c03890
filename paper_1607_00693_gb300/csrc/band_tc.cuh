// Banded Cholesky of the FP32 cell problems with the trailing update on the
// tensor cores: one system per warp, column blocks of NB = 8, half
// bandwidth b <= 40.
//
// The active part of the matrix -- rows and columns [K, K + 8 + b) of the
// band, lower triangle -- lives in registers, laid out as the accumulator
// fragments of mma.m16n8k8 (16-row tiles T0..T2 by 8-column tiles C0..C5;
// lane (g, t) holds rows 16 i + g and 16 i + g + 8, columns 8 j + 2 t and
// 8 j + 2 t + 1 of tile (i, j)).  Per block:
//   1. the panel (columns K..K+7 of every window row) is written to shared
//      memory and factorised there with one or two rows per lane (column
//      pairs, as in band_block.cuh); the right-hand sides ride along as
//      extra columns, which is the forward substitution;
//   2. the trailing update A22 -= L21 L21^T runs on the tensor cores:
//      nine 16 x 8 tiles, K = 8, with each FP32 operand split into TF32
//      parts (TERMS = 3: x = h + m + l exactly, six products accumulated
//      in FP32, the dropped ones below 2^-33 of a product; TERMS = 2:
//      x = hi + lo + O(2^-22 x), three products, about 2^-21 per product,
//      several times the FP32 rounding), without the shared-memory
//      read-modify-write of the window that the FP32 FMA update needs;
//   3. the window moves down by 8 rows and 8 columns: within each lane a
//      register renaming (row 16 i + g + 8 becomes row 16 i + g of the same
//      tile, row 16 (i+1) + g becomes row 16 i + g + 8);
//   4. the 8 rows that enter are generated from the coefficient (row
//      values prefetched one block ahead) into a small shared image of
//      their band, from which each lane picks its fragment entries.
// Entries outside the band stay exactly zero (zero operands contribute
// exactly zero), so the band structure is kept without masks.  Factor
// blocks go to global scratch in the (NB + bmax) x NB layout that
// blk_backward / blk_forward_stored (band_block.cuh, NB = 8, 32 lanes)
// read back.
#pragma once
#include "band_block.cuh"

namespace stomsfem {

constexpr int kTcNB = 8;
constexpr int kTcBMax = 40;                // largest half bandwidth held in registers
constexpr int kTcRows = kTcNB + kTcBMax;   // 48 window rows: three 16-row tiles
constexpr int kTcTiles = 12;               // stored tiles: T0 x C0..1, T1 x C0..3, T2 x C0..5
constexpr int kTcPP = 12;                  // panel buffer pitch (floats): conflict-free row loads
constexpr int kTcIP = 56;                  // image pitch (floats): conflict-free fragment loads
constexpr int kTcRW = kTcRows;             // right-hand-side ring rows (a multiple of NB)

__host__ __device__ constexpr int tc_tile(int i, int j) { return (i == 0 ? 0 : (i == 1 ? 2 : 6)) + j; }
__host__ __device__ constexpr int tc_ncol(int i) { return 2 * i + 2; }

// Shared memory of one warp (bytes, 128-byte multiple): panel [48][12],
// image [8][56], ring [48][4] (float), broadcast [32] (float), raw [8][4]
// (double).  The back substitution reuses panel + image as its two staging
// buffers of (8 + bmax) x 8 floats (3072 bytes at bmax = 40).
constexpr size_t kTcOffPn = 0;
constexpr size_t kTcOffImg = kTcOffPn + sizeof(float) * kTcRows * kTcPP;      // 2304
constexpr size_t kTcOffRhs = kTcOffImg + sizeof(float) * kTcNB * kTcIP;       // 4096
constexpr size_t kTcOffLb = kTcOffRhs + sizeof(float) * kTcRW * 4;            // 4864
constexpr size_t kTcOffRaw = kTcOffLb + sizeof(float) * 32;                   // 4992
constexpr size_t kTcSmemBytes = kTcOffRaw + sizeof(double) * kTcNB * 4;        // 5248
constexpr size_t kTcSmemWarp = (kTcSmemBytes + 127) & ~size_t(127);             // 5248
static_assert(kTcOffRhs >= 2 * sizeof(float) * kTcRows * kTcNB, "staging fits in panel + image");

struct TcSmem {
  float* pn;
  float* img;
  float* rhs;
  float* lb;
  double* raw;
};

__device__ inline TcSmem make_tc(unsigned char* base) {
  TcSmem s;
  s.pn = reinterpret_cast<float*>(base + kTcOffPn);
  s.img = reinterpret_cast<float*>(base + kTcOffImg);
  s.rhs = reinterpret_cast<float*>(base + kTcOffRhs);
  s.lb = reinterpret_cast<float*>(base + kTcOffLb);
  s.raw = reinterpret_cast<double*>(base + kTcOffRaw);
  return s;
}

// View for the substitutions of band_block.cuh: staging in panel + image,
// solution ring = the right-hand-side ring.
__device__ inline BlkSmem<float> tc_blk_view(const TcSmem& t) {
  BlkSmem<float> s;
  s.wnd = t.pn;
  s.tb = t.pn;
  s.rhs = t.rhs;
  s.lb = t.lb;
  s.raw = t.raw;
  s.RW = kTcRW;
  s.PW = 0;
  s.RP = 0;
  s.RAWD = 4;
  return s;
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// x = hi + lo + O(2^-22 |x|), both TF32
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// x as TERMS TF32 parts, each the rounded remainder of the previous ones:
// two parts leave a remainder below 2^-22 |x|, three parts represent an FP32
// value exactly (3 x 11 significant bits >= 24).
template <int TERMS>
__device__ __forceinline__ void tf32_parts(float x, uint32_t (&p)[TERMS]) {
  float r = x;
#pragma unroll
  for (int q = 0; q < TERMS; ++q) {
    p[q] = tf32_rna(r);
    r -= __uint_as_float(p[q]);
  }
}

// C -= A B with A, B given by their TF32 parts, smallest products first.
// The products go into a zero accumulator D, which is then subtracted from C
// with FP32 operations: the tensor core's own accumulation (truncating, not
// rounding to nearest) then errs relative to the update, not to the window
// entry it updates.  TERMS = 2: hi*lo, lo*hi, hi*hi (drops lo*lo and the
// parts' remainders: about 2^-21 of each product).  TERMS = 3: the six
// products whose parts' exponents sum to at most 2 (h = 0, m = 1, l = 2),
// dropping those below about 2^-33 of the product.
template <int TERMS>
__device__ __forceinline__ void tc_tile_update(float (&c)[4], const uint32_t (&a)[TERMS][4],
                                               const uint32_t (&b)[TERMS][2]) {
  float d[4] = {0.f, 0.f, 0.f, 0.f};
  if constexpr (TERMS == 2) {
    mma_tf32(d, a[1], b[0]);
    mma_tf32(d, a[0], b[1]);
    mma_tf32(d, a[0], b[0]);
  } else {
    static_assert(TERMS == 3, "two or three TF32 parts");
    mma_tf32(d, a[2], b[0]);
    mma_tf32(d, a[0], b[2]);
    mma_tf32(d, a[1], b[1]);
    mma_tf32(d, a[1], b[0]);
    mma_tf32(d, a[0], b[1]);
    mma_tf32(d, a[0], b[0]);
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) c[e] -= d[e];
}

// Rows [wr0, wr0 + 8) of the window (absolute rows r0 + q, r0 = K + wr0):
// band entries into the image, right-hand sides into the ring, then each
// lane copies the image row it holds into its fragment entries.  Lanes
// 0..7 generate (raw values in `raw`, from gen.load or the prefetch).
template <int NR, class Gen>
__device__ __forceinline__ void tc_fill(const Gen& gen, const TcSmem& s, float (&W)[kTcTiles][4], int K, int wr0,
                                        int n, int lane, const typename Gen::Raw& raw) {
  const int g = lane >> 2, t = lane & 3;
  const int mx = gen.mx;
  const int r = K + wr0 + lane;
  if (lane < kTcNB && r < n) {
    float e[5], rh[NR];
    gen.template make<float, NR>(r, raw, e, rh);
    float* row = s.img + lane * kTcIP;
    const int wr = wr0 + lane;  // window row; its band reaches back to column wr - mx - 1 >= 0
    row[wr] = e[0];
    if (r >= 1) row[wr - 1] = e[1];
    if (r >= mx - 1) row[wr - mx + 1] = e[2];
    if (r >= mx) row[wr - mx] = e[3];
    if (r >= mx + 1) row[wr - mx - 1] = e[4];
    st_row4<NR>(s.rhs + (r % kTcRW) * 4, rh);
  }
  __syncwarp();
  // the lane's rows are g + 8 k (k = 0..5); exactly one lies in [wr0, wr0 + 8)
  const int k = (wr0 + 7 - g) >> 3;  // g + 8 k in [wr0, wr0 + 8)
  const float* src = s.img + (g + 8 * k - wr0) * kTcIP + 2 * t;
#define TC_FILL_ROW(I, H)                                                        \
  {                                                                              \
    _Pragma("unroll") for (int j = 0; j < tc_ncol(I); ++j) {                     \
      const float2 v = *reinterpret_cast<const float2*>(src + 8 * j);            \
      W[tc_tile(I, j)][2 * (H)] = v.x;                                           \
      W[tc_tile(I, j)][2 * (H) + 1] = v.y;                                       \
    }                                                                            \
  }
  switch (k) {
    case 0: TC_FILL_ROW(0, 0) break;
    case 1: TC_FILL_ROW(0, 1) break;
    case 2: TC_FILL_ROW(1, 0) break;
    case 3: TC_FILL_ROW(1, 1) break;
    case 4: TC_FILL_ROW(2, 0) break;
    default: TC_FILL_ROW(2, 1) break;
  }
#undef TC_FILL_ROW
  __syncwarp();
  // clear what the generating lanes wrote
  if (lane < kTcNB && r < n) {
    float* row = s.img + lane * kTcIP;
    const int wr = wr0 + lane;
    row[wr] = 0.f;
    if (r >= 1) row[wr - 1] = 0.f;
    if (r >= mx - 1) row[wr - mx + 1] = 0.f;
    if (r >= mx) row[wr - mx] = 0.f;
    if (r >= mx + 1) row[wr - mx - 1] = 0.f;
  }
}

// Factorise (and forward-substitute NR right-hand sides).  n rows, half
// bandwidth b <= kTcBMax, bmax >= b the factor-block stride parameter; the
// generator's mx must be at least 3 (distinct stencil offsets).  Lg
// receives the factor blocks ((8 + bmax) x 8, the diagonal as 1 / L_jj),
// yg[k * NR + c] the forward solution.  FWD_ONLY (NR = 4): nothing is
// stored; lane 0..7 add the products of the forward solution's components
// into yy[0..8] as in blk_factor.  Returns -1 or the first failing pivot.
template <int NR, bool FWD_ONLY, class Gen, typename TS, int TERMS = 3>
__device__ int tc_factor(const Gen& gen, int n, int b, int bmax, const TcSmem& s, float* __restrict__ Lg,
                         TS* __restrict__ yg, int lane, double* yy = nullptr) {
  constexpr int NB = kTcNB;
  const int g = lane >> 2, t = lane & 3;
  const int LBS = (NB + bmax) * NB;
  float W[kTcTiles][4];
#pragma unroll
  for (int q = 0; q < kTcTiles; ++q) W[q][0] = W[q][1] = W[q][2] = W[q][3] = 0.f;
  // the image starts (and is kept) zero
  blk_zero16<32>(s.img, kTcNB * kTcIP / 4, lane);
  __syncwarp();
  int fail = -1;
  // first window: rows [0, min(n, 8 + b)), 8 at a time
  const int first = min(n, NB + b);
  for (int wr0 = 0; wr0 < first; wr0 += NB) {
    typename Gen::Raw raw;
    if (lane < NB && wr0 + lane < n) gen.load(wr0 + lane, raw);
    tc_fill<NR>(gen, s, W, 0, wr0, n, lane, raw);
  }
  // raw values of the rows entering after block 0
  if (lane < NB && NB + b + lane < n) gen.prefetch(NB + b + lane, s.raw + 4 * lane);
  cp_async_commit();
  for (int K = 0, kb = 0; K < n; K += NB, ++kb) {
    const int nb = min(NB, n - K);
    const int np = min(nb + b, n - K);
    __syncwarp();
    // ---- 1. panel columns (tile column 0) to shared memory
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      *reinterpret_cast<float2*>(s.pn + (16 * i + g) * kTcPP + 2 * t) = make_float2(W[tc_tile(i, 0)][0], W[tc_tile(i, 0)][1]);
      *reinterpret_cast<float2*>(s.pn + (16 * i + g + 8) * kTcPP + 2 * t) = make_float2(W[tc_tile(i, 0)][2], W[tc_tile(i, 0)][3]);
    }
    __syncwarp();
    {
      float pr[2][NB];
      float rh[2][NR];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int i = lane + 32 * q;
        const bool in = i < np;  // np <= 48
        const float* row = s.pn + (in ? i : 0) * kTcPP;
        const float4 v0 = reinterpret_cast<const float4*>(row)[0], v1 = reinterpret_cast<const float4*>(row)[1];
        const float pv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
        for (int p = 0; p < NB; ++p) pr[q][p] = (in && p < nb) ? pv[p] : 0.f;
        float x4[4];
        ld_row4(s.rhs + ((K + (in ? i : 0)) % kTcRW) * 4, x4);
#pragma unroll
        for (int c = 0; c < NR; ++c) rh[q][c] = in ? x4[c] : 0.f;
      }
      if (nb == NB)
        panel_pair<0, 32, float, NR, 2, NB>(pr, rh, s.lb, lane, K, fail);
      else
        panel_col<0, 32, float, NR, 2, NB>(pr, rh, s.lb, lane, nb, np, K, fail);
      __syncwarp();
      float* Lb = Lg + (size_t)kb * LBS;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int i = lane + 32 * q;
        if (i < np) {
          if constexpr (!FWD_ONLY) {
            float4* dst = reinterpret_cast<float4*>(Lb + i * NB);
            dst[0] = make_float4(0 <= i ? pr[q][0] : 0.f, 1 <= i ? pr[q][1] : 0.f, 2 <= i ? pr[q][2] : 0.f,
                                 3 <= i ? pr[q][3] : 0.f);
            dst[1] = make_float4(4 <= i ? pr[q][4] : 0.f, 5 <= i ? pr[q][5] : 0.f, 6 <= i ? pr[q][6] : 0.f,
                                 7 <= i ? pr[q][7] : 0.f);
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
            st_row4<NR>(s.rhs + ((K + i) % kTcRW) * 4, rh[q]);
          }
        }
        // multipliers of the rows below the diagonal block, for the update
        // (rows past np are zero)
        if (i >= NB && i < kTcRows) {
          float4* d = reinterpret_cast<float4*>(s.pn + i * kTcPP);
          d[0] = make_float4(pr[q][0], pr[q][1], pr[q][2], pr[q][3]);
          d[1] = make_float4(pr[q][4], pr[q][5], pr[q][6], pr[q][7]);
        }
      }
    }
    __syncwarp();
    // ---- 2. trailing update on the tensor cores: tiles (i, j), j >= 1
    if (np > nb) {
      // A operand of row tile i: L[16 i + m][k] (m16n8k8 layout a0 = (g, t),
      // a1 = (g + 8, t), a2 = (g, t + 4), a3 = (g + 8, t + 4)), split into
      // TF32 parts.  The B operand of column tile j, B[k][n] = L[8 j + n][k]
      // (b0 = (k = t, n = g), b1 = (t + 4, g)), is the same data: (a0, a2)
      // of row tile j / 2 for even j, (a1, a3) for odd j.
      uint32_t ap[3][TERMS][4];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float* r0 = s.pn + (16 * i + g) * kTcPP;
        const float* r1 = r0 + 8 * kTcPP;
        const float x[4] = {r0[t], r1[t], r0[t + 4], r1[t + 4]};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          uint32_t part[TERMS];
          tf32_parts<TERMS>(x[e], part);
#pragma unroll
          for (int q = 0; q < TERMS; ++q) ap[i][q][e] = part[q];
        }
      }
#pragma unroll
      for (int j = 1; j < 6; ++j) {
        uint32_t bp[TERMS][2];
#pragma unroll
        for (int q = 0; q < TERMS; ++q) {
          bp[q][0] = ap[j / 2][q][(j & 1) ? 1 : 0];
          bp[q][1] = ap[j / 2][q][(j & 1) ? 3 : 2];
        }
        // rows 0..7 of row tile 0 are the panel's own rows: their results
        // are never used (the shift discards them)
#pragma unroll
        for (int i = (j - 1) / 2; i < 3; ++i) tc_tile_update<TERMS>(W[tc_tile(i, j)], ap[i], bp);
      }
    }
    // ---- 3. the window moves down and right by 8
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int j = 0; j < tc_ncol(i); ++j) {
        float* w = W[tc_tile(i, j)];
        if (j + 1 < tc_ncol(i)) {
          w[0] = W[tc_tile(i, j + 1)][2];
          w[1] = W[tc_tile(i, j + 1)][3];
        } else {
          w[0] = w[1] = 0.f;  // above the diagonal
        }
        if (i + 1 < 3) {
          w[2] = W[tc_tile(i + 1, j + 1)][0];
          w[3] = W[tc_tile(i + 1, j + 1)][1];
        } else {
          w[2] = w[3] = 0.f;  // filled below when inside the matrix
        }
      }
    }
    // ---- 4. the rows entering the next window: K + 8 + b + 0..7
    const int Kn = K + NB;
    if (Kn < n) {
      cp_async_wait<0>();
      __syncwarp();
      typename Gen::Raw raw;
      if (lane < NB) gen.from_smem(s.raw + 4 * lane, raw);
      if (Kn + b < n) tc_fill<NR>(gen, s, W, Kn, b, n, lane, raw);
      __syncwarp();
      if (lane < NB && Kn + NB + b + lane < n) gen.prefetch(Kn + NB + b + lane, s.raw + 4 * lane);
      cp_async_commit();
    }
  }
  cp_async_wait<0>();
  __syncwarp();
  return fail;
}

}  // namespace stomsfem
