// Global MGARD levels on the gathered block-coarse grid G (Sec. III-B hybrid
// hierarchy: L local levels, then M whole-grid levels).  Each level is a
// handful of whole-grid passes: coefficients, three restriction passes (one
// per dimension, shrinking it: the band product I^T M_f and the tridiagonal
// solve with M_c of that dimension) and the coarse correction; the inverse
// runs them backwards.
// Node coordinates are physical (block offset plus the node's in-block
// coordinate), so every per-dimension operator comes from a host-built table.
#pragma once

#include "bm_common.cuh"

namespace bm {

template <typename T>
struct GDim {
  int n, c;
  const int* cidx;      // [c] fine index of coarse node J
  const int* jlo;       // [n] coarse index of the left interpolation node (= J at coarse nodes)
  const int* jhi;       // [n] right node
  const T* wl;          // [n] interpolation weights (1, 0 at coarse nodes)
  const T* wr;
  const int* cb;        // [n] number of coarse indices below i
  const uint8_t* isc;   // [n] 1 at coarse nodes
  const T* P;           // [c x n] row-major projection M_c^{-1} I^T M_f
  const int* f0;        // [c] first fine column of row J of I^T M_f
  const T* band;        // [5c] row J of I^T M_f over fine columns f0[J] .. f0[J]+4
  const T* tm;          // [c] Thomas factors of M_c: y_J = r_J - tm_J y_{J-1},
  const T* tib;         //     z_J = (y_J - tsup_J z_{J+1}) tib_J
  const T* tsup;
  const T* md;          // [n] diagonal of M_f
  const T* mo;          // [n] mo[i] = M_f(i, i+1)
  int ident;            // 1: the identity of n nodes (c = n); the tables above are not used
};

// Index tables of a dimension, the identity's computed in place.
template <typename T> __device__ __forceinline__ int g_cidx(const GDim<T>& D, int i) { return D.ident ? i : D.cidx[i]; }
template <typename T> __device__ __forceinline__ int g_jlo(const GDim<T>& D, int i) { return D.ident ? i : D.jlo[i]; }
template <typename T> __device__ __forceinline__ int g_jhi(const GDim<T>& D, int i) { return D.ident ? i : D.jhi[i]; }
template <typename T> __device__ __forceinline__ T g_wl(const GDim<T>& D, int i) { return D.ident ? T(1) : D.wl[i]; }
template <typename T> __device__ __forceinline__ T g_wr(const GDim<T>& D, int i) { return D.ident ? T(0) : D.wr[i]; }
template <typename T> __device__ __forceinline__ int g_cb(const GDim<T>& D, int i) { return D.ident ? i : D.cb[i]; }
template <typename T> __device__ __forceinline__ bool g_isc(const GDim<T>& D, int i) { return D.ident || D.isc[i]; }

template <typename T>
struct GLevel {
  GDim<T> d[3];
  int64_t sym_off;    // first symbol of the level in the stream order
  int64_t blk_extra;  // added per index of dimension 0: 0 for global levels; for the in-cache levels
                      // of the block-major grid, the symbols of a block's other levels (block-major order)
  // Blocked levels (the in-cache levels of the padded grid of a round's
  // blocks, block-diagonal operators): coefficients are stored block by
  // block, bpb symbols per block, each block's level row-major over its own
  // non-coarse nodes; be / bce: a block's extent and coarse count per
  // dimension, bnb: blocks per dimension.  bmode = 0 otherwise.
  int bmode;
  int be[3], bce[3], bnb[3];
  int64_t bpb;
};

// Block (row-major over the block grid) of a node of a blocked level.
template <typename T>
__device__ __forceinline__ int64_t blk_of(const GLevel<T>& L, int i0, int i1, int i2) {
  return ((int64_t)(i0 / L.be[0]) * L.bnb[1] + i1 / L.be[1]) * L.bnb[2] + i2 / L.be[2];
}

// Stream position of a non-coarse node of a blocked level.
template <typename T>
__device__ __forceinline__ int64_t blk_pos(const GLevel<T>& L, int i0, int i1, int i2) {
  const int b0 = i0 / L.be[0], b1 = i1 / L.be[1], b2 = i2 / L.be[2];
  const int k0 = i0 - b0 * L.be[0], k1 = i1 - b1 * L.be[1], k2 = i2 - b2 * L.be[2];
  // coarse nodes of the block before the node: from the line tables, whose
  // coarse counts run over the whole padded line
  const int64_t c0 = L.d[0].cb[i0] - (int64_t)b0 * L.bce[0];
  const int64_t c1 = L.d[1].cb[i1] - (int64_t)b1 * L.bce[1];
  const int64_t c2 = L.d[2].cb[i2] - (int64_t)b2 * L.bce[2];
  int64_t before = c0 * L.bce[1] * L.bce[2];
  if (L.d[0].isc[i0]) {
    before += c1 * L.bce[2];
    if (L.d[1].isc[i1]) before += c2;
  }
  const int64_t flat = ((int64_t)k0 * L.be[1] + k1) * L.be[2] + k2;
  const int64_t b = ((int64_t)b0 * L.bnb[1] + b1) * L.bnb[2] + b2;
  return L.sym_off + b * L.bpb + flat - before;
}

template <typename T>
__device__ __forceinline__ bool all_coarse(const GLevel<T>& L, int i0, int i1, int i2) {
  return g_isc(L.d[0], i0) && g_isc(L.d[1], i1) && g_isc(L.d[2], i2);
}

// Stream position of the coefficient at (i0, i1, i2), flat index `flat`:
// its rank among the level's non-coarse nodes (row-major) plus the level's
// offset and, per index of dimension 0, blk_extra.
template <typename T>
__device__ __forceinline__ int64_t nc_pos(const GLevel<T>& L, int i0, int i1, int i2, int64_t flat) {
  if (L.bmode) return blk_pos(L, i0, i1, i2);
  const int64_t c1 = L.d[1].c, c2 = L.d[2].c;
  int64_t before = (int64_t)g_cb(L.d[0], i0) * c1 * c2;
  if (g_isc(L.d[0], i0)) {
    before += (int64_t)g_cb(L.d[1], i1) * c2;
    if (g_isc(L.d[1], i1)) before += g_cb(L.d[2], i2);
  }
  return L.sym_off + flat - before + (int64_t)i0 * L.blk_extra;
}

// Coefficients of one global level: D = U - I(U|C) at every node (0 at
// all-coarse nodes, exactly), written to Dfull; the non-coarse ones are
// quantised (mode 0; a histogram pass counts the symbols afterwards) or stored
// (mode 1) at their stream position.  One warp
// per grid row (i0, i1): the row's interpolation sources, weights and stream
// offset are computed once, the lanes walk i2.
// With tier != null (the in-cache levels of the block-major grid), the
// quantiser width of row (i0, i1) is rq_ptr[tier[i0] * tstride] (the block's
// ROI tier); otherwise rq_ptr[0].
template <typename T, int MODE>
__global__ void __launch_bounds__(256) gl_fwd_detail(GLevel<T> L, const T* __restrict__ U, T* __restrict__ Dfull,
                                                     uint16_t* sym, int32_t* esc, T* coef, const T* rq_ptr,
                                                     int radius, Scalars* sc, const uint8_t* tier = nullptr,
                                                     int tstride = 0) {
  const GDim<T>&D0 = L.d[0], &D1 = L.d[1], &D2 = L.d[2];
  const int n1 = D1.n, n2 = D2.n;
  const int64_t rows = (int64_t)D0.n * n1, c12 = (int64_t)D1.c * D2.c;
  const unsigned dict = 2u * (unsigned)radius;
  bool ovf = false;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows; row += nwarps) {
    const int i0 = (int)(row / n1), i1 = (int)(row - (int64_t)i0 * n1);
    const T rq_row = MODE == 0 && !L.bmode ? rq_ptr[tier ? (int)tier[i0] * tstride : 0] : T(0);
    const int a0 = g_cidx(D0, g_jlo(D0, i0)), b0 = g_cidx(D0, g_jhi(D0, i0));
    const int a1 = g_cidx(D1, g_jlo(D1, i1)), b1 = g_cidx(D1, g_jhi(D1, i1));
    const T wl0 = g_wl(D0, i0), wr0 = g_wr(D0, i0), wl1 = g_wl(D1, i1), wr1 = g_wr(D1, i1);
    const T* r00 = U + ((int64_t)a0 * n1 + a1) * n2;
    const T* r01 = U + ((int64_t)a0 * n1 + b1) * n2;
    const T* r10 = U + ((int64_t)b0 * n1 + a1) * n2;
    const T* r11 = U + ((int64_t)b0 * n1 + b1) * n2;
    const bool cc01 = g_isc(D0, i0) && g_isc(D1, i1);  // the row holds all-coarse nodes
    // stream rank of the row's first node: flat index minus the all-coarse nodes before it
    int64_t before = (int64_t)g_cb(D0, i0) * c12;
    if (g_isc(D0, i0)) before += (int64_t)g_cb(D1, i1) * D2.c;
    const int64_t rbase = L.sym_off + row * n2 - before + (int64_t)i0 * L.blk_extra;
    for (int i2 = lane; i2 < n2; i2 += 32) {
      const int a2 = g_cidx(D2, g_jlo(D2, i2)), b2 = g_cidx(D2, g_jhi(D2, i2));
      const T wl2 = g_wl(D2, i2), wr2 = g_wr(D2, i2);
      const T ta = fma(wl1, fma(wl2, r00[a2], wr2 * r00[b2]), wr1 * fma(wl2, r01[a2], wr2 * r01[b2]));
      const T tb = fma(wl1, fma(wl2, r10[a2], wr2 * r10[b2]), wr1 * fma(wl2, r11[a2], wr2 * r11[b2]));
      const T e = fma(wl0, ta, wr0 * tb);
      const int64_t idx = row * n2 + i2;
      const T dv = U[idx] - e;
      Dfull[idx] = dv;
      if (cc01 && g_isc(D2, i2)) continue;  // all-coarse node: no coefficient
      int64_t pos;
      T rq = rq_row;
      if (L.bmode) {  // block-major order; the block's ROI tier
        pos = blk_pos(L, i0, i1, i2);
        if (MODE == 0) rq = rq_ptr[tier ? (int)tier[blk_of(L, i0, i1, i2)] * tstride : 0];
      } else {
        pos = rbase + i2 - (cc01 ? g_cb(D2, i2) : 0);
      }
      if (MODE == 0) {
        const int code = quantize(dv, rq, ovf);
        const unsigned u = (unsigned)(code + radius);
        const bool in = u - 1u < dict - 1u;
        const unsigned sv = in ? u : 0u;
        sym[pos] = (uint16_t)sv;
        if (!in) esc[pos] = code;
      } else {
        coef[pos] = dv;
      }
    }
  }
  if (MODE == 0 && ovf) atomicOr(&sc->status, ST_OVERFLOW);
}

// One restriction pass of a global level as a dense contraction with the
// level's projection P = M_c^{-1} I^T M_f (c x n) along dimension DIM:
//   out[b][J][col] = sum_i P[J][i] in[b][i][col]
// (the same operator as band products followed by the tridiagonal solve).
// A CTA owns 64 columns of one batch; 32 x 64 tiles of `in` (its unit-stride
// index varying fastest across threads) and 32 x 32 tiles of P are staged in
// shared memory; a thread keeps 8 outputs of each 32-row tile of J.
//   DIM 2: in (n0,n1,n2) -> out (n0,n1,c2), columns = lines (n0*n1)
//   DIM 1: in (n0,n1,c2) -> out (n0,c1,c2), batches i0, columns j2
//   DIM 0: in (n0,c1,c2) -> out (c0,c1,c2), columns (j1,j2); FINAL 1: out =
//          U|C + z (forward), FINAL 2: out = U - z (inverse, U compact)
struct ApplyShape {
  int64_t nb, ncol;
  int64_t in_b, in_i, in_c;
  int64_t out_b, out_j, out_c;
};

template <typename T>
ApplyShape apply_shape(const GLevel<T>& L, int dim) {
  const int64_t n0 = L.d[0].n, n1 = L.d[1].n, n2 = L.d[2].n, c1 = L.d[1].c, c2 = L.d[2].c;
  ApplyShape S{};
  if (dim == 2) {
    S.nb = 1; S.ncol = n0 * n1; S.in_i = 1; S.in_c = n2; S.out_j = 1; S.out_c = c2;
  } else if (dim == 1) {
    S.nb = n0; S.ncol = c2; S.in_b = n1 * c2; S.in_i = c2; S.in_c = 1; S.out_b = c1 * c2; S.out_j = c2; S.out_c = 1;
  } else {
    S.nb = 1; S.ncol = c1 * c2; S.in_i = c1 * c2; S.in_c = 1; S.out_j = c1 * c2; S.out_c = 1;
  }
  return S;
}

constexpr int kApplyCols = 64, kApplyK = 32, kApplyJ = 32;

template <typename T, int DIM, int FINAL>
__global__ void __launch_bounds__(256) gl_apply(GLevel<T> L, ApplyShape S, const T* __restrict__ in,
                                                T* __restrict__ out, const T* __restrict__ U) {
  __shared__ T s_in[kApplyK][kApplyCols + 1];
  __shared__ T s_p[kApplyJ][kApplyK + 1];
  const GDim<T>& D = L.d[DIM];
  const int n = D.n, c = D.c;
  const int64_t tiles = (S.ncol + kApplyCols - 1) / kApplyCols;
  const int64_t b = blockIdx.x / tiles;
  const int64_t col0 = (blockIdx.x - b * tiles) * kApplyCols;
  const int tid = threadIdx.x, tc = tid & (kApplyCols - 1), jg = tid >> 6;
  const T* inb = in + b * S.in_b;
  const bool unit_i = S.in_i == 1;
  for (int jt = 0; jt < c; jt += kApplyJ) {
    T acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = T(0);
    for (int i0 = 0; i0 < n; i0 += kApplyK) {
      __syncthreads();  // the previous tile has been consumed
#pragma unroll
      for (int r = 0; r < kApplyK * kApplyCols / 256; ++r) {
        const int e = tid + 256 * r;
        const int ii = unit_i ? (e & (kApplyK - 1)) : (e >> 6);
        const int cc = unit_i ? (e >> 5) : (e & (kApplyCols - 1));
        const int64_t col = col0 + cc;
        T v = T(0);
        if (i0 + ii < n && col < S.ncol) v = inb[(int64_t)(i0 + ii) * S.in_i + col * S.in_c];
        s_in[ii][cc] = v;
      }
#pragma unroll
      for (int r = 0; r < kApplyJ * kApplyK / 256; ++r) {
        const int e = tid + 256 * r, ii = e & (kApplyK - 1), jj = e >> 5;
        s_p[jj][ii] = (jt + jj < c && i0 + ii < n) ? D.P[(int64_t)(jt + jj) * n + i0 + ii] : T(0);
      }
      __syncthreads();
#pragma unroll 8
      for (int ii = 0; ii < kApplyK; ++ii) {
        const T x = s_in[ii][tc];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = fma(s_p[jg * 8 + q][ii], x, acc[q]);
      }
    }
    const int64_t col = col0 + tc;
    if (col < S.ncol) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int J = jt + jg * 8 + q;
        if (J >= c) break;
        const int64_t o = b * S.out_b + (int64_t)J * S.out_j + col * S.out_c;
        if (FINAL == 1) {
          const int c2 = L.d[2].c, j1 = (int)(col / c2), j2 = (int)(col - (int64_t)j1 * c2);
          const int64_t u = ((int64_t)L.d[0].cidx[J] * L.d[1].n + L.d[1].cidx[j1]) * L.d[2].n + L.d[2].cidx[j2];
          out[o] = U[u] + acc[q];
        } else if (FINAL == 2) {
          out[o] = U[o] - acc[q];
        } else {
          out[o] = acc[q];
        }
      }
    }
  }
}

// One restriction pass of a global level, line by line along dimension DIM:
// r = I^T M_f d (five-point band), then M_c z = r by the Thomas recurrences,
// each evaluated as a warp scan of affine maps (lane l owns the E coarse rows
// l*E .. l*E+E-1, composes their maps, combines them across the warp with
// shuffles, then replays its rows from the combined input).  The same
// operator as the dense projection in gl_apply, in O(n) work per line.
// A CTA stages kLineTile lines (one 128-byte row of columns) in shared memory,
// read coalesced along the line when it is contiguous (DIM 2) and across the
// lines otherwise; eight warps take one line at a time.  Shapes and FINAL as
// for gl_apply.  E is odd, so the lanes' rows of a segment never share a bank.
template <typename T>
constexpr int line_tile() {
  return 128 / (int)sizeof(T);
}
inline int line_segment(int c) {  // rows per lane (0: the line is too long for gl_line)
  const int e = (c + 31) / 32;
  return e <= 1 ? 1 : e <= 3 ? 3 : e <= 9 ? 9 : e <= 17 ? 17 : 0;
}
template <typename T>
size_t line_smem(int n, int c) {
  return (size_t)line_tile<T>() * (size_t)((n | 1) + (c | 1)) * sizeof(T);
}

template <typename T, int DIM, int FINAL, int E>
__global__ void __launch_bounds__(256) gl_line(GLevel<T> L, ApplyShape S, const T* __restrict__ in,
                                               T* __restrict__ out, const T* __restrict__ U) {
  constexpr int LT = line_tile<T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GDim<T>& D = L.d[DIM];
  const int n = D.n, c = D.c, sn = n | 1, sc = c | 1;
  T* s_in = reinterpret_cast<T*>(smem_raw);  // [LT][sn] the lines
  T* s_out = s_in + LT * sn;                  // [LT][sc] r, then z
  const int64_t tiles = (S.ncol + LT - 1) / LT;
  const int64_t b = blockIdx.x / tiles;
  const int64_t col0 = (blockIdx.x - b * tiles) * LT;
  const int nl = (int)(S.ncol - col0 < LT ? S.ncol - col0 : LT);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T* inb = in + b * S.in_b;
  if (S.in_i == 1) {
    for (int w = warp; w < nl; w += 8)
      for (int i = lane; i < n; i += 32) s_in[w * sn + i] = inb[(col0 + w) * S.in_c + i];
  } else {
    for (int e = threadIdx.x; e < n * LT; e += 256) {
      const int i = e / LT, w = e - i * LT;
      if (w < nl) s_in[w * sn + i] = inb[(int64_t)i * S.in_i + (col0 + w) * S.in_c];
    }
  }
  __syncthreads();
  for (int w = warp; w < nl; w += 8) {
    const T* x = s_in + w * sn;
    T* r = s_out + w * sc;
    if (c == n) {  // a dimension of at most two nodes is not coarsened
      for (int J = lane; J < c; J += 32) r[J] = x[J];
      continue;
    }
    for (int J = lane; J < c; J += 32) {
      const int f = D.f0[J];
      T v = T(0);
#pragma unroll
      for (int m = 0; m < 5; ++m)
        if (f + m < n) v = fma(D.band[5 * J + m], x[f + m], v);
      r[J] = v;
    }
    __syncwarp();
    const int j0 = lane * E;
    T y[E];
    // forward recurrence y_J = r_J - tm_J y_{J-1} (y_{-1} = 0)
    T a = T(0), m = T(1);
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int J = j0 + k;
      if (J < c) {
        const T t = D.tm[J];
        a = fma(-t, a, r[J]);
        m = -t * m;
      }
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const T pa = __shfl_up_sync(0xffffffffu, a, off), pm = __shfl_up_sync(0xffffffffu, m, off);
      if (lane >= off) {
        a = fma(m, pa, a);
        m *= pm;
      }
    }
    T prev = __shfl_up_sync(0xffffffffu, a, 1);
    if (lane == 0) prev = T(0);
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int J = j0 + k;
      if (J < c) {
        y[k] = fma(-D.tm[J], prev, r[J]);
        prev = y[k];
      }
    }
    // backward recurrence z_J = (y_J - tsup_J z_{J+1}) tib_J (z_c = 0)
    a = T(0);
    m = T(1);
#pragma unroll
    for (int k = E - 1; k >= 0; --k) {
      const int J = j0 + k;
      if (J < c) {
        const T ib = D.tib[J], q = -D.tsup[J] * ib;
        a = fma(q, a, y[k] * ib);
        m = q * m;
      }
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const T pa = __shfl_down_sync(0xffffffffu, a, off), pm = __shfl_down_sync(0xffffffffu, m, off);
      if (lane + off < 32) {
        a = fma(m, pa, a);
        m *= pm;
      }
    }
    T next = __shfl_down_sync(0xffffffffu, a, 1);
    if (lane == 31) next = T(0);
    __syncwarp();  // every lane has read its r before any z overwrites it
#pragma unroll
    for (int k = E - 1; k >= 0; --k) {
      const int J = j0 + k;
      if (J < c) {
        next = fma(-D.tsup[J], next, y[k]) * D.tib[J];
        r[J] = next;
      }
    }
  }
  __syncthreads();
  auto emit = [&](int J, int w) {
    const int64_t col = col0 + w;
    const int64_t o = b * S.out_b + (int64_t)J * S.out_j + col * S.out_c;
    const T z = s_out[w * sc + J];
    if (FINAL == 1) {
      const int c2 = L.d[2].c, j1 = (int)(col / c2), j2 = (int)(col - (int64_t)j1 * c2);
      const int64_t u = ((int64_t)L.d[0].cidx[J] * L.d[1].n + L.d[1].cidx[j1]) * L.d[2].n + L.d[2].cidx[j2];
      out[o] = U[u] + z;
    } else if (FINAL == 2) {
      out[o] = U[o] - z;
    } else {
      out[o] = z;
    }
  };
  if (S.out_j == 1) {
    for (int w = warp; w < nl; w += 8)
      for (int J = lane; J < c; J += 32) emit(J, w);
  } else {
    for (int e = threadIdx.x; e < c * LT; e += 256) {
      const int J = e / LT, w = e - J * LT;
      if (w < nl) emit(J, w);
    }
  }
}

// The restriction pass along an identity dimension 0 (the block index of
// the block-major grid): z = in, elementwise, with FINAL as for gl_apply
// (1: out = U|C + z; 2: out = U - z; 0: out = z).  in, out: (n0, c1, c2).
template <typename T, int FINAL>
__global__ void __launch_bounds__(256) gl_ident0(GLevel<T> L, const T* __restrict__ in, T* __restrict__ out,
                                                 const T* __restrict__ U) {
  const int n0 = L.d[0].n, c1 = L.d[1].c, c2 = L.d[2].c, n1 = L.d[1].n, n2 = L.d[2].n;
  const int64_t total = (int64_t)n0 * c1 * c2;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
    const T z = in[o];
    if (FINAL == 1) {
      const int j2 = (int)(o % c2);
      const int64_t t = o / c2;
      const int j1 = (int)(t % c1);
      const int i0 = (int)(t / c1);
      out[o] = U[((int64_t)i0 * n1 + g_cidx(L.d[1], j1)) * n2 + g_cidx(L.d[2], j2)] + z;
    } else if (FINAL == 2) {
      out[o] = U[o] - z;
    } else {
      out[o] = z;
    }
  }
}

// Between a grid and its blocks in block-major order: block b (row-major
// over the block grid nb) of edges e[3] (1 along dimensions of extent 1) is
// stored as a contiguous E1 x E2 tile, its axes the grid dimensions ax[0] and
// ax[1] (ax[0] = -1: E1 = 1).  DIR 0 gathers (nodes outside the grid read as
// zero), DIR 1 scatters the nodes inside the grid.
struct Reblock {
  int64_t g[3];   // grid shape
  int e[3];       // block edge per dimension
  int nb[3];      // blocks per dimension
  int ax[2];      // grid dimension of tile axis 1 and 2 (-1: none)
  int E1, E2;     // tile extents
  int64_t nblk;
};

template <typename T, int DIR>
__global__ void __launch_bounds__(256) reblock_kernel(Reblock R, T* __restrict__ grid, T* __restrict__ blocked) {
  const int64_t total = R.nblk * R.E1 * R.E2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k2 = (int)(idx % R.E2);
    const int64_t t = idx / R.E2;
    const int k1 = (int)(t % R.E1);
    const int64_t b = t / R.E1;
    const int b2 = (int)(b % R.nb[2]);
    const int64_t t2 = b / R.nb[2];
    const int b1 = (int)(t2 % R.nb[1]);
    const int b0 = (int)(t2 / R.nb[1]);
    int64_t c[3] = {(int64_t)b0 * R.e[0], (int64_t)b1 * R.e[1], (int64_t)b2 * R.e[2]};
    if (R.ax[0] >= 0) c[R.ax[0]] += k1;
    c[R.ax[1]] += k2;
    const bool in = c[0] < R.g[0] && c[1] < R.g[1] && c[2] < R.g[2];
    const int64_t gi = (c[0] * R.g[1] + c[1]) * R.g[2] + c[2];
    if (DIR == 0) blocked[idx] = in ? grid[gi] : T(0);
    else if (in) grid[gi] = blocked[idx];
  }
}

// Between a grid of shape S and its zero-padded copy of shape P (P >= S per
// dimension, the padding at the high end): DIR 0 pads (dst = padded),
// DIR 1 crops (dst = the grid).
template <typename T, int DIR>
__global__ void __launch_bounds__(256) pad_kernel(const T* __restrict__ src, T* __restrict__ dst, int64_t s0,
                                                  int64_t s1, int64_t s2, int64_t p0, int64_t p1, int64_t p2) {
  const int64_t total = DIR == 0 ? p0 * p1 * p2 : s0 * s1 * s2;
  const int64_t n1 = DIR == 0 ? p1 : s1, n2 = DIR == 0 ? p2 : s2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i2 = idx % n2, t = idx / n2, i1 = t % n1, i0 = t / n1;
    if (DIR == 0) dst[idx] = (i0 < s0 && i1 < s1 && i2 < s2) ? src[(i0 * s1 + i1) * s2 + i2] : T(0);
    else dst[idx] = src[(i0 * p1 + i1) * p2 + i2];
  }
}

// Inverse: dequantised coefficients into a full grid (0 at all-coarse nodes).
// With tier != null (the in-cache levels of the block-major grid), the
// quantiser width of the nodes with index i0 is q_ptr[tier[i0] * tstride];
// the tier byte is range-checked against ntiers (a corrupt stream flags sc).
template <typename T, int MODE>
__global__ void gl_inv_dequant(GLevel<T> L, const uint16_t* __restrict__ sym, const int32_t* __restrict__ esc,
                               const T* __restrict__ coef, const double* q_ptr, int radius, T* __restrict__ Dfull,
                               const uint8_t* tier = nullptr, int tstride = 0, int ntiers = 1, Scalars* sc = nullptr) {
  const int n0 = L.d[0].n, n1 = L.d[1].n, n2 = L.d[2].n;
  const int64_t total = (int64_t)n0 * n1 * n2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i2 = (int)(idx % n2);
    const int64_t t = idx / n2;
    const int i1 = (int)(t % n1);
    const int i0 = (int)(t / n1);
    T v = T(0);
    if (!all_coarse(L, i0, i1, i2)) {
      const int64_t pos = nc_pos(L, i0, i1, i2, idx);
      int tr = tier ? (int)tier[L.bmode ? blk_of(L, i0, i1, i2) : (int64_t)i0] : 0;
      if (tr >= ntiers) {
        if (sc) atomicOr(&sc->status, ST_CORRUPT);
        tr = 0;
      }
      const T q = MODE == 0 ? (T)q_ptr[tr * tstride] : T(0);
      if (MODE == 0) {
        const unsigned s = sym[pos];
        const int code = s ? (int)s - radius : esc[pos];
        v = dequant(code, q);
      } else {
        v = coef[pos];
      }
    }
    Dfull[idx] = v;
  }
}

// Inverse: U = I(Uc) + D in place (Dfull holds D on entry, U on exit).
template <typename T>
__global__ void gl_inv_interp(GLevel<T> L, const T* __restrict__ Uc, T* __restrict__ Dfull) {
  const int n0 = L.d[0].n, n1 = L.d[1].n, n2 = L.d[2].n;
  const int c1 = L.d[1].c, c2 = L.d[2].c;
  const int64_t total = (int64_t)n0 * n1 * n2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i2 = (int)(idx % n2);
    const int64_t t = idx / n2;
    const int i1 = (int)(t % n1);
    const int i0 = (int)(t / n1);
    const int a0 = g_jlo(L.d[0], i0), b0 = g_jhi(L.d[0], i0);
    const int a1 = g_jlo(L.d[1], i1), b1 = g_jhi(L.d[1], i1);
    const int a2 = g_jlo(L.d[2], i2), b2 = g_jhi(L.d[2], i2);
    const T wl0 = g_wl(L.d[0], i0), wr0 = g_wr(L.d[0], i0);
    const T wl1 = g_wl(L.d[1], i1), wr1 = g_wr(L.d[1], i1);
    const T wl2 = g_wl(L.d[2], i2), wr2 = g_wr(L.d[2], i2);
    auto s = [&](int x0, int x1) {
      const T* row = Uc + ((int64_t)x0 * c1 + x1) * c2;
      return fma(wl2, row[a2], wr2 * row[b2]);
    };
    const T ta = fma(wl1, s(a0, a1), wr1 * s(a0, b1));
    const T tb = fma(wl1, s(b0, a1), wr1 * s(b0, b1));
    const T e = fma(wl0, ta, wr0 * tb);
    Dfull[idx] = e + Dfull[idx];
  }
}

// Coarsest array: quantised directly (mode 0) or stored (mode 1).
template <typename T, int MODE>
__global__ void coarsest_fwd(const T* __restrict__ U, int64_t count, int64_t sym_off, uint16_t* sym, int32_t* esc,
                             T* coef, const T* rq_ptr, int radius, Scalars* sc) {
  const T rq = MODE == 0 ? *rq_ptr : T(0);
  bool ovf = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    if (MODE == 0) {
      const int code = quantize(U[i], rq, ovf);
      const bool in = code > -radius && code < radius;
      const unsigned sv = in ? (unsigned)(code + radius) : 0u;
      sym[sym_off + i] = (uint16_t)sv;
      if (!in) esc[sym_off + i] = code;
    } else {
      coef[sym_off + i] = U[i];
    }
  }
  if (MODE == 0 && ovf) atomicOr(&sc->status, ST_OVERFLOW);
}

template <typename T, int MODE>
__global__ void coarsest_inv(T* __restrict__ U, int64_t count, int64_t sym_off, const uint16_t* sym, const int32_t* esc,
                             const T* coef, const double* q_ptr, int radius) {
  const T q = MODE == 0 ? (T)*q_ptr : T(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    if (MODE == 0) {
      const unsigned s = sym[sym_off + i];
      const int code = s ? (int)s - radius : esc[sym_off + i];
      U[i] = dequant(code, q);
    } else {
      U[i] = coef[sym_off + i];
    }
  }
}

}  // namespace bm
