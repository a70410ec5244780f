// Global MGARD levels on the gathered block-coarse grid G (Sec. III-B hybrid
// hierarchy: L local levels, then M whole-grid levels).  Each level is a
// handful of whole-grid passes: coefficients, three restriction+solve passes
// (one per dimension, shrinking it) and the coarse correction; the inverse
// runs them backwards.  Node coordinates are physical (block offset plus the
// node's in-block coordinate), so every per-dimension operator comes from a
// host-built table.
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
  const int* f0;        // [c] first fine column of row J of I^T M_f
  const T* band;        // [5c] that row's entries f0 .. f0+4 (zero past n)
  const T* tm;          // [c] Thomas multipliers of M_c
  const T* tib;         // [c] inverse pivots
  const T* tsup;        // [c] super-diagonal
};

template <typename T>
struct GLevel {
  GDim<T> d[3];
  int64_t sym_off;  // first symbol of the level in the stream order
};

__device__ __forceinline__ bool all_coarse(const uint8_t* a, const uint8_t* b, const uint8_t* c, int i0, int i1,
                                           int i2) {
  return a[i0] && b[i1] && c[i2];
}

template <typename T>
__device__ __forceinline__ int64_t nc_rank(const GLevel<T>& L, int i0, int i1, int i2, int64_t flat) {
  const int64_t c1 = L.d[1].c, c2 = L.d[2].c;
  int64_t before = (int64_t)L.d[0].cb[i0] * c1 * c2;
  if (L.d[0].isc[i0]) {
    before += (int64_t)L.d[1].cb[i1] * c2;
    if (L.d[1].isc[i1]) before += L.d[2].cb[i2];
  }
  return flat - before;
}

// Coefficients of one global level: D = U - I(U|C) at every node (0 at
// all-coarse nodes, exactly), written to Dfull; the non-coarse ones are
// quantised (mode 0) or stored (mode 1) at their stream position.
template <typename T, int MODE>
__global__ void gl_fwd_detail(GLevel<T> L, const T* __restrict__ U, T* __restrict__ Dfull, uint16_t* sym,
                              int32_t* esc, T* coef, const T* rq_ptr, unsigned* hist, int radius, Scalars* sc) {
  __shared__ unsigned hloc[kHistWin];
  if (MODE == 0)
    for (int i = threadIdx.x; i < kHistWin; i += blockDim.x) hloc[i] = 0;
  __syncthreads();
  const int n0 = L.d[0].n, n1 = L.d[1].n, n2 = L.d[2].n;
  const int64_t total = (int64_t)n0 * n1 * n2;
  const T rq = MODE == 0 ? *rq_ptr : T(0);
  bool ovf = false;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i2 = (int)(idx % n2);
    const int64_t t = idx / n2;
    const int i1 = (int)(t % n1);
    const int i0 = (int)(t / n1);
    const int a0 = L.d[0].cidx[L.d[0].jlo[i0]], b0 = L.d[0].cidx[L.d[0].jhi[i0]];
    const int a1 = L.d[1].cidx[L.d[1].jlo[i1]], b1 = L.d[1].cidx[L.d[1].jhi[i1]];
    const int a2 = L.d[2].cidx[L.d[2].jlo[i2]], b2 = L.d[2].cidx[L.d[2].jhi[i2]];
    const T wl0 = L.d[0].wl[i0], wr0 = L.d[0].wr[i0];
    const T wl1 = L.d[1].wl[i1], wr1 = L.d[1].wr[i1];
    const T wl2 = L.d[2].wl[i2], wr2 = L.d[2].wr[i2];
    auto s = [&](int x0, int x1) {
      const T* row = U + ((int64_t)x0 * n1 + x1) * n2;
      return fma(wl2, row[a2], wr2 * row[b2]);
    };
    const T ta = fma(wl1, s(a0, a1), wr1 * s(a0, b1));
    const T tb = fma(wl1, s(b0, a1), wr1 * s(b0, b1));
    const T e = fma(wl0, ta, wr0 * tb);
    const T dv = U[idx] - e;
    Dfull[idx] = dv;
    if (!all_coarse(L.d[0].isc, L.d[1].isc, L.d[2].isc, i0, i1, i2)) {
      const int64_t pos = L.sym_off + nc_rank(L, i0, i1, i2, idx);
      if (MODE == 0) {
        const int code = quantize(dv, rq, ovf);
        const bool in = code > -radius && code < radius;
        const unsigned sv = in ? (unsigned)(code + radius) : 0u;
        sym[pos] = (uint16_t)sv;
        if (!in) esc[pos] = code;
        const int bin = (int)sv - (radius - kHistWin / 2);
        if (bin >= 0 && bin < kHistWin) atomicAdd(hloc + bin, 1u);
        else atomicAdd(hist + sv, 1u);
      } else {
        coef[pos] = dv;
      }
    }
  }
  if (MODE == 0) {
    if (ovf) atomicOr(&sc->status, ST_OVERFLOW);
    __syncthreads();
    const int lo = radius - kHistWin / 2;
    for (int i = threadIdx.x; i < kHistWin; i += blockDim.x) {
      const unsigned v = hloc[i];
      if (v && lo + i >= 0 && lo + i < 2 * radius) atomicAdd(hist + lo + i, v);
    }
  }
}

// Restriction + tridiagonal solve along dimension DIM, one thread per line.
//   DIM 2: in (n0,n1,n2) -> out (n0,n1,c2)
//   DIM 1: in (n0,n1,c2) -> out (n0,c1,c2)
//   DIM 0: in (n0,c1,c2) -> out (c0,c1,c2); FINAL = 1: out = U|C + z (forward),
//          FINAL = 2: out = out - z (inverse, out holds the coarse values)
template <typename T, int DIM, int FINAL>
__global__ void gl_restrict(GLevel<T> L, const T* __restrict__ in, T* out, const T* __restrict__ U) {
  const GDim<T>& D = L.d[DIM];
  const int n0 = L.d[0].n, n1 = L.d[1].n, n2 = L.d[2].n;
  const int c1 = L.d[1].c, c2 = L.d[2].c;
  int64_t nlines;
  if (DIM == 2) nlines = (int64_t)n0 * n1;
  else if (DIM == 1) nlines = (int64_t)n0 * c2;
  else nlines = (int64_t)c1 * c2;
  for (int64_t line = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; line < nlines;
       line += (int64_t)gridDim.x * blockDim.x) {
    int64_t ibase, istride, obase, ostride;
    int x, y;  // the two fixed indices of the line
    if (DIM == 2) {
      ibase = line * n2; istride = 1; obase = line * c2; ostride = 1; x = 0; y = 0;
    } else if (DIM == 1) {
      const int64_t i0 = line / c2, j2 = line % c2;
      ibase = i0 * n1 * c2 + j2; istride = c2; obase = i0 * (int64_t)c1 * c2 + j2; ostride = c2; x = 0; y = 0;
    } else {
      const int j1 = (int)(line / c2), j2 = (int)(line % c2);
      ibase = (int64_t)j1 * c2 + j2; istride = (int64_t)c1 * c2; obase = ibase; ostride = istride; x = j1; y = j2;
    }
    const int n = D.n, c = D.c;
    // band products r_J of the whole line first: independent loads that can
    // be in flight together
#pragma unroll 4
    for (int J = 0; J < c; ++J) {
      const int f = D.f0[J];
      T r = T(0);
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        const int col = f + m;
        if (col < n) r = fma(D.band[5 * J + m], in[ibase + col * istride], r);
      }
      out[obase + J * ostride] = r;
    }
    // forward sweep: y_J = r_J - tm_J y_{J-1}, in place
    T yprev = out[obase];
    for (int J = 1; J < c; ++J) {
      const T yv = fma(-D.tm[J], yprev, out[obase + J * ostride]);
      out[obase + J * ostride] = yv;
      yprev = yv;
    }
    // backward sweep
    T znext = T(0);
    for (int J = c - 1; J >= 0; --J) {
      const T yv = out[obase + J * ostride];
      const T z = (J == c - 1 ? yv : fma(-D.tsup[J], znext, yv)) * D.tib[J];
      znext = z;
      if (FINAL == 1) {
        const int64_t u = ((int64_t)L.d[0].cidx[J] * n1 + L.d[1].cidx[x]) * n2 + L.d[2].cidx[y];
        out[obase + J * ostride] = U[u] + z;
      } else if (FINAL == 2) {
        // inverse: the coarse values live in U (compact); out aliases nothing
        out[obase + J * ostride] = U[obase + J * ostride] - z;
      } else {
        out[obase + J * ostride] = z;
      }
    }
  }
}

// Inverse: dequantised coefficients into a full grid (0 at all-coarse nodes).
template <typename T, int MODE>
__global__ void gl_inv_dequant(GLevel<T> L, const uint16_t* __restrict__ sym, const int32_t* __restrict__ esc,
                               const T* __restrict__ coef, const double* q_ptr, int radius, T* __restrict__ Dfull) {
  const int n0 = L.d[0].n, n1 = L.d[1].n, n2 = L.d[2].n;
  const int64_t total = (int64_t)n0 * n1 * n2;
  const T q = MODE == 0 ? (T)*q_ptr : T(0);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i2 = (int)(idx % n2);
    const int64_t t = idx / n2;
    const int i1 = (int)(t % n1);
    const int i0 = (int)(t / n1);
    T v = T(0);
    if (!all_coarse(L.d[0].isc, L.d[1].isc, L.d[2].isc, i0, i1, i2)) {
      const int64_t pos = L.sym_off + nc_rank(L, i0, i1, i2, idx);
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
    const int a0 = L.d[0].jlo[i0], b0 = L.d[0].jhi[i0];
    const int a1 = L.d[1].jlo[i1], b1 = L.d[1].jhi[i1];
    const int a2 = L.d[2].jlo[i2], b2 = L.d[2].jhi[i2];
    const T wl0 = L.d[0].wl[i0], wr0 = L.d[0].wr[i0];
    const T wl1 = L.d[1].wl[i1], wr1 = L.d[1].wr[i1];
    const T wl2 = L.d[2].wl[i2], wr2 = L.d[2].wr[i2];
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
                             T* coef, const T* rq_ptr, unsigned* hist, int radius, Scalars* sc) {
  __shared__ unsigned hloc[kHistWin];
  if (MODE == 0)
    for (int i = threadIdx.x; i < kHistWin; i += blockDim.x) hloc[i] = 0;
  __syncthreads();
  const T rq = MODE == 0 ? *rq_ptr : T(0);
  bool ovf = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    if (MODE == 0) {
      const int code = quantize(U[i], rq, ovf);
      const bool in = code > -radius && code < radius;
      const unsigned sv = in ? (unsigned)(code + radius) : 0u;
      sym[sym_off + i] = (uint16_t)sv;
      if (!in) esc[sym_off + i] = code;
      const int bin = (int)sv - (radius - kHistWin / 2);
      if (bin >= 0 && bin < kHistWin) atomicAdd(hloc + bin, 1u);
      else atomicAdd(hist + sv, 1u);
    } else {
      coef[sym_off + i] = U[i];
    }
  }
  if (MODE == 0) {
    if (ovf) atomicOr(&sc->status, ST_OVERFLOW);
    __syncthreads();
    const int lo = radius - kHistWin / 2;
    for (int i = threadIdx.x; i < kHistWin; i += blockDim.x) {
      const unsigned v = hloc[i];
      if (v && lo + i >= 0 && lo + i < 2 * radius) atomicAdd(hist + lo + i, v);
    }
  }
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
