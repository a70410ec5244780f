// Adjoints (transposes) of the decomposition and the recomposition.
//
// One level (Sec. II-B) maps the level grid u to (D_F, c):
//   D = (Id - I R_C) u   (zero at the all-coarse nodes),   D_F = S_F D,
//   c = R_C u + P D,      P = P_0 (x) P_1 (x) P_2,  P_k = M_c^-1 I^T M_f,
// with I the tensor interpolation from the all-coarse nodes, R_C the
// injection onto them and S_F the selection of the other nodes.  Its
// transpose, given gradients (g_D, g_c), is
//   v = S_F^T g_D + P^T g_c,   P_k^T = M_f I M_c^-1   (both mass matrices are symmetric),
//   g_u = v + R_C^T (g_c - I^T v).
// The recomposition (c - P D, then I(.) + D) is the inverse of the level; the
// transpose of that inverse, given g_u, is
//   g_c = I^T g_u,   g_D = S_F (g_u - P^T g_c).
// Both are built from two line operators applied one dimension at a time:
// "expand" (M_f I M_c^-1, coarse line to fine line) and "restrict"
// (I^T, fine line to coarse line).  The In-cache Block levels run them in
// shared memory with the compile-time tables of the forward kernels; the
// global levels run them as whole-grid passes with the plan's tables.
#pragma once

#include <atomic>

#include "bm_block.cuh"
#include "bm_global.cuh"

namespace bm {

// ---------------------------------------------------------------------------
// Block levels (uniform unit spacing, N odd, C = (N+1)/2)
// ---------------------------------------------------------------------------

// out = M_f I M_c^-1 z for one line; z[J] at in[J * stride].
template <typename T, int N>
__device__ __forceinline__ void expand_line(const BlockLevel<T, N>& tb, const T* in, int stride, T (&out)[N]) {
  constexpr int C = (N + 1) / 2;
  T y[C];
  y[0] = in[0];
#pragma unroll
  for (int i = 1; i < C; ++i) y[i] = fma(-tb.tm[i], y[i - 1], in[i * stride]);
  T z[C];
  z[C - 1] = y[C - 1] * tb.tib[C - 1];
#pragma unroll
  for (int i = C - 2; i >= 0; --i) z[i] = fma(-tb.tsup[i], z[i + 1], y[i]) * tb.tib[i];
  T w[N];
#pragma unroll
  for (int k = 0; k < N; ++k) w[k] = (k & 1) ? T(0.5) * (z[k / 2] + z[k / 2 + 1]) : z[k / 2];
  // fine mass matrix of unit spacing: diagonal 2/3 (1/3 at the ends), off-diagonal 1/6
  const T third = T(1) / T(3), sixth = T(1) / T(6);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    T v = ((k == 0 || k == N - 1) ? third : T(2) * third) * w[k];
    if (k > 0) v = fma(sixth, w[k - 1], v);
    if (k < N - 1) v = fma(sixth, w[k + 1], v);
    out[k] = v;
  }
}

// r = I^T v for one line: r[J] = v[2J] + (v[2J-1] + v[2J+1]) / 2; v[k] at in[k * stride].
template <typename T, int N>
__device__ __forceinline__ void restrict_line(const T* in, int stride, T (&r)[(N + 1) / 2]) {
  constexpr int C = (N + 1) / 2;
#pragma unroll
  for (int J = 0; J < C; ++J) {
    T s = T(0);
    if (2 * J - 1 >= 0) s += in[(2 * J - 1) * stride];
    if (2 * J + 1 < N) s += in[(2 * J + 1) * stride];
    r[J] = fma(T(0.5), s, in[2 * J * stride]);
  }
}

// Expansion of a C^3 array to N^3 in shared memory: dim 0 (gc -> Y1, N C C),
// dim 1 (Y1 -> Y2, N N C); the dim-2 pass is left to the caller (`last`
// receives each (i0, i1) line's N values).
template <typename T, int N, class Last>
__device__ __forceinline__ void expand3(const T* gc, T* Y1, T* Y2, Last last) {
  constexpr int C = (N + 1) / 2;
  const auto& tb = block_tab<T, N>();
  for (int L = threadIdx.x; L < C * C; L += blockDim.x) {  // L = J1*C + J2
    T o[N];
    expand_line<T, N>(tb, gc + L, C * C, o);
#pragma unroll
    for (int i = 0; i < N; ++i) Y1[i * C * C + L] = o[i];
  }
  __syncthreads();
  for (int L = threadIdx.x; L < N * C; L += blockDim.x) {  // L = i0*C + J2
    const int i0 = L / C, j2 = L - i0 * C;
    T o[N];
    expand_line<T, N>(tb, Y1 + i0 * C * C + j2, C, o);
#pragma unroll
    for (int i = 0; i < N; ++i) Y2[(i0 * N + i) * C + j2] = o[i];
  }
  __syncthreads();
  for (int L = threadIdx.x; L < N * N; L += blockDim.x) {  // L = i0*N + i1
    T o[N];
    expand_line<T, N>(tb, Y2 + L * C, 1, o);
    last(L, o);
  }
  __syncthreads();
}

// Restriction of an N^3 array X to C^3 (out) through Y2 (N N C) and Y1 (N C C).
template <typename T, int N>
__device__ __forceinline__ void restrict3(const T* X, T* Y1, T* Y2, T* out) {
  constexpr int C = (N + 1) / 2;
  for (int L = threadIdx.x; L < N * N; L += blockDim.x) {
    T r[C];
    restrict_line<T, N>(X + L * N, 1, r);
#pragma unroll
    for (int J = 0; J < C; ++J) Y2[L * C + J] = r[J];
  }
  __syncthreads();
  for (int L = threadIdx.x; L < N * C; L += blockDim.x) {  // L = i0*C + J2
    const int i0 = L / C, j2 = L - i0 * C;
    T r[C];
    restrict_line<T, N>(Y2 + i0 * N * C + j2, C, r);
#pragma unroll
    for (int J = 0; J < C; ++J) Y1[(i0 * C + J) * C + j2] = r[J];
  }
  __syncthreads();
  for (int L = threadIdx.x; L < C * C; L += blockDim.x) {  // L = J1*C + J2
    T r[C];
    restrict_line<T, N>(Y1 + L, C * C, r);
#pragma unroll
    for (int J = 0; J < C; ++J) out[J * C * C + L] = r[J];
  }
  __syncthreads();
}

// Stream position of node k of line (i0, i1) inside its level, or -1 at an
// all-coarse node (the same order as the forward level).
template <int N>
__device__ __forceinline__ int level_pos(int L, int k) {
  constexpr int C = (N + 1) / 2;
  const int i0 = L / N, i1 = L - i0 * N;
  const bool cc = !(i0 & 1) && !(i1 & 1);
  if (cc && !(k & 1)) return -1;
  const int cc_before = ((i0 + 1) / 2) * C + ((i0 & 1) ? 0 : (i1 + 1) / 2);
  return L * N - cc_before * C + (cc ? k / 2 : k);
}

// Transposed decomposition level: gc (C^3) and the level's coefficient
// gradients (at gcoef + lvl_off) give g_u in X (N^3).  R is C^3 scratch.
template <typename T, int N>
__device__ __forceinline__ void level_adj_decompose(T* X, T* Y1, T* Y2, const T* gc, T* R, const T* gcoef,
                                                    int lvl_off) {
  constexpr int C = (N + 1) / 2;
  expand3<T, N>(gc, Y1, Y2, [&](int L, const T (&o)[N]) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int p = level_pos<N>(L, k);
      X[L * N + k] = p >= 0 ? o[k] + gcoef[lvl_off + p] : o[k];
    }
  });
  restrict3<T, N>(X, Y1, Y2, R);
  for (int e = threadIdx.x; e < C * C * C; e += blockDim.x) {
    const int j0 = e / (C * C), r = e - j0 * C * C, j1 = r / C, j2 = r - j1 * C;
    X[((2 * j0) * N + 2 * j1) * N + 2 * j2] += gc[e] - R[e];
  }
  __syncthreads();
}

// Transposed recomposition level: X (N^3, g_u) gives gc (C^3) and the
// level's coefficient gradients (written at gcoef + lvl_off).
template <typename T, int N>
__device__ __forceinline__ void level_adj_recompose(const T* X, T* Y1, T* Y2, T* gc, T* gcoef, int lvl_off) {
  restrict3<T, N>(X, Y1, Y2, gc);
  expand3<T, N>(gc, Y1, Y2, [&](int L, const T (&o)[N]) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int p = level_pos<N>(L, k);
      if (p >= 0) gcoef[lvl_off + p] = X[L * N + k] - o[k];
    }
  });
}

template <typename T, int N, int L, int B>
struct AdjDecLevels {  // levels L, L-1, ..., 0 (level L has N nodes)
  __device__ __forceinline__ static void run(const LevelBufs<T>& bufs, T* Y1, T* Y2, T* R, const T* gcoef) {
    level_adj_decompose<T, N>(bufs(L), Y1, Y2, bufs(L + 1), R, gcoef, lvl_offset(B, L));
    if constexpr (L > 0) AdjDecLevels<T, 2 * N - 1, L - 1, B>::run(bufs, Y1, Y2, R, gcoef);
  }
};

template <typename T, int N, int L, int K, int B>
struct AdjRecLevels {  // levels L, L+1, ..., K-1
  __device__ __forceinline__ static void run(const LevelBufs<T>& bufs, T* Y1, T* Y2, T* gcoef) {
    level_adj_recompose<T, N>(bufs(L), Y1, Y2, bufs(L + 1), gcoef, lvl_offset(B, L));
    if constexpr (L + 1 < K) AdjRecLevels<T, (N + 1) / 2, L + 1, K, B>::run(bufs, Y1, Y2, gcoef);
  }
};

template <typename T, int B, int K>
struct AdjCfg {
  using Cfg = BlockCfg<T, B, K>;
  // A (B^3), Y2 (B^2 C1), Y1 (B C1^2), cb0 (C1^3), cb1 (C2^3), R (C1^3)
  static constexpr size_t smem = sizeof(T) * (Cfg::A + Cfg::T1 + Cfg::T2 + 2 * Cfg::CB0 + Cfg::CB1);
};

// DIR 0: transposed decomposition (a.coef: coefficient gradients, a.G: block
// coarse gradients -> a.field: field gradients at the in-domain nodes).
// DIR 1: transposed recomposition (a.field -> a.coef, a.G).
template <typename T, int B, int K, int DIR>
__global__ void __launch_bounds__(BlockCfg<T, B, K>::NT_INV) block_adj_kernel(BlockArgs<T> a) {
  using Cfg = BlockCfg<T, B, K>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* Y2 = A + Cfg::A;
  T* Y1 = Y2 + Cfg::T1;
  T* cb0 = Y1 + Cfg::T2;
  T* cb1 = cb0 + Cfg::CB0;
  T* R = cb1 + Cfg::CB1;
  LevelBufs<T> bufs{A, cb0, cb1};
  constexpr int M = Cfg::M;
  for (int64_t b = blockIdx.x; b < a.nblocks; b += gridDim.x) {
    const BlockCoord bc(b, a.nb1, a.nb2);
    T* gcoef = a.coef + b * (int64_t)Cfg::PB;
    T* g = a.G + (((int64_t)bc.b0 * M) * a.g1 + (int64_t)bc.b1 * M) * a.g2 + (int64_t)bc.b2 * M;
    T* cf = bufs(K);
    if (DIR == 0) {
      for (int e = threadIdx.x; e < M * M * M; e += blockDim.x) {
        const int j0 = e / (M * M), r = e - j0 * M * M, j1 = r / M, j2 = r - j1 * M;
        cf[e] = g[((int64_t)j0 * a.g1 + j1) * a.g2 + j2];
      }
      __syncthreads();
      AdjDecLevels<T, M * 2 - 1, K - 1, B>::run(bufs, Y1, Y2, R, gcoef);
      store_block<T, B>(BlockSpan<T, B>(a.field, a.n0, a.n1, a.n2, bc), A, a.n1, a.n2);
    } else {
      issue_block_load<T, B>(A, a.field, BlockSpan<const T, B>(a.field, a.n0, a.n1, a.n2, bc), a.n1, a.n2);
      cp_async_commit();
      cp_async_wait<0>();
      __syncthreads();
      AdjRecLevels<T, B, 0, K, B>::run(bufs, Y1, Y2, gcoef);
      for (int e = threadIdx.x; e < M * M * M; e += blockDim.x) {
        const int j0 = e / (M * M), r = e - j0 * M * M, j1 = r / M, j2 = r - j1 * M;
        g[((int64_t)j0 * a.g1 + j1) * a.g2 + j2] = cf[e];
      }
    }
    __syncthreads();
  }
}

template <typename T, int B, int K>
cudaError_t launch_adj_one(int dir, const BlockArgs<T>& a, cudaStream_t s, int nsm) {
  using Cfg = BlockCfg<T, B, K>;
  const void* fn = dir == 0 ? (const void*)block_adj_kernel<T, B, K, 0> : (const void*)block_adj_kernel<T, B, K, 1>;
  const size_t smem = AdjCfg<T, B, K>::smem;
  static std::atomic<int> cached[2][64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int per_sm = dev < 64 ? cached[dir][dev].load() : 0;
  if (per_sm <= 0) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, Cfg::NT_INV, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (dev < 64) cached[dir][dev].store(per_sm);
  }
  int64_t grid = (int64_t)per_sm * nsm;
  if (grid > a.nblocks) grid = a.nblocks;
  if (grid < 1) return cudaSuccess;
  if (dir == 0) block_adj_kernel<T, B, K, 0><<<(unsigned)grid, Cfg::NT_INV, smem, s>>>(a);
  else block_adj_kernel<T, B, K, 1><<<(unsigned)grid, Cfg::NT_INV, smem, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Global levels (physical coordinates, plan tables), one thread per line
// ---------------------------------------------------------------------------

// A line pass along one dimension between a grid with n nodes on it (fine
// side) and one with c (coarse side).  Shapes as in apply_shape: lines are
// (batch b, column col); node i of the fine line is at
// fine + b*f_b + i*f_i + col*f_c, node J of the coarse line likewise.
struct LineShape {
  int64_t nb, ncol;
  int64_t f_b, f_i, f_c;
  int64_t c_b, c_i, c_c;
};

template <typename T>
LineShape line_shape(const GLevel<T>& L, int dim) {
  const ApplyShape A = apply_shape(L, dim);  // fine -> coarse restriction layout
  return LineShape{A.nb, A.ncol, A.in_b, A.in_i, A.in_c, A.out_b, A.out_j, A.out_c};
}

// fine line = M_f I M_c^-1 (coarse line): Thomas sweeps with the coarse
// values kept in the fine line's coarse slots, then the fine slots by
// interpolation, then the mass matrix with a rolling window (in place).
template <typename T>
__global__ void __launch_bounds__(256) gl_expand(GDim<T> D, LineShape S, const T* __restrict__ coarse,
                                                  T* __restrict__ fine) {
  const int n = D.n, c = D.c;
  const int64_t lines = S.nb * S.ncol;
  for (int64_t line = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; line < lines;
       line += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = line / S.ncol, col = line - b * S.ncol;
    const T* x = coarse + b * S.c_b + col * S.c_c;
    T* y = fine + b * S.f_b + col * S.f_c;
    const int64_t so = S.f_i, si = S.c_i;
    if (c == n) {  // a dimension of at most two nodes is not coarsened
      for (int i = 0; i < n; ++i) y[i * so] = x[i * si];
      continue;
    }
    T yv = x[0];
    y[(int64_t)D.cidx[0] * so] = yv;
    for (int J = 1; J < c; ++J) {
      yv = fma(-D.tm[J], yv, x[J * si]);
      y[(int64_t)D.cidx[J] * so] = yv;
    }
    T z = yv * D.tib[c - 1];
    y[(int64_t)D.cidx[c - 1] * so] = z;
    for (int J = c - 2; J >= 0; --J) {
      z = fma(-D.tsup[J], z, y[(int64_t)D.cidx[J] * so]) * D.tib[J];
      y[(int64_t)D.cidx[J] * so] = z;
    }
    for (int i = 0; i < n; ++i)
      if (!D.isc[i])
        y[i * so] = fma(D.wl[i], y[(int64_t)D.cidx[D.jlo[i]] * so], D.wr[i] * y[(int64_t)D.cidx[D.jhi[i]] * so]);
    T wm = T(0), w0 = y[0];
    for (int i = 0; i < n; ++i) {
      const T wp = i + 1 < n ? y[(i + 1) * so] : T(0);
      T v = D.md[i] * w0;
      if (i > 0) v = fma(D.mo[i - 1], wm, v);
      if (i + 1 < n) v = fma(D.mo[i], wp, v);
      y[i * so] = v;
      wm = w0;
      w0 = wp;
    }
  }
}

// coarse line = I^T (fine line): each coarse node gathers itself and its
// fine neighbours with their interpolation weights.
template <typename T>
__global__ void __launch_bounds__(256) gl_restrict_interp(GDim<T> D, LineShape S, const T* __restrict__ fine,
                                                           T* __restrict__ coarse) {
  const int n = D.n, c = D.c;
  const int64_t total = S.nb * S.ncol * c;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    // e = (b * c + J) * ncol + col: consecutive threads take consecutive columns
    const int64_t col = e % S.ncol, t = e / S.ncol;
    const int J = (int)(t % c);
    const int64_t b = t / c;
    const T* x = fine + b * S.f_b + col * S.f_c;
    const int i = D.cidx[J];
    T v = x[i * S.f_i];
    if (c != n) {
      if (i > 0 && !D.isc[i - 1]) v = fma(D.wr[i - 1], x[(i - 1) * S.f_i], v);
      if (i + 1 < n && !D.isc[i + 1]) v = fma(D.wl[i + 1], x[(i + 1) * S.f_i], v);
    }
    coarse[b * S.c_b + (int64_t)J * S.c_i + col * S.c_c] = v;
  }
}

template <typename T>
__global__ void gl_axpy(T* __restrict__ y, const T* __restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}

// g_u at the all-coarse nodes: += g_c - I^T v.
template <typename T>
__global__ void gl_adj_correct(GLevel<T> L, T* __restrict__ U, const T* __restrict__ gc, const T* __restrict__ r) {
  const int c0 = L.d[0].c, c1 = L.d[1].c, c2 = L.d[2].c, n1 = L.d[1].n, n2 = L.d[2].n;
  const int64_t total = (int64_t)c0 * c1 * c2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j2 = (int)(e % c2);
    const int64_t t = e / c2;
    const int j1 = (int)(t % c1), j0 = (int)(t / c1);
    const int64_t u = ((int64_t)L.d[0].cidx[j0] * n1 + L.d[1].cidx[j1]) * n2 + L.d[2].cidx[j2];
    U[u] += gc[e] - r[e];
  }
}

// Coefficient gradients of a level: g - t at the non all-coarse nodes, in
// stream order.
template <typename T>
__global__ void gl_adj_gather(GLevel<T> L, const T* __restrict__ g, const T* __restrict__ t, T* __restrict__ coef) {
  const int n0 = L.d[0].n, n1 = L.d[1].n, n2 = L.d[2].n;
  const int64_t total = (int64_t)n0 * n1 * n2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i2 = (int)(idx % n2);
    const int64_t q = idx / n2;
    const int i1 = (int)(q % n1), i0 = (int)(q / n1);
    if (all_coarse(L, i0, i1, i2)) continue;
    coef[nc_pos(L, i0, i1, i2, idx)] = g[idx] - t[idx];
  }
}

}  // namespace bm
