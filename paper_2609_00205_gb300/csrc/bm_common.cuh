// Shared device-side definitions of the BlockMGARD CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bm {

// ---------------------------------------------------------------------------
// Status bits written by kernels (never a trap): the host reads them back.
// ---------------------------------------------------------------------------
enum : unsigned {
  ST_OVERFLOW = 1u,   // a quantisation code did not fit in 30 bits (or NaN)
  ST_CORRUPT = 2u,    // decoding ran past a chunk / table bound
  ST_CAPACITY = 4u,   // a write would pass the output capacity
  ST_RAW = 8u,        // the stream must fall back to a raw copy
  ST_TIMEOUT = 16u,   // a bounded wait gave up (never expected on a healthy GPU)
};

constexpr int kHeaderBytes = 256;
constexpr uint32_t kMagic = 0x31474D42u;  // "BMG1"
constexpr int kMaxDict = 65536;          // symbols (2 * radius): 16-bit symbols
constexpr int kMaxLen = 32;              // longest Huffman code

__host__ __device__ inline uint64_t pad8(uint64_t x) { return (x + 7) & ~uint64_t(7); }

// Scalars shared by the kernels of one compress call (device scratch).
struct Scalars {
  unsigned long long maxabs_bits;  // max |u| as IEEE bits (float bits in the low word for FP32)
  unsigned status;                 // ST_* bits
  unsigned skip;                   // set before the encoder when the stream is already known to be raw
  unsigned long long n_words;      // Huffman words of the whole stream
  unsigned long long n_outliers;
  unsigned long long codebook_bytes;
  unsigned long long n_runs;
  unsigned long long off_bits;     // stream offsets decided on the device
  unsigned long long off_chunk_esc;
  unsigned long long off_outliers;
  unsigned long long total;
  double max_abs;
  double margin;
  unsigned long long max_len;
  unsigned long long esc_seen;     // escapes the encoder met (must equal n_outliers)
  unsigned maxabs_done;            // CTAs of the max|u| pass that have finished
  unsigned enc_lo;                 // first symbol of the encoder's shared-memory code window
  unsigned enc_mode;               // the encoder's table: 0 small window, 3 large window, 1 large window + global
                                   // table, 2 global table
  unsigned qready;                 // batched forward kernel: 1 once the quantiser table is written
  unsigned enc_n;                  // entries of the encoder's window that a met symbol can reach
};

// ---------------------------------------------------------------------------
// Compile-time tables of one uniform block level with N (odd) nodes.
//
// Block-local coordinates of level 1 are x_j = j; every deeper level keeps
// every other node, so each level is a uniform grid and its operators are
// those of N equally spaced nodes (the projection is scale invariant).
// Coarse nodes are the even indices (N odd), interpolation weights are 1/2.
//   rs[J][m]  band of row J of I^T M_f over fine columns 2J-2 .. 2J+2
//   tm, tib, tsup  LU factors of the coarse mass matrix M_c (Thomas):
//             forward y_i = r_i - tm_i y_{i-1}; back z_i = (y_i - tsup_i z_{i+1}) tib_i
// ---------------------------------------------------------------------------
template <typename T, int N>
struct BlockLevel {
  static constexpr int n = N;
  static constexpr int c = (N + 1) / 2;
  T rs[(N + 1) / 2][5];
  T tm[(N + 1) / 2];
  T tib[(N + 1) / 2];
  T tsup[(N + 1) / 2];
};

template <typename T, int N>
constexpr BlockLevel<T, N> make_block_level() {
  static_assert(N % 2 == 1 && N >= 3, "block levels need an odd node count >= 3");
  constexpr int C = (N + 1) / 2;
  BlockLevel<T, N> t{};
  // fine mass matrix (unit spacing): diag 2/3 (1/3 at the ends), off-diagonal 1/6
  double md[N] = {}, mo[N] = {};  // mo[i] = M(i, i+1)
  for (int i = 0; i < N; ++i) md[i] = (i == 0 || i == N - 1) ? 1.0 / 3.0 : 2.0 / 3.0;
  for (int i = 0; i + 1 < N; ++i) mo[i] = 1.0 / 6.0;
  for (int J = 0; J < C; ++J) {
    for (int m = 0; m < 5; ++m) {
      const int col = 2 * J - 2 + m;
      double v = 0.0;
      if (col >= 0 && col < N) {
        // rows contributing to coarse J: fine 2J (weight 1), 2J-1 and 2J+1 (weight 1/2)
        for (int dr = -1; dr <= 1; ++dr) {
          const int row = 2 * J + dr;
          if (row < 0 || row >= N) continue;
          const double w = dr == 0 ? 1.0 : 0.5;
          double mrc = 0.0;
          if (row == col) mrc = md[row];
          else if (row + 1 == col) mrc = mo[row];
          else if (col + 1 == row) mrc = mo[col];
          v += w * mrc;
        }
      }
      t.rs[J][m] = (T)v;
    }
  }
  // coarse mass matrix (spacing 2): diag 4/3 (2/3 at the ends), off-diagonal 1/3
  double b[C] = {}, a[C] = {}, cs[C] = {};
  for (int i = 0; i < C; ++i) {
    b[i] = (i == 0 || i == C - 1) ? 2.0 / 3.0 : 4.0 / 3.0;
    a[i] = i > 0 ? 1.0 / 3.0 : 0.0;
    cs[i] = i + 1 < C ? 1.0 / 3.0 : 0.0;
  }
  double bp = b[0];
  t.tm[0] = (T)0;
  t.tib[0] = (T)(1.0 / bp);
  for (int i = 1; i < C; ++i) {
    const double mul = a[i] / bp;
    bp = b[i] - mul * cs[i - 1];
    t.tm[i] = (T)mul;
    t.tib[i] = (T)(1.0 / bp);
  }
  for (int i = 0; i < C; ++i) t.tsup[i] = (T)cs[i];
  return t;
}

// Restriction + tridiagonal solve of one line held in registers:
// z = M_c^{-1} (I^T M_f d), all coefficients compile-time constants.
template <typename T, int N, class Tab>
__device__ __forceinline__ void restrict_solve(const Tab& tb, const T (&d)[N], T (&z)[(N + 1) / 2]) {
  constexpr int C = (N + 1) / 2;
  T r[C];
#pragma unroll
  for (int J = 0; J < C; ++J) {
    T s = T(0);
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      const int col = 2 * J - 2 + m;
      if (col >= 0 && col < N) s = fma(tb.rs[J][m], d[col], s);
    }
    r[J] = s;
  }
#pragma unroll
  for (int i = 1; i < C; ++i) r[i] = fma(-tb.tm[i], r[i - 1], r[i]);
  z[C - 1] = r[C - 1] * tb.tib[C - 1];
#pragma unroll
  for (int i = C - 2; i >= 0; --i) z[i] = fma(-tb.tsup[i], z[i + 1], r[i]) * tb.tib[i];
}

// ---------------------------------------------------------------------------
// Quantiser: code = floor(c * rq + 1/2) in the field's precision (one fused
// multiply-add, round to nearest); |code| must stay below 2^30.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int quantize(float c, float rq, bool& ovf) {
  const float y = __fmaf_rn(c, rq, 0.5f);
  if (!(fabsf(y) < 1073741824.0f)) { ovf = true; return 0; }
  return __float2int_rd(y);
}
__device__ __forceinline__ int quantize(double c, double rq, bool& ovf) {
  const double y = __fma_rn(c, rq, 0.5);
  if (!(fabs(y) < 1073741824.0)) { ovf = true; return 0; }
  return __double2int_rd(y);
}
__device__ __forceinline__ float dequant(int code, float q) { return __int2float_rn(code) * q; }
__device__ __forceinline__ double dequant(int code, double q) { return __int2double_rn(code) * q; }

// Asynchronous global->shared copy of one element with zero fill
// (cp.async; src_bytes = 0 fills zeros without reading).
template <int BYTES>
__device__ __forceinline__ void cp_async_zfill(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int src = valid ? BYTES : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(gmem), "n"(BYTES), "r"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int NLEFT>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NLEFT)); }

// Bulk asynchronous copies (cp.async.bulk, global -> shared) completing on a
// shared-memory mbarrier: the barrier's phase ends when every expected thread
// has arrived and all bytes announced with expect_tx have landed.  Addresses
// and sizes must be multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of the given parity to end; gives up after about 2^31
// SM cycles (a second at GB300 clocks) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// Orders this thread's earlier generic-proxy accesses of shared memory before
// later bulk copies into it (issued after a CTA barrier).
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Histogram bins kept in shared memory by the kernels that count symbols: a
// window of kHistWin symbols centred on the dictionary's middle (code 0), so
// the frequent symbols never go to a global atomic before the per-CTA flush
// (a single hot global bin serialises on one L2 slice); symbols outside the
// window (large codes, spread thinly over the dictionary) are counted with
// global atomics.  A dictionary of at most kHistWin symbols lies wholly in it.
constexpr int kHistWin = 8192;

}  // namespace bm
