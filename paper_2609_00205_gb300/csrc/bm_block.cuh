// In-cache Block kernels (Sec. III-A, III-D): one CTA keeps a B^3 block in
// shared memory through K decomposition levels, quantises the coefficients on
// the spot and writes only symbols (u16), the codes of escaping symbols and
// the block's coarse values.
//
// Level structure (Sec. II-B): for a level of N (odd) nodes per dimension
//   Phase A  lines (i0,i1) along dim 2: coefficients d = u - I(u|C) at every
//            node (zero at all-coarse nodes), emitted as symbols or values;
//            then z2 = M_c^-1 I^T M_f d along the line     -> T1, stored (i0,j2,i1)
//   Phase B  lines (i0,j2) along dim 1                      -> T2, stored (j1,j2,i0)
//   Phase C  lines (j1,j2) along dim 0, coarse = u|C + z    -> out (C,C,C)
// T1 and T2 are stored transposed so that every thread of phases B and C
// reads its line contiguously (stride N between threads: no bank conflicts).
// The forward pass copies u|C into `out` during phase A, after which the
// level's input is dead, so T2 takes the input's place in shared memory.
// The shrinking arrays N^3 -> N^2 C -> N C^2 -> C^3 are the paper's
// 8x8x8 -> 5x8x8 -> 5x5x8 -> 5x5x5 sequence for the block size used.
#pragma once

#include "bm_common.cuh"
#include "bm_internal.h"
#include "bm_qtab.cuh"

// Build-time choices of the forward kernel: whether it keeps the symbol
// histogram itself (BM_FWD_HIST; otherwise a separate pass counts the
// symbols), its threads per CTA (BM_FWD_THREADS; 0 = one per
// line of the first pass, B^2 rounded up to whole warps) and the CTAs per SM
// it is compiled for (BM_FWD_MIN_CTAS, capped by what shared memory holds);
// BM_INV_THREADS and BM_INV_MIN_CTAS are the last two for the inverse.  The
// defaults are the fastest measured on GB300 for the 513^3 FP32 workload: the
// in-kernel histogram's shared atomics and its 32 KB cost more than a separate
// pass, prefetching costs more than it hides, and five-warp CTAs (two lines of
// the first pass per thread, four or more CTAs per SM) let one CTA's barrier
// waits overlap the others' work.
#ifndef BM_FWD_HIST
#define BM_FWD_HIST 0
#endif
#ifndef BM_FWD_MIN_CTAS
#define BM_FWD_MIN_CTAS 4
#endif
#ifndef BM_FWD_THREADS
#define BM_FWD_THREADS 160
#endif
#ifndef BM_INV_THREADS
#define BM_INV_THREADS 160
#endif
#ifndef BM_INV_MIN_CTAS
#define BM_INV_MIN_CTAS 4
#endif
// BM_INV_CODES: the inverse turns symbols and escapes into int32 codes while
// loading a block (coalesced escape loads, 4 bytes per staged code) instead of
// reading each escape's code from the escape array where it is needed.
#ifndef BM_INV_CODES
#define BM_INV_CODES 1
#endif
// BM_FWD_BULK: 1 = the forward kernel stages a block that lies wholly inside
// the field with one bulk copy (cp.async.bulk, completing on an mbarrier) per
// row of B elements, rounded out to 16-byte boundaries, into shared memory
// that is dead at a block's start (the transposed and coarse arrays and the
// symbol staging area), then compacts the rows; blocks on the field's far
// faces keep the element-wise zero-filling cp.async.  0 (default) =
// element-wise cp.async for every block: a warp's 32 consecutive elements of
// a row go out as coalesced requests, and on GB300 (513^3 FP32, B = 17, K = 2)
// the kernel took 0.477 ms against 0.531 ms with 1 (289 bulk requests of 80
// bytes per block plus the compaction).  Prefetching the next block's rows
// into slots of their own (three CTAs per SM instead of four) took 0.590 ms.
#ifndef BM_FWD_BULK
#define BM_FWD_BULK 0
#endif

namespace bm {

// __constant__ tables, one per (dtype, level size), built at compile time.
#define BM_TAB(T, N) \
  static __constant__ BlockLevel<T, N> c_tab_##T##_##N = make_block_level<T, N>();
BM_TAB(float, 3)
BM_TAB(float, 5)
BM_TAB(float, 9)
BM_TAB(float, 17)
BM_TAB(double, 3)
BM_TAB(double, 5)
BM_TAB(double, 9)
BM_TAB(double, 17)
#undef BM_TAB

template <typename T, int N>
__device__ __forceinline__ const BlockLevel<T, N>& block_tab();
#define BM_TABREF(T, N) \
  template <>           \
  __device__ __forceinline__ const BlockLevel<T, N>& block_tab<T, N>() { return c_tab_##T##_##N; }
BM_TABREF(float, 3)
BM_TABREF(float, 5)
BM_TABREF(float, 9)
BM_TABREF(float, 17)
BM_TABREF(double, 3)
BM_TABREF(double, 5)
BM_TABREF(double, 9)
BM_TABREF(double, 17)
#undef BM_TABREF

constexpr int lvl_n(int B, int l) { return l == 0 ? B : (lvl_n(B, l - 1) + 1) / 2; }
constexpr int cube(int x) { return x * x * x; }
constexpr int per_block_count(int B, int K) {
  return K == 0 ? 0 : cube(B) - cube((B + 1) / 2) + per_block_count((B + 1) / 2, K - 1);
}
constexpr int lvl_offset(int B, int l) {  // first symbol of level l inside a block
  return l == 0 ? 0 : cube(lvl_n(B, l - 1)) - cube(lvl_n(B, l)) + lvl_offset(B, l - 1);
}

// Staging of a code in the forward kernel's 16-bit shared-memory array:
// code + kStageBias, or kStageWide for a code outside [-(2^15 - 1), 2^15 - 1].
// Every staged code has |code| < 2^15, so it becomes a symbol for any radius
// up to 2^15 (the largest dictionary: code 2^15 - 1 is symbol 2^16 - 1); a
// wide code has |code| >= 2^15 and always escapes.
constexpr int kStageBias = (1 << 15) - 1;
constexpr unsigned kStageWide = 0xFFFFu;

template <typename T, int B, int K>
struct BlockCfg {
  static constexpr int NT = ((B * B + 31) / 32) * 32;
  static constexpr int NT_FWD = (BM_FWD_THREADS > 0 && BM_FWD_THREADS < NT) ? BM_FWD_THREADS : NT;
  static constexpr int NT_INV = (BM_INV_THREADS > 0 && BM_INV_THREADS < NT) ? BM_INV_THREADS : NT;
  static constexpr int C1 = (B + 1) / 2;
  static constexpr int C2 = (C1 + 1) / 2;
  static constexpr int A = B * B * B;
  static constexpr int T1 = B * B * C1;
  static constexpr int T2 = B * C1 * C1;
  static constexpr int CB0 = C1 * C1 * C1;
  static constexpr int CB1 = C2 * C2 * C2;
  static constexpr int PB = per_block_count(B, K);
  static constexpr int M = lvl_n(B, K);
  // byte offsets: the symbol staging area and the histogram start on 16-byte
  // boundaries (the staging area is copied out with 8-byte vectors)
  static constexpr size_t up16(size_t x) { return (x + 15) / 16 * 16; }
  static constexpr size_t fwd_stage_off = up16(sizeof(T) * (A + T1 + CB0 + CB1));  // T2 overlays A
  static constexpr size_t fwd_hist_off = up16(fwd_stage_off + 2 * PB);
  static constexpr size_t fwd_hist_end = fwd_hist_off + (BM_FWD_HIST ? 4 * kHistWin : 0);
  // bulk staging: B^2 row slots of RP bytes (a row of B elements starting
  // anywhere on an element boundary, rounded out to 16-byte boundaries) from
  // the end of the block array on (over T1, the coarse buffers and the symbol
  // staging area; after the histogram when the kernel keeps one), then the
  // copies' mbarrier
  static constexpr int RP = (int)((B * sizeof(T) + 16 - sizeof(T) + 15) / 16 * 16);
  static constexpr size_t fwd_stg_off = BM_FWD_HIST ? up16(fwd_hist_end) : up16(sizeof(T) * A);
  // used unless the slots would cut the CTAs an SM holds (228 KB, 1 KB
  // reserved per CTA) below 16: FP64 with B = 17 keeps the element-wise copy
  static constexpr size_t fwd_stg_end = fwd_stg_off + (size_t)B * B * RP;
  static constexpr size_t fwd_bar_off = up16(fwd_stg_end > fwd_hist_end ? fwd_stg_end : fwd_hist_end);
  static constexpr int fit_of(size_t bytes) { return (int)((228u * 1024u) / (bytes + 1024u)); }
  static constexpr bool BULK = BM_FWD_BULK &&
                               (fit_of(fwd_bar_off + 16) >= fit_of(fwd_hist_end) || fit_of(fwd_bar_off + 16) >= 16);
  static constexpr size_t fwd_smem = BULK ? fwd_bar_off + 16 : fwd_hist_end;
  static constexpr size_t inv_stage_off = up16(sizeof(T) * (A + T1 + T2 + CB0 + CB1));
  static constexpr size_t inv_smem(int mode) {
    return inv_stage_off + up16((mode ? sizeof(T) : (BM_INV_CODES ? 4 : 2)) * PB);
  }
  // CTAs per SM the forward kernel is compiled for: BM_FWD_MIN_CTAS, or as many
  // as the shared memory of an SM holds (228 KB, 1 KB reserved per CTA) when
  // fewer, so the register budget is not cut for residency that cannot happen.
  static constexpr int fwd_fit = (int)((228u * 1024u) / (fwd_smem + 1024u));
  static constexpr int FWD_MIN_CTAS = fwd_fit < 1 ? 1 : (fwd_fit < BM_FWD_MIN_CTAS ? fwd_fit : BM_FWD_MIN_CTAS);
  static constexpr int inv_fit = (int)((228u * 1024u) / (inv_smem(1) + 1024u));
  static constexpr int INV_MIN_CTAS = inv_fit < 1 ? 1 : (inv_fit < BM_INV_MIN_CTAS ? inv_fit : BM_INV_MIN_CTAS);
};

// Histogram of one CTA: a window of kHistWin symbols around the centre in
// shared memory, global atomics outside it; the centre symbol (code 0, most
// of the symbols at loose tolerances) is counted in a register per thread and
// added once at the end.
__device__ __forceinline__ void hist_count(unsigned* hloc, unsigned* hglob, int radius, unsigned s, unsigned& centre) {
  if (s == (unsigned)radius) {
    ++centre;
    return;
  }
  const int bin = (int)s - (radius - kHistWin / 2);
  if (bin >= 0 && bin < kHistWin) atomicAdd(hloc + bin, 1u);
  else atomicAdd(hglob + s, 1u);
}

// ---------------------------------------------------------------------------
// Forward level
// ---------------------------------------------------------------------------
template <typename T, int N, int MODE>
__device__ __forceinline__ void level_fwd(T* X, T* __restrict__ T1, T* __restrict__ out, const int lvl_off, const T rq,
                                          uint16_t* stage, int32_t* __restrict__ esc_blk, T* __restrict__ coef_blk,
                                          bool& ovf, const bool full) {
  constexpr int C = (N + 1) / 2;
  const auto& tb = block_tab<T, N>();
  for (int L = threadIdx.x; L < N * N; L += blockDim.x) {
    const int i0 = L / N, i1 = L - i0 * N;
    const bool f0 = i0 & 1, f1 = i1 & 1;
    const int lo0 = f0 ? i0 - 1 : i0, hi0 = f0 ? i0 + 1 : i0;
    const int lo1 = f1 ? i1 - 1 : i1, hi1 = f1 ? i1 + 1 : i1;
    const T* r00 = X + (lo0 * N + lo1) * N;
    const T* r01 = X + (lo0 * N + hi1) * N;
    const T* r10 = X + (hi0 * N + lo1) * N;
    const T* r11 = X + (hi0 * N + hi1) * N;
    T w[C];
#pragma unroll
    for (int J = 0; J < C; ++J) w[J] = T(0.25) * ((r00[2 * J] + r01[2 * J]) + (r10[2 * J] + r11[2 * J]));
    T d[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const T u = X[L * N + k];
      const T e = (k & 1) ? T(0.5) * (w[k / 2] + w[k / 2 + 1]) : w[k / 2];
      d[k] = u - e;
    }
    const bool cc = !f0 && !f1;
    if (cc) {  // u|C of this line: the start of the coarse values (phase C adds z)
#pragma unroll
      for (int J = 0; J < C; ++J) out[((i0 / 2) * C + i1 / 2) * C + J] = X[L * N + 2 * J];
    }
    const int cc_before = ((i0 + 1) / 2) * C + (f0 ? 0 : (i1 + 1) / 2);
    const int base = lvl_off + L * N - cc_before * C;
    if (MODE == 0) {
      // the quantisation codes staged in the block's order as code + 2^15 - 1
      // (store_codes turns them into symbols and escapes when the block is
      // done); a code outside [-(2^15 - 1), 2^15 - 1] is staged as 0xFFFF and
      // goes to the escape array at once (a predicated store).  With the full
      // dictionary (`full`: radius 2^15) those wide codes are exactly the
      // escapes, so the staged value is the symbol itself: code + 2^15, or 0
      // A line with a wide code writes every code of the line to the escape
      // array (entries at other positions are never read): the lines of a
      // warp are consecutive positions, so its stores fill whole sectors
      // instead of leaving partly written ones to be merged from DRAM.
      const unsigned sadd = full ? 1u : 0u, swide = full ? 0u : kStageWide;
      int codes[N];
      bool anyw = false;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        if ((k & 1) || !cc) {
          const int pos = base + (cc ? k / 2 : k);
          const int code = quantize(d[k], rq, ovf);
          const unsigned b = (unsigned)(code + kStageBias);
          const bool wide = b >= kStageWide;
          stage[pos] = (uint16_t)(wide ? swide : b + sadd);
          codes[k] = code;
          anyw |= wide;
        }
      }
      if (anyw) {
#pragma unroll
        for (int k = 0; k < N; ++k)
          if ((k & 1) || !cc) esc_blk[base + (cc ? k / 2 : k)] = codes[k];
      }
    } else {
#pragma unroll
      for (int k = 0; k < N; ++k)
        if ((k & 1) || !cc) coef_blk[base + (cc ? k / 2 : k)] = d[k];
    }
    T z[C];
    restrict_solve<T, N>(tb, d, z);
#pragma unroll
    for (int j = 0; j < C; ++j) T1[(i0 * C + j) * N + i1] = z[j];
  }
  __syncthreads();
  T* T2 = X;
  for (int L = threadIdx.x; L < N * C; L += blockDim.x) {  // L = i0*C + j2
    const int i0 = L / C, j2 = L - i0 * C;
    T d[N];
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = T1[L * N + i];
    T z[C];
    restrict_solve<T, N>(tb, d, z);
#pragma unroll
    for (int j = 0; j < C; ++j) T2[(j * C + j2) * N + i0] = z[j];
  }
  __syncthreads();
  for (int L = threadIdx.x; L < C * C; L += blockDim.x) {  // L = j1*C + j2
    const int j1 = L / C, j2 = L - j1 * C;
    T d[N];
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = T2[L * N + i];
    T z[C];
    restrict_solve<T, N>(tb, d, z);
#pragma unroll
    for (int J = 0; J < C; ++J) out[(J * C + j1) * C + j2] += z[J];
  }
  __syncthreads();
}

// Buffer of level output j (0 = the block itself): ping-pong between two
// coarse buffers so a level never writes the array it reads.
template <typename T>
struct LevelBufs {
  T* A;
  T* cb0;
  T* cb1;
  __device__ __forceinline__ T* operator()(int j) const { return j == 0 ? A : ((j & 1) ? cb0 : cb1); }
};

template <typename T, int N, int L, int K, int B, int MODE>
struct FwdLevels {
  __device__ __forceinline__ static void run(const LevelBufs<T>& bufs, T* T1, const T* rq, uint16_t* stage,
                                             int32_t* esc_blk, T* coef_blk, bool& ovf, const bool full) {
    level_fwd<T, N, MODE>(bufs(L), T1, bufs(L + 1), lvl_offset(B, L), rq[L], stage, esc_blk, coef_blk, ovf, full);
    if constexpr (L + 1 < K)
      FwdLevels<T, (N + 1) / 2, L + 1, K, B, MODE>::run(bufs, T1, rq, stage, esc_blk, coef_blk, ovf, full);
  }
};

// Block coordinates (b0, b1, b2) of linear block index b: two 32-bit divisions
// per block (the block grid has fewer than 2^31 blocks).
struct BlockCoord {
  int b0, b1, b2;
  __device__ __forceinline__ BlockCoord(int64_t b, int nb1, int nb2) {
    const unsigned ub = (unsigned)b, q2 = ub / (unsigned)nb2, q1 = q2 / (unsigned)nb1;
    b2 = (int)(ub - q2 * (unsigned)nb2);
    b1 = (int)(q2 - q1 * (unsigned)nb1);
    b0 = (int)q1;
  }
};

// First element of block (b0, b1, b2) in the field, and its in-domain extents.
template <typename T, int B>
struct BlockSpan {
  T* base;
  int lim0, lim1, lim2;
  __device__ __forceinline__ BlockSpan(T* field, int64_t n0, int64_t n1, int64_t n2, const BlockCoord& c) {
    base = field + ((int64_t)c.b0 * B * n1 + (int64_t)c.b1 * B) * n2 + (int64_t)c.b2 * B;
    const int64_t r0 = n0 - (int64_t)c.b0 * B, r1 = n1 - (int64_t)c.b1 * B, r2 = n2 - (int64_t)c.b2 * B;
    lim0 = r0 < B ? (int)r0 : B;
    lim1 = r1 < B ? (int)r1 : B;
    lim2 = r2 < B ? (int)r2 : B;
  }
};

// Copy of one B^3 block into shared memory (row-major), zero filled outside the
// domain.  Work item t < B(B+1) (threads stride over the items) owns column
// k = t % B and the rows r0 + (B+1) j of the block (r0 = t / B, j < B): each
// step moves one plane down and one row
// on (i0+1, i1+1, i1 wrapping once), so the source advances by the constant
// s0 + n2, corrected once by s0 - B n2 at the wrap, and the destination by
// B(B+1) elements.  Consecutive threads read consecutive elements of a row.
template <typename T, int B>
__device__ __forceinline__ void issue_block_load(T* dst, const T* __restrict__ field, const BlockSpan<const T, B>& sp,
                                                 int64_t n1, int64_t n2) {
  for (int t = threadIdx.x; t < B * (B + 1); t += blockDim.x) {
    const int k = t % B, r0 = t / B, jc = B - r0;
    const int64_t s0 = n1 * n2, D = s0 + n2, E = s0 - (int64_t)B * n2;
    const T* p = sp.base + (int64_t)r0 * n2 + k;
    T* q = dst + t;
    if ((sp.lim0 == B) & (sp.lim1 == B) & (sp.lim2 == B)) {  // interior block
#pragma unroll
      for (int j = 0; j < B; ++j) {
        if (j < B - 1 || r0 == 0) cp_async_zfill<sizeof(T)>(q + j * B * (B + 1), p + (j >= jc ? E : 0), true);
        p += D;
      }
    } else {
#pragma unroll
      for (int j = 0; j < B; ++j) {
        if (j < B - 1 || r0 == 0) {
          const int carry = j >= jc;
          const int i0 = j + carry, i1 = r0 + j - (carry ? B : 0);
          const bool ok = (i0 < sp.lim0) & (i1 < sp.lim1) & (k < sp.lim2);
          cp_async_zfill<sizeof(T)>(q + j * B * (B + 1), ok ? p + (carry ? E : 0) : field, ok);
        }
        p += D;
      }
    }
  }
}

// Bulk staging of a block that lies wholly inside the field: row (i0, i1)
// starts at byte address p = base + (i0 s0 + i1 n2) sizeof(T); the copy takes
// [p rounded down to 16, p + B sizeof(T) rounded up to 16) into slot
// i0 B + i1 (RP bytes).  Every 16-byte segment of that span holds an element
// of the row, so it never leaves the pages of the field.  Every thread
// arrives once on the barrier, announcing the bytes of its own rows.
template <typename T, int B, int K>
__device__ __forceinline__ void issue_block_bulk(unsigned char* stg, uint64_t* bar, const T* base, int64_t s0,
                                                 int64_t n2) {
  using Cfg = BlockCfg<T, B, K>;
  constexpr int NR = B * B, IT = (NR + Cfg::NT_FWD - 1) / Cfg::NT_FWD;
  const uintptr_t b0 = reinterpret_cast<uintptr_t>(base);
  uintptr_t lo[IT];
  unsigned nb[IT];
  unsigned bytes = 0;
#pragma unroll
  for (int j = 0; j < IT; ++j) {
    const int r = threadIdx.x + j * Cfg::NT_FWD;
    nb[j] = 0;
    lo[j] = 0;
    if (r < NR) {
      const int i0 = r / B, i1 = r - i0 * B;
      const uintptr_t p = b0 + (uintptr_t)(((int64_t)i0 * s0 + (int64_t)i1 * n2) * (int64_t)sizeof(T));
      lo[j] = p & ~(uintptr_t)15;
      nb[j] = (unsigned)(((p + B * sizeof(T) + 15) & ~(uintptr_t)15) - lo[j]);
      bytes += nb[j];
    }
  }
  mbar_arrive_expect_tx(bar, bytes);
#pragma unroll
  for (int j = 0; j < IT; ++j)
    if (nb[j]) bulk_g2s(stg + (size_t)(threadIdx.x + j * Cfg::NT_FWD) * Cfg::RP, reinterpret_cast<const void*>(lo[j]),
                        nb[j], bar);
}

// Staged rows -> the block array (row-major B^3): a thread per row reads its
// slot as 16-byte vectors and drops the m = (p mod 16) / sizeof(T) leading
// elements with a two-step select (m & 2, then m & 1), so no register array
// is indexed at run time.  Slot reads (stride RP) and row writes (stride B)
// are free of bank conflicts.
template <typename T, int B, int K>
__device__ __forceinline__ void compact_block_rows(T* X, const unsigned char* stg, const T* base, int64_t s0,
                                                   int64_t n2) {
  using Cfg = BlockCfg<T, B, K>;
  constexpr int W = Cfg::RP / (int)sizeof(T);  // elements per slot
  const uintptr_t b0 = reinterpret_cast<uintptr_t>(base);
  for (int r = threadIdx.x; r < B * B; r += blockDim.x) {
    const int i0 = r / B, i1 = r - i0 * B;
    const uintptr_t p = b0 + (uintptr_t)(((int64_t)i0 * s0 + (int64_t)i1 * n2) * (int64_t)sizeof(T));
    const unsigned m = (unsigned)(p & 15) / (unsigned)sizeof(T);
    T v[W];
    const uint4* src = reinterpret_cast<const uint4*>(stg + (size_t)r * Cfg::RP);
#pragma unroll
    for (int g = 0; g < Cfg::RP / 16; ++g) {
      const uint4 q = src[g];
      if constexpr (sizeof(T) == 4) {
        v[4 * g] = __uint_as_float(q.x);
        v[4 * g + 1] = __uint_as_float(q.y);
        v[4 * g + 2] = __uint_as_float(q.z);
        v[4 * g + 3] = __uint_as_float(q.w);
      } else {
        v[2 * g] = __hiloint2double((int)q.y, (int)q.x);
        v[2 * g + 1] = __hiloint2double((int)q.w, (int)q.z);
      }
    }
    if constexpr (sizeof(T) == 4) {
      const bool s2 = m & 2u;
#pragma unroll
      for (int k = 0; k < W - 2; ++k) v[k] = s2 ? v[k + 2] : v[k];
    }
    const bool s1 = m & 1u;
#pragma unroll
    for (int k = 0; k < B; ++k) v[k] = s1 ? v[k + 1] : v[k];
    T* d = X + r * B;
#pragma unroll
    for (int k = 0; k < B; ++k) d[k] = v[k];
  }
}

// The inverse copy: the in-domain part of the block from shared memory to the
// field, with the same thread-to-element assignment.
template <typename T, int B>
__device__ __forceinline__ void store_block(const BlockSpan<T, B>& sp, const T* src, int64_t n1, int64_t n2) {
  for (int t = threadIdx.x; t < B * (B + 1); t += blockDim.x) {
    const int k = t % B, r0 = t / B, jc = B - r0;
    const int64_t s0 = n1 * n2, D = s0 + n2, E = s0 - (int64_t)B * n2;
    T* p = sp.base + (int64_t)r0 * n2 + k;
    const T* q = src + t;
    if ((sp.lim0 == B) & (sp.lim1 == B) & (sp.lim2 == B)) {
#pragma unroll
      for (int j = 0; j < B; ++j) {
        if (j < B - 1 || r0 == 0) p[j >= jc ? E : 0] = q[j * B * (B + 1)];
        p += D;
      }
    } else {
#pragma unroll
      for (int j = 0; j < B; ++j) {
        if (j < B - 1 || r0 == 0) {
          const int carry = j >= jc;
          const int i0 = j + carry, i1 = r0 + j - (carry ? B : 0);
          if ((i0 < sp.lim0) & (i1 < sp.lim1) & (k < sp.lim2)) p[carry ? E : 0] = q[j * B * (B + 1)];
        }
        p += D;
      }
    }
  }
}

// Copy of n u16 symbols from shared to global memory with the widest aligned
// stores the per-block offset allows.
// A block's staged codes -> symbols: code + radius for |code| < radius, else
// the escape symbol 0 with the code kept at the same position of the escape
// array.  Consecutive threads take consecutive groups of four codes, so the
// symbol stores (8 bytes) and the escape stores (the whole 16-byte group
// whenever one of its codes escapes) are coalesced; escape-array entries at
// other positions are never read.  A group holding a wide code (already in
// the escape array) stores its other escapes one by one.
template <int PB>
__device__ __forceinline__ void store_codes(uint16_t* __restrict__ sym, int32_t* __restrict__ esc,
                                            const uint16_t* __restrict__ st, const int radius, unsigned* hloc,
                                            unsigned* hglob, unsigned& centre) {
  const unsigned span = (unsigned)(2 * radius - 1);
  auto to_sym = [&](unsigned b) {  // b: staged value; wide codes always escape
    const unsigned u = (unsigned)((int)b - kStageBias + radius);
    return (b != kStageWide && (u - 1u) < span) ? u : 0u;
  };
  bool vec = false;
  if constexpr (PB % 4 == 0)
    vec = ((reinterpret_cast<uintptr_t>(sym) & 7) | (reinterpret_cast<uintptr_t>(esc) & 15)) == 0;
  if (vec) {
    const uint2* s2 = reinterpret_cast<const uint2*>(st);
    uint2* d2 = reinterpret_cast<uint2*>(sym);
    int4* e4 = reinterpret_cast<int4*>(esc);
    for (int i = threadIdx.x; i < PB / 4; i += blockDim.x) {
      const uint2 w = s2[i];
      const unsigned b[4] = {w.x & 0xFFFFu, w.x >> 16, w.y & 0xFFFFu, w.y >> 16};
      unsigned a[4];
      bool any_esc = false, any_wide = false;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        a[j] = to_sym(b[j]);
        any_esc |= a[j] == 0u;
        any_wide |= b[j] == kStageWide;
      }
      d2[i] = make_uint2(a[0] | (a[1] << 16), a[2] | (a[3] << 16));
      if (any_esc) {
        if (!any_wide) {
          e4[i] = make_int4((int)b[0] - kStageBias, (int)b[1] - kStageBias, (int)b[2] - kStageBias,
                            (int)b[3] - kStageBias);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (a[j] == 0u && b[j] != kStageWide) esc[4 * i + j] = (int)b[j] - kStageBias;
        }
      }
      if (BM_FWD_HIST)
#pragma unroll
        for (int j = 0; j < 4; ++j) hist_count(hloc, hglob, radius, a[j], centre);
    }
  } else {
    for (int i = threadIdx.x; i < PB; i += blockDim.x) {
      const unsigned b = st[i];
      const unsigned a = to_sym(b);
      sym[i] = (uint16_t)a;
      if (!a && b != kStageWide) esc[i] = (int)b - kStageBias;
      if (BM_FWD_HIST) hist_count(hloc, hglob, radius, a, centre);
    }
  }
}

// A block's staged symbols (full dictionary: escapes are already in the
// escape array) to global memory: 8-byte vectors when the block's first
// symbol is 8-byte aligned.
template <int PB>
__device__ __forceinline__ void copy_symbols(uint16_t* __restrict__ sym, const uint16_t* __restrict__ st) {
  if (PB % 4 == 0 && (reinterpret_cast<uintptr_t>(sym) & 7) == 0) {
    const uint2* s2 = reinterpret_cast<const uint2*>(st);
    uint2* d2 = reinterpret_cast<uint2*>(sym);
    for (int i = threadIdx.x; i < PB / 4; i += blockDim.x) d2[i] = s2[i];
  } else {
    for (int i = threadIdx.x; i < PB; i += blockDim.x) sym[i] = st[i];
  }
}

// Shared memory of the forward kernels.
template <typename T, int B, int K>
struct FwdSmem {
  T* A;            // the block (B^3), then T2 over it
  T* T1;           // first-pass results (B^2 C)
  T* cb0;          // coarse values of odd levels (C^3)
  T* cb1;          // coarse values of even levels
  uint16_t* stage;  // the block's staged codes
  unsigned* hloc;  // histogram window (BM_FWD_HIST)
  uint64_t* bar;   // bulk-copy barrier (BM_FWD_BULK)
  unsigned char* stg;  // bulk-copy row slots
  __device__ __forceinline__ explicit FwdSmem(unsigned char* raw) {
    using Cfg = BlockCfg<T, B, K>;
    A = reinterpret_cast<T*>(raw);
    T1 = A + Cfg::A;
    cb0 = T1 + Cfg::T1;
    cb1 = cb0 + Cfg::CB0;
    stage = reinterpret_cast<uint16_t*>(raw + Cfg::fwd_stage_off);
    hloc = reinterpret_cast<unsigned*>(raw + Cfg::fwd_hist_off);
    bar = reinterpret_cast<uint64_t*>(raw + Cfg::fwd_bar_off);
    stg = raw + Cfg::fwd_stg_off;
  }
};

template <typename T, int B, int K>
__device__ __forceinline__ void fwd_init(const FwdSmem<T, B, K>& S) {
  if (BlockCfg<T, B, K>::BULK) {
    if (threadIdx.x == 0) {
      mbar_init(S.bar, BlockCfg<T, B, K>::NT_FWD);
      mbar_fence_init();
    }
    __syncthreads();
  }
}

// One block of the forward pass: staged into shared memory (zero filled
// outside the domain), K levels with the codes quantised on the spot, the
// block's coarse values to the gathered grid G, its symbols and escapes out.
// The quantiser table is read around L1 (the batched kernel writes it in the
// same launch).  Returns false when the block's bulk copies never completed:
// the status is set and the CTA must stop.
template <typename T, int B, int K, int MODE>
__device__ __forceinline__ bool fwd_block(const BlockArgs<T>& a, int64_t b, const FwdSmem<T, B, K>& S,
                                          unsigned& phase, bool& ovf, unsigned& centre) {
  using Cfg = BlockCfg<T, B, K>;
  const BlockCoord bc(b, a.nb1, a.nb2);
  const BlockSpan<const T, B> sp(a.field, a.n0, a.n1, a.n2, bc);
  if (Cfg::BULK && (sp.lim0 == B) & (sp.lim1 == B) & (sp.lim2 == B)) {
    const int64_t s0 = a.n1 * a.n2;
    issue_block_bulk<T, B, K>(S.stg, S.bar, sp.base, s0, a.n2);
    const bool late = !mbar_wait_bounded(S.bar, phase);
    compact_block_rows<T, B, K>(S.A, S.stg, sp.base, s0, a.n2);
    if (__syncthreads_or(late)) {  // the copies never completed: report, drain (bounded), stop
      if (threadIdx.x == 0 && a.sc) atomicOr(&a.sc->status, ST_TIMEOUT);
      mbar_wait_bounded(S.bar, phase);
      return false;
    }
    phase ^= 1u;
  } else {
    issue_block_load<T, B>(S.A, a.field, sp, a.n1, a.n2);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
  }
  T rq[K];
  const int tier = a.tier ? a.tier[b] : 0;
#pragma unroll
  for (int l = 0; l < K; ++l) rq[l] = MODE == 0 ? __ldcg(a.rq + tier * K + l) : T(0);
  const int64_t sbase = b * (int64_t)Cfg::PB;
  const LevelBufs<T> bufs{S.A, S.cb0, S.cb1};
  const bool full = MODE == 0 && a.radius == (1 << 15) && !BM_FWD_HIST;
  FwdLevels<T, B, 0, K, B, MODE>::run(bufs, S.T1, rq, S.stage, a.esc + (MODE == 0 ? sbase : 0),
                                      a.coef + (MODE == 1 ? sbase : 0), ovf, full);
  {  // block coarse values -> gathered grid G
    constexpr int M = Cfg::M;
    const T* cf = bufs(K);
    T* g = a.G + (((int64_t)bc.b0 * M) * a.g1 + (int64_t)bc.b1 * M) * a.g2 + (int64_t)bc.b2 * M;
    for (int e = threadIdx.x; e < M * M * M; e += blockDim.x) {
      const int j0 = e / (M * M), r = e - j0 * M * M, j1 = r / M, j2 = r - j1 * M;
      g[((int64_t)j0 * a.g1 + j1) * a.g2 + j2] = cf[e];
    }
  }
  if (MODE == 0) {
    if (full) copy_symbols<Cfg::PB>(a.sym + sbase, S.stage);
    else store_codes<Cfg::PB>(a.sym + sbase, a.esc + sbase, S.stage, a.radius, S.hloc, a.hist, centre);
  }
  if (Cfg::BULK) fence_proxy_async_smem();  // the next block's bulk copies overwrite what was read here
  __syncthreads();
  return true;
}

// Forward: persistent CTAs walk the blocks of one field.  (A variant that
// prefetched the next block into a second buffer with element-wise cp.async
// cost more than it hid: twice the block array per CTA.)
template <typename T, int B, int K, int MODE>
__global__ void __launch_bounds__(BlockCfg<T, B, K>::NT_FWD, BlockCfg<T, B, K>::FWD_MIN_CTAS)
    block_fwd_kernel(BlockArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FwdSmem<T, B, K> S(smem_raw);
  if (MODE == 0 && BM_FWD_HIST)
    for (int i = threadIdx.x; i < kHistWin; i += blockDim.x) S.hloc[i] = 0;
  fwd_init(S);
  bool ovf = false;
  unsigned centre = 0, phase = 0;
  for (int64_t b = blockIdx.x; b < a.nblocks; b += gridDim.x)
    if (!fwd_block<T, B, K, MODE>(a, b, S, phase, ovf, centre)) return;
  if (MODE == 0 && ovf) atomicOr(&a.sc->status, ST_OVERFLOW);
  if (MODE == 0 && BM_FWD_HIST) {
#pragma unroll
    for (int o = 16; o; o >>= 1) centre += __shfl_xor_sync(0xffffffffu, centre, o);
    if ((threadIdx.x & 31) == 0 && centre) atomicAdd(S.hloc + (kHistWin / 2), centre);
    __syncthreads();
    const int lo = a.radius - kHistWin / 2;
    for (int i = threadIdx.x; i < kHistWin; i += blockDim.x) {
      const unsigned v = S.hloc[i];
      if (v && lo + i >= 0 && lo + i < 2 * a.radius) atomicAdd(a.hist + lo + i, v);
    }
  }
}

// ---------------------------------------------------------------------------
// Batched forward (Sec. III-B / III-D: many fields per launch): one persistent
// launch drains a device-side queue of work items spanning every field of a
// batch that shares (dtype, B, K).  Items are taken in ticket order from one
// global counter: first the max|u| items of every field (a slice of
// kBatchMaxChunk elements each), then one item per block.  The CTA that
// finishes a field's last max|u| item computes that field's quantiser table
// and raises its ready flag; a CTA taking a block of the field waits for the
// flag (bounded, acquire).  Every max|u| item holds a lower ticket than every
// block item and is done by a running CTA without waiting, so the wait ends.
// ---------------------------------------------------------------------------
constexpr int64_t kBatchMaxChunk = 65536;

template <typename T>
struct BatchField {
  BlockArgs<T> a;             // the field's block arguments (MODE 0)
  QtabArgs qa;                // its quantiser table (qa.sc: the field's scalars)
  int64_t nel;                // elements of the field
  unsigned long long max0;    // first max|u| ticket
  unsigned long long blk0;    // first block ticket
};

struct BatchQueue {
  unsigned long long* ticket;  // zeroed before the launch
  unsigned long long n_max;    // max|u| items of all fields (tickets [0, n_max))
  unsigned long long n_all;    // all items
  int nfields;
};

// Field of ticket t: the last field whose first ticket (of the item's kind)
// is <= t (binary search over the descriptors, one thread).
template <typename T>
__device__ __forceinline__ int batch_field_of(const BatchField<T>* f, int n, unsigned long long t, bool blk) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const unsigned long long v = blk ? __ldg(&f[mid].blk0) : __ldg(&f[mid].max0);
    if (v <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// max|u| of elements [lo, hi) of u, 16-byte loads over the aligned middle.
template <typename T>
__device__ __forceinline__ void maxabs_slice(const T* __restrict__ u, int64_t lo, int64_t hi, T& m, bool& bad) {
  constexpr int V = 16 / sizeof(T);
  const uintptr_t pa = reinterpret_cast<uintptr_t>(u + lo);
  int64_t h = (int64_t)(((16 - (pa & 15)) & 15) / sizeof(T));
  if (h > hi - lo) h = hi - lo;
  const int64_t nv = (hi - lo - h) / V;
  const uint4* pv = reinterpret_cast<const uint4*>(u + lo + h);
  for (int64_t i = threadIdx.x; i < nv; i += blockDim.x) {
    const uint4 q = __ldg(pv + i);
    const T* t = reinterpret_cast<const T*>(&q);
#pragma unroll
    for (int j = 0; j < V; ++j) maxabs_acc(t[j], m, bad);
  }
  for (int64_t i = threadIdx.x; i < h; i += blockDim.x) maxabs_acc(u[lo + i], m, bad);
  for (int64_t i = lo + h + nv * V + threadIdx.x; i < hi; i += blockDim.x) maxabs_acc(u[i], m, bad);
}

template <typename T, int B, int K>
__global__ void __launch_bounds__(BlockCfg<T, B, K>::NT_FWD, BlockCfg<T, B, K>::FWD_MIN_CTAS)
    block_fwd_batch_kernel(const BatchField<T>* __restrict__ fields, BatchQueue q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FwdSmem<T, B, K> S(smem_raw);
  __shared__ unsigned long long s_t;
  __shared__ int s_ok;
  __shared__ T s_m[32];
  __shared__ int s_bad;
  fwd_init(S);
  unsigned phase = 0, centre = 0;
  while (true) {
    if (threadIdx.x == 0) s_t = atomicAdd(q.ticket, 1ull);
    __syncthreads();
    const unsigned long long t = s_t;
    if (t >= q.n_all) break;
    if (t < q.n_max) {  // a slice of max|u|
      const int f = batch_field_of(fields, q.nfields, t, false);
      const BatchField<T>& F = fields[f];
      const int64_t lo = (int64_t)(t - F.max0) * kBatchMaxChunk;
      const int64_t hi = lo + kBatchMaxChunk < F.nel ? lo + kBatchMaxChunk : F.nel;
      T m = T(0);
      bool bad = false;
      maxabs_slice(F.a.field, lo, hi, m, bad);
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const T y = __shfl_xor_sync(0xffffffffu, m, o);
        m = y > m ? y : m;
      }
      bad = __any_sync(0xffffffffu, bad);
      if (threadIdx.x == 0) s_bad = 0;
      __syncthreads();
      if ((threadIdx.x & 31) == 0) {
        s_m[threadIdx.x >> 5] = m;
        if (bad) s_bad = 1;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = s_m[w] > m ? s_m[w] : m;
        Scalars* sc = F.qa.sc;
        if (sizeof(T) == 4) atomicMax(&sc->maxabs_bits, (unsigned long long)__float_as_uint((float)m));
        else atomicMax(&sc->maxabs_bits, (unsigned long long)__double_as_longlong((double)m));
        if (s_bad) atomicOr(&sc->status, ST_RAW);
        __threadfence();
        const unsigned n_items = (unsigned)((F.nel + kBatchMaxChunk - 1) / kBatchMaxChunk);
        if (atomicAdd(&sc->maxabs_done, 1u) == n_items - 1) {  // the field's last slice: its table
          __threadfence();
          qtab_compute(F.qa);
          __threadfence();
          asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(&sc->qready), "r"(1u) : "memory");
        }
      }
      __syncthreads();
    } else {  // one block
      const int f = batch_field_of(fields, q.nfields, t, true);
      const BatchField<T>& F = fields[f];
      if (threadIdx.x == 0) {
        const unsigned* flag = &F.qa.sc->qready;
        unsigned v = 0;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(flag) : "memory");
        if (!v) {
          const long long t0 = clock64();
          do {
            __nanosleep(256);
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(flag) : "memory");
          } while (!v && clock64() - t0 < (1ll << 31));
        }
        s_ok = v != 0;
        if (!v) atomicOr(&F.qa.sc->status, ST_TIMEOUT);
      }
      __syncthreads();
      if (!s_ok) continue;  // the field's table never came: reported, block skipped
      bool ovf = false;
      if (!fwd_block<T, B, K, 0>(F.a, (int64_t)(t - F.blk0), S, phase, ovf, centre)) return;
      if (ovf) atomicOr(&F.a.sc->status, ST_OVERFLOW);
    }
  }
}

// Symbols and escapes of a block -> int32 codes in shared memory (the inverse
// of store_codes): consecutive threads take consecutive groups of four, and a
// group with an escape symbol loads its four escape-array entries as one
// coalesced 16-byte load.
template <int PB>
__device__ __forceinline__ void load_codes(const uint16_t* __restrict__ sym, const int32_t* __restrict__ esc,
                                           int32_t* __restrict__ st, const int radius) {
  bool vec = false;
  if constexpr (PB % 4 == 0)
    vec = ((reinterpret_cast<uintptr_t>(sym) & 7) | (reinterpret_cast<uintptr_t>(esc) & 15)) == 0;
  if (vec) {
    const uint2* s2 = reinterpret_cast<const uint2*>(sym);
    const int4* e4 = reinterpret_cast<const int4*>(esc);
    int4* d4 = reinterpret_cast<int4*>(st);
    for (int i = threadIdx.x; i < PB / 4; i += blockDim.x) {
      const uint2 w = __ldg(s2 + i);
      const int a0 = (int)(w.x & 0xFFFFu), a1 = (int)(w.x >> 16), a2 = (int)(w.y & 0xFFFFu), a3 = (int)(w.y >> 16);
      int4 c = make_int4(0, 0, 0, 0);
      if (!(a0 && a1 && a2 && a3)) c = __ldg(e4 + i);
      d4[i] = make_int4(a0 ? a0 - radius : c.x, a1 ? a1 - radius : c.y, a2 ? a2 - radius : c.z,
                        a3 ? a3 - radius : c.w);
    }
  } else {
    for (int i = threadIdx.x; i < PB; i += blockDim.x) {
      const int a = (int)sym[i];
      st[i] = a ? a - radius : esc[i];
    }
  }
}

// ---------------------------------------------------------------------------
// Inverse level: coarse values `cin` (C^3) and the level's coefficients give
// the N^3 values in X.  z = P D (three passes), u|C = c - z, u = I u|C + D.
// ---------------------------------------------------------------------------
template <typename T, int N, int MODE>
__device__ __forceinline__ void level_inv(T* __restrict__ X, T* __restrict__ T1, T* __restrict__ T2,
                                          T* __restrict__ cin, const int lvl_off, const T q,
                                          const void* stage, const int32_t* __restrict__ esc_blk, const int radius) {
  constexpr int C = (N + 1) / 2;
  const auto& tb = block_tab<T, N>();
  for (int L = threadIdx.x; L < N * N; L += blockDim.x) {
    const int i0 = L / N, i1 = L - i0 * N;
    const bool f0 = i0 & 1, f1 = i1 & 1;
    const bool cc = !f0 && !f1;
    const int cc_before = ((i0 + 1) / 2) * C + (f0 ? 0 : (i1 + 1) / 2);
    const int base = lvl_off + L * N - cc_before * C;
    T d[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      T v = T(0);
      if ((k & 1) || !cc) {
        const int pos = base + (cc ? k / 2 : k);
        if (MODE == 0) {
#if BM_INV_CODES
          const int code = reinterpret_cast<const int32_t*>(stage)[pos];
#else
          const unsigned s = reinterpret_cast<const uint16_t*>(stage)[pos];
          const int code = s ? (int)s - radius : esc_blk[pos];
#endif
          v = dequant(code, q);
        } else {
          v = reinterpret_cast<const T*>(stage)[pos];
        }
      }
      d[k] = v;
      X[L * N + k] = v;
    }
    T z[C];
    restrict_solve<T, N>(tb, d, z);
#pragma unroll
    for (int j = 0; j < C; ++j) T1[(i0 * C + j) * N + i1] = z[j];
  }
  __syncthreads();
  for (int L = threadIdx.x; L < N * C; L += blockDim.x) {  // L = i0*C + j2
    const int i0 = L / C, j2 = L - i0 * C;
    T d[N];
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = T1[L * N + i];
    T z[C];
    restrict_solve<T, N>(tb, d, z);
#pragma unroll
    for (int j = 0; j < C; ++j) T2[(j * C + j2) * N + i0] = z[j];
  }
  __syncthreads();
  for (int L = threadIdx.x; L < C * C; L += blockDim.x) {  // L = j1*C + j2
    const int j1 = L / C, j2 = L - j1 * C;
    T d[N];
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = T2[L * N + i];
    T z[C];
    restrict_solve<T, N>(tb, d, z);
#pragma unroll
    for (int J = 0; J < C; ++J) cin[(J * C + j1) * C + j2] -= z[J];
  }
  __syncthreads();
  for (int L = threadIdx.x; L < N * N; L += blockDim.x) {
    const int i0 = L / N, i1 = L - i0 * N;
    const int a0 = i0 >> 1, b0 = (i0 + 1) >> 1, a1 = i1 >> 1, b1 = (i1 + 1) >> 1;
    const T* r00 = cin + (a0 * C + a1) * C;
    const T* r01 = cin + (a0 * C + b1) * C;
    const T* r10 = cin + (b0 * C + a1) * C;
    const T* r11 = cin + (b0 * C + b1) * C;
    T w[C];
#pragma unroll
    for (int J = 0; J < C; ++J) w[J] = T(0.25) * ((r00[J] + r01[J]) + (r10[J] + r11[J]));
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const T e = (k & 1) ? T(0.5) * (w[k / 2] + w[k / 2 + 1]) : w[k / 2];
      X[L * N + k] = e + X[L * N + k];
    }
  }
  __syncthreads();
}

template <typename T, int N, int L, int B, int MODE>
struct InvLevels {  // recompose levels L, L-1, ..., 0 (level L has N nodes)
  __device__ __forceinline__ static void run(const LevelBufs<T>& bufs, T* T1, T* T2, const double* q, int K,
                                             const void* stage, const int32_t* esc_blk, int radius) {
    const T qv = MODE == 0 ? (T)q[L] : T(0);
    level_inv<T, N, MODE>(bufs(L), T1, T2, bufs(L + 1), lvl_offset(B, L), qv, stage, esc_blk, radius);
    if constexpr (L > 0) InvLevels<T, 2 * N - 1, L - 1, B, MODE>::run(bufs, T1, T2, q, K, stage, esc_blk, radius);
  }
};

template <typename T, int B, int K, int MODE>
__global__ void __launch_bounds__(BlockCfg<T, B, K>::NT_INV, BlockCfg<T, B, K>::INV_MIN_CTAS)
    block_inv_kernel(BlockArgs<T> a) {
  using Cfg = BlockCfg<T, B, K>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* T1 = A + Cfg::A;
  T* T2 = T1 + Cfg::T1;
  T* cb0 = T2 + Cfg::T2;
  T* cb1 = cb0 + Cfg::CB0;
  void* stage = smem_raw + Cfg::inv_stage_off;
  LevelBufs<T> bufs{A, cb0, cb1};
  constexpr int M = Cfg::M;
  for (int64_t b = blockIdx.x; b < a.nblocks; b += gridDim.x) {
    const BlockCoord bc(b, a.nb1, a.nb2);
    const int64_t sbase = b * (int64_t)Cfg::PB;
    if (MODE == 0) {
#if BM_INV_CODES
      load_codes<Cfg::PB>(a.sym + sbase, a.esc + sbase, reinterpret_cast<int32_t*>(stage), a.radius);
#else
      uint16_t* st = reinterpret_cast<uint16_t*>(stage);
      const uint16_t* src = a.sym + sbase;
      if ((reinterpret_cast<uintptr_t>(src) & 3) == 0) {
        const uint32_t* s32 = reinterpret_cast<const uint32_t*>(src);
        uint32_t* d32 = reinterpret_cast<uint32_t*>(st);
        for (int i = threadIdx.x; i < Cfg::PB / 2; i += blockDim.x) d32[i] = __ldg(s32 + i);
        if ((Cfg::PB & 1) && threadIdx.x == 0) st[Cfg::PB - 1] = src[Cfg::PB - 1];
      } else {
        for (int i = threadIdx.x; i < Cfg::PB; i += blockDim.x) st[i] = src[i];
      }
#endif
    } else {
      T* st = reinterpret_cast<T*>(stage);
      for (int i = threadIdx.x; i < Cfg::PB; i += blockDim.x) st[i] = a.coef[sbase + i];
    }
    T* cf = bufs(K);
    const T* g = a.G + (((int64_t)bc.b0 * M) * a.g1 + (int64_t)bc.b1 * M) * a.g2 + (int64_t)bc.b2 * M;
    for (int e = threadIdx.x; e < M * M * M; e += blockDim.x) {
      const int j0 = e / (M * M), r = e - j0 * M * M, j1 = r / M, j2 = r - j1 * M;
      cf[e] = g[((int64_t)j0 * a.g1 + j1) * a.g2 + j2];
    }
    __syncthreads();
    int tier = (MODE == 0 && a.tier) ? a.tier[b] : 0;
    if (tier >= a.ntiers) {  // corrupt stream: keep the q reads inside the table
      if (threadIdx.x == 0 && a.sc) atomicOr(&a.sc->status, ST_CORRUPT);
      tier = 0;
    }
    InvLevels<T, M * 2 - 1, K - 1, B, MODE>::run(bufs, T1, T2, a.q + tier * K, K, stage,
                                                  MODE == 0 ? a.esc + sbase : nullptr, a.radius);
    store_block<T, B>(BlockSpan<T, B>(a.field, a.n0, a.n1, a.n2, bc), A, a.n1, a.n2);
    __syncthreads();
  }
}

}  // namespace bm
