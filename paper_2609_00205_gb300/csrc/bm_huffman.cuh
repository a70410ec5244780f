// Huffman stage (the lossless stage of the pipeline, Sec. III-B: outlier
// handling, histogram, codebook, encoding, concatenation of chunk codes).
//
// Codebook: code lengths of the two-queue Huffman construction (leaves sorted
// by (frequency, symbol); on equal weight a leaf goes before an internal
// node; internal nodes in creation order), canonical codes by (length,
// symbol), lengths above 32 bits avoided by re-running on max(1, f >> t).
// The GPU builds exactly that tree in parallel rounds: with X the sum of the
// two lightest remaining nodes, every remaining node of weight <= X is
// consumed, in merged order, before any node created from now on (new nodes
// weigh >= X and lose ties), so all those pairs are formed at once.
#pragma once

#include <stddef.h>

#include <cooperative_groups.h>

#include "bm_common.cuh"

namespace bm {

constexpr int kCbThreads = 1024;
constexpr int kLutBits = 14;
// Entries of the code table the encoder keeps in shared memory (a window of
// the dictionary), 4 bytes each.  When every present symbol lies within
// kEncWinSmall consecutive symbols, the window holds them all in CTAs of
// eight warps, four per SM (the rest of the SM's shared memory stays L1 for
// the symbol loads in flight).  Otherwise the window of the variant with
// global look-ups beside it has kEncWin entries in one CTA of kEncWarps warps
// per SM: 57,344 entries (224 KB) serve all but the far tails of a
// 65,536-symbol dictionary.  The encoder of caller-supplied symbols keeps
// kEncWinSmall entries.
#ifndef BM_ENC_WIN
#define BM_ENC_WIN 57344
#endif
constexpr int kEncWin = BM_ENC_WIN;
constexpr int kEncWarps = kEncWin > 8192 ? 32 : 8;
constexpr int kEncWinSmall = 8192;
// The window variant with global look-ups beside it is taken while its
// window (and the escape symbol's registers) serve at least BM_ENC_WIN_PCT
// percent of a call's symbols and fewer than BM_ENC_ESC_PCT percent escape.
// When escapes dominate, the other symbols are the far tails spread over the
// whole dictionary, and the global-table variant, which leaves all of L1 to
// the table, was faster on GB300 (513^3 GRF, 1e-5, 56 % escapes: 1.08 against
// 1.68 ms for the large window); at 1e-4 (no symbol spans fewer than 57,344)
// the large window took 0.52 ms, against 0.84 for the 8,192-entry one.
#ifndef BM_ENC_WIN_PCT
#define BM_ENC_WIN_PCT 50
#endif
#ifndef BM_ENC_ESC_PCT
#define BM_ENC_ESC_PCT 20
#endif
// The encoder's table entry of a symbol: its code in the low kPackBits bits
// and its length above them.  A code longer than kPackBits bits (a few
// symbols of singleton counts in fields of 10^8 symbols and more) keeps only
// its length there, and the encoder reads the code from the full code table.
constexpr unsigned kPackBits = 26;
__host__ __device__ constexpr unsigned enc_entry(unsigned code, unsigned len) {
  return (len <= kPackBits ? code : 0u) | (len << kPackBits);
}
// Shared memory of the encoder with a window of `win` entries; the variant
// for wide code distributions keeps no table in shared memory.
template <int TAB>
__host__ __device__ constexpr size_t enc_smem(int win = kEncWin) { return TAB == 2 ? 0 : (size_t)win * 4; }
// Every chunk is split into eight equal runs; the stream stores the bit
// offsets of runs 1..7 so that eight decoders can work on one chunk.
constexpr int kSplits = 8;

// Canonical-code tables shared by encoder and decoder.
struct CanonTables {
  unsigned first_code[kMaxLen + 2];
  unsigned first_pos[kMaxLen + 2];
  unsigned count[kMaxLen + 2];
  unsigned long long limit[kMaxLen + 2];  // (first_code + count) << (32 - L), left-justified
  unsigned n;                             // present symbols
  unsigned max_len;
};

struct DecodeTables {
  CanonTables ct;
  // sym | len << 16 for codes of <= kLutBits bits; for a prefix of longer
  // codes, L0 << 16 with L0 > kLutBits the length of the prefix's first code
  // (kMaxLen + 1: no code has the prefix)
  alignas(16) unsigned lut[1 << kLutBits];
  uint16_t canon[kMaxDict];     // symbols in canonical order
  // construction arrays for more present symbols than shared memory holds
  uint8_t big_clen[kMaxDict];
  uint16_t big_csym[kMaxDict];
  uint16_t big_canon[kMaxDict];
};

// ---------------------------------------------------------------------------
// Block-wide helpers (blockDim.x == kCbThreads)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* warp_tot, unsigned* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    unsigned t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;  // inclusive
  }
  __syncthreads();
  const unsigned before = (wid ? warp_tot[wid - 1] : 0u) + x - v;
  if (total && threadIdx.x == 0) *total = warp_tot[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

// Exclusive scan over the warps of a block of one count per warp (every lane
// of a warp passes the same value); returns the sum of the warps before this
// one to every lane, and the total in *total.  scan_tmp: 32 u32.
__device__ __forceinline__ unsigned warp_excl_scan_block(unsigned v, unsigned* scan_tmp, unsigned* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) scan_tmp[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const unsigned c = lane < nw ? scan_tmp[lane] : 0u;
    unsigned x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane < nw) scan_tmp[lane] = x - c;
    if (lane == 31 && total) *total = x;
  }
  __syncthreads();
  const unsigned r = scan_tmp[wid];
  __syncthreads();
  return r;
}

// Per-warp running counts of a counting pass, stored by (digit, warp) with
// the warp index swizzled by the digit so that the lanes of a warp reading
// counts of different digits hit different banks.
__device__ __forceinline__ int wc_idx(unsigned d, int w) { return (int)(d * 32u + ((unsigned)w ^ (d & 31u))); }

// Stable LSD radix sort (8-bit digits) of n <= kMaxDict (key, payload) pairs
// by key, one block of kCbThreads threads.  Warp w owns the contiguous rows
// w*rows .. w*rows+rows-1 of 32 pairs, so (warp, row, lane) is index order.
// Each pass: a counting walk (every warp ranks its rows by digit with
// __match_any_sync, keeping a running count per (digit, warp)), one block
// scan over (digit, warp) for every group's start, and a scatter walk over
// the same rows in the same order that recomputes each pair's rank (so no
// per-row state is kept in registers and n is not limited by them).  As many
// passes as maxkey has bytes.  Input in (ka, sa); returns 0 when the sorted
// pairs are in (ka, sa), 1 when in (kb, sb).  wcnt: 256 * 32 u32 of scratch.
__device__ int radix_sort_pairs(unsigned* ka, uint16_t* sa, unsigned* kb, uint16_t* sb, unsigned* wcnt, int n,
                                unsigned maxkey, unsigned* scan_tmp) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int rows = (n + kCbThreads - 1) / kCbThreads;
  const int seg = rows * 32;
  int passes = 1;
  while (passes < 4 && (maxkey >> (8 * passes)) != 0u) ++passes;
  int cur = 0;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    const unsigned* kin = cur ? kb : ka;
    const uint16_t* sin = cur ? sb : sa;
    unsigned* kout = cur ? ka : kb;
    uint16_t* sout = cur ? sa : sb;
    for (int i = threadIdx.x; i < 256 * 32; i += blockDim.x) wcnt[i] = 0u;
    __syncthreads();
    for (int r0 = 0; r0 < rows; r0 += 8) {  // counting walk, eight rows' keys loaded ahead
      unsigned kk[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int i = wid * seg + (r0 + t) * 32 + lane;
        kk[t] = (r0 + t < rows && i < n) ? kin[i] : 0u;
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (r0 + t >= rows) break;
        const int i = wid * seg + (r0 + t) * 32 + lane;
        const bool ok = i < n;
        const unsigned d = (kk[t] >> shift) & 255u;
        const unsigned m = __match_any_sync(0xffffffffu, ok ? d : 256u + (unsigned)lane);
        if (ok && (m & ((1u << lane) - 1u)) == 0u) wcnt[wc_idx(d, wid)] += (unsigned)__popc(m);
        __syncwarp();
      }
    }
    __syncthreads();
    // exclusive scan in (digit, warp) order: thread t owns entries 8t .. 8t+7
    unsigned v[8], sum = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = threadIdx.x * 8 + j;
      v[j] = wcnt[wc_idx((unsigned)k >> 5, k & 31)];
      sum += v[j];
    }
    unsigned pre = block_excl_scan(sum, scan_tmp, nullptr);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = threadIdx.x * 8 + j;
      wcnt[wc_idx((unsigned)k >> 5, k & 31)] = pre;
      pre += v[j];
    }
    __syncthreads();
    for (int r0 = 0; r0 < rows; r0 += 8) {  // scatter walk, eight rows loaded ahead
      unsigned kk[8];
      uint16_t pp[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int i = wid * seg + (r0 + t) * 32 + lane;
        const bool ok = r0 + t < rows && i < n;
        kk[t] = ok ? kin[i] : 0u;
        pp[t] = ok ? sin[i] : (uint16_t)0;
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (r0 + t >= rows) break;
        const int i = wid * seg + (r0 + t) * 32 + lane;
        const bool ok = i < n;
        const unsigned d = (kk[t] >> shift) & 255u;
        const unsigned m = __match_any_sync(0xffffffffu, ok ? d : 256u + (unsigned)lane);
        const unsigned lt = m & ((1u << lane) - 1u);
        const unsigned base = ok ? wcnt[wc_idx(d, wid)] : 0u;
        if (ok) {
          const unsigned dst = base + (unsigned)__popc(lt);
          kout[dst] = kk[t];
          sout[dst] = pp[t];
        }
        __syncwarp();
        if (ok && lt == 0u) wcnt[wc_idx(d, wid)] = base + (unsigned)__popc(m);
        __syncwarp();
      }
    }
    __syncthreads();
    cur ^= 1;
  }
  return cur;
}

__device__ __forceinline__ int upper_bound_u32(const unsigned* a, int lo, int hi, unsigned v) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}
// upper_bound by the 32 lanes of a warp (all lanes call it with the same
// arguments and get the same result): each step probes the last element of 32
// equal segments and keeps the first segment whose last element exceeds v.
__device__ __forceinline__ int warp_upper_bound_u32(const unsigned* a, int lo, int hi, unsigned v) {
  const int lane = threadIdx.x & 31;
  while (hi - lo > 32) {
    const int step = (hi - lo + 31) / 32;
    const int p = min(lo + (lane + 1) * step, hi) - 1;
    const unsigned m = __ballot_sync(0xffffffffu, a[p] > v);
    if (m == 0u) return hi;
    const int f = __ffs(m) - 1;
    const int nlo = lo + f * step;
    hi = min(nlo + step, hi);
    lo = nlo;
  }
  const unsigned m = __ballot_sync(0xffffffffu, lane < hi - lo && a[lo + lane] > v);
  return m ? lo + __ffs(m) - 1 : hi;
}
// upper_bound over the sorted a[lo, hi) by the 32 lanes of a warp, with
// samples smp[k] = a[64 k + 63] in shared memory for the blocks k < nfull (a
// last block shorter than 64 elements, if any, follows them unsampled): a
// 32-ary search of the samples finds the block that holds the bound, then one
// coalesced read of that block (the search's only global round trip).
__device__ __forceinline__ int warp_upper_bound_sampled(const unsigned* a, const unsigned* smp, int lo, int hi,
                                                        int nfull, unsigned v) {
  const int lane = threadIdx.x & 31;
  if (lo >= hi) return hi;
  int klo = lo >> 6, khi = nfull;  // the first block in [klo, khi) whose sample exceeds v, else khi
  while (khi - klo > 32) {
    const int step = (khi - klo + 31) / 32;
    const int p = min(klo + (lane + 1) * step, khi) - 1;
    const unsigned m = __ballot_sync(0xffffffffu, smp[p] > v);
    if (m == 0u) {
      klo = khi;
      break;
    }
    const int f = __ffs(m) - 1;
    const int nlo = klo + f * step;
    khi = min(nlo + step, khi);
    klo = nlo;
  }
  if (klo < khi) {
    const unsigned m = __ballot_sync(0xffffffffu, lane < khi - klo && smp[klo + lane] > v);
    klo = m ? klo + __ffs(m) - 1 : khi;
  }
  const int b0 = max(lo, klo << 6), b1 = min(hi, (klo << 6) + 64);
  if (b0 >= b1) return hi;
  const int i0 = b0 + lane, i1 = b0 + 32 + lane;
  const unsigned x0 = i0 < b1 ? a[i0] : 0u, x1 = i1 < b1 ? a[i1] : 0u;
  const unsigned m0 = __ballot_sync(0xffffffffu, i0 < b1 && x0 > v);
  if (m0) return b0 + __ffs(m0) - 1;
  const unsigned m1 = __ballot_sync(0xffffffffu, i1 < b1 && x1 > v);
  return m1 ? b0 + 32 + __ffs(m1) - 1 : hi;
}
// Merge path split by the 32 lanes of a warp: the number of A elements among
// the first d of merge(A[0..na), B[0..nb)) when A's element goes first on
// equal weight, i.e. the first i in [max(0, d - nb), min(d, na)] with
// A[i] > B[d - 1 - i] (a 32-ary search: each step probes 32 equal segments).
__device__ __forceinline__ int warp_merge_split(const unsigned* A, int na, const unsigned* B, int nb, int d) {
  const int lane = threadIdx.x & 31;
  int lo = max(0, d - nb), hi = min(d, na);
  auto after = [&](int i) { return A[i] > B[d - 1 - i]; };  // A[i] is not among the first d
  while (hi - lo > 32) {
    const int step = (hi - lo + 31) / 32;
    const int p = min(lo + (lane + 1) * step, hi) - 1;
    const unsigned m = __ballot_sync(0xffffffffu, after(p));
    if (m == 0u) return hi;
    const int f = __ffs(m) - 1;
    const int nlo = lo + f * step;
    hi = min(nlo + step, hi);
    lo = nlo;
  }
  const unsigned m = __ballot_sync(0xffffffffu, lane < hi - lo && after(lo + lane));
  return m ? lo + __ffs(m) - 1 : hi;
}

__device__ __forceinline__ int lower_bound_u32(const unsigned* a, int lo, int hi, unsigned v) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// First codes, first positions, left-justified limits, the symbol count and
// the longest length of canonical codes from the count of codes of each
// length (ct->count[1..kMaxLen], count[kMaxLen + 1] = 0); one thread.
__device__ inline void canon_from_counts(CanonTables* ct) {
  unsigned code = 0, p = 0, maxl = 0;
  ct->count[0] = 0;
  for (int L = 1; L <= kMaxLen + 1; ++L) {
    code = (code + (L > 1 ? ct->count[L - 1] : 0u)) << 1;
    if (L == 1) code = 0;
    ct->first_code[L] = code;
    ct->first_pos[L] = p;
    p += ct->count[L];
    if (ct->count[L]) maxl = L;
  }
  for (int L = 1; L <= kMaxLen; ++L) ct->limit[L] = ((unsigned long long)ct->first_code[L] + ct->count[L]) << (32 - L);
  ct->limit[kMaxLen + 1] = 1ull << 32;
  ct->n = p;
  ct->max_len = maxl;
}

// Canonical-code tables from the code lengths of the n present symbols held
// in symbol order (len[i]: length of the i-th present symbol): canon[] gets
// the indices i in (length, symbol) order, by one stable counting pass over
// the lengths (at most kMaxLen): warps rank their rows of 32 as in
// radix_sort_pairs (counting walk, scan, ranking walk), warp L-1 scans length
// L's counts over the warps, and each index lands at first_pos[len] + (indices
// of its length before it).  wcnt is scratch of at least (kMaxLen + 1) * 32 u32.
__device__ void build_canonical(const uint8_t* len, int n, unsigned* wcnt, uint16_t* canon, CanonTables* ct) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x < kMaxLen + 2) ct->count[threadIdx.x] = 0;
  for (int i = threadIdx.x; i < (kMaxLen + 1) * 32; i += blockDim.x) wcnt[i] = 0u;
  __syncthreads();
  const int rows = (n + kCbThreads - 1) / kCbThreads;
  const int seg = rows * 32;
  for (int r0 = 0; r0 < rows; r0 += 8) {
    unsigned ll[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int i = wid * seg + (r0 + t) * 32 + lane;
      ll[t] = (r0 + t < rows && i < n) ? len[i] : 0u;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if (r0 + t >= rows) break;
      const unsigned L = ll[t];
      const bool ok = L != 0u && L <= (unsigned)kMaxLen;
      const unsigned m = __match_any_sync(0xffffffffu, ok ? L : 64u + (unsigned)lane);
      if (ok && (m & ((1u << lane) - 1u)) == 0u) wcnt[wc_idx(L, wid)] += (unsigned)__popc(m);
      __syncwarp();
    }
  }
  __syncthreads();
  if (wid < kMaxLen) {  // length L = wid + 1: exclusive scan of its counts over the warps
    const unsigned L = (unsigned)wid + 1u;
    const unsigned c = wcnt[wc_idx(L, lane)];
    unsigned x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    wcnt[wc_idx(L, lane)] = x - c;
    if (lane == 31) ct->count[L] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) canon_from_counts(ct);
  __syncthreads();
  for (int r0 = 0; r0 < rows; r0 += 8) {
    unsigned ll[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int i = wid * seg + (r0 + t) * 32 + lane;
      ll[t] = (r0 + t < rows && i < n) ? len[i] : 0u;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if (r0 + t >= rows) break;
      const int i = wid * seg + (r0 + t) * 32 + lane;
      const unsigned L = ll[t];
      const bool ok = L != 0u && L <= (unsigned)kMaxLen;
      const unsigned m = __match_any_sync(0xffffffffu, ok ? L : 64u + (unsigned)lane);
      const unsigned lt = m & ((1u << lane) - 1u);
      const unsigned base = ok ? wcnt[wc_idx(L, wid)] : 0u;
      if (ok) canon[ct->first_pos[L] + base + (unsigned)__popc(lt)] = (uint16_t)i;
      __syncwarp();
      if (ok && lt == 0u) wcnt[wc_idx(L, wid)] = base + (unsigned)__popc(m);
      __syncwarp();
    }
  }
  __syncthreads();
}

struct CodebookArgs {
  const unsigned* hist;  // [dict]
  int dict;
  uint8_t* lens;         // [dict] out
  unsigned* codes;       // [dict] out
  uint8_t* out;          // stream base (codebook runs written at out + off), may be null
  unsigned long long off;
  unsigned long long capacity;
  Scalars* sc;
  int esc_mode;                  // symbol 0 is the escape of an outlier code
  unsigned long long nch;        // chunks
  unsigned long long raw_total;  // size of the raw stream (~0: no raw fallback)
  unsigned char* big;            // global scratch for more than kCbSmemSyms present symbols (cb_big_bytes())
  unsigned* packed;              // [dict] out (nullable): the encoder's entries, enc_entry(code, len)
  int presorted;                 // cb_presort_kernel ran: tables cleared, symbols compacted into the
                                 // global arrays and, above kCbSmemSyms of them, sorted
};

// Present symbols the codebook keeps in shared memory; more use global
// scratch (L2-resident) with the same code.
constexpr int kCbSmemSyms = 8192;

// Arrays of the codebook construction over the n present symbols, indexed by
// their rank in symbol order ("compact index"); node ids of the Huffman tree
// are leaves 0..n-1 (sorted order) and internal nodes n.. (creation order).
template <typename IdT>
struct CbArrays {
  uint16_t* csym;      // [n] symbol of compact index
  uint8_t* clen;       // [n] code length of compact index
  unsigned* ka;        // [n] sort keys -> sorted leaf weights (lw)
  uint16_t* sa;        // [n] compact indices -> sorted leaf order (ls)
  unsigned* kb;        // [n] sort buffer (aliases iw in shared memory)
  uint16_t* sb;        // [n] sort buffer (aliases parent in shared memory)
  unsigned* iw;        // [n] internal weights
  IdT* parent;         // [2n]
  uint8_t* depth;      // [2n]
  unsigned* wcnt;      // [256*32] sort counts (aliases round_end in shared memory)
  IdT* round_end;      // [n] internal nodes created up to the end of each round
  uint16_t* canon;     // [n] compact indices in canonical order (aliases iw)
  unsigned* run_start; // [n] compact index of each run's first symbol (aliases ka)
  unsigned* run_end;   // [n] one past its last (aliases iw, after the canonical codes are out)
  unsigned* run_off;   // [n] byte offset of the run in the codebook section (aliases wcnt)
};

// Shared-memory layout for at most kCbSmemSyms present symbols (16-bit ids).
struct CbSmem {
  unsigned ka[kCbSmemSyms];                 // 32 KB  } global-scratch variant: a tile of the
  unsigned iw[kCbSmemSyms];                 // 32 KB  } two queues (sort: kb; later canon)
  unsigned wcnt[256 * 32];                  // 32 KB (rounds: round_end u16[N])
  uint16_t parent[2 * kCbSmemSyms];         // 32 KB (sort: sb)
  uint8_t depth[2 * kCbSmemSyms];           // 16 KB
  uint16_t sa[kCbSmemSyms];                 // 16 KB
  uint16_t csym[kCbSmemSyms];               // 16 KB
  uint8_t clen[kCbSmemSyms];                //  8 KB
  unsigned scan_tmp[64];
  CanonTables ct;
};
static_assert(sizeof(CbSmem) <= 227 * 1024, "codebook shared memory");
static_assert(256 * 32 >= kCbSmemSyms, "run offsets over the sort counts");

// Shared memory of the global-scratch variant's rounds, in the arrays only
// the shared-memory variant uses: the samples of its two queues (samp, in
// parent), and per tile of merged ranks the new parent of each leaf and
// internal node taken (pa, pb: tile-relative pair index, in depth and sa)
// and the weights of the new nodes (wk, in csym), so that the global arrays
// are written with coalesced stores; after the rounds, the leaves' lengths
// (lens, over all of these arrays), copied out in compact-index order.
struct CbTileScratch {
  unsigned* samp;
  uint16_t* pa;
  uint16_t* pb;
  unsigned* wk;
  uint8_t* lens;
};
static_assert(sizeof(CbSmem::parent) >= 2 * (kMaxDict / 64) * sizeof(unsigned), "queue samples");
static_assert(sizeof(CbSmem::depth) >= kCbSmemSyms * sizeof(uint16_t) && sizeof(CbSmem::sa) >= kCbSmemSyms * 2 &&
                  sizeof(CbSmem::csym) >= kCbSmemSyms / 2 * sizeof(unsigned),
              "tile scratch");
static_assert(offsetof(CbSmem, clen) + sizeof(CbSmem::clen) - offsetof(CbSmem, parent) >= kMaxDict,
              "a length byte per leaf from parent to clen");
__device__ __forceinline__ CbTileScratch cb_tile_scratch(CbSmem& S) {
  return {reinterpret_cast<unsigned*>(S.parent), reinterpret_cast<uint16_t*>(S.depth), S.sa,
          reinterpret_cast<unsigned*>(S.csym), reinterpret_cast<uint8_t*>(S.parent)};
}

// Global scratch of the large variant: n <= kMaxDict present symbols, 32-bit ids.
constexpr int kPreCtas = 64;  // CTAs of cb_presort_kernel
// Counts of the multi-CTA presort, after the arrays in the global scratch.
struct CbPre {
  unsigned n, maxk, passes, pad;
  unsigned cnt[kPreCtas];          // present symbols of each CTA's dictionary segment
  unsigned dcnt[kPreCtas * 256];   // per (CTA, digit) keys of the current pass; then per (CTA, length) codes
  unsigned rcnt[kPreCtas];         // run starts of each CTA's segment of compact indices
  unsigned bsum[kPreCtas];         // codebook-section bytes of each CTA's runs
  unsigned long long bits, all, win;  // sums of f len, f, f served by the encoder's window
};
__host__ __device__ constexpr size_t cb_big_bytes() {
  return (size_t)kMaxDict * (2 + 1 + 4 + 2 + 4 + 2 + 4 + 4 * 2 + 2 + 4 + 2) + 3 * 4 * (size_t)kMaxDict + 16 * 256 +
         sizeof(CbPre) + 256;
}

__device__ __forceinline__ CbArrays<uint16_t> cb_small(CbSmem& S) {
  CbArrays<uint16_t> v;
  v.csym = S.csym; v.clen = S.clen; v.ka = S.ka; v.sa = S.sa;
  v.kb = S.iw; v.sb = S.parent; v.iw = S.iw; v.parent = S.parent; v.depth = S.depth;
  v.wcnt = S.wcnt;
  v.round_end = reinterpret_cast<uint16_t*>(S.wcnt);
  v.canon = reinterpret_cast<uint16_t*>(S.iw);
  v.run_start = S.ka;
  v.run_end = S.iw;
  v.run_off = S.wcnt;
  return v;
}

__device__ __forceinline__ CbArrays<unsigned> cb_big(unsigned char* g, unsigned* smem_wcnt) {
  auto take = [&](size_t bytes) {
    unsigned char* p = g;
    g += (bytes + 255) & ~size_t(255);
    return p;
  };
  const size_t N = kMaxDict;
  CbArrays<unsigned> v;
  v.csym = reinterpret_cast<uint16_t*>(take(2 * N));
  v.clen = take(N);
  v.ka = reinterpret_cast<unsigned*>(take(4 * N));
  v.sa = reinterpret_cast<uint16_t*>(take(2 * N));
  v.kb = reinterpret_cast<unsigned*>(take(4 * N));
  v.sb = reinterpret_cast<uint16_t*>(take(2 * N));
  v.iw = reinterpret_cast<unsigned*>(take(4 * N));
  v.parent = reinterpret_cast<unsigned*>(take(4 * 2 * N));
  v.depth = take(2 * N);
  v.round_end = reinterpret_cast<unsigned*>(take(4 * N));
  v.canon = reinterpret_cast<uint16_t*>(take(2 * N));
  v.run_start = reinterpret_cast<unsigned*>(take(4 * N));
  v.run_end = reinterpret_cast<unsigned*>(take(4 * N));
  v.run_off = reinterpret_cast<unsigned*>(take(4 * N));
  v.wcnt = smem_wcnt;  // the counting passes stay in shared memory
  return v;
}
// The presort's counts: after the arrays of cb_big.
__device__ __forceinline__ CbPre* cb_pre(unsigned char* g) {
  const size_t N = kMaxDict;
  size_t off = 0;
  const size_t parts[] = {2 * N, N, 4 * N, 2 * N, 4 * N, 2 * N, 4 * N, 8 * N, 2 * N, 4 * N, 2 * N, 4 * N, 4 * N, 4 * N};
  for (size_t b : parts) off += (b + 255) & ~size_t(255);
  return reinterpret_cast<CbPre*>(g + off);
}

// The codebook over the compact arrays V (n present symbols, already in
// V.csym): Huffman lengths into V.clen.  The lengths are those of the
// sequential two-queue construction; lengths above kMaxLen are avoided by
// re-running on max(1, f >> t), t = 1, 2, ...
// Ranks of a round's merged order handled per shared-memory tile by the
// global-scratch variant.
constexpr int kCbTile = 8192;
static_assert(kCbTile == kCbSmemSyms, "a tile of each queue fills ka, then iw (adjacent)");
static_assert(2 * kCbTile * sizeof(unsigned) >= kMaxDict, "the staging holds a depth byte per internal node");

// Pairs of the ranks [d0, d1) of merge(A[0..na), B[0..nb)) (A first on equal
// weight), d0 even, whose first i0 = split(d0) ranks came from A: appends
// the pairs' weights to iw at qe + rank/2 and sets the parents.  Ids: A[i] is
// node aid0 + i, B[j] is node bid0 + j.
template <typename IdT>
__device__ __forceinline__ unsigned merge_pairs(const unsigned* A, int na, const unsigned* B, int nb, int d0, int d1,
                                                int i, int aid0, int bid0, int qe, int rank0, unsigned* iw,
                                                IdT* parent, int n) {
  unsigned leaves = 0;
  int j = d0 - i;
  for (int d = d0; d < d1; d += 2) {
    int id[2];
    unsigned w[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (i < na && (j >= nb || A[i] <= B[j])) { w[t] = A[i]; id[t] = aid0 + i; ++i; ++leaves; }
      else { w[t] = B[j]; id[t] = bid0 + j; ++j; }
    }
    const int k = (rank0 + d) >> 1;
    iw[qe + k] = w[0] + w[1];
    parent[id[0]] = (IdT)(n + qe + k);
    parent[id[1]] = (IdT)(n + qe + k);
  }
  return leaves;
}
// The same pairs within one tile, their results in shared memory: pa[i] /
// pb[j], the tile-relative index of the new parent of A[i] / B[j]; wk[k], the
// weight of the tile's k-th new node.
__device__ __forceinline__ unsigned merge_pairs_tile(const unsigned* A, int na, const unsigned* B, int nb, int d0,
                                                     int d1, int i, uint16_t* pa, uint16_t* pb, unsigned* wk) {
  unsigned leaves = 0;
  int j = d0 - i;
  for (int d = d0; d < d1; d += 2) {
    unsigned w[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (i < na && (j >= nb || A[i] <= B[j])) { w[t] = A[i]; pa[i] = (uint16_t)(d >> 1); ++i; ++leaves; }
      else { w[t] = B[j]; pb[j] = (uint16_t)(d >> 1); ++j; }
    }
    wk[d >> 1] = w[0] + w[1];
  }
  return leaves;
}

// stage (global-scratch variant): shared memory for the tiles of the two
// queues; ts: its other shared memory, the samples of both queues (which turn
// each bound search into one global round trip) and the tile's results.
template <typename IdT>
__device__ void codebook_lengths(const CodebookArgs& a, CbArrays<IdT> V, int n, unsigned* scan_tmp,
                                 unsigned* stage, int pre_passes = -1, const CbTileScratch* ts = nullptr) {
  unsigned* const samp = ts ? ts->samp : nullptr;
  __shared__ unsigned s_lp, s_qp, s_qe, s_pl, s_pq, s_leaves, s_rounds, s_maxd, s_maxk;
  __shared__ int s_split;
  if (n <= 1) {
    if (n == 1 && threadIdx.x == 0) V.clen[0] = 1;
    __syncthreads();
    return;
  }
  for (int shift = 0;; ++shift) {
    const bool presorted = shift == 0 && pre_passes > 0;  // pairs sorted by cb_presort_kernel
    if (presorted && (pre_passes & 1)) {  // the sorted pairs are in (kb, sb)
      unsigned* tk = V.ka;
      V.ka = V.kb;
      V.kb = tk;
      uint16_t* ts = V.sa;
      V.sa = V.sb;
      V.sb = ts;
    }
    // 1. (freq', compact index) pairs in symbol order
    if (threadIdx.x == 0) s_maxk = 0;
    __syncthreads();
    if (!presorted) {
    unsigned mk = 0;
    for (int i0 = threadIdx.x; i0 < n; i0 += 8 * blockDim.x) {  // eight loads in flight
      unsigned sy[8], f[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int i = i0 + t * (int)blockDim.x;
        sy[t] = i < n ? (unsigned)V.csym[i] : 0u;
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) f[t] = i0 + t * (int)blockDim.x < n ? a.hist[sy[t]] : 0u;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int i = i0 + t * (int)blockDim.x;
        if (i < n) {
          const unsigned fs = shift ? max(1u, f[t] >> shift) : f[t];
          V.ka[i] = fs;
          V.sa[i] = (uint16_t)i;
          V.clen[i] = 0;
          mk = max(mk, fs);
        }
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) mk = max(mk, __shfl_xor_sync(0xffffffffu, mk, o));
    if ((threadIdx.x & 31) == 0 && mk) atomicMax(&s_maxk, mk);
    __syncthreads();
    // leaves by ascending weight, ties in symbol order, into (ka, sa) = (lw, ls)
    const int which = radix_sort_pairs(V.ka, V.sa, V.kb, V.sb, V.wcnt, n, s_maxk, scan_tmp);
    if (which) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        V.ka[i] = V.kb[i];
        V.sa[i] = V.sb[i];
      }
    }
    }  // !presorted
    const unsigned* lw = V.ka;
    const uint16_t* ls = V.sa;
    unsigned* isamp = samp ? samp + kMaxDict / 64 : nullptr;
    if (samp) {  // the leaves' samples (the last block's is the last leaf), once the sort's copies are in
      __syncthreads();
      for (int k = threadIdx.x; k < (n + 63) >> 6; k += blockDim.x) samp[k] = lw[min(64 * k + 63, n - 1)];
    }
    if (threadIdx.x == 0) { s_lp = 0; s_qp = 0; s_qe = 0; s_rounds = 0; s_leaves = 0; }
    __syncthreads();
    // 2. parallel rounds of the two-queue construction.  Warp 0 folds the
    // previous round into the queue state and picks this round's pairs: all
    // nodes of weight <= X (X = the two smallest weights summed), found by
    // warp-wide searches of both sorted queues.
    int np_prev = 0;
    while (true) {
      if (threadIdx.x == 0 && np_prev) {
        s_lp += s_leaves;
        s_qp += 2 * np_prev - s_leaves;
        s_qe += np_prev;
        V.round_end[s_rounds++] = (IdT)s_qe;
        s_leaves = 0;
      }
      __syncthreads();
      // warps 0 and 1 find, side by side, how many leaves and how many
      // internal nodes weigh at most X (both compute X)
      if (threadIdx.x < 64) {
        unsigned lp = s_lp, qp = s_qp;
        const unsigned qe = s_qe;
        if (qe < (unsigned)(n - 1)) {
          // the two smallest remaining weights: the first two of each queue,
          // read together (a weight is below 2^31, so ~0u marks an empty slot)
          const unsigned c0 = lp < (unsigned)n ? lw[lp] : ~0u, c1 = lp + 1 < (unsigned)n ? lw[lp + 1] : ~0u;
          const unsigned d0 = qp < qe ? V.iw[qp] : ~0u, d1 = qp + 1 < qe ? V.iw[qp + 1] : ~0u;
          const unsigned X = c0 <= d0 ? c0 + min(c1, d0) : d0 + min(c0, d1);
          if (threadIdx.x < 32) {
            const int pl = (samp ? warp_upper_bound_sampled(lw, samp, (int)lp, n, (n + 63) >> 6, X)
                                 : warp_upper_bound_u32(lw, (int)lp, n, X)) - (int)lp;
            if (threadIdx.x == 0) s_pl = (unsigned)pl;
          } else {
            const int pq = (samp ? warp_upper_bound_sampled(V.iw, isamp, (int)qp, (int)qe, (int)(qe >> 6), X)
                                 : warp_upper_bound_u32(V.iw, (int)qp, (int)qe, X)) - (int)qp;
            if (threadIdx.x == 32) s_pq = (unsigned)pq;
          }
        }
      }
      __syncthreads();
      if (s_qe >= (unsigned)(n - 1)) break;
      const int lp = s_lp, qp = s_qp, qe = s_qe, pl = s_pl, pq = s_pq;
      const int npairs = (pl + pq) >> 1;
      // the first 2*npairs nodes of the merged order (leaf first on equal
      // weight) pair up in order.  Merge path: thread t takes the ranks
      // [d0, d1) (d0 even), finds how many of the first d0 are leaves by one
      // binary search, then walks its ranks sequentially and forms its pairs.
      const unsigned* A = lw + lp;
      const unsigned* Bq = V.iw + qp;
      const int T = 2 * npairs;
      unsigned leaves = 0;
      if (stage == nullptr) {  // arrays in shared memory: one split per thread
        const int seg = 2 * ((npairs + (int)blockDim.x - 1) / (int)blockDim.x);
        const int d0 = min(T, (int)threadIdx.x * seg), d1 = min(T, d0 + seg);
        if (d0 < d1) {
          int lo = max(0, d0 - pq), hi = min(d0, pl);
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (A[mid] <= Bq[d0 - 1 - mid]) lo = mid + 1; else hi = mid;
          }
          leaves = merge_pairs<IdT>(A, pl, Bq, pq, d0, d1, lo, lp, n + qp, qe, 0, V.iw, V.parent, n);
        }
      } else {  // arrays in global memory: tiles of kCbTile ranks staged in shared memory
        unsigned* sA = stage;
        unsigned* sB = stage + kCbTile;
        int ia = 0;
        for (int tb = 0; tb < T; tb += kCbTile) {
          const int te = min(T, tb + kCbTile);
          if (te == pl + pq) {  // every node of both queues
            if (threadIdx.x == 0) s_split = pl;
          } else if (te == T) {  // all but the last of the merged order (A first on equal weight)
            if (threadIdx.x == 0) s_split = pq == 0 ? pl - 1 : pl == 0 ? 0 : A[pl - 1] <= Bq[pq - 1] ? pl : pl - 1;
          } else if (threadIdx.x < 32) {
            const int ib = warp_merge_split(A, pl, Bq, pq, te);
            if (threadIdx.x == 0) s_split = ib;
          }
          __syncthreads();
          const int ib = s_split, ja = tb - ia, jb = te - ib;
          for (int k0 = threadIdx.x; k0 < ib - ia; k0 += 8 * blockDim.x) {  // eight loads in flight
            unsigned x[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              const int k = k0 + t * (int)blockDim.x;
              x[t] = k < ib - ia ? A[ia + k] : 0u;
            }
#pragma unroll
            for (int t = 0; t < 8; ++t)
              if (k0 + t * (int)blockDim.x < ib - ia) sA[k0 + t * blockDim.x] = x[t];
          }
          for (int k0 = threadIdx.x; k0 < jb - ja; k0 += 8 * blockDim.x) {
            unsigned x[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              const int k = k0 + t * (int)blockDim.x;
              x[t] = k < jb - ja ? Bq[ja + k] : 0u;
            }
#pragma unroll
            for (int t = 0; t < 8; ++t)
              if (k0 + t * (int)blockDim.x < jb - ja) sB[k0 + t * blockDim.x] = x[t];
          }
          __syncthreads();
          const int tl = te - tb, na = ib - ia, nb = jb - ja;
          const int seg = 2 * ((tl / 2 + (int)blockDim.x - 1) / (int)blockDim.x);
          const int d0 = min(tl, (int)threadIdx.x * seg), d1 = min(tl, d0 + seg);
          if (d0 < d1) {
            int lo = max(0, d0 - nb), hi = min(d0, na);
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (sA[mid] <= sB[d0 - 1 - mid]) lo = mid + 1; else hi = mid;
            }
            leaves += merge_pairs_tile(sA, na, sB, nb, d0, d1, lo, ts->pa, ts->pb, ts->wk);
          }
          __syncthreads();
          // the tile's parents and new weights, coalesced
          const int kb0 = qe + (tb >> 1);
          for (int k = threadIdx.x; k < na; k += blockDim.x) V.parent[lp + ia + k] = (IdT)(n + kb0 + ts->pa[k]);
          for (int k = threadIdx.x; k < nb; k += blockDim.x) V.parent[n + qp + ja + k] = (IdT)(n + kb0 + ts->pb[k]);
          for (int k = threadIdx.x; k < (tl >> 1); k += blockDim.x) {
            const unsigned w = ts->wk[k];
            V.iw[kb0 + k] = w;
            if (((kb0 + k) & 63) == 63) isamp[(kb0 + k) >> 6] = w;
          }
          ia = ib;
          __syncthreads();
        }
      }
      if (leaves) atomicAdd(&s_leaves, leaves);
      np_prev = npairs;
      __syncthreads();
    }
    // 3. depths, rounds in reverse (a parent is always created in a later
    // round).  The global-scratch variant keeps the internal nodes' depths in
    // the tile staging's shared memory (one byte each: a depth stays below 64
    // for counts below 2^32), indexed by creation order.
    const int root = 2 * n - 2;
    uint8_t* const dsh = stage ? reinterpret_cast<uint8_t*>(stage) : nullptr;
    if (threadIdx.x == 0) {
      if (dsh) dsh[n - 2] = 0;
      else V.depth[root] = 0;
      s_maxd = 0;
    }
    __syncthreads();
    for (int r = (int)s_rounds - 1; r >= 0; --r) {
      const int jb = r ? (int)V.round_end[r - 1] : 0, je = (int)V.round_end[r];
      for (int j = jb + threadIdx.x; j < je; j += blockDim.x) {
        const int v = n + j;
        if (v != root) {
          if (dsh) dsh[j] = (uint8_t)(dsh[(int)V.parent[v] - n] + 1);
          else V.depth[v] = V.depth[V.parent[v]] + 1;
        }
      }
      __syncthreads();
    }
    unsigned md = 0;
    for (int i0 = threadIdx.x; i0 < n; i0 += 8 * blockDim.x) {  // eight loads in flight
      unsigned pa[8], li[8], dd[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int i = i0 + t * (int)blockDim.x;
        pa[t] = i < n ? (unsigned)V.parent[i] : 0u;
        li[t] = i < n ? (unsigned)ls[i] : 0u;
      }
#pragma unroll
      for (int t = 0; t < 8; ++t)
        dd[t] = i0 + t * (int)blockDim.x < n ? (unsigned)(dsh ? dsh[pa[t] - (unsigned)n] : V.depth[pa[t]]) + 1u : 0u;
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (i0 + t * (int)blockDim.x < n) {
          // the global-scratch variant gathers the lengths in shared memory
          // (scattered byte stores), then copies them out in order
          if (ts) ts->lens[li[t]] = (uint8_t)min(dd[t], 255u);
          else V.clen[li[t]] = (uint8_t)min(dd[t], 255u);
          md = max(md, dd[t]);
        }
    }
    if (md) atomicMax(&s_maxd, md);
    __syncthreads();
    if (ts) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) V.clen[i] = ts->lens[i];
      __syncthreads();
    }
    if (s_maxd <= (unsigned)kMaxLen) break;
    __syncthreads();
  }
}

// The codebook's decisions (one thread): section sizes and offsets, the
// encoder's table and window, the lower bound on the stream size and the
// raw-copy decision.  smin / smax: the smallest and largest present symbol;
// bits, all, win: sum of f_s len_s, of f_s, and of f_s over the symbols the
// encoder's centred window (or the escape registers) serves.
__device__ inline void codebook_decide(const CodebookArgs& a, unsigned smin, unsigned smax, unsigned long long total,
                                       int nruns, unsigned max_len, unsigned long long bits, unsigned long long all,
                                       unsigned long long win, bool fits) {
  const unsigned wlo_c =
      a.dict <= kEncWin ? 0u : (unsigned)min(max(a.dict / 2 - kEncWin / 2, 0), a.dict - kEncWin);
  {
    Scalars* sc = a.sc;
    sc->codebook_bytes = total;
    sc->n_runs = (unsigned long long)nruns;
    sc->max_len = max_len;
    // the encoder's shared-memory window of the code table: every present
    // symbol when they span at most kEncWinSmall symbols, or at most kEncWin
    // (a larger window in a larger CTA); else kEncWin entries centred on the dictionary's middle (code 0) while they and the
    // escape symbol serve at least BM_ENC_WIN_PCT percent of the symbols met
    // and escapes are fewer than BM_ENC_ESC_PCT percent (the rest looked up
    // in the global table); else no window (the global-table variant, with
    // all of L1 for the table)
    unsigned wn = kEncWin;
    if (smax - smin < (unsigned)kEncWinSmall) {
      sc->enc_lo = a.dict <= kEncWinSmall ? 0u : min(smin, (unsigned)(a.dict - kEncWinSmall));
      sc->enc_mode = 0;
      wn = kEncWinSmall;
    } else if (smax - smin < (unsigned)kEncWin) {
      sc->enc_lo = a.dict <= kEncWin ? 0u : min(smin, (unsigned)(a.dict - kEncWin));
      sc->enc_mode = 3;
    } else if (win * 100ull >= (unsigned long long)BM_ENC_WIN_PCT * all &&
               (unsigned long long)a.hist[0] * 100ull < (unsigned long long)BM_ENC_ESC_PCT * all) {
      sc->enc_lo = wlo_c;
      sc->enc_mode = 1;
    } else {
      sc->enc_lo = 0;
      sc->enc_mode = 2;
    }
    // the window's entries above the largest present symbol are never read
    sc->enc_n = smax >= sc->enc_lo ? min(wn, smax + 1u - sc->enc_lo) : 0u;
    if (a.out && !fits) atomicOr(&sc->status, ST_CAPACITY | ST_RAW);
    const unsigned long long nout = a.esc_mode ? (unsigned long long)a.hist[0] : 0ull;
    const unsigned long long off_ce = a.off + pad8(total);
    const unsigned long long off_out = off_ce + (nout ? pad8(4ull * a.nch) : 0ull);
    const unsigned long long off_bits = off_out + pad8(4ull * nout);
    const unsigned long long min_total = off_bits + pad8(4ull * ((bits + 31ull) / 32ull));
    sc->n_outliers = nout;
    sc->off_chunk_esc = off_ce;
    sc->off_outliers = off_out;
    sc->off_bits = off_bits;
    // a quantisation overflow, a size bound at or above the raw copy, or sections
    // that do not fit all make the stream a raw copy: skip the encoder
    if ((sc->status & ST_OVERFLOW) || min_total >= a.raw_total || off_bits > a.capacity) atomicOr(&sc->status, ST_RAW);
    sc->skip = (sc->status & ST_RAW) ? 1u : 0u;
  }
}

// Canonical codes, the lookup tables of the encoder, the codebook section of
// the stream and the offsets of the sections after it, from the lengths.
template <typename IdT>
__device__ void codebook_emit(const CodebookArgs& a, CbArrays<IdT> V, int n, unsigned* scan_tmp, CanonTables* ct) {
  __shared__ unsigned s_total, s_nruns;
  __shared__ unsigned long long s_bits, s_all, s_win;
  if (threadIdx.x == 0) { s_bits = 0; s_all = 0; s_win = 0; }
  // 4. canonical codes (the counting pass in the sort counts' shared memory)
  build_canonical(V.clen, n, V.wcnt, V.canon, ct);
  const bool pk = a.packed != nullptr;
  const int nc = (int)ct->n;
  for (int i0 = threadIdx.x; i0 < nc; i0 += 8 * blockDim.x) {  // eight loads in flight
    unsigned ci[8], L[8], sy[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int i = i0 + t * (int)blockDim.x;
      ci[t] = i < nc ? (unsigned)V.canon[i] : 0u;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const bool ok = i0 + t * (int)blockDim.x < nc;
      L[t] = ok ? (unsigned)V.clen[ci[t]] : 0u;
      sy[t] = ok ? (unsigned)V.csym[ci[t]] : 0u;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int i = i0 + t * (int)blockDim.x;
      if (i < nc) {
        const unsigned c = ct->first_code[L[t]] + (unsigned)(i - (int)ct->first_pos[L[t]]);
        a.codes[sy[t]] = c;
        if (pk) a.packed[sy[t]] = enc_entry(c, L[t]);
        a.lens[sy[t]] = (uint8_t)L[t];
      }
    }
  }
  // 5. codebook runs {u32 first, u32 count, u8 len[count], pad to 4}: a run
  // starts at every present symbol whose predecessor is absent.  Warp w walks
  // its contiguous rows of 32 compact indices (coalesced loads): run starts
  // by ballot, one scan over the warps, then each start's run index.
  unsigned* run_start = V.run_start;
  unsigned* run_end = V.run_end;
  unsigned* run_off = V.run_off;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int rows = (n + 31) / 32, rpw = (rows + nwarps - 1) / nwarps;
  const int r0 = wid * rpw, r1 = min(rows, r0 + rpw);
  // run-start masks of eight rows at once (sixteen loads in flight)
  auto start_masks = [&](int r, unsigned (&m)[8]) {
    unsigned c[8], p[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int i = (r + t) * 32 + lane;
      const bool ok = r + t < r1 && i < n;
      c[t] = ok ? (unsigned)V.csym[i] : 0u;
      p[t] = ok && i > 0 ? (unsigned)V.csym[i - 1] : 0u;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int i = (r + t) * 32 + lane;
      m[t] = __ballot_sync(0xffffffffu, r + t < r1 && i < n && (i == 0 || c[t] != p[t] + 1u));
    }
  };
  unsigned nst = 0;
  for (int r = r0; r < r1; r += 8) {
    unsigned m[8];
    start_masks(r, m);
#pragma unroll
    for (int t = 0; t < 8; ++t) nst += (unsigned)__popc(m[t]);
  }
  const unsigned rbase = warp_excl_scan_block(nst, scan_tmp, &s_nruns);
  {
    unsigned q = rbase;
    for (int r = r0; r < r1; r += 8) {
      unsigned m[8];
      start_masks(r, m);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if ((m[t] >> lane) & 1u)
          run_start[q + (unsigned)__popc(m[t] & ((1u << lane) - 1u))] = (unsigned)((r + t) * 32 + lane);
        q += (unsigned)__popc(m[t]);
      }
    }
  }
  __syncthreads();
  const int nruns = (int)s_nruns;
  for (int q = threadIdx.x; q < nruns; q += blockDim.x) run_end[q] = q + 1 < nruns ? run_start[q + 1] : (unsigned)n;
  __syncthreads();
  unsigned my_bytes = 0;
  const int rper = (nruns + blockDim.x - 1) / blockDim.x;
  const int q0 = threadIdx.x * rper;
  for (int q = q0; q < q0 + rper && q < nruns; ++q) my_bytes += 8u + (((run_end[q] - run_start[q]) + 3u) & ~3u);
  unsigned off = block_excl_scan(my_bytes, scan_tmp, &s_total);
  for (int q = q0; q < q0 + rper && q < nruns; ++q) {
    run_off[q] = off;
    off += 8u + (((run_end[q] - run_start[q]) + 3u) & ~3u);
  }
  __syncthreads();
  const unsigned long long total = s_total;
  const bool fits = a.out && a.off + pad8(total) <= a.capacity;
  if (fits) {
    for (int q = threadIdx.x; q < nruns; q += blockDim.x) {
      const unsigned first = run_start[q], cntq = run_end[q] - first;
      uint8_t* p = a.out + a.off + run_off[q];
      *reinterpret_cast<unsigned*>(p) = (unsigned)V.csym[first];
      *reinterpret_cast<unsigned*>(p + 4) = cntq;
      for (unsigned t = cntq; t < ((cntq + 3u) & ~3u); ++t) p[8 + t] = 0;
    }
    // length bytes: compact index i of run q goes to run_off[q] + 8 + (i -
    // run_start[q]), q = (run starts up to i) - 1, from the same row walk
    unsigned q = rbase;
    for (int r = r0; r < r1; r += 8) {
      unsigned m[8], qi[8], ro[8], rs[8], cl[8];
      start_masks(r, m);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        qi[t] = q + (unsigned)__popc(m[t] & ((2u << lane) - 1u)) - 1u;
        q += (unsigned)__popc(m[t]);
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int i = (r + t) * 32 + lane;
        const bool ok = r + t < r1 && i < n;
        ro[t] = ok ? run_off[qi[t]] : 0u;
        rs[t] = ok ? run_start[qi[t]] : 0u;
        cl[t] = ok ? (unsigned)V.clen[i] : 0u;
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int i = (r + t) * 32 + lane;
        if (r + t < r1 && i < n) a.out[a.off + ro[t] + 8 + (i - rs[t])] = (uint8_t)cl[t];
      }
    }
    if (threadIdx.x == 0)
      for (unsigned long long t = total; t < pad8(total); ++t) a.out[a.off + t] = 0;
  }
  // 6. layout of the rest of the stream (escape counts, outlier codes, then
  // the bitstream) and a lower bound on its size: the bitstream holds exactly
  // sum_s f_s len_s bits plus the padding of each chunk to whole words
  // (and the symbols met that the encoder's window centred on code 0, or the
  // escape symbol's registers, serve)
  const unsigned wlo_c =
      a.dict <= kEncWin ? 0u : (unsigned)min(max(a.dict / 2 - kEncWin / 2, 0), a.dict - kEncWin);
  unsigned long long my_bits = 0, my_all = 0, my_win = 0;
  for (int i0 = threadIdx.x; i0 < n; i0 += 8 * blockDim.x) {  // eight loads in flight
    unsigned sy[8], cl[8], f[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int i = i0 + t * (int)blockDim.x;
      sy[t] = i < n ? (unsigned)V.csym[i] : 0u;
      cl[t] = i < n ? (unsigned)V.clen[i] : 0u;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) f[t] = i0 + t * (int)blockDim.x < n ? a.hist[sy[t]] : 0u;
#pragma unroll
    for (int t = 0; t < 8; ++t)
      if (i0 + t * (int)blockDim.x < n) {
        my_bits += (unsigned long long)f[t] * cl[t];
        my_all += f[t];
        if (sy[t] - wlo_c < (unsigned)kEncWin || sy[t] == 0u) my_win += f[t];
      }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    my_bits += __shfl_xor_sync(0xffffffffu, my_bits, o);
    my_all += __shfl_xor_sync(0xffffffffu, my_all, o);
    my_win += __shfl_xor_sync(0xffffffffu, my_win, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (my_bits) atomicAdd(&s_bits, my_bits);
    if (my_all) atomicAdd(&s_all, my_all);
    if (my_win) atomicAdd(&s_win, my_win);
  }
  __syncthreads();
  if (threadIdx.x == 0)
    codebook_decide(a, n ? V.csym[0] : 0u, n ? V.csym[n - 1] : 0u, total, nruns, ct->max_len, s_bits, s_all, s_win,
                    fits);
}

// Multi-CTA start of the codebook for wide code distributions: one
// cooperative launch of kPreCtas CTAs with grid-wide barriers between the
// phases.  It clears the code tables, compacts the present symbols (symbol
// order) into the global arrays with their frequencies as keys, the compact
// index as payload and zero lengths, and, when more than kCbSmemSyms symbols
// are present, sorts the pairs by key, stably, with 8-bit LSD passes: each
// CTA owns a contiguous segment of the pairs; a pass counts the segment's
// digits, and after the barrier thread d of each CTA walks its segment (staged
// in shared memory) in order and places the keys of digit d at the digit's
// global offset (all keys of smaller digits, then those of digit d in the
// CTAs before), so equal keys keep their order.  The sorted pairs are in
// (ka, sa) after an even number of passes and in (kb, sb) after an odd one
// (CbPre::passes; 0 when the codebook kernel sorts in shared memory itself).
constexpr int kPreThreads = 256;
constexpr int kPreSeg = kMaxDict / kPreCtas;  // pairs per CTA at most
__global__ void __launch_bounds__(kPreThreads) cb_presort_kernel(CodebookArgs a) {
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  CbPre* pre = cb_pre(a.big);
  const CbArrays<unsigned> V = cb_big(a.big, nullptr);
  const int dict = a.dict, c = blockIdx.x, G = gridDim.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ unsigned s_red[kPreThreads / 32];
  __shared__ unsigned s_scan[kPreThreads];
  __shared__ unsigned s_dc[256];
  __shared__ unsigned s_key[kPreSeg];
  __shared__ uint16_t s_val[kPreSeg];
  __shared__ unsigned s_base, s_n, s_maxk;
  auto block_sum = [&](unsigned v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    unsigned t = 0;
    for (int w = 0; w < kPreThreads / 32; ++w) t += s_red[w];
    return t;
  };
  auto block_excl = [&](unsigned v, unsigned* total) {  // exclusive scan over the block's threads
    s_scan[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kPreThreads; o <<= 1) {
      const unsigned y = threadIdx.x >= (unsigned)o ? s_scan[threadIdx.x - o] : 0u;
      __syncthreads();
      s_scan[threadIdx.x] += y;
      __syncthreads();
    }
    const unsigned incl = s_scan[threadIdx.x];
    if (total) *total = s_scan[kPreThreads - 1];
    __syncthreads();
    return incl - v;
  };
  // 0. tables cleared; present symbols of this CTA's dictionary segment counted
  for (int s = c * kPreThreads + threadIdx.x; s < dict; s += G * kPreThreads) {
    a.lens[s] = 0;
    a.codes[s] = 0;
    if (a.packed) a.packed[s] = 0;
  }
  const int dseg = (dict + G - 1) / G, d0 = min(dict, c * dseg), d1 = min(dict, d0 + dseg);
  unsigned my = 0;
  for (int s = d0 + threadIdx.x; s < d1; s += kPreThreads) my += a.hist[s] != 0u;
  const unsigned cnt = block_sum(my);
  if (threadIdx.x == 0) {
    pre->cnt[c] = cnt;
    if (c == 0) {
      pre->maxk = 0;
      pre->bits = 0;
      pre->all = 0;
      pre->win = 0;
    }
  }
  grid.sync();
  // 1. compaction in symbol order: (frequency, compact index) pairs
  if (threadIdx.x == 0) {
    unsigned b = 0, t = 0;
    for (int k = 0; k < G; ++k) {
      const unsigned v = pre->cnt[k];
      if (k < c) b += v;
      t += v;
    }
    s_base = b;
    s_n = t;
  }
  __syncthreads();
  unsigned pos = s_base, mk = 0;
  for (int s0 = d0; s0 < d1; s0 += kPreThreads) {
    const int s = s0 + threadIdx.x;
    const unsigned f = s < d1 ? a.hist[s] : 0u;
    unsigned tot = 0;
    const unsigned r = block_excl(f != 0u ? 1u : 0u, &tot);
    if (f) {
      const unsigned i = pos + r;
      V.csym[i] = (uint16_t)s;
      V.clen[i] = 0;
      V.ka[i] = f;
      V.sa[i] = (uint16_t)i;
      mk = max(mk, f);
    }
    pos += tot;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) mk = max(mk, __shfl_xor_sync(0xffffffffu, mk, o));
  if (lane == 0 && mk) atomicMax(&pre->maxk, mk);
  if (c == 0 && threadIdx.x == 0) pre->n = s_n;
  grid.sync();
  const int n = (int)s_n;
  if (threadIdx.x == 0) s_maxk = pre->maxk;
  __syncthreads();
  int passes = 0;
  if (n > kCbSmemSyms) {
    passes = 1;
    while (passes < 4 && (s_maxk >> (8 * passes)) != 0u) ++passes;
  }
  if (c == 0 && threadIdx.x == 0) pre->passes = (unsigned)passes;
  const int pseg = (n + G - 1) / G, p0 = min(n, c * pseg), p1 = min(n, p0 + pseg);
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    const unsigned* kin = (p & 1) ? V.kb : V.ka;
    const uint16_t* sin = (p & 1) ? V.sb : V.sa;
    unsigned* kout = (p & 1) ? V.ka : V.kb;
    uint16_t* sout = (p & 1) ? V.sa : V.sb;
    // the segment staged, its digits counted
    s_dc[threadIdx.x] = 0u;
    __syncthreads();
    for (int i = p0 + threadIdx.x; i < p1; i += kPreThreads) {
      const unsigned k = kin[i];
      s_key[i - p0] = k;
      s_val[i - p0] = sin[i];
      atomicAdd(&s_dc[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    pre->dcnt[c * 256 + threadIdx.x] = s_dc[threadIdx.x];
    grid.sync();
    // offsets of digit d (thread d): keys of smaller digits, then of digit d
    // in the CTAs before this one
    const unsigned d = threadIdx.x;
    unsigned col = 0, part = 0;
    for (int k = 0; k < G; ++k) {
      const unsigned v = pre->dcnt[k * 256 + d];
      if (k < c) part += v;
      col += v;
    }
    unsigned off = block_excl(col, nullptr) + part;
    for (int i = 0; i < p1 - p0; ++i) {
      const unsigned k = s_key[i];
      if (((k >> shift) & 255u) == d) {
        kout[off] = k;
        sout[off] = s_val[i];
        ++off;
      }
    }
    grid.sync();
  }
}

// Multi-CTA end of the codebook for wide code distributions (after the one-CTA
// tree, above kCbSmemSyms present symbols; cooperative launch of kPreCtas
// CTAs, grid-wide barriers between the phases): what codebook_emit does, each
// CTA over its segment of compact indices.  Canonical order: per-(CTA,
// length) counts, then thread L of each CTA places its segment's indices of
// length L in order (symbol order within a length).  Runs of consecutive
// present symbols: per-CTA start counts give each start's run index; the
// runs' section bytes are summed per CTA for their offsets.  The sums of the
// size bound and of the encoder's window go to global atomics; CTA 0 makes
// the decisions.
__global__ void __launch_bounds__(kPreThreads) cb_emit_kernel(CodebookArgs a) {
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  CbPre* pre = cb_pre(a.big);
  const CbArrays<unsigned> V = cb_big(a.big, nullptr);
  const int n = (int)pre->n;
  if (n <= kCbSmemSyms) return;  // the one-CTA kernel emitted everything (the same for every CTA)
  const int c = blockIdx.x, G = gridDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  __shared__ uint8_t s_len[kPreSeg];
  __shared__ uint16_t s_sym[kPreSeg];
  __shared__ unsigned s_lc[kMaxLen + 2];
  __shared__ unsigned s_scan[kPreThreads];
  __shared__ unsigned s_red[kPreThreads / 32];
  __shared__ unsigned long long s_r64[3][kPreThreads / 32];
  __shared__ CanonTables s_ct;
  __shared__ unsigned s_prev, s_rbase, s_nruns, s_boff, s_total;
  auto block_excl = [&](unsigned v, unsigned* total) {
    s_scan[tid] = v;
    __syncthreads();
    for (int o = 1; o < kPreThreads; o <<= 1) {
      const unsigned y = tid >= o ? s_scan[tid - o] : 0u;
      __syncthreads();
      s_scan[tid] += y;
      __syncthreads();
    }
    const unsigned incl = s_scan[tid];
    if (total) *total = s_scan[kPreThreads - 1];
    __syncthreads();
    return incl - v;
  };
  const int pseg = (n + G - 1) / G, e0 = min(n, c * pseg), e1 = min(n, e0 + pseg), m = e1 - e0;
  // E0: the segment staged; its length counts, run starts and size sums
  if (tid < kMaxLen + 2) s_lc[tid] = 0u;
  if (tid == 0) s_prev = e0 > 0 ? (unsigned)V.csym[e0 - 1] : 0u;
  __syncthreads();
  const unsigned wlo_c =
      a.dict <= kEncWin ? 0u : (unsigned)min(max(a.dict / 2 - kEncWin / 2, 0), a.dict - kEncWin);
  unsigned long long my_bits = 0, my_all = 0, my_win = 0;
  for (int i = tid; i < m; i += kPreThreads) {
    const unsigned L = V.clen[e0 + i], sy = V.csym[e0 + i];
    s_len[i] = (uint8_t)L;
    s_sym[i] = (uint16_t)sy;
    if (L >= 1u && L <= (unsigned)kMaxLen) atomicAdd(&s_lc[L], 1u);
    const unsigned long long f = a.hist[sy];
    my_bits += f * L;
    my_all += f;
    if (sy - wlo_c < (unsigned)kEncWin || sy == 0u) my_win += f;
  }
  __syncthreads();
  auto is_start = [&](int i) {  // i: index within the segment
    return e0 + i == 0 || (unsigned)s_sym[i] != (i ? (unsigned)s_sym[i - 1] : s_prev) + 1u;
  };
  unsigned my_st = 0;
  for (int i = tid; i < m; i += kPreThreads) my_st += is_start(i);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    my_bits += __shfl_xor_sync(0xffffffffu, my_bits, o);
    my_all += __shfl_xor_sync(0xffffffffu, my_all, o);
    my_win += __shfl_xor_sync(0xffffffffu, my_win, o);
    my_st += __shfl_xor_sync(0xffffffffu, my_st, o);
  }
  if (lane == 0) {
    s_r64[0][wid] = my_bits;
    s_r64[1][wid] = my_all;
    s_r64[2][wid] = my_win;
    s_red[wid] = my_st;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long b = 0, al = 0, w = 0;
    unsigned st = 0;
    for (int k = 0; k < kPreThreads / 32; ++k) {
      b += s_r64[0][k];
      al += s_r64[1][k];
      w += s_r64[2][k];
      st += s_red[k];
    }
    atomicAdd(&pre->bits, b);
    atomicAdd(&pre->all, al);
    atomicAdd(&pre->win, w);
    pre->rcnt[c] = st;
  }
  if (tid < kMaxLen + 2) pre->dcnt[c * 256 + tid] = s_lc[tid];
  grid.sync();
  // E1: canonical tables (every CTA, the same), this segment's canonical
  // positions; run bases
  unsigned part = 0;
  if (tid <= kMaxLen + 1) {
    unsigned tot = 0;
    for (int k = 0; k < G; ++k) {
      const unsigned v = pre->dcnt[k * 256 + tid];
      if (k < c) part += v;
      tot += v;
    }
    s_ct.count[tid] = tid == 0 || tid == kMaxLen + 1 ? 0u : tot;
  }
  if (tid == 0) {
    unsigned rb = 0, rt = 0;
    for (int k = 0; k < G; ++k) {
      const unsigned v = pre->rcnt[k];
      if (k < c) rb += v;
      rt += v;
    }
    s_rbase = rb;
    s_nruns = rt;
  }
  __syncthreads();
  if (tid == 0) canon_from_counts(&s_ct);
  __syncthreads();
  if (tid >= 1 && tid <= kMaxLen) {
    unsigned pos = s_ct.first_pos[tid] + part;
    for (int i = 0; i < m; ++i)
      if (s_len[i] == (unsigned)tid) V.canon[pos++] = (uint16_t)(e0 + i);
  }
  const int nruns = (int)s_nruns;
  {  // run starts of the segment at their run indices
    unsigned q = s_rbase;
    for (int i0 = 0; i0 < m; i0 += kPreThreads) {
      const int i = i0 + tid;
      const bool st = i < m && is_start(i);
      unsigned tot = 0;
      const unsigned r = block_excl(st ? 1u : 0u, &tot);
      if (st) V.run_start[q + r] = (unsigned)(e0 + i);
      q += tot;
    }
  }
  grid.sync();
  // E2: code tables over the canonical order; section bytes of this CTA's runs
  const bool pk = a.packed != nullptr;
  for (int i = c * kPreThreads + tid; i < n; i += G * kPreThreads) {
    const unsigned ci = V.canon[i];
    const unsigned L = V.clen[ci];
    const unsigned cd = s_ct.first_code[L] + (unsigned)(i - (int)s_ct.first_pos[L]);
    const unsigned sy = V.csym[ci];
    a.codes[sy] = cd;
    if (pk) a.packed[sy] = enc_entry(cd, L);
    a.lens[sy] = (uint8_t)L;
  }
  const int rq = (nruns + G - 1) / G, q0 = min(nruns, c * rq), q1 = min(nruns, q0 + rq);
  unsigned my_b = 0;
  for (int q = q0 + tid; q < q1; q += kPreThreads) {
    const unsigned st = V.run_start[q], en = q + 1 < nruns ? V.run_start[q + 1] : (unsigned)n;
    V.run_end[q] = en;
    my_b += 8u + (((en - st) + 3u) & ~3u);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) my_b += __shfl_xor_sync(0xffffffffu, my_b, o);
  if (lane == 0) s_red[wid] = my_b;
  __syncthreads();
  if (tid == 0) {
    unsigned t = 0;
    for (int k = 0; k < kPreThreads / 32; ++k) t += s_red[k];
    pre->bsum[c] = t;
  }
  grid.sync();
  // E3: run offsets and headers
  if (tid == 0) {
    unsigned b = 0, t = 0;
    for (int k = 0; k < G; ++k) {
      const unsigned v = pre->bsum[k];
      if (k < c) b += v;
      t += v;
    }
    s_boff = b;
    s_total = t;
  }
  __syncthreads();
  const unsigned long long total = s_total;
  const bool fits = a.out && a.off + pad8(total) <= a.capacity;
  {
    unsigned off = s_boff;
    for (int qb = q0; qb < q1; qb += kPreThreads) {
      const int q = qb + tid;
      const unsigned st = q < q1 ? V.run_start[q] : 0u, en = q < q1 ? V.run_end[q] : 0u;
      const unsigned bq = q < q1 ? 8u + (((en - st) + 3u) & ~3u) : 0u;
      unsigned tot = 0;
      const unsigned r = block_excl(bq, &tot);
      if (q < q1) {
        V.run_off[q] = off + r;
        if (fits) {
          uint8_t* p = a.out + a.off + off + r;
          *reinterpret_cast<unsigned*>(p) = (unsigned)V.csym[st];
          *reinterpret_cast<unsigned*>(p + 4) = en - st;
          for (unsigned t = en - st; t < (((en - st) + 3u) & ~3u); ++t) p[8 + t] = 0;
        }
      }
      off += tot;
    }
  }
  grid.sync();
  // E4: the length bytes, each at its run's offset; CTA 0's decisions
  if (fits) {
    unsigned q = s_rbase;  // run index of the next start
    for (int i0 = 0; i0 < m; i0 += kPreThreads) {
      const int i = i0 + tid;
      const bool st = i < m && is_start(i);
      unsigned tot = 0;
      const unsigned r = block_excl(st ? 1u : 0u, &tot);
      if (i < m) {
        const unsigned qi = q + r + (st ? 1u : 0u) - 1u;  // starts up to and including i, minus one
        a.out[a.off + V.run_off[qi] + 8 + ((unsigned)(e0 + i) - V.run_start[qi])] = s_len[i];
      }
      q += tot;
    }
    if (c == 0 && tid == 0)
      for (unsigned long long t = total; t < pad8(total); ++t) a.out[a.off + t] = 0;
  }
  if (c == 0 && tid == 0)
    codebook_decide(a, V.csym[0], V.csym[n - 1], total, nruns, s_ct.max_len, pre->bits, pre->all, pre->win, fits);
}

// The codebook of one compress call, built by one CTA (the whole block).
__device__ void codebook_block(const CodebookArgs& a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CbSmem& S = *reinterpret_cast<CbSmem*>(smem_raw);
  __shared__ unsigned s_n;
  const int dict = a.dict;
  if (a.presorted) {  // cb_presort_kernel cleared the tables and compacted the symbols
    const CbPre* pre = cb_pre(a.big);
    const int n = (int)pre->n;
    const int passes = (int)pre->passes;
    if (n <= kCbSmemSyms) {
      const uint16_t* gsym = cb_big(a.big, S.wcnt).csym;
      for (int i = threadIdx.x; i < n; i += blockDim.x) S.csym[i] = gsym[i];
      __syncthreads();
      const CbArrays<uint16_t> V = cb_small(S);
      codebook_lengths<uint16_t>(a, V, n, S.scan_tmp, nullptr);
      codebook_emit<uint16_t>(a, V, n, S.scan_tmp, &S.ct);
    } else {  // the tree here; cb_emit_kernel emits the codes on many CTAs afterwards
      const CbArrays<unsigned> V = cb_big(a.big, S.wcnt);
      const CbTileScratch ts = cb_tile_scratch(S);
      codebook_lengths<unsigned>(a, V, n, S.scan_tmp, S.ka, passes, &ts);
    }
    return;
  }
  // 0. every dictionary entry starts without a code
  for (int s = threadIdx.x; s < dict; s += blockDim.x) {
    a.lens[s] = 0;
    a.codes[s] = 0;
    if (a.packed) a.packed[s] = 0;
  }
  // present symbols, in symbol order, compacted: warp w walks its contiguous
  // rows of 32 symbols (coalesced loads, eight rows in flight), counting by
  // ballot; one scan over the warps; a second walk writes each present
  // symbol at its warp's offset plus its rank in the row
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int rows = (dict + 31) / 32, rpw = (rows + nwarps - 1) / nwarps;
  const int r0 = wid * rpw, r1 = min(rows, r0 + rpw);
  unsigned cnt = 0;
  for (int r = r0; r < r1; r += 8) {
    unsigned f[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int s = (r + k) * 32 + lane;
      f[k] = (r + k < r1 && s < dict) ? a.hist[s] : 0u;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) cnt += (unsigned)__popc(__ballot_sync(0xffffffffu, f[k] != 0u));
  }
  if (lane == 0) S.scan_tmp[32 + wid] = cnt;
  __syncthreads();
  if (wid == 0) {
    const unsigned c = lane < nwarps ? S.scan_tmp[32 + lane] : 0u;
    unsigned x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane < nwarps) S.scan_tmp[lane] = x - c;
    if (lane == 31) s_n = x;
  }
  __syncthreads();
  const int n = (int)s_n;
  const bool small = n <= kCbSmemSyms;
  uint16_t* csym = small ? S.csym : cb_big(a.big, S.wcnt).csym;
  unsigned pos = S.scan_tmp[wid];
  for (int r = r0; r < r1; r += 8) {
    unsigned f[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int s = (r + k) * 32 + lane;
      f[k] = (r + k < r1 && s < dict) ? a.hist[s] : 0u;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const unsigned m = __ballot_sync(0xffffffffu, f[k] != 0u);
      if (f[k]) csym[pos + (unsigned)__popc(m & ((1u << lane) - 1u))] = (uint16_t)((r + k) * 32 + lane);
      pos += (unsigned)__popc(m);
    }
  }
  __syncthreads();
  if (small) {
    const CbArrays<uint16_t> V = cb_small(S);
    codebook_lengths<uint16_t>(a, V, n, S.scan_tmp, nullptr);
    codebook_emit<uint16_t>(a, V, n, S.scan_tmp, &S.ct);
  } else {
    const CbArrays<unsigned> V = cb_big(a.big, S.wcnt);
    // S.ka and S.iw (adjacent) stage the tiles
    const CbTileScratch ts = cb_tile_scratch(S);
    codebook_lengths<unsigned>(a, V, n, S.scan_tmp, S.ka, -1, &ts);
    codebook_emit<unsigned>(a, V, n, S.scan_tmp, &S.ct);
  }
}

__global__ void __launch_bounds__(kCbThreads) codebook_kernel(CodebookArgs a) { codebook_block(a); }

// The codebooks of several compress calls (a batch), one CTA each.
__global__ void __launch_bounds__(kCbThreads) codebook_batch_kernel(const CodebookArgs* __restrict__ args) {
  const CodebookArgs a = args[blockIdx.x];
  codebook_block(a);
}

// Histogram of a symbol array (stand-alone Huffman entry point): a shared
// window of kHistWin bins around the dictionary's middle, global atomics
// outside it; symbols not below dict are flagged.
__global__ void __launch_bounds__(256) hist_kernel(const uint16_t* __restrict__ sym, unsigned long long n, int dict,
                                                   unsigned* hist, Scalars* sc) {
  __shared__ unsigned hs[kHistWin];
  const int lo = max(0, min(dict / 2 - kHistWin / 2, dict - kHistWin));
  const int w = min(dict, kHistWin);
  for (int i = threadIdx.x; i < w; i += blockDim.x) hs[i] = 0;
  __syncthreads();
  bool bad = false;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned s = sym[i];
    const unsigned k = s - (unsigned)lo;
    if (k < (unsigned)w) atomicAdd(hs + k, 1u);
    else if (s < (unsigned)dict) atomicAdd(hist + s, 1u);
    else bad = true;
  }
  if (bad) atomicOr(&sc->status, ST_CORRUPT);
  __syncthreads();
  for (int i = threadIdx.x; i < w; i += blockDim.x)
    if (hs[i]) atomicAdd(hist + lo + i, hs[i]);
}

// Histogram of a symbol range [s0, s1) with 16-byte loads.  Build-time choice
// BM_HIST_METHOD: 1 = the centre symbol (code 0) counted in a register, the
// rest with shared atomics; 7 = the seven symbols around the centre in
// registers; 0 = equal symbols of a warp instruction merged first
// (__match_any_sync), one shared atomic per distinct symbol.  Shared bins
// cover kHistWin symbols around the centre; the rest go to global atomics.
#ifndef BM_HIST_METHOD
#define BM_HIST_METHOD 1
#endif
#ifndef BM_HIST_INFLIGHT
#define BM_HIST_INFLIGHT 8
#endif
__global__ void __launch_bounds__(256) hist_range_kernel(const uint16_t* __restrict__ sym, unsigned long long s0,
                                                         unsigned long long s1, int dict, unsigned centre_sym,
                                                         unsigned* hist) {
  __shared__ unsigned hs[kHistWin];
  const unsigned wlo = (unsigned)max(0, min((int)centre_sym - kHistWin / 2, dict - kHistWin));
  const unsigned wn = (unsigned)min(dict, kHistWin);
  for (int i = threadIdx.x; i < (int)wn; i += blockDim.x) hs[i] = 0;
  __syncthreads();
  constexpr int NC = BM_HIST_METHOD == 7 ? 7 : 1;
  unsigned cnt[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) cnt[j] = 0;
  unsigned n_esc = 0;  // the escape symbol 0: outside the window for large dictionaries, and frequent
  const unsigned lo = centre_sym - (NC / 2);
  auto bin = [&](unsigned s, unsigned c) {
    const unsigned k = s - wlo;
    if (k < wn) atomicAdd(hs + k, c);
    else if (s < (unsigned)dict) atomicAdd(hist + s, c);
  };
  auto count = [&](unsigned s) {
    if (BM_HIST_METHOD == 0) {
      const unsigned m = __match_any_sync(__activemask(), s);
      if ((unsigned)(threadIdx.x & 31) == (unsigned)(__ffs(m) - 1)) bin(s, __popc(m));
      return;
    }
    const unsigned d = s - lo;
#pragma unroll
    for (int j = 0; j < NC; ++j) cnt[j] += d == (unsigned)j;
    n_esc += s == 0u;
    if (d >= (unsigned)NC && s != 0u) bin(s, 1u);
  };
  const unsigned long long a0 = min(s1, (s0 + 7) & ~7ull);  // 16-byte aligned start
  const unsigned long long tid = blockIdx.x * 256ull + threadIdx.x, nth = gridDim.x * 256ull;
  for (unsigned long long i = s0 + tid; i < a0; i += nth) count(sym[i]);
  const unsigned long long nv = (s1 - a0) / 8;
  const uint4* pv = reinterpret_cast<const uint4*>(sym + a0);
  // BM_HIST_INFLIGHT 16-byte loads per thread are issued before any is counted
  constexpr int NF = BM_HIST_INFLIGHT;
  for (unsigned long long v = tid; v < nv; v += NF * nth) {
    uint4 q[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const unsigned long long vf = v + f * nth;
      q[f] = vf < nv ? __ldg(pv + vf) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      if (v + f * nth >= nv) break;
      const unsigned w4[4] = {q[f].x, q[f].y, q[f].z, q[f].w};
#pragma unroll
      for (int h = 0; h < 4; ++h) { count(w4[h] & 0xFFFFu); count(w4[h] >> 16); }
    }
  }
  for (unsigned long long i = a0 + nv * 8 + tid; i < s1; i += nth) count(sym[i]);
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    unsigned c = cnt[j];
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (BM_HIST_METHOD != 0 && (threadIdx.x & 31) == 0 && c) bin(lo + j, c);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) n_esc += __shfl_xor_sync(0xffffffffu, n_esc, o);
  if ((threadIdx.x & 31) == 0 && n_esc) bin(0u, n_esc);
  __syncthreads();
  for (int i = threadIdx.x; i < (int)wn; i += blockDim.x)
    if (hs[i]) atomicAdd(hist + wlo + i, hs[i]);
}

// Histogram of a symbol range [s0, s1) for dictionaries larger than the
// small window: one CTA of kHistWideThreads threads per SM keeps a private
// window of hist_wide_bins(dict) bins centred on the centre symbol (as much
// of the dictionary as fits in shared memory: at most kHistWideMax bins) and
// counts with shared atomics; symbols outside it (thin tails of very wide
// code distributions) go to global atomics; the centre and the escape symbol
// 0 are counted in registers.  Symbols not below dict are flagged (sc, when
// given).  Measured on GB300 faster than spreading the whole dictionary over
// a thread-block cluster in distributed shared memory (remote reductions on
// the frequent bins serialise at their owner).
constexpr int kHistWideThreads = 1024;
constexpr int kHistWideMax = 49152;
__host__ __device__ constexpr int hist_wide_bins(int dict) { return dict < kHistWideMax ? dict : kHistWideMax; }

__global__ void __launch_bounds__(kHistWideThreads)
    hist_wide_kernel(const uint16_t* __restrict__ sym, unsigned long long s0, unsigned long long s1, int dict,
                     unsigned centre_sym, unsigned* hist, Scalars* sc) {
  extern __shared__ __align__(16) unsigned hw[];
  const int W = hist_wide_bins(dict);
  const unsigned wlo = (unsigned)max(0, min((int)centre_sym - W / 2, dict - W));
  for (int i = threadIdx.x; i < W; i += blockDim.x) hw[i] = 0;
  __syncthreads();
  unsigned n_centre = 0, n_esc = 0;
  bool bad = false;
  auto count = [&](unsigned s) {
    n_centre += s == centre_sym;
    n_esc += s == 0u;
    if (s == centre_sym || s == 0u) return;
    const unsigned k = s - wlo;
    if (k < (unsigned)W) atomicAdd(hw + k, 1u);
    else if (s < (unsigned)dict) atomicAdd(hist + s, 1u);
    else bad = true;
  };
  const unsigned long long a0 = min(s1, (s0 + 7) & ~7ull);  // 16-byte aligned start
  const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  const unsigned long long nth = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = s0 + tid; i < a0; i += nth) count(sym[i]);
  const unsigned long long nv = (s1 - a0) / 8;
  const uint4* pv = reinterpret_cast<const uint4*>(sym + a0);
  constexpr int NF = 4;
  for (unsigned long long v = tid; v < nv; v += NF * nth) {
    uint4 q[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const unsigned long long vf = v + f * nth;
      q[f] = vf < nv ? __ldg(pv + vf) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      if (v + f * nth >= nv) break;
      const unsigned w4[4] = {q[f].x, q[f].y, q[f].z, q[f].w};
#pragma unroll
      for (int h = 0; h < 4; ++h) { count(w4[h] & 0xFFFFu); count(w4[h] >> 16); }
    }
  }
  for (unsigned long long i = a0 + nv * 8 + tid; i < s1; i += nth) count(sym[i]);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    n_centre += __shfl_xor_sync(0xffffffffu, n_centre, o);
    n_esc += __shfl_xor_sync(0xffffffffu, n_esc, o);
  }
  if ((threadIdx.x & 31) == 0) {  // the window always holds the centre (it is centred on it, or holds all)
    if (n_centre) atomicAdd(hw + (centre_sym - wlo), n_centre);
    if (n_esc) atomicAdd(hist, n_esc);
  }
  if (bad && sc) atomicOr(&sc->status, ST_CORRUPT);
  __syncthreads();
  for (int i = threadIdx.x; i < W; i += blockDim.x) {
    const unsigned v = hw[i];
    if (v) atomicAdd(hist + wlo + i, v);
  }
}

// ---------------------------------------------------------------------------
// Single-pass encoder (decoupled look-back, Merrill & Garland 2016)
// ---------------------------------------------------------------------------
// Status word of a chunk for the look-back: [flag:2][words:31][escapes:31],
// so one load sees a consistent pair (inputs hold fewer than 2^31 symbols).
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagIncl = 2ull << 62;
constexpr unsigned long long kM31 = (1ull << 31) - 1;
constexpr long kSpinLimit = 1l << 24;
__device__ __forceinline__ unsigned long long pack_status(unsigned long long flag, unsigned long long w,
                                                          unsigned long long e) {
  return flag | ((w & kM31) << 31) | (e & kM31);
}

struct FusedEncodeArgs {
  const uint16_t* sym;
  const int32_t* esc;            // codes of escaped symbols (stream mode) or null
  unsigned long long n;
  int chunk;                     // multiple of 32
  const uint8_t* lens;
  const unsigned* codes;
  const unsigned* packed;        // [dict] enc_entry(code, len) per symbol (written by the codebook)
  int dict;
  unsigned long long nch;
  unsigned* ticket;              // zeroed before launch
  unsigned long long* st;        // [nch] look-back status words (zeroed)
  unsigned* chunk_words;         // stream chunk table
  uint16_t* splits;              // stream split offsets [nch][7]
  uint8_t* out;                  // stream base; the codebook kernel put the section offsets in sc
  unsigned long long capacity;
  Scalars* sc;
  int win;                       // entries of the shared-memory window (dynamic shared memory: 4 per entry)
};

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

constexpr int kEncGroups = 8;  // a lane's slice: up to 8 groups of 8 symbols (chunk <= 2048)

__device__ __forceinline__ unsigned sym_of(const uint4* q, int i) {
  const unsigned w = (i & 4) ? ((i & 2) ? q[i >> 3].w : q[i >> 3].z) : ((i & 2) ? q[i >> 3].y : q[i >> 3].x);
  return (i & 1) ? (w >> 16) : (w & 0xFFFFu);
}

// The encoder's code table, entries enc_entry(code, len): a window of
// `wn` entries in shared memory (sc) starting at symbol `lo`, and the
// whole table in global memory (gp), read through L1; gc holds the full codes
// of the rare codes longer than kPackBits bits.  The escape symbol 0's code
// and length are in registers.
struct EncTab {
  const unsigned* sc;
  unsigned lo, wn;  // first symbol and entries of the window
  const unsigned* gc;
  const unsigned* gp;
  unsigned c0, l0;  // code and length of symbol 0
};

// A global load issued only where `pred` holds (a predicated instruction,
// not a branch: the warp does not diverge); v keeps its value elsewhere.
__device__ __forceinline__ unsigned ld_nc_if(const unsigned* p, bool pred, unsigned v) {
  asm("{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n @q ld.global.nc.u32 %0, [%1];\n}\n"
      : "+r"(v)
      : "l"(p), "r"((unsigned)pred));
  return v;
}
// Table of a lookup: TAB 0 = the shared-memory window only (it holds every
// symbol met), 1 = the window with the global table for symbols outside it,
// 2 = the global table only.
template <int TAB>
__device__ __forceinline__ unsigned entry_of(const EncTab& t, unsigned s) {
  if (TAB == 0) return t.sc[s - t.lo];
  if (TAB == 1) {  // the window's entry, or (rare) the global table's by a predicated load
    const unsigned k = s - t.lo;
    const bool in = k < t.wn;
    const unsigned ew = t.sc[in ? k : 0u];
    const unsigned eg = ld_nc_if(t.gp + s, !in && s != 0u, enc_entry(t.c0, t.l0));
    return in ? ew : eg;
  }
  return s == 0u ? enc_entry(t.c0, t.l0) : __ldg(t.gp + s);
}
template <int TAB>
__device__ __forceinline__ void code_of(const EncTab& t, unsigned s, unsigned& c, unsigned& L) {
  const unsigned e = entry_of<TAB>(t, s);
  c = e & ((1u << kPackBits) - 1u);
  L = e >> kPackBits;
  if (L > kPackBits) c = s == 0u ? t.c0 : __ldg(t.gc + s);  // a long code (rare)
}
// Without long codes in the warp's slices: the entry alone.
template <int TAB>
__device__ __forceinline__ void code_of_short(const EncTab& t, unsigned s, unsigned& c, unsigned& L) {
  const unsigned e = entry_of<TAB>(t, s);
  c = e & ((1u << kPackBits) - 1u);
  L = e >> kPackBits;
}
template <int TAB>
__device__ __forceinline__ unsigned len_of(const EncTab& t, unsigned s) {
  return entry_of<TAB>(t, s) >> kPackBits;
}
// An entry at or above this one has a code longer than kPackBits bits.
constexpr unsigned kLongEntry = (kPackBits + 1u) << kPackBits;

// Symbols of a slice, streamed past L1 (the global code table of the GLOB
// variant keeps L1 to itself).
__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}

// Bits, escape mask and largest table entry of a lane's vector slice (G
// groups held in registers).  CLAMP: symbols may be out of the dictionary
// (caller-supplied) and are clamped; the compressor's own symbols are in
// range by construction.
template <int TAB, bool CLAMP, int GC>
__device__ __forceinline__ void slice_bits(const uint4* q, int G, unsigned dmax, const EncTab& tab, unsigned& bits,
                                           unsigned long long& emask, unsigned& emax) {
  bits = 0;
  emax = 0;
  unsigned nz = 0;
#pragma unroll
  for (int i = 0; i < 8 * kEncGroups; ++i) {
    if ((i >> 3) < (GC ? GC : G)) {
      const unsigned s = CLAMP ? min(sym_of(q, i), dmax) : sym_of(q, i);
      const unsigned e = entry_of<TAB>(tab, s);
      bits += e >> kPackBits;
      emax = max(emax, e);
      nz += s == 0;
    }
  }
  emask = 0;
  if (nz) {  // escapes (symbol 0): their positions, for the outlier codes
    unsigned em[2] = {0u, 0u};
#pragma unroll
    for (int i = 0; i < 8 * kEncGroups; ++i)
      if ((i >> 3) < (GC ? GC : G)) em[i >> 5] |= (unsigned)(sym_of(q, i) == 0) << (i & 31);
    emask = ((unsigned long long)em[1] << 32) | em[0];
  }
}

// MSB-first packing of a lane's vector slice.  `acc` holds the pending bits in
// its low `nb` bits (garbage above is shifted out and never stored); every
// word is stored through `wp` as soon as it fills.  The lane's first word may
// start with the previous lane's last bits: it is stored with zeros there and
// the previous lane ORs its bits in afterwards.
template <int TAB, bool CLAMP, int GC, bool LONG>
__device__ __forceinline__ void slice_pack(const uint4* q, int G, unsigned dmax, const EncTab& tab, unsigned* wp,
                                           unsigned nb, unsigned long long& acc_out, unsigned& nb_out,
                                           unsigned*& wp_out) {
  // acc = hi:lo holds at most 31 pending bits, so a code of up to 32 bits
  // fits; each shift is one clamped funnel shift (a shift by 32 moves the
  // whole low word up).  LONG: the warp's slices hold codes longer than
// kPackBits bits, read from the full code table.
  unsigned hi = 0, lo = 0;
#pragma unroll
  for (int i = 0; i < 8 * kEncGroups; ++i) {
    if ((i >> 3) < (GC ? GC : G)) {
      const unsigned s = CLAMP ? min(sym_of(q, i), dmax) : sym_of(q, i);
      unsigned c, L;
      if (LONG) code_of<TAB>(tab, s, c, L);
      else code_of_short<TAB>(tab, s, c, L);
      hi = __funnelshift_lc(lo, hi, L);
      lo = __funnelshift_lc(0u, lo, L) | c;
      nb += L;
      if (nb >= 32u) {
        nb -= 32u;
        *wp++ = __funnelshift_r(lo, hi, nb);
      }
    }
  }
  acc_out = ((unsigned long long)hi << 32) | lo;
  nb_out = nb;
  wp_out = wp;
}

// The instantiation of a slice function picked at run time (full
// default-size slices or not; for packing, long codes in the warp or not);
// TAB is the kernel's.
#define BM_ENC_DISPATCH(FN, ...)                                  \
  do {                                                            \
    if (G == kEncGroups) FN<TAB, CLAMP, kEncGroups>(__VA_ARGS__); \
    else FN<TAB, CLAMP, 0>(__VA_ARGS__);                          \
  } while (0)
#define BM_ENC_DISPATCH_PACK(FN, ...)                                                  \
  do {                                                                                 \
    if (G == kEncGroups) {                                                             \
      if (wlong) FN<TAB, CLAMP, kEncGroups, true>(__VA_ARGS__);                        \
      else FN<TAB, CLAMP, kEncGroups, false>(__VA_ARGS__);                             \
    } else {                                                                           \
      if (wlong) FN<TAB, CLAMP, 0, true>(__VA_ARGS__);                                 \
      else FN<TAB, CLAMP, 0, false>(__VA_ARGS__);                                      \
    }                                                                                  \
  } while (0)

// The codebook's choice of table (sc->enc_mode, the kernel's MODE): 0 when
// every symbol met lies in a window of kEncWinSmall entries, 3 when they all
// lie in one of kEncWin entries, 1 when that window serves most of them and
// the global table the rest, 2 (the global table only) otherwise; modes 0 and
// 3 look up the window alone (TAB 0).  For the compressor's own symbols
// (CLAMP = false) all four are launched, the ones that do not match returning
// at once; for caller-supplied symbols the host picks by dictionary size.
// Warps take chunks in ticket order.  A warp codes its chunk's bit count from
// the symbols it holds in registers, publishes the chunk's (words, escapes)
// aggregate, walks back over its predecessors until one has published an
// inclusive prefix (bounded wait), publishes its own inclusive prefix and then
// packs its codes at the now known word offset.  Each lane stores its full
// words; a word shared by two lanes is completed by an atomic OR of the
// earlier lane's last bits.
template <int WARPS, bool CLAMP, int MODE>
__global__ void __launch_bounds__(WARPS * 32, 32 / WARPS) encode_fused_kernel(FusedEncodeArgs a) {
  constexpr int TAB = MODE == 3 ? 0 : MODE;
  extern __shared__ __align__(16) unsigned char enc_smem_raw[];
  const int WN = TAB == 2 ? 0 : a.win;
  unsigned* ent = reinterpret_cast<unsigned*>(enc_smem_raw);  // [WN] the window's entries
  Scalars* sc = a.sc;
  if (sc->skip) return;  // the stream is already known to be a raw copy
  if (!CLAMP && (unsigned)MODE != sc->enc_mode) return;
  const unsigned wlo = sc->enc_lo;
  // the compressor's symbols lie below enc_lo + enc_n: the rest is never read
  const int nfill = CLAMP ? WN : min(WN, (int)sc->enc_n);
  for (int i = threadIdx.x; i < nfill; i += blockDim.x) {
    const unsigned s = wlo + (unsigned)i;
    ent[i] = s < (unsigned)a.dict ? a.packed[s] : 0u;
  }
  const EncTab tab{ent, wlo, (unsigned)WN, a.codes, a.packed, a.codes[0], a.lens[0]};
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const unsigned dmax = (unsigned)(a.dict - 1);
  const unsigned long long off_bits = sc->off_bits;
  const unsigned long long n_out = sc->n_outliers;
  unsigned* words = reinterpret_cast<unsigned*>(a.out + off_bits);
  unsigned* chunk_esc = (a.esc && n_out) ? reinterpret_cast<unsigned*>(a.out + sc->off_chunk_esc) : nullptr;
  int32_t* ocode = reinterpret_cast<int32_t*>(a.out + sc->off_outliers);
  const unsigned long long word_cap = a.capacity > off_bits ? (a.capacity - off_bits) / 4 : 0ull;
  const int per = a.chunk / 32;
  const int G = per / 8;
  while (true) {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(a.ticket, 1u);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c >= a.nch) break;
    const unsigned long long cb = c * (unsigned long long)a.chunk;
    const unsigned long long ce = min(a.n, cb + (unsigned long long)a.chunk);
    const unsigned long long s0 = min(ce, cb + (unsigned long long)lane * per);
    const unsigned long long s1 = min(ce, s0 + per);
    const int cnt = (int)(s1 - s0);
    // vector slices: whole groups of 8 symbols, 16-byte aligned, every lane
    // full with at least 32 symbols (so at least 32 bits: a word never has
    // more than two owners)
    const bool warp_vec = __all_sync(0xffffffffu, (per & 7) == 0 && per >= 32 && cnt == per && (s0 & 7ull) == 0 &&
                                                      (reinterpret_cast<uintptr_t>(a.sym) & 15) == 0);
    uint4 q[kEncGroups];
    // pass 1: bits and escapes of the slice
    unsigned bits = 0, nesc = 0, emax = 0;
    unsigned long long emask = 0;
    if (warp_vec) {
      const uint4* p = reinterpret_cast<const uint4*>(a.sym + s0);
#pragma unroll
      for (int g = 0; g < kEncGroups; ++g)
        q[g] = g < G ? (TAB == 2 ? ld_stream(p + g) : __ldg(p + g)) : make_uint4(0, 0, 0, 0);
      // G is 8 at the default chunk of 2048 symbols: a fully unrolled slice
      BM_ENC_DISPATCH(slice_bits, q, G, dmax, tab, bits, emask, emax);
      nesc = __popcll(emask);
    } else {
      for (int t = 0; t < cnt; ++t) {
        const unsigned s = CLAMP ? min((unsigned)a.sym[s0 + t], dmax) : (unsigned)a.sym[s0 + t];
        bits += len_of<TAB>(tab, s);
        nesc += s == 0;
      }
    }
    if (!a.esc) nesc = 0;
    unsigned xb = bits, xe = nesc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned yb = __shfl_up_sync(0xffffffffu, xb, o);
      const unsigned ye = __shfl_up_sync(0xffffffffu, xe, o);
      if (lane >= o) { xb += yb; xe += ye; }
    }
    const unsigned tot_bits = __shfl_sync(0xffffffffu, xb, 31);
    const unsigned tot_esc = __shfl_sync(0xffffffffu, xe, 31);
    const unsigned W = (tot_bits + 31u) >> 5;
    // publish the aggregate, then look back (a window of 32 predecessors per
    // step, one per lane) until an inclusive prefix is found
    unsigned long long pw = 0, pe = 0;
    int timed_out = 0;
    if (c == 0) {
      if (lane == 0) atomicExch(a.st + 0, pack_status(kFlagIncl, W, tot_esc));
    } else {
      if (lane == 0) atomicExch(a.st + c, pack_status(kFlagAgg, W, tot_esc));
      long long top = (long long)c - 1;  // highest predecessor not yet summed
      long spins = 0;
      while (top >= 0) {
        const long long pidx = top - lane;
        const unsigned long long sv = pidx >= 0 ? ld_volatile_u64(a.st + pidx) : kFlagIncl;  // before chunk 0: prefix 0
        const unsigned flag = (unsigned)(sv >> 62);
        // only the lanes up to the first unpublished one can be used
        const unsigned unpub = __ballot_sync(0xffffffffu, flag == 0);
        const unsigned incl = __ballot_sync(0xffffffffu, flag == 2);
        const int first_incl = incl ? __ffs(incl) - 1 : 32;
        const int first_unpub = unpub ? __ffs(unpub) - 1 : 32;
        if (first_unpub <= first_incl && first_unpub < 32) {
          if (first_unpub == 0) {  // nearest predecessor not published yet: wait
            if (++spins > kSpinLimit) { timed_out = 1; break; }
            __nanosleep(32);
            continue;
          }
        }
        const int take = min(first_incl + 1, first_unpub);  // lanes [0, take) are summed
        unsigned long long w = 0, e = 0;
        if (lane < take && pidx >= 0) { w = (sv >> 31) & kM31; e = sv & kM31; }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          w += __shfl_xor_sync(0xffffffffu, w, o);
          e += __shfl_xor_sync(0xffffffffu, e, o);
        }
        pw += w;
        pe += e;
        if (first_incl < take) break;  // reached an inclusive prefix (or the start)
        top -= take;
      }
      timed_out = __shfl_sync(0xffffffffu, timed_out, 0);
      if (!timed_out && lane == 0) {
        __threadfence();
        atomicExch(a.st + c, pack_status(kFlagIncl, pw + W, pe + tot_esc));
      }
    }
    if (lane == 0) {
      a.chunk_words[c] = W;
      if (chunk_esc) chunk_esc[c] = tot_esc;
      if (c == a.nch - 1) {
        sc->n_words = pw + W;
        sc->esc_seen = pe + tot_esc;
      }
    }
    timed_out = __shfl_sync(0xffffffffu, timed_out, 0);
    if (timed_out) {
      if (lane == 0) atomicOr(&sc->status, ST_TIMEOUT | ST_RAW);
      break;
    }
    pw = __shfl_sync(0xffffffffu, pw, 0);
    pe = __shfl_sync(0xffffffffu, pe, 0);
    if (pw + W > word_cap) {  // the stream would not fit: it becomes a raw copy
      if (lane == 0) atomicOr(&sc->status, ST_RAW);
      continue;
    }
    // outlier codes of the slice, in stream order
    unsigned long long epos = pe + (xe - nesc);
    if (a.esc && warp_vec && (per & 31) == 0 && tot_esc * 8u >= (unsigned)a.chunk) {
      // many escapes: the warp copies them together, 32 consecutive symbols of
      // one lane's slice at a time (that lane's escape mask, broadcast), so
      // the loads of the escaped codes and the stores of the outliers are
      // coalesced rather than one line per lane
      unsigned long long ep = pe;
      for (int l = 0; l < 32; ++l) {
        const unsigned long long ml = __shfl_sync(0xffffffffu, emask, l);
        const unsigned long long sl = cb + (unsigned long long)l * per;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const unsigned m = (unsigned)(ml >> (32 * h));
          if (32 * h < per && m) {
            const unsigned r = __popc(m & ((1u << lane) - 1u));
            if (((m >> lane) & 1u) && ep + r < n_out) ocode[ep + r] = __ldg(a.esc + sl + 32 * h + lane);
            ep += __popc(m);
          }
        }
      }
    } else if (a.esc && nesc) {
      if (warp_vec) {
        unsigned long long m = emask;
        while (m) {
          int idx[4];
          int k = 0;
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            idx[t] = m ? __ffsll((long long)m) - 1 : -1;
            m &= m ? m - 1 : 0ull;
            k += idx[t] >= 0;
          }
          int32_t v[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) v[t] = idx[t] >= 0 ? __ldg(a.esc + s0 + idx[t]) : 0;
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (idx[t] >= 0 && epos + t < n_out) ocode[epos + t] = v[t];
          epos += k;
        }
      } else {
        for (int t = 0; t < cnt; ++t)
          if (a.sym[s0 + t] == 0) {
            if (epos < n_out) ocode[epos] = a.esc[s0 + t];
            ++epos;
          }
      }
    }
    if ((lane & 3) == 0 && lane) a.splits[c * (kSplits - 1) + (lane >> 2) - 1] = (uint16_t)(xb - bits);
    // pass 2: pack MSB-first
    const unsigned bit0 = xb - bits;
    const unsigned long long head_idx = pw + (bit0 >> 5);
    const bool head_partial = (bit0 & 31u) != 0;
    if (warp_vec) {
      unsigned long long acc;
      unsigned nb;
      unsigned* wp;
      unsigned* const w0 = words + head_idx;
      const unsigned nb0 = bit0 & 31u;
      const bool wlong = __any_sync(0xffffffffu, emax >= kLongEntry);
      BM_ENC_DISPATCH_PACK(slice_pack, q, G, dmax, tab, w0, nb0, acc, nb, wp);
      // every lane holds >= 32 bits, so the word of its last bits is the next
      // lane's first word (already stored, zeros in these bits); the last
      // lane's last word is its own
      __syncwarp();
      if (nb) {
        const unsigned tail = (unsigned)(acc << (32 - nb));
        if (lane == 31) *wp = tail;
        else atomicOr(wp, tail);
      }
    } else {  // a partial chunk: zero its words, shared words are ORed
      for (unsigned w = lane; w < W; w += 32) words[pw + w] = 0u;
      __syncwarp();
      unsigned long long acc = 0, widx = head_idx;
      unsigned nb = bit0 & 31u, head = 0;
      bool pending_head = head_partial;
      for (int t = 0; t < cnt; ++t) {
        const unsigned s = CLAMP ? min((unsigned)a.sym[s0 + t], dmax) : (unsigned)a.sym[s0 + t];
        unsigned c, L;
        code_of<TAB>(tab, s, c, L);
        acc = (acc << L) | c;
        nb += L;
        if (nb >= 32u) {
          nb -= 32u;
          const unsigned word = (unsigned)(acc >> nb);
          if (pending_head) head = word;
          else words[widx] = word;
          pending_head = false;
          ++widx;
        }
      }
      __syncwarp();
      if (head_partial && !pending_head) atomicOr(words + head_idx, head);
      if (nb) atomicOr(words + widx, (unsigned)(acc << (32 - nb)));
    }
  }
}

// After the fused encoder (one thread): stream length and the raw decision.
__device__ __forceinline__ void encode_finish(unsigned long long raw_total, unsigned long long capacity, Scalars* sc) {
  if (sc->skip) return;  // already raw
  const unsigned long long total = sc->off_bits + pad8(4ull * sc->n_words);
  sc->total = total;
  if (sc->esc_seen != sc->n_outliers) atomicOr(&sc->status, ST_CORRUPT | ST_RAW);
  if (total >= raw_total || total > capacity || (sc->status & ST_OVERFLOW)) atomicOr(&sc->status, ST_RAW);
}
__global__ void encode_finish_kernel(unsigned long long raw_total, unsigned long long capacity, Scalars* sc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) encode_finish(raw_total, capacity, sc);
}

// ---------------------------------------------------------------------------
// Decoding
// ---------------------------------------------------------------------------
// Present symbols the decoder-table builder keeps in shared memory; more use
// the global arrays of DecodeTables.
constexpr int kDtSmemSyms = 8192;

struct DtSmem {
  uint8_t clen[kDtSmemSyms];    // code length of each present symbol (symbol order)
  uint16_t csym[kDtSmemSyms];   // its symbol
  uint16_t canon[kDtSmemSyms];  // present-symbol indices in canonical order
  unsigned key32[kDtSmemSyms];  // the codebook section (when it fits), then counting scratch
  unsigned scan_tmp[64];
  CanonTables ct;
  unsigned rfirst[512], rcount[512], roff[512];
};

// Build decode tables from the stream's codebook runs (one CTA of
// kCbThreads threads, DtSmem in its dynamic shared memory).  The runs list
// the present symbols in symbol order: run q's t-th symbol is present symbol
// (symbols of the runs before q) + t.
__device__ __forceinline__ void decode_tables_block(const uint8_t* runs, unsigned long long nbytes,
                                                    unsigned long long n_runs, int dict, DecodeTables* out,
                                                    Scalars* sc, unsigned char* smem_raw) {
  DtSmem& S = *reinterpret_cast<DtSmem*>(smem_raw);
  __shared__ unsigned s_bad;
  __shared__ unsigned long long s_kr;
  __shared__ unsigned s_total, s_n;
  if (threadIdx.x == 0) { s_bad = 0; s_kr = 0; s_n = 0; }
  // every present symbol takes at least one length byte after its run's
  // 8-byte header: this bounds their count and picks the arrays
  const unsigned long long nbound = nbytes > 8ull * n_runs ? nbytes - 8ull * n_runs : 0ull;
  const bool small = nbound <= (unsigned long long)kDtSmemSyms;
  const unsigned cap = small ? (unsigned)kDtSmemSyms : (unsigned)kMaxDict;
  uint8_t* clen = small ? S.clen : out->big_clen;
  uint16_t* csym = small ? S.csym : out->big_csym;
  uint16_t* canon = small ? S.canon : out->big_canon;
  // the codebook section is walked serially: read it from shared memory when
  // it fits in the key scratch (free until build_canonical)
  const uint8_t* rbase = runs;
  if (nbytes <= sizeof(S.key32) && (reinterpret_cast<uintptr_t>(runs) & 3) == 0) {
    const unsigned* src = reinterpret_cast<const unsigned*>(runs);
    const unsigned nw = (unsigned)(nbytes / 4);
    for (unsigned i = threadIdx.x; i < nw; i += blockDim.x) S.key32[i] = src[i];
    uint8_t* kb = reinterpret_cast<uint8_t*>(S.key32);
    for (unsigned i = 4 * nw + threadIdx.x; i < (unsigned)nbytes; i += blockDim.x) kb[i] = runs[i];
    rbase = kb;
  }
  __syncthreads();
  // walk the run headers (serial, 512 at a time), then every thread copies
  // lengths and symbols of the batch (rcount holds each run's first index in
  // the batch)
  unsigned long long off = 0;
  unsigned prev_end = 0;  // runs must be ascending and must not overlap
  for (unsigned long long rb = 0; rb < n_runs; rb += 512) {
    const int nb = (int)min(512ull, n_runs - rb);
    if (threadIdx.x == 0) {
      unsigned tot = 0;
      for (int q = 0; q < nb; ++q) {
        if (off + 8 > nbytes) { s_bad = 1; break; }
        const unsigned first = *reinterpret_cast<const unsigned*>(rbase + off);
        const unsigned cnt = *reinterpret_cast<const unsigned*>(rbase + off + 4);
        if ((unsigned long long)first + cnt > (unsigned long long)dict || off + 8 + cnt > nbytes ||
            (rb + q > 0 && first < prev_end) || (unsigned long long)s_n + tot + cnt > cap) {
          s_bad = 1;
          break;
        }
        S.rfirst[q] = first; S.rcount[q] = tot; S.roff[q] = (unsigned)off;
        tot += cnt;
        prev_end = first + cnt;
        off += 8ull + ((cnt + 3u) & ~3u);
      }
      s_total = tot;
    }
    __syncthreads();
    if (s_bad) break;
    const unsigned tot = s_total, base = s_n;
    for (unsigned e = threadIdx.x; e < tot; e += blockDim.x) {
      const int q = upper_bound_u32(S.rcount, 0, nb, e) - 1;
      const unsigned t = e - S.rcount[q];
      clen[base + e] = rbase[S.roff[q] + 8 + t];
      csym[base + e] = (uint16_t)(S.rfirst[q] + t);
    }
    __syncthreads();
    if (threadIdx.x == 0) s_n = base + tot;
    __syncthreads();
  }
  const int n = (int)s_n;
  // Kraft sum (exact, in units of 2^-32) and the length bound
  unsigned long long kr = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const unsigned L = clen[i];
    if (L > (unsigned)kMaxLen) s_bad = 1;
    else if (L) kr += 1ull << (32 - L);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) kr += __shfl_xor_sync(0xffffffffu, kr, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&s_kr, kr);
  __syncthreads();
  if (s_kr > (1ull << 32)) s_bad = 1;
  __syncthreads();
  if (s_bad) {
    if (threadIdx.x == 0) atomicOr(&sc->status, ST_CORRUPT);
    return;
  }
  build_canonical(clen, n, S.key32, canon, &S.ct);
  for (int i = threadIdx.x; i < (int)S.ct.n; i += blockDim.x) out->canon[i] = csym[canon[i]];
  __syncthreads();
  // every LUT entry from its own bits: the length is the first whose
  // left-justified limit lies above them (canonical order), the symbol that
  // code's canonical rank; a prefix of longer codes keeps the length of its
  // first code, where the decoder's search for the length starts
  for (int p = threadIdx.x; p < (1 << kLutBits); p += blockDim.x) {
    const unsigned long long peek = (unsigned long long)p << (32 - kLutBits);
    unsigned L = 1;
    while (L <= (unsigned)kMaxLen && peek >= S.ct.limit[L]) ++L;
    unsigned e = L << 16;
    if (L <= (unsigned)kLutBits) {
      const unsigned idx = S.ct.first_pos[L] + (((unsigned)peek >> (32 - L)) - S.ct.first_code[L]);
      e = idx < S.ct.n ? ((unsigned)csym[canon[idx]] | (L << 16)) : ((unsigned)(kMaxLen + 1) << 16);
    }
    out->lut[p] = e;
  }
  if (threadIdx.x == 0) out->ct = S.ct;
}

struct DecodeArgs {
  const unsigned* words;               // bitstream
  unsigned long long n_words;
  const unsigned long long* word_off;  // [nch+1]
  const uint16_t* splits;              // [nch][7] bit offsets of runs 1..7
  unsigned long long nch;
  unsigned long long n;
  int chunk;
  const DecodeTables* tab;
  uint16_t* sym;
  Scalars* sc;
};

// One thread per run (an eighth of a chunk): table-driven canonical decoding
// with a 64-bit window refilled a word at a time from registers loaded ahead
// in 16-byte groups, sixteen symbols per step stored as one 32-byte sector.
// Codes of at most kLutBits bits take one shared-memory lookup; for a longer
// one the lookup gives the length of the first code of its prefix, from
// which the left-justified limits are walked (one or two steps).  A run must end exactly where the next one
// starts (the last run of a chunk within the chunk); reading past the chunk
// reads zeros and shows in that check.  Persistent CTAs: the tables are
// staged once per CTA.
// Threads per decoder CTA: the lookup table (64 KB) is staged once per CTA,
// so larger CTAs keep more warps per SM on one table.  On GB300 (513^3 FP32
// streams, 1e-2 .. 1e-5) 512 took 0.399 / 0.501 / 0.723 / 1.186 ms against
// 0.451 / 0.566 / 0.749 / 1.189 with 256 and 0.682 / 0.903 / 1.180 / 1.586
// with 128.
#ifndef BM_DEC_THREADS
#define BM_DEC_THREADS 512
#endif
constexpr int kDecThreads = BM_DEC_THREADS;
constexpr size_t kDecSmem = sizeof(unsigned) * (1u << kLutBits) + sizeof(unsigned long long) * (kMaxLen + 2) +
                            2 * sizeof(unsigned) * (kMaxLen + 2);

__global__ void __launch_bounds__(kDecThreads) decode_kernel(DecodeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned* lut = reinterpret_cast<unsigned*>(smem_raw);
  unsigned long long* limit = reinterpret_cast<unsigned long long*>(lut + (1 << kLutBits));
  unsigned* fcode = reinterpret_cast<unsigned*>(limit + kMaxLen + 2);
  unsigned* fpos = fcode + kMaxLen + 2;
  const DecodeTables* T = a.tab;
  {
    const uint4* src = reinterpret_cast<const uint4*>(T->lut);
    uint4* dst = reinterpret_cast<uint4*>(lut);
    for (int i = threadIdx.x; i < (1 << kLutBits) / 4; i += blockDim.x) dst[i] = src[i];
  }
  if (threadIdx.x < kMaxLen + 2) {
    limit[threadIdx.x] = T->ct.limit[threadIdx.x];
    fcode[threadIdx.x] = T->ct.first_code[threadIdx.x];
    fpos[threadIdx.x] = T->ct.first_pos[threadIdx.x];
  }
  const unsigned nsym = T->ct.n;
  const uint16_t* canon = T->canon;
  __syncthreads();
  const unsigned long long nruns = a.nch * kSplits;
  const int sub = a.chunk / kSplits;
  for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < nruns;
       r += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long c = r / kSplits;
    const int k = (int)(r % kSplits);
    const unsigned long long cw0 = a.word_off[c], cw1 = a.word_off[c + 1];
    if (cw1 < cw0 || cw1 > a.n_words) { atomicOr(&a.sc->status, ST_CORRUPT); continue; }
    const unsigned long long cbits = (cw1 - cw0) * 32ull;
    const unsigned long long b0 = k ? a.splits[c * (kSplits - 1) + k - 1] : 0ull;
    const unsigned long long b1 = k < kSplits - 1 ? a.splits[c * (kSplits - 1) + k] : cbits;
    if (b0 > b1 || b1 > cbits) { atomicOr(&a.sc->status, ST_CORRUPT); continue; }
    const unsigned long long s0 = c * (unsigned long long)a.chunk + (unsigned long long)k * sub;
    const int cnt = (int)(min(a.n, s0 + (unsigned long long)sub) - s0);
    // words enter the window from a queue (c0..c3, cl of them valid) filled
    // from aligned 16-byte groups, the next group (n) in flight; a group is
    // read as one vector unless it reaches past the bitstream (words past a
    // chunk's end are never consumed by a valid run and show in the check below)
    const unsigned* const wall = a.words + a.n_words;
    auto ld = [&](const unsigned* q) { return q < wall ? __ldg(q) : 0u; };
    auto ld4 = [&](const unsigned* g) {
      if (g + 4 <= wall) return __ldg(reinterpret_cast<const uint4*>(g));
      return make_uint4(ld(g), ld(g + 1), ld(g + 2), ld(g + 3));
    };
    const unsigned* gp = a.words + cw0 + (b0 >> 5);
    const unsigned w0 = ld(gp), w1 = ld(gp + 1);
    gp += 2;
    const int m = (int)((reinterpret_cast<uintptr_t>(gp) >> 2) & 3);
    const unsigned* gq = gp - m;  // 16-byte aligned
    const uint4 A = ld4(gq);
    uint4 n = ld4(gq + 4);
    gq += 8;
    unsigned c0 = m == 0 ? A.x : m == 1 ? A.y : m == 2 ? A.z : A.w;
    unsigned c1 = m == 0 ? A.y : m == 1 ? A.z : A.w;
    unsigned c2 = m == 0 ? A.z : A.w;
    unsigned c3 = A.w;
    int cl = 4 - m;
    const int skip = (int)(b0 & 31);
    unsigned long long buf = (((unsigned long long)w0 << 32) | w1) << skip;
    int nbits = 64 - skip;
    unsigned nwords = 2;  // words entered into the window
    bool bad = false;
    auto one = [&]() -> unsigned {
      // a word into the window when 32 bits or fewer are left: selects, so
      // that lanes refilling at different symbols do not diverge; only the
      // reload of the queue (every fourth word) branches
      const bool need = nbits <= 32;
      const int sh = need ? 32 - nbits : 0;
      buf |= need ? (unsigned long long)c0 << sh : 0ull;
      nbits += need ? 32 : 0;
      nwords += need ? 1u : 0u;
      c0 = need ? c1 : c0;
      c1 = need ? c2 : c1;
      c2 = need ? c3 : c2;
      cl -= need ? 1 : 0;
      if (cl == 0) {
        c0 = n.x;
        c1 = n.y;
        c2 = n.z;
        c3 = n.w;
        n = ld4(gq);
        gq += 4;
        cl = 4;
      }
      const unsigned peek = (unsigned)(buf >> 32);
      unsigned e = lut[peek >> (32 - kLutBits)];
      unsigned L = e >> 16;
      if (L > (unsigned)kLutBits) {  // a longer code: its length from its prefix's first on
        while (L <= (unsigned)kMaxLen && (unsigned long long)peek >= limit[L]) ++L;
        const unsigned idx = L <= (unsigned)kMaxLen ? fpos[L] + ((peek >> (32 - L)) - fcode[L]) : nsym;
        if (idx >= nsym) {
          bad = true;
          L = 1;
          e = 0;
        } else {
          e = (unsigned)canon[idx];
        }
      }
      buf <<= L;
      nbits -= (int)L;
      return e & 0xFFFFu;
    };
    uint16_t* out = a.sym + s0;
    int i = 0;
    if ((reinterpret_cast<uintptr_t>(out) & 31) == 0) {  // sixteen symbols: one whole 32-byte sector
      for (; i + 16 <= cnt; i += 16) {
        unsigned v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const unsigned lo = one();
          v[t] = lo | (one() << 16);
        }
        uint4* o = reinterpret_cast<uint4*>(out + i);
        o[0] = make_uint4(v[0], v[1], v[2], v[3]);
        o[1] = make_uint4(v[4], v[5], v[6], v[7]);
      }
    }
    for (; i < cnt; ++i) out[i] = (uint16_t)one();
    // bits consumed from the chunk start
    const unsigned long long used = b0 + (unsigned long long)nwords * 32ull - (unsigned long long)skip - nbits;
    if (bad || (k < kSplits - 1 ? used != b1 : used > b1)) atomicOr(&a.sc->status, ST_CORRUPT);
  }
}

// Escaped symbols (symbol 0) take the outlier codes in stream order: one
// warp per chunk, each lane a slice of chunk/32 (<= 64) symbols read as 16-byte
// vectors when the slices allow it; a lane's escapes are a 64-bit mask.
__global__ void __launch_bounds__(256) escape_fixup_kernel(const uint16_t* sym, unsigned long long n, int chunk,
                                                           unsigned long long nch, const unsigned long long* esc_off,
                                                           const int32_t* ocode, unsigned long long n_out,
                                                           int32_t* esc, Scalars* sc) {
  const int lane = threadIdx.x & 31;
  const int per = chunk / 32;
  const int G = per / 8;
  for (unsigned long long c = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) / 32; c < nch;
       c += (unsigned long long)gridDim.x * blockDim.x / 32) {
    const unsigned long long cb = c * (unsigned long long)chunk;
    const unsigned long long s0 = min(n, cb + (unsigned long long)lane * per), s1 = min(n, s0 + per);
    const int cnt = (int)(s1 - s0);
    const bool vec = __all_sync(0xffffffffu, (per & 7) == 0 && cnt == per && (s0 & 7ull) == 0);
    unsigned long long m = 0;
    if (vec) {
      const uint4* p = reinterpret_cast<const uint4*>(sym + s0);
      uint4 q[kEncGroups];
#pragma unroll
      for (int g = 0; g < kEncGroups; ++g) q[g] = g < G ? __ldg(p + g) : make_uint4(1u, 1u, 1u, 1u);
#pragma unroll
      for (int i = 0; i < 8 * kEncGroups; ++i)
        if ((i >> 3) < G) m |= (unsigned long long)(sym_of(q, i) == 0) << i;
    } else {
      for (int t = 0; t < cnt; ++t) m |= (unsigned long long)(sym[s0 + t] == 0) << t;
    }
    const unsigned ne = __popcll(m);
    unsigned x = ne;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const unsigned total = __shfl_sync(0xffffffffu, x, 31);
    const unsigned long long e0 = esc_off[c], e1 = esc_off[c + 1];
    if (e0 + total != e1 || e1 > n_out) {  // the outlier reads stay inside the outlier section
      if (lane == 0) atomicOr(&sc->status, ST_CORRUPT);
      continue;
    }
    unsigned long long e = e0 + (x - ne);
    if (vec && (reinterpret_cast<uintptr_t>(esc + s0) & 15) == 0) {
      // groups of four positions: one 16-byte store for each group holding an
      // escape (entries of the other positions are never read)
      int4* e4 = reinterpret_cast<int4*>(esc + s0);
      for (int g = 0; g < per / 4 && m; ++g) {
        const unsigned bits = (unsigned)(m >> (4 * g)) & 15u;
        if (!bits) continue;
        int v[4];
        unsigned r = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const bool on = (bits >> t) & 1u;
          v[t] = on ? __ldg(ocode + e + r) : 0;
          r += on;
        }
        e4[g] = make_int4(v[0], v[1], v[2], v[3]);
        e += r;
      }
    } else {
      while (m) {
        int idx[4];
        int k = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          idx[t] = m ? __ffsll((long long)m) - 1 : -1;
          m &= m ? m - 1 : 0ull;
          k += idx[t] >= 0;
        }
        int32_t v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) v[t] = idx[t] >= 0 ? __ldg(ocode + e + t) : 0;
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (idx[t] >= 0) esc[s0 + idx[t]] = v[t];
        e += k;
      }
    }
  }
}

__global__ void codes_from_symbols_kernel(const uint16_t* sym, const int32_t* esc, unsigned long long n, int radius,
                                          int32_t* out) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned s = sym[i];
    out[i] = s ? (int)s - radius : esc[i];
  }
}

}  // namespace bm
