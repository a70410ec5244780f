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

#include "bm_common.cuh"

namespace bm {

constexpr int kCbThreads = 1024;
constexpr int kLutBits = 12;

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
  unsigned lut[1 << kLutBits];  // sym | len << 16 for codes of <= kLutBits bits, 0 otherwise
  uint16_t canon[kMaxDict];     // symbols in canonical order
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

template <typename K>
__device__ void bitonic_sort(K* keys, int P) {
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const K a = keys[i], b = keys[ixj];
          const bool up = (i & k) == 0;
          if ((a > b) == up) { keys[i] = b; keys[ixj] = a; }
        }
      }
      __syncthreads();
    }
}

__device__ __forceinline__ int upper_bound_u32(const unsigned* a, int lo, int hi, unsigned v) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int lower_bound_u32(const unsigned* a, int lo, int hi, unsigned v) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Canonical tables from a length array len[0..dict) in shared memory.
// key32 is scratch of >= next_pow2(dict) u32.  Writes canon order into canon.
__device__ void build_canonical(const uint8_t* len, int dict, unsigned* key32, uint16_t* canon, CanonTables* ct,
                                unsigned* scan_tmp) {
  __shared__ unsigned s_n;
  if (threadIdx.x < kMaxLen + 2) ct->count[threadIdx.x] = 0;
  __syncthreads();
  // compact present symbols as (len << 13 | sym) keys
  const int per = (dict + blockDim.x - 1) / blockDim.x;
  const int s0 = threadIdx.x * per;
  unsigned cnt = 0;
  for (int s = s0; s < s0 + per && s < dict; ++s) cnt += len[s] ? 1u : 0u;
  unsigned pos = block_excl_scan(cnt, scan_tmp, &s_n);
  for (int s = s0; s < s0 + per && s < dict; ++s)
    if (len[s]) {
      key32[pos++] = ((unsigned)len[s] << 13) | (unsigned)s;
      atomicAdd(&ct->count[len[s]], 1u);
    }
  __syncthreads();
  const int n = (int)s_n;
  int P = 1;
  while (P < n) P <<= 1;
  for (int i = n + threadIdx.x; i < P; i += blockDim.x) key32[i] = 0xFFFFFFFFu;
  __syncthreads();
  bitonic_sort(key32, P);
  for (int i = threadIdx.x; i < n; i += blockDim.x) canon[i] = (uint16_t)(key32[i] & 8191u);
  if (threadIdx.x == 0) {
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
    for (int L = 1; L <= kMaxLen; ++L)
      ct->limit[L] = ((unsigned long long)ct->first_code[L] + ct->count[L]) << (32 - L);
    ct->limit[kMaxLen + 1] = 1ull << 32;
    ct->n = (unsigned)n;
    ct->max_len = maxl;
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
};

// Shared memory of the codebook kernel (dynamic).
struct CbSmem {
  unsigned long long keys[kMaxDict];  // sort keys; later merged order / round ends
  unsigned lw[kMaxDict];              // leaf weights (sorted)
  unsigned iw[kMaxDict];              // internal weights (creation order)
  uint16_t ls[kMaxDict];              // leaf symbols
  uint16_t parent[2 * kMaxDict];
  uint8_t depth[2 * kMaxDict];
  uint8_t len[kMaxDict];
  unsigned scan_tmp[64];
  CanonTables ct;
};

__global__ void __launch_bounds__(kCbThreads) codebook_kernel(CodebookArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CbSmem& S = *reinterpret_cast<CbSmem*>(smem_raw);
  __shared__ unsigned s_n, s_lp, s_qp, s_qe, s_pl, s_pq, s_leaves, s_rounds, s_maxd, s_total;
  const int dict = a.dict;
  uint16_t* merged = reinterpret_cast<uint16_t*>(S.keys);                      // [2*kMaxDict]
  uint16_t* round_end = reinterpret_cast<uint16_t*>(S.keys) + 2 * kMaxDict;    // [kMaxDict]
  for (int shift = 0;; ++shift) {
    // 1. present symbols as (freq' << 13 | sym) keys
    const int per = (dict + blockDim.x - 1) / blockDim.x;
    const int s0 = threadIdx.x * per;
    unsigned cnt = 0;
    for (int s = s0; s < s0 + per && s < dict; ++s) cnt += a.hist[s] ? 1u : 0u;
    unsigned pos = block_excl_scan(cnt, S.scan_tmp, &s_n);
    for (int s = s0; s < s0 + per && s < dict; ++s) {
      const unsigned f = a.hist[s];
      if (f) {
        const unsigned fs = shift ? max(1u, f >> shift) : f;
        S.keys[pos++] = ((unsigned long long)fs << 13) | (unsigned long long)s;
      }
    }
    for (int s = threadIdx.x; s < dict; s += blockDim.x) S.len[s] = 0;
    __syncthreads();
    const int n = (int)s_n;
    if (n <= 1) {
      if (n == 1 && threadIdx.x == 0) S.len[S.keys[0] & 8191ull] = 1;
      __syncthreads();
      break;
    }
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = n + threadIdx.x; i < P; i += blockDim.x) S.keys[i] = ~0ull;
    __syncthreads();
    bitonic_sort(S.keys, P);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      S.lw[i] = (unsigned)(S.keys[i] >> 13);
      S.ls[i] = (uint16_t)(S.keys[i] & 8191ull);
    }
    if (threadIdx.x == 0) { s_lp = 0; s_qp = 0; s_qe = 0; s_rounds = 0; s_leaves = 0; }
    __syncthreads();
    // 2. parallel rounds of the two-queue construction
    while (s_qe < (unsigned)(n - 1)) {
      if (threadIdx.x == 0) {
        unsigned lp = s_lp, qp = s_qp;
        const unsigned qe = s_qe;
        unsigned w[2];
        for (int t = 0; t < 2; ++t) {
          if (lp < (unsigned)n && (qp >= qe || S.lw[lp] <= S.iw[qp])) w[t] = S.lw[lp++];
          else w[t] = S.iw[qp++];
        }
        const unsigned X = w[0] + w[1];
        s_pl = (unsigned)upper_bound_u32(S.lw, s_lp, n, X) - s_lp;
        s_pq = (unsigned)upper_bound_u32(S.iw, s_qp, qe, X) - s_qp;
      }
      __syncthreads();
      const int lp = s_lp, qp = s_qp, qe = s_qe, pl = s_pl, pq = s_pq;
      const int npairs = (pl + pq) >> 1;
      for (int e = threadIdx.x; e < pl + pq; e += blockDim.x) {
        int rank, id;
        if (e < pl) {
          const int i = lp + e;
          rank = e + (lower_bound_u32(S.iw, qp, qp + pq, S.lw[i]) - qp);
          id = i;
        } else {
          const int j = qp + (e - pl);
          rank = (e - pl) + (upper_bound_u32(S.lw, lp, lp + pl, S.iw[j]) - lp);
          id = n + j;
        }
        if (rank < 2 * npairs) merged[rank] = (uint16_t)id;
      }
      __syncthreads();
      unsigned leaves = 0;
      for (int k = threadIdx.x; k < npairs; k += blockDim.x) {
        const int x = merged[2 * k], y = merged[2 * k + 1];
        const unsigned wx = x < n ? S.lw[x] : S.iw[x - n];
        const unsigned wy = y < n ? S.lw[y] : S.iw[y - n];
        S.iw[qe + k] = wx + wy;
        S.parent[x] = (uint16_t)(n + qe + k);
        S.parent[y] = (uint16_t)(n + qe + k);
        leaves += (x < n) + (y < n);
      }
      if (leaves) atomicAdd(&s_leaves, leaves);
      __syncthreads();
      if (threadIdx.x == 0) {
        s_lp += s_leaves;
        s_qp += 2 * npairs - s_leaves;
        s_qe += npairs;
        round_end[s_rounds++] = (uint16_t)s_qe;
        s_leaves = 0;
      }
      __syncthreads();
    }
    // 3. depths, rounds in reverse (a parent is always created in a later round)
    const int root = 2 * n - 2;
    if (threadIdx.x == 0) { S.depth[root] = 0; s_maxd = 0; }
    __syncthreads();
    for (int r = (int)s_rounds - 1; r >= 0; --r) {
      const int jb = r ? round_end[r - 1] : 0, je = round_end[r];
      for (int j = jb + threadIdx.x; j < je; j += blockDim.x) {
        const int v = n + j;
        if (v != root) S.depth[v] = S.depth[S.parent[v]] + 1;
      }
      __syncthreads();
    }
    unsigned md = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const unsigned d = S.depth[S.parent[i]] + 1u;
      S.len[S.ls[i]] = (uint8_t)min(d, 255u);
      md = max(md, d);
    }
    if (md) atomicMax(&s_maxd, md);
    __syncthreads();
    if (s_maxd <= (unsigned)kMaxLen) break;
    __syncthreads();
  }
  // 4. canonical codes
  unsigned* key32 = reinterpret_cast<unsigned*>(S.lw);  // lw/iw no longer needed
  uint16_t* canon = reinterpret_cast<uint16_t*>(S.iw);
  build_canonical(S.len, dict, key32, canon, &S.ct, S.scan_tmp);
  for (int i = threadIdx.x; i < (int)S.ct.n; i += blockDim.x) {
    const int s = canon[i];
    const int L = S.len[s];
    a.codes[s] = S.ct.first_code[L] + (unsigned)(i - (int)S.ct.first_pos[L]);
  }
  for (int s = threadIdx.x; s < dict; s += blockDim.x) {
    a.lens[s] = S.len[s];
    if (!S.len[s]) a.codes[s] = 0;
  }
  // 5. codebook runs {u32 first, u32 count, u8 len[count], pad to 4}
  unsigned* run_start = reinterpret_cast<unsigned*>(S.keys);            // [kMaxDict/2+1]
  unsigned* run_end = run_start + (kMaxDict / 2 + 1);                    // one past the last symbol
  unsigned* run_off = run_end + (kMaxDict / 2 + 1);
  const int per = (dict + blockDim.x - 1) / blockDim.x;
  const int s0 = threadIdx.x * per;
  auto is_start = [&](int s) { return S.len[s] && (s == 0 || !S.len[s - 1]); };
  auto is_end = [&](int s) { return S.len[s] && (s == dict - 1 || !S.len[s + 1]); };
  unsigned nst = 0, nen = 0;
  for (int s = s0; s < s0 + per && s < dict; ++s) { nst += is_start(s); nen += is_end(s); }
  unsigned r = block_excl_scan(nst, S.scan_tmp, &s_n);
  for (int s = s0; s < s0 + per && s < dict; ++s)
    if (is_start(s)) run_start[r++] = (unsigned)s;
  unsigned r2 = block_excl_scan(nen, S.scan_tmp, nullptr);
  for (int s = s0; s < s0 + per && s < dict; ++s)
    if (is_end(s)) run_end[r2++] = (unsigned)s + 1u;
  __syncthreads();
  const int nruns = (int)s_n;
  unsigned my_bytes = 0;
  const int rper = (nruns + blockDim.x - 1) / blockDim.x;
  const int r0 = threadIdx.x * rper;
  for (int q = r0; q < r0 + rper && q < nruns; ++q) my_bytes += 8u + (((run_end[q] - run_start[q]) + 3u) & ~3u);
  unsigned off = block_excl_scan(my_bytes, S.scan_tmp, &s_total);
  for (int q = r0; q < r0 + rper && q < nruns; ++q) {
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
      *reinterpret_cast<unsigned*>(p) = first;
      *reinterpret_cast<unsigned*>(p + 4) = cntq;
      for (unsigned t = cntq; t < ((cntq + 3u) & ~3u); ++t) p[8 + t] = 0;
    }
    // length bytes: symbol s of run q goes to run_off[q] + 8 + (s - first)
    for (int s = threadIdx.x; s < dict; s += blockDim.x) {
      if (!S.len[s]) continue;
      const int q = upper_bound_u32(run_start, 0, nruns, (unsigned)s) - 1;
      a.out[a.off + run_off[q] + 8 + (s - run_start[q])] = S.len[s];
    }
    if (threadIdx.x == 0)
      for (unsigned long long t = total; t < pad8(total); ++t) a.out[a.off + t] = 0;
  }
  if (threadIdx.x == 0) {
    a.sc->codebook_bytes = total;
    a.sc->n_runs = (unsigned long long)nruns;
    a.sc->max_len = S.ct.max_len;
    if (a.out && !fits) atomicOr(&a.sc->status, ST_CAPACITY | ST_RAW);
  }
}

// Histogram of a symbol array (stand-alone Huffman entry point).
__global__ void hist_kernel(const uint16_t* __restrict__ sym, unsigned long long n, int dict, unsigned* hist,
                            Scalars* sc) {
  extern __shared__ unsigned hs[];
  for (int i = threadIdx.x; i < dict; i += blockDim.x) hs[i] = 0;
  __syncthreads();
  bool bad = false;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned s = sym[i];
    if (s < (unsigned)dict) atomicAdd(hs + s, 1u);
    else bad = true;
  }
  if (bad) atomicOr(&sc->status, ST_CORRUPT);
  __syncthreads();
  for (int i = threadIdx.x; i < dict; i += blockDim.x)
    if (hs[i]) atomicAdd(hist + i, hs[i]);
}

// ---------------------------------------------------------------------------
// Encoding: one warp per chunk; lane j codes a contiguous slice of the chunk.
// ---------------------------------------------------------------------------
struct EncodeArgs {
  const uint16_t* sym;
  const int32_t* esc;          // codes of escaped symbols (symbol 0), or null
  unsigned long long n;
  int chunk;
  const uint8_t* lens;
  const unsigned* codes;
  int dict;
  unsigned* chunk_words;       // [nch] (stream section)
  unsigned* chunk_esc;         // [nch] scratch
  unsigned long long* word_off;  // [nch+1]
  unsigned long long* esc_off;   // [nch+1]
  unsigned long long nch;
  uint8_t* out;                // stream base
  Scalars* sc;
};

__device__ __forceinline__ void lane_slice(const EncodeArgs& a, unsigned long long c, int lane,
                                           unsigned long long& s0, unsigned long long& s1) {
  const int per = a.chunk / 32;
  const unsigned long long cb = c * (unsigned long long)a.chunk;
  s0 = cb + (unsigned long long)lane * per;
  s1 = s0 + per;
  const unsigned long long ce = min(a.n, cb + (unsigned long long)a.chunk);
  if (s0 > ce) s0 = ce;
  if (s1 > ce) s1 = ce;
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) chunk_bits_kernel(EncodeArgs a) {
  __shared__ uint8_t lens[kMaxDict];
  for (int i = threadIdx.x; i < a.dict; i += blockDim.x) lens[i] = a.lens[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (unsigned long long c = blockIdx.x * (unsigned long long)WARPS + (threadIdx.x >> 5); c < a.nch;
       c += (unsigned long long)gridDim.x * WARPS) {
    unsigned long long s0, s1;
    lane_slice(a, c, lane, s0, s1);
    unsigned bits = 0, esc = 0;
    for (unsigned long long i = s0; i < s1; ++i) {
      const unsigned s = min((unsigned)a.sym[i], (unsigned)(a.dict - 1));
      bits += lens[s];
      esc += (s == 0);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      bits += __shfl_xor_sync(0xffffffffu, bits, o);
      esc += __shfl_xor_sync(0xffffffffu, esc, o);
    }
    if (lane == 0) {
      if (a.chunk_words) a.chunk_words[c] = (bits + 31u) >> 5;
      a.chunk_esc[c] = a.esc ? esc : 0u;
    }
  }
}

// Exclusive scans of the chunk word counts and escape counts (one CTA), then
// the stream offsets of the bitstream, the per-chunk escape counts (present
// only when there are escapes) and the outlier codes.
__global__ void __launch_bounds__(kCbThreads) chunk_scan_kernel(const unsigned* chunk_words, const unsigned* chunk_esc,
                                                                unsigned long long nch, unsigned long long* word_off,
                                                                unsigned long long* esc_off, Scalars* sc,
                                                                unsigned long long off_codebook,
                                                                unsigned long long raw_total,
                                                                unsigned long long capacity, uint8_t* out) {
  __shared__ unsigned long long wt[32], et[32];
  __shared__ unsigned long long carry_w, carry_e;
  __shared__ int s_write;
  if (threadIdx.x == 0) { carry_w = 0; carry_e = 0; }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (unsigned long long base = 0; base < nch; base += blockDim.x) {
    const unsigned long long i = base + threadIdx.x;
    unsigned long long w = i < nch ? chunk_words[i] : 0ull;
    unsigned long long e = i < nch ? chunk_esc[i] : 0ull;
    unsigned long long xw = w, xe = e;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long yw = __shfl_up_sync(0xffffffffu, xw, o);
      const unsigned long long ye = __shfl_up_sync(0xffffffffu, xe, o);
      if (lane >= o) { xw += yw; xe += ye; }
    }
    if (lane == 31) { wt[wid] = xw; et[wid] = xe; }
    __syncthreads();
    if (wid == 0) {
      unsigned long long tw = wt[lane], te = et[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long yw = __shfl_up_sync(0xffffffffu, tw, o);
        const unsigned long long ye = __shfl_up_sync(0xffffffffu, te, o);
        if (lane >= o) { tw += yw; te += ye; }
      }
      wt[lane] = tw;
      et[lane] = te;
    }
    __syncthreads();
    const unsigned long long bw = carry_w + (wid ? wt[wid - 1] : 0ull) + xw - w;
    const unsigned long long be = carry_e + (wid ? et[wid - 1] : 0ull) + xe - e;
    if (i < nch) { word_off[i] = bw; esc_off[i] = be; }
    __syncthreads();
    if (threadIdx.x == 0) { carry_w += wt[31]; carry_e += et[31]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    word_off[nch] = carry_w;
    esc_off[nch] = carry_e;
    sc->n_words = carry_w;
    sc->n_outliers = carry_e;
    const unsigned long long off_bits = off_codebook + pad8(sc->codebook_bytes);
    const unsigned long long off_ce = off_bits + pad8(4ull * carry_w);
    const unsigned long long off_out = off_ce + (carry_e ? pad8(4ull * nch) : 0ull);
    const unsigned long long total = off_out + pad8(4ull * carry_e);
    sc->off_bits = off_bits;
    sc->off_chunk_esc = off_ce;
    sc->off_outliers = off_out;
    sc->total = total;
    if (total >= raw_total || total > capacity) atomicOr(&sc->status, ST_RAW);
    if (sc->status & ST_OVERFLOW) atomicOr(&sc->status, ST_RAW);
    s_write = out && carry_e && !(sc->status & ST_RAW);
  }
  __syncthreads();
  if (s_write) {
    unsigned* dst = reinterpret_cast<unsigned*>(out + sc->off_chunk_esc);
    for (unsigned long long i = threadIdx.x; i < nch; i += blockDim.x) dst[i] = chunk_esc[i];
  }
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) encode_kernel(EncodeArgs a) {
  __shared__ uint8_t lens[kMaxDict];
  __shared__ unsigned codes[kMaxDict];
  if (a.sc && (a.sc->status & ST_RAW)) return;
  for (int i = threadIdx.x; i < a.dict; i += blockDim.x) { lens[i] = a.lens[i]; codes[i] = a.codes[i]; }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  unsigned* words = reinterpret_cast<unsigned*>(a.out + a.sc->off_bits);
  int32_t* ocode = reinterpret_cast<int32_t*>(a.out + a.sc->off_outliers);
  for (unsigned long long c = blockIdx.x * (unsigned long long)WARPS + (threadIdx.x >> 5); c < a.nch;
       c += (unsigned long long)gridDim.x * WARPS) {
    unsigned long long s0, s1;
    lane_slice(a, c, lane, s0, s1);
    unsigned bits = 0, esc = 0;
    for (unsigned long long i = s0; i < s1; ++i) {
      const unsigned s = min((unsigned)a.sym[i], (unsigned)(a.dict - 1));
      bits += lens[s];
      esc += (s == 0);
    }
    unsigned xb = bits, xe = esc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned yb = __shfl_up_sync(0xffffffffu, xb, o);
      const unsigned ye = __shfl_up_sync(0xffffffffu, xe, o);
      if (lane >= o) { xb += yb; xe += ye; }
    }
    const unsigned bit0 = xb - bits, esc0 = xe - esc;
    const unsigned long long wbase = a.word_off[c];
    const unsigned nw = (unsigned)(a.word_off[c + 1] - wbase);
    for (unsigned w = lane; w < nw; w += 32) words[wbase + w] = 0u;
    __syncwarp();
    unsigned long long acc = 0;
    unsigned nb = bit0 & 31u;
    unsigned long long widx = wbase + (bit0 >> 5);
    bool shared_first = (bit0 & 31u) != 0;
    unsigned long long epos = a.esc_off[c] + esc0;
    for (unsigned long long i = s0; i < s1; ++i) {
      const unsigned s = min((unsigned)a.sym[i], (unsigned)(a.dict - 1));
      const unsigned L = lens[s];
      acc = (acc << L) | codes[s];
      nb += L;
      if (nb >= 32) {
        const unsigned word = (unsigned)(acc >> (nb - 32));
        if (shared_first) { atomicOr(words + widx, word); shared_first = false; }
        else words[widx] = word;
        ++widx;
        nb -= 32;
        acc &= (nb ? ((1ull << nb) - 1ull) : 0ull);
      }
      if (s == 0 && a.esc) ocode[epos++] = a.esc[i];
    }
    if (nb) atomicOr(words + widx, (unsigned)(acc << (32 - nb)));
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Decoding
// ---------------------------------------------------------------------------
struct DtSmem {
  uint8_t len[kMaxDict];
  unsigned key32[kMaxDict];
  uint16_t canon[kMaxDict];
  unsigned scan_tmp[64];
  CanonTables ct;
  unsigned rfirst[512], rcount[512], roff[512];
};

// Build decode tables from the stream's codebook runs (one CTA).
__global__ void __launch_bounds__(kCbThreads) decode_tables_kernel(const uint8_t* runs, unsigned long long nbytes,
                                                                   unsigned long long n_runs, int dict,
                                                                   DecodeTables* out, Scalars* sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DtSmem& S = *reinterpret_cast<DtSmem*>(smem_raw);
  __shared__ unsigned s_bad;
  __shared__ unsigned long long s_kr;
  if (threadIdx.x == 0) { s_bad = 0; s_kr = 0; }
  for (int s = threadIdx.x; s < dict; s += blockDim.x) S.len[s] = 0;
  __syncthreads();
  // walk the run headers (serial over runs, parallel over each run's bytes)
  unsigned long long off = 0;
  for (unsigned long long rb = 0; rb < n_runs; rb += 512) {
    const int nb = (int)min(512ull, n_runs - rb);
    if (threadIdx.x == 0) {
      for (int q = 0; q < nb; ++q) {
        if (off + 8 > nbytes) { s_bad = 1; break; }
        const unsigned first = *reinterpret_cast<const unsigned*>(runs + off);
        const unsigned cnt = *reinterpret_cast<const unsigned*>(runs + off + 4);
        if ((unsigned long long)first + cnt > (unsigned long long)dict || off + 8 + cnt > nbytes) { s_bad = 1; break; }
        S.rfirst[q] = first; S.rcount[q] = cnt; S.roff[q] = (unsigned)off;
        off += 8ull + ((cnt + 3u) & ~3u);
      }
    }
    __syncthreads();
    if (s_bad) break;
    for (int q = 0; q < nb; ++q)
      for (unsigned t = threadIdx.x; t < S.rcount[q]; t += blockDim.x) S.len[S.rfirst[q] + t] = runs[S.roff[q] + 8 + t];
    __syncthreads();
  }
  // Kraft sum (exact, in units of 2^-32) and the length bound
  unsigned long long kr = 0;
  for (int s = threadIdx.x; s < dict; s += blockDim.x) {
    const unsigned L = S.len[s];
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
  build_canonical(S.len, dict, S.key32, S.canon, &S.ct, S.scan_tmp);
  for (int i = threadIdx.x; i < (1 << kLutBits); i += blockDim.x) out->lut[i] = 0;
  for (int i = threadIdx.x; i < (int)S.ct.n; i += blockDim.x) out->canon[i] = S.canon[i];
  __syncthreads();
  for (int i = threadIdx.x; i < (int)S.ct.n; i += blockDim.x) {
    const int s = S.canon[i];
    const unsigned L = S.len[s];
    if (L <= (unsigned)kLutBits) {
      const unsigned code = S.ct.first_code[L] + (unsigned)(i - (int)S.ct.first_pos[L]);
      const unsigned b0 = code << (kLutBits - L), cnt = 1u << (kLutBits - L);
      for (unsigned t = 0; t < cnt; ++t) out->lut[b0 + t] = (unsigned)s | (L << 16);
    }
  }
  if (threadIdx.x == 0) out->ct = S.ct;
}

struct DecodeArgs {
  const unsigned* words;            // bitstream
  unsigned long long n_words;
  const unsigned long long* esc_off;  // [nch+1] first outlier of each chunk, or null without outliers
  const int32_t* ocode;               // outlier codes in stream order
  int32_t* esc;                       // codes of escaped symbols, indexed like sym
  int stream_mode;                    // symbol 0 is the escape symbol (must have an outlier code)
  const unsigned long long* word_off;  // [nch+1]
  unsigned long long nch;
  unsigned long long n;
  int chunk;
  const DecodeTables* tab;
  uint16_t* sym;
  Scalars* sc;
};

// One thread per chunk, table-driven canonical decoding with a 64-bit window.
__global__ void __launch_bounds__(256) decode_kernel(DecodeArgs a) {
  __shared__ unsigned lut[1 << kLutBits];
  __shared__ uint16_t canon[kMaxDict];
  __shared__ unsigned long long limit[kMaxLen + 2];
  __shared__ unsigned fcode[kMaxLen + 2], fpos[kMaxLen + 2];
  const DecodeTables* T = a.tab;
  for (int i = threadIdx.x; i < (1 << kLutBits); i += blockDim.x) lut[i] = T->lut[i];
  const unsigned nsym = T->ct.n;
  for (int i = threadIdx.x; i < (int)nsym; i += blockDim.x) canon[i] = T->canon[i];
  if (threadIdx.x < kMaxLen + 2) {
    limit[threadIdx.x] = T->ct.limit[threadIdx.x];
    fcode[threadIdx.x] = T->ct.first_code[threadIdx.x];
    fpos[threadIdx.x] = T->ct.first_pos[threadIdx.x];
  }
  __syncthreads();
  for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < a.nch;
       c += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long w = a.word_off[c];
    const unsigned long long wend = a.word_off[c + 1];
    if (wend < w || wend > a.n_words) { atomicOr(&a.sc->status, ST_CORRUPT); continue; }
    const unsigned long long s0 = c * (unsigned long long)a.chunk;
    const unsigned long long s1 = min(a.n, s0 + (unsigned long long)a.chunk);
    unsigned long long buf = 0;
    int nbits = 0;
    bool bad = false;
    unsigned long long epos = a.esc_off ? a.esc_off[c] : 0ull;
    const unsigned long long eend = a.esc_off ? a.esc_off[c + 1] : 0ull;
    for (unsigned long long i = s0; i < s1; ++i) {
      while (nbits <= 32 && w < wend) {
        buf |= (unsigned long long)a.words[w++] << (32 - nbits);
        nbits += 32;
      }
      const unsigned peek = (unsigned)(buf >> 32);
      const unsigned e = lut[peek >> (32 - kLutBits)];
      unsigned s, L;
      if (e >> 16) {
        L = e >> 16;
        s = e & 0xFFFFu;
      } else {
        L = kLutBits + 1;
        while (L <= (unsigned)kMaxLen && (unsigned long long)peek >= limit[L]) ++L;
        if (L > (unsigned)kMaxLen) { bad = true; break; }
        const unsigned idx = fpos[L] + ((peek >> (32 - L)) - fcode[L]);
        if (idx >= nsym) { bad = true; break; }
        s = canon[idx];
      }
      if ((int)L > nbits) { bad = true; break; }
      buf <<= L;
      nbits -= (int)L;
      a.sym[i] = (uint16_t)s;
      if (s == 0 && a.stream_mode) {
        if (epos >= eend) { bad = true; break; }
        a.esc[i] = a.ocode[epos++];
      }
    }
    if (a.esc_off && !bad && epos != eend) bad = true;
    if (bad) atomicOr(&a.sc->status, ST_CORRUPT);
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
