/*
 * blockmgard.h — C ABI of the GB300 (sm_103a) BlockMGARD compressor.
 *
 * The library implements the data-parallel hot path of BlockMGARD (SC26):
 *   (a) In-cache Block multilevel decomposition of fixed B^3 blocks held in
 *       shared memory (Sec. III-A), fused with (c) quantisation (Sec. III-D);
 *   (b) the hybrid hand-off: M global MGARD levels on the gathered
 *       block-coarse nodes (Sec. III-B);
 *   (c) ROI-aware, level-scaled quantisation with per-block tolerances and
 *       tau_global = min_i tau_i (Sec. II-B error shares, Sec. III-C);
 *   (d) Huffman coding of the quantised symbols (Sec. III-B lossless stage);
 * and the inverse of all four.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are device pointers (cudaMalloc'd or torch-owned) on
 *     the current CUDA device; h_* are host pointers.  The caller owns every
 *     buffer it passes.  The library allocates only internal scratch, cached
 *     per CUDA stream and released by bm_release_workspace().
 *   - `stream` is a cudaStream_t passed as void* (0 = legacy default stream).
 *     All device work is ordered on that stream.  Calls that return sizes
 *     (bm_compress) synchronise the stream before returning.  A call's own
 *     small transfers (tolerance tables, status block, stream header) are done
 *     by a kernel through the device mapping of the library's pinned staging
 *     memory, not by copy-engine copies, so a call does not wait behind bulk
 *     copies the caller has queued on other streams.
 *   - Fields have ndim = 1, 2 or 3 dimensions, row-major (C order) with the
 *     last extent varying fastest; `shape` holds ndim extents, each >= 1, at
 *     least two values in all.  A field is handled as 3-D with leading extents
 *     of 1, and a dimension of extent 1 is neither blocked nor coarsened (its
 *     blocks are one node thick), so a 1-D or 2-D field gets the 1-D or 2-D
 *     transform.  dtype: BM_F32 or BM_F64.
 *   - Every call returns a bm_status.  On failure a readable message is
 *     available from bm_last_error_detail() (thread-local); no output buffer
 *     is guaranteed to hold meaningful data.  Invalid arguments are rejected
 *     on the host before any device work is issued.
 *   - The library is not re-entrant on the same stream from several host
 *     threads at once; distinct streams may be used concurrently.
 */
#ifndef BLOCKMGARD_H
#define BLOCKMGARD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { BM_F32 = 0, BM_F64 = 1 } bm_dtype;

typedef enum {
  BM_OK = 0,
  BM_ERR_ARG = 1,          /* invalid argument (shape, tolerance, parameters) */
  BM_ERR_CUDA = 2,         /* a CUDA runtime call failed                      */
  BM_ERR_CAPACITY = 3,     /* output buffer smaller than needed               */
  BM_ERR_CORRUPT = 4,      /* input stream malformed or truncated             */
  BM_ERR_UNSUPPORTED = 5,  /* valid but not supported by this build           */
  BM_ERR_OOM = 6           /* scratch allocation failed                       */
} bm_status;

/* Tolerance mode: BM_ABS = tol is absolute; BM_REL = tol (and every ROI entry)
 * is relative to max|u| (the paper's L-inf relative bound, Sec. IV-A). */
typedef enum { BM_ABS = 0, BM_REL = 1 } bm_tol_mode;

/* Hierarchy parameters (Sec. III-A block size, Sec. III-B L/M; the paper's L
 * is incache_levels here).  Zero-initialised fields take the defaults. */
typedef struct {
  int block_nodes;     /* B: nodes per block edge; this build supports 9, 17 (default 17) */
  int incache_levels;  /* K >= 1: levels done while the block is resident (default 2)    */
  int global_levels;   /* M >= 0: MGARD levels on the gathered coarse grid (default 2;
                          -1 selects 0)                                                  */
  int chunk_symbols;   /* Huffman chunk length in symbols, multiple of 32, 64..2048
                          (default 2048)                                                 */
  int dict_radius;     /* quantisation codes with |code| < radius become 16-bit symbols
                          code + radius; others are outliers.  16..32768 (default 32768) */
  int rounds;          /* R, 1..8 (0 = 1): re-blocking rounds of K in-cache levels each;
                          round r+1 re-blocks round r's gathered coarse values and takes
                          the strictest tolerance among the blocks each new block holds
                          coarse values of (Sec. III-C).  With R > 1 the global levels use
                          index coordinates; the adjoint entry points need R = 1.  R > 1
                          needs a 3-D field without extents of 1.                       */
} bm_params;

/* Upper bound on the stream size for a field of this shape and dtype: the raw
 * fallback (256-byte header + the field) always fits.  0 on invalid input. */
size_t bm_compress_bound(int ndim, const int64_t* shape, bm_dtype dtype);

/* Compress one field (Sec. III, the whole pipeline of Fig. 1).
 *   d_field     device pointer to the field, shape[0]*shape[1]*shape[2] values
 *               of `dtype`, row-major.
 *   tol         error tolerance (> 0, finite); absolute or relative (tol_mode).
 *   h_roi_tol   optional host array with one tolerance per block (B nodes along
 *               every dimension of extent > 1), row-major over the block grid
 *               ceil(shape[d]/B); same mode as tol.  Block i's tolerance is min(tol, h_roi_tol[i]) (Sec. III-C
 *               block-wise tolerance assignment).  NULL = uniform.  At most 255
 *               distinct values.
 *   d_out       device buffer for the stream; out_capacity bytes (use
 *               bm_compress_bound()).
 *   out_bytes   receives the stream length (host pointer).
 * Guarantee: decompression reproduces every node of block i within its
 * tolerance (L-inf), including floating-point round-off, or the stream is a
 * raw copy of the field (when the field holds non-finite values, the tolerance
 * is too close to round-off, or coding would not shrink it). */
bm_status bm_compress(const void* d_field, int ndim, const int64_t* shape, bm_dtype dtype, double tol,
                      bm_tol_mode tol_mode, const double* h_roi_tol, const bm_params* params, void* d_out,
                      size_t out_capacity, size_t* out_bytes, void* stream);

/* Header of a stream (the first 256 bytes, host or device memory: set
 * `in_is_device`).  Any output pointer may be NULL; shape receives the
 * field's ndim extents (unused entries 0). */
bm_status bm_stream_info(const void* in, size_t in_bytes, int in_is_device, int* ndim, int64_t shape[3],
                         bm_dtype* dtype, size_t* n_coeffs);

/* Decompress a stream produced by bm_compress into d_field (device, sized by
 * bm_stream_info).  Inverse of every stage (Sec. III; Huffman decode,
 * dequantisation, global then In-cache Block recomposition).  Malformed
 * streams give BM_ERR_CORRUPT; device-side decoding checks every read against
 * the stream bounds and reports through a status word rather than trapping. */
bm_status bm_decompress(const void* d_in, size_t in_bytes, void* d_field, void* stream);

/* Performance model of the compress pipeline on this GPU (Sec. III-B): the
 * In-cache Block stage follows Eq. 1 (time of N blocks = 1/Slope +
 * N/TP_peak, i.e. TP(N) = N / (1/Slope + N/TP_peak)); the global levels, the
 * histogram and the encoder are straight lines in their size; the codebook and
 * the remaining small stages are constants.  Times in ms. */
typedef struct {
  double block_latency_ms;      /* 1/Slope */
  double block_peak_per_ms;     /* TP_peak, blocks per ms */
  double global_ms, global_ms_per_node;       /* per global level */
  double hist_ms, hist_ms_per_symbol;         /* max of the two */
  double codebook_ms;
  double encode_ms, encode_ms_per_symbol;     /* max of the two */
  double other_ms;
  int block_nodes, incache_levels;            /* configuration the fit was taken with */
  bm_dtype dtype;
} bm_perf_model;

/* Fits the model by compressing synthetic fields of 1^3 .. 22^3 blocks of
 * block_nodes nodes (default levels) on `stream` with stage timing; allocates
 * and frees its own buffers (up to ~1.6 GB for FP32, B = 17).  Synchronous. */
bm_status bm_perf_model_fit(bm_dtype dtype, int block_nodes, bm_perf_model* model, void* stream);
/* Block count at which Eq. 1 reaches `fraction` (0..1) of TP_peak (the knee). */
double bm_perf_model_knee(const bm_perf_model* model, double fraction);
/* Predicted compress time of one field with these parameters. */
bm_status bm_predict_ms(const bm_perf_model* model, int ndim, const int64_t* shape, const bm_params* params,
                        double* ms);
/* Alg. 1: among the (in-cache levels K, global levels M) pairs whose
 * predicted time is within budget_ms, the largest in (M, -K) (more global
 * levels first, then fewer in-cache levels); block size as in the model.
 * BM_ERR_UNSUPPORTED when no pair fits. */
bm_status bm_select_params(const bm_perf_model* model, int ndim, const int64_t* shape, double budget_ms,
                           bm_params* out, double* predicted_ms);

/* One field of a batched compress: the arguments of bm_compress for it. */
typedef struct {
  const void* d_field;
  int ndim;
  int64_t shape[3];
  bm_dtype dtype;
  double tol;
  bm_tol_mode tol_mode;
  const double* h_roi_tol; /* nullable, as for bm_compress */
  bm_params params;
  void* d_out;
  size_t out_capacity;
} bm_batch_item;

/* Compresses n independent fields (Sec. III-B throughput model, Sec. III-D:
 * many fields per launch).  Every 3-D field (no extent of 1) with B in
 * {9, 17} and one round has its max|u| pass, quantiser table and In-cache
 * Block stage done by one persistent kernel launch per (dtype, B, K), whose
 * CTAs take work items (slices of max|u|, then single blocks) from a
 * device-side queue spanning all those fields; a block waits, with a bounded
 * wait (status BM_ERR_CUDA if it ever ran out), for its field's quantiser
 * table.  The other stages, and whole pipelines of the other fields, are
 * queued on a pool of the library's streams, forked from and joined back
 * into `stream`, without any host synchronisation until all are queued; then
 * one synchronisation and the per-field sizes in out_bytes[i] (host array of
 * n).  Each field gives the same stream, byte for byte, as bm_compress with
 * the same arguments.  Device scratch for the batched fields (their symbols,
 * escape codes and levels at once) is kept by the library between calls.
 * item_status (host array of n, nullable) receives each field's status; the
 * return value is the first non-OK status, or BM_OK.  Buffers are owned by
 * the caller; fields and outputs must not overlap. */
bm_status bm_compress_batch(int n, const bm_batch_item* items, size_t* out_bytes, bm_status* item_status,
                            void* stream);

/* Multilevel decomposition only (Sec. II-B / III-A / III-B), no quantisation:
 * writes the n_coeffs full-precision coefficients to d_coeffs (same dtype as
 * the field) in stream order: blocks row-major; inside a block levels finest
 * to coarsest, each level's non-coarse nodes row-major; then the global
 * levels finest to coarsest (row-major); then the coarsest grid (row-major).
 * n_coeffs comes from bm_coeff_count(). */
bm_status bm_decompose(const void* d_field, int ndim, const int64_t* shape, bm_dtype dtype,
                       const bm_params* params, void* d_coeffs, void* stream);

/* Inverse of bm_decompose (recomposition, Sec. II-B): coefficients in stream
 * order to the field. */
bm_status bm_recompose(const void* d_coeffs, int ndim, const int64_t* shape, bm_dtype dtype,
                       const bm_params* params, void* d_field, void* stream);

/* Adjoints (transposes) of the two linear operators above, for gradients
 * (Sec. II-B: each level is linear; its transpose is built from M_f I M_c^-1
 * and I^T along each dimension).  bm_decompose_adjoint: d_coeff_grad
 * (n_coeffs values, stream order, read) -> d_field_grad (the field's shape,
 * written; nodes outside the domain of a padded block have no field entry
 * and receive nothing).  bm_recompose_adjoint: d_field_grad (read) ->
 * d_coeff_grad (n_coeffs, written).  Same dtype, parameters and errors as
 * bm_decompose, except that they need a 3-D field without extents of 1
 * (BM_ERR_UNSUPPORTED otherwise); both run asynchronously on `stream` and
 * allocate nothing beyond the cached workspace. */
bm_status bm_decompose_adjoint(const void* d_coeff_grad, int ndim, const int64_t* shape, bm_dtype dtype,
                               const bm_params* params, void* d_field_grad, void* stream);
bm_status bm_recompose_adjoint(const void* d_field_grad, int ndim, const int64_t* shape, bm_dtype dtype,
                               const bm_params* params, void* d_coeff_grad, void* stream);

/* Number of coefficients (= quantised symbols) for a shape and parameters. */
bm_status bm_coeff_count(int ndim, const int64_t* shape, const bm_params* params, size_t* n_coeffs);

/* Integer quantisation codes of a (non-raw) stream, decoded on the device:
 * d_codes receives n_coeffs int32 values in stream order (outliers applied). */
bm_status bm_stream_codes(const void* d_in, size_t in_bytes, int32_t* d_codes, void* stream);

/* Stand-alone Huffman stage (Sec. III-B lossless stage; cuSZ-style chunked
 * coding, "deflate" = concatenation of chunk codes): encodes n uint16 symbols
 * (each < dict_size, dict_size <= 65536; n < 2^31) into the section layout used inside
 * streams: u32 chunk word counts | u16 split offsets (bit offsets of the
 * eighths 1..7 of every chunk) | codebook runs | u32 code words, each part
 * padded to 8 bytes.  chunk_symbols: multiple of 32 in [64, 2048].  sizes_out[0..4] = codebook bytes, runs, chunks, words,
 * total bytes.  Synchronises the stream. */
bm_status bm_huffman_encode(const uint16_t* d_symbols, uint64_t n, int dict_size, int chunk_symbols,
                            void* d_out, size_t out_capacity, uint64_t sizes_out[5], void* stream);

/* Allocation-free variant of bm_huffman_encode (this entry point has no
 * counterpart in the paper).  Same arguments, same output bytes, but it calls
 * no cudaMalloc/cudaFree and no allocating library routine.  It is meant for
 * callers that cannot allocate device memory: a process whose device memory
 * is entirely reserved by another allocator (a framework's caching pool that
 * took the whole GPU up front), or a latency-critical loop that cannot accept
 * the device-wide synchronisation a cudaMalloc or cudaFree may imply.
 * Its scratch is one static device array of 1 MiB per GPU that loads this
 * library, held until the process exits; it limits a call to at most 16384
 * chunks (n <= 16384 * chunk_symbols), larger requests return BM_ERR_ARG.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it for the life of the process; the cached
 * address does not survive cudaDeviceReset, so do not call this entry point
 * after resetting a device.  Every call shares the array and it keeps the
 * last call's contents (the call clears what must start at zero), so calls
 * whose GPU work overlaps in time (different streams, different host
 * threads) race and must be serialised by the caller.
 * The call ends by copying its status to the host and synchronising the
 * stream, so it must not be issued on a stream that is being captured into a
 * CUDA graph: on a capturing stream it returns BM_ERR_ARG before enqueuing
 * anything. */
bm_status bm_huffman_encode_noalloc(const uint16_t* d_symbols, uint64_t n, int dict_size, int chunk_symbols,
                                    void* d_out, size_t out_capacity, uint64_t sizes_out[5], void* stream);

/* Inverse of bm_huffman_encode: sizes as returned by it; writes n symbols. */
bm_status bm_huffman_decode(const void* d_section, const uint64_t sizes[5], uint64_t n, int dict_size,
                            int chunk_symbols, uint16_t* d_symbols, void* stream);

/* Free the scratch cached for `stream` (NULL/0 = every stream). */
void bm_release_workspace(void* stream);

/* Instrumentation: when enabled, every stage records CUDA events on the
 * call's stream; bm_stage_times() returns the last call's per-stage
 * milliseconds (names[i] static strings), up to max_stages entries. */
void bm_set_timing(int enabled);
int bm_stage_times(const char** names, float* ms, int max_stages);
/* The same, plus each stage's start in milliseconds after the start of the
 * call's first stage (stages on the second stream overlap the others). */
int bm_stage_timeline(const char** names, float* ms, float* start_ms, int max_stages);
/* Test hook: cap the persistent grid of the In-cache Block kernels at
 * max_ctas CTAs (0 = the occupancy-based default), so that small fields also
 * make every CTA walk several blocks.  Process-wide; results do not depend on
 * it. */
void bm_set_block_grid_limit(int max_ctas);
/* Count of kernels this library has launched since load (monotonic). */
uint64_t bm_launch_count(void);

const char* bm_error_string(bm_status s);
const char* bm_last_error_detail(void);

#ifdef __cplusplus
}
#endif
#endif /* BLOCKMGARD_H */
