// Launchers shared between the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "bm_common.cuh"

namespace bm {

template <typename T>
struct BlockArgs {
  T* field;  // fwd: input (read); inv: output (written)
  int64_t n0, n1, n2;
  int nb0, nb1, nb2;
  int64_t nblocks;
  T* G;  // gathered block-coarse grid, row-major (nb0*m, nb1*m, nb2*m)
  int64_t g1, g2;
  uint16_t* sym;  // symbols, per_block per block (mode 0)
  int32_t* esc;   // codes of escaped symbols, indexed like sym
  T* coef;        // coefficients (mode 1)
  const uint8_t* tier;  // per block tier or null
  const T* rq;          // fwd: 1/q per [tier*K + level]
  const double* q;      // inv: q per [tier*K + level]
  unsigned* hist;       // global histogram [2*radius]
  int radius;
  Scalars* sc;
  int ntiers;           // inv: tiers in the q table (a block tier at or above it is corrupt)
};


// In-cache Block kernels for one (dtype, B): dir 0 = decompose (+quantise),
// dir 1 = recompose; mode 0 = symbols, 1 = full-precision coefficients.
// Returns cudaErrorInvalidValue for an unsupported K.
// max_grid > 0 caps the persistent grid (several blocks per CTA at any size).
cudaError_t launch_block_f32_b9(int dir, int K, int mode, const BlockArgs<float>& a, cudaStream_t s, int nsm,
                                int max_grid);
cudaError_t launch_block_f32_b17(int dir, int K, int mode, const BlockArgs<float>& a, cudaStream_t s, int nsm,
                                 int max_grid);
cudaError_t launch_block_f64_b9(int dir, int K, int mode, const BlockArgs<double>& a, cudaStream_t s, int nsm,
                                int max_grid);
cudaError_t launch_block_f64_b17(int dir, int K, int mode, const BlockArgs<double>& a, cudaStream_t s, int nsm,
                                 int max_grid);

// Batched forward In-cache Block kernel (max|u|, quantiser tables and the
// blocks of every field of a batch sharing dtype, B and K; mode 0).
template <typename T>
struct BatchField;
struct BatchQueue;
cudaError_t launch_block_batch_f32_b9(int K, const BatchField<float>* fields, const BatchQueue& q, cudaStream_t s,
                                      int nsm);
cudaError_t launch_block_batch_f32_b17(int K, const BatchField<float>* fields, const BatchQueue& q, cudaStream_t s,
                                       int nsm);
cudaError_t launch_block_batch_f64_b9(int K, const BatchField<double>* fields, const BatchQueue& q, cudaStream_t s,
                                      int nsm);
cudaError_t launch_block_batch_f64_b17(int K, const BatchField<double>* fields, const BatchQueue& q, cudaStream_t s,
                                       int nsm);

// Transposed In-cache Block levels: dir 0 = transposed decomposition
// (coefficient and block-coarse gradients -> field gradients), dir 1 =
// transposed recomposition (field gradients -> coefficient and block-coarse
// gradients).  cudaErrorInvalidValue for an unsupported (B, K).
cudaError_t launch_block_adj_f32(int dir, int B, int K, const BlockArgs<float>& a, cudaStream_t s, int nsm);
cudaError_t launch_block_adj_f64(int dir, int B, int K, const BlockArgs<double>& a, cudaStream_t s, int nsm);

}  // namespace bm
