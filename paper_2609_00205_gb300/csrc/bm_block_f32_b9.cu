// In-cache Block kernels instantiated for float fields and 9-node blocks.
#include "bm_block_launch.cuh"

namespace bm {

cudaError_t launch_block_f32_b9(int dir, int K, int mode, const BlockArgs<float>& a, cudaStream_t s, int nsm,
                                 int max_grid) {
  switch (K) {
    case 1: return launch_mode<float, 9, 1>(dir, mode, a, s, nsm, max_grid);
    case 2: return launch_mode<float, 9, 2>(dir, mode, a, s, nsm, max_grid);
    case 3: return launch_mode<float, 9, 3>(dir, mode, a, s, nsm, max_grid);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_block_batch_f32_b9(int K, const BatchField<float>* fields, const BatchQueue& q, cudaStream_t s,
                                    int nsm) {
  return launch_batch_k<float, 9>(K, fields, q, s, nsm);
}

}  // namespace bm
