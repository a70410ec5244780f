// In-cache Block kernels instantiated for double fields and 17-node blocks.
#include "bm_block_launch.cuh"

namespace bm {

cudaError_t launch_block_f64_b17(int dir, int K, int mode, const BlockArgs<double>& a, cudaStream_t s, int nsm,
                                 int max_grid) {
  switch (K) {
    case 1: return launch_mode<double, 17, 1>(dir, mode, a, s, nsm, max_grid);
    case 2: return launch_mode<double, 17, 2>(dir, mode, a, s, nsm, max_grid);
    case 3: return launch_mode<double, 17, 3>(dir, mode, a, s, nsm, max_grid);
    case 4: return launch_mode<double, 17, 4>(dir, mode, a, s, nsm, max_grid);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_block_batch_f64_b17(int K, const BatchField<double>* fields, const BatchQueue& q, cudaStream_t s,
                                    int nsm) {
  return launch_batch_k<double, 17>(K, fields, q, s, nsm);
}

}  // namespace bm
