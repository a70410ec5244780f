// Transposed block levels instantiated for float fields.
#include "bm_adjoint.cuh"

namespace bm {

cudaError_t launch_block_adj_f32(int dir, int B, int K, const BlockArgs<float>& a, cudaStream_t s, int nsm) {
  if (B == 9) {
    switch (K) {
      case 1: return launch_adj_one<float, 9, 1>(dir, a, s, nsm);
      case 2: return launch_adj_one<float, 9, 2>(dir, a, s, nsm);
      case 3: return launch_adj_one<float, 9, 3>(dir, a, s, nsm);
      default: return cudaErrorInvalidValue;
    }
  }
  if (B == 17) {
    switch (K) {
      case 1: return launch_adj_one<float, 17, 1>(dir, a, s, nsm);
      case 2: return launch_adj_one<float, 17, 2>(dir, a, s, nsm);
      case 3: return launch_adj_one<float, 17, 3>(dir, a, s, nsm);
      case 4: return launch_adj_one<float, 17, 4>(dir, a, s, nsm);
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace bm
