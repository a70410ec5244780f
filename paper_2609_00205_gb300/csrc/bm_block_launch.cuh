// Launch helpers of the In-cache Block kernels for one (dtype, block size).
#pragma once

#include <atomic>

#include "bm_block.cuh"
#include "bm_internal.h"

namespace bm {

template <typename T, int B, int K, int MODE>
cudaError_t launch_one(int dir, const BlockArgs<T>& a, cudaStream_t s, int nsm, int max_grid) {
  using Cfg = BlockCfg<T, B, K>;
  const void* fn = dir == 0 ? (const void*)block_fwd_kernel<T, B, K, MODE> : (const void*)block_inv_kernel<T, B, K, MODE>;
  const size_t smem = dir == 0 ? Cfg::fwd_smem : Cfg::inv_smem(MODE);
  // shared-memory attribute and occupancy, once per device and direction
  static std::atomic<int> cached[2][64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int per_sm = dev < 64 ? cached[dir][dev].load() : 0;
  if (per_sm <= 0) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, dir == 0 ? Cfg::NT_FWD : Cfg::NT_INV, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (dev < 64) cached[dir][dev].store(per_sm);
  }
  int64_t grid = (int64_t)per_sm * nsm;
  if (max_grid > 0 && grid > max_grid) grid = max_grid;
  if (grid > a.nblocks) grid = a.nblocks;
  if (grid < 1) return cudaSuccess;
  if (dir == 0) block_fwd_kernel<T, B, K, MODE><<<(unsigned)grid, Cfg::NT_FWD, smem, s>>>(a);
  else block_inv_kernel<T, B, K, MODE><<<(unsigned)grid, Cfg::NT_INV, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int B, int K>
cudaError_t launch_mode(int dir, int mode, const BlockArgs<T>& a, cudaStream_t s, int nsm, int max_grid) {
  return mode == 0 ? launch_one<T, B, K, 0>(dir, a, s, nsm, max_grid) : launch_one<T, B, K, 1>(dir, a, s, nsm, max_grid);
}

}  // namespace bm
