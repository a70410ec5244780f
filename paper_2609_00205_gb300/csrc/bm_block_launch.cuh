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

// The batched forward kernel over a queue of fields (persistent grid: as
// many CTAs as the SMs hold, at most one per item).
template <typename T, int B, int K>
cudaError_t launch_batch_one(const BatchField<T>* fields, const BatchQueue& q, cudaStream_t s, int nsm) {
  using Cfg = BlockCfg<T, B, K>;
  const void* fn = (const void*)block_fwd_batch_kernel<T, B, K>;
  static std::atomic<int> cached[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int per_sm = dev < 64 ? cached[dev].load() : 0;
  if (per_sm <= 0) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::fwd_smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, Cfg::NT_FWD, Cfg::fwd_smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (dev < 64) cached[dev].store(per_sm);
  }
  int64_t grid = (int64_t)per_sm * nsm;
  if (grid > (int64_t)q.n_all) grid = (int64_t)q.n_all;
  if (grid < 1) return cudaSuccess;
  block_fwd_batch_kernel<T, B, K><<<(unsigned)grid, Cfg::NT_FWD, Cfg::fwd_smem, s>>>(fields, q);
  return cudaGetLastError();
}

// K levels need a level of at least 3 nodes last (B = 9: K <= 3).
template <typename T, int B>
cudaError_t launch_batch_k(int K, const BatchField<T>* fields, const BatchQueue& q, cudaStream_t s, int nsm) {
  switch (K) {
    case 1: return launch_batch_one<T, B, 1>(fields, q, s, nsm);
    case 2: return launch_batch_one<T, B, 2>(fields, q, s, nsm);
    case 3:
      if constexpr (lvl_n(B, 2) >= 3) return launch_batch_one<T, B, 3>(fields, q, s, nsm);
      return cudaErrorInvalidValue;
    case 4:
      if constexpr (lvl_n(B, 3) >= 3) return launch_batch_one<T, B, 4>(fields, q, s, nsm);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int B, int K>
cudaError_t launch_mode(int dir, int mode, const BlockArgs<T>& a, cudaStream_t s, int nsm, int max_grid) {
  return mode == 0 ? launch_one<T, B, K, 0>(dir, a, s, nsm, max_grid) : launch_one<T, B, K, 1>(dir, a, s, nsm, max_grid);
}

}  // namespace bm
