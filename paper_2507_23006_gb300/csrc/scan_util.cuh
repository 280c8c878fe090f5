// Block-level scan helpers shared by the chained-scan kernels.
#pragma once

#include <cuda/atomic>

#include "gsr_internal.cuh"

namespace gsr {

// 256-thread exclusive scan of one value per thread; returns the block total through *total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* total) {
  __shared__ uint32_t warp_sums[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_sums[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t s = lane < nw ? warp_sums[lane] : 0u;
    uint32_t si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += y;
    }
    if (lane < nw) warp_sums[lane] = si - s;
    if (lane == nw - 1) warp_sums[31] = si;
  }
  __syncthreads();
  const uint32_t r = warp_sums[wid] + inc - x;
  *total = warp_sums[31];
  __syncthreads();
  return r;
}

// Decoupled look-back for block `bid`: publishes the block aggregate, waits (bounded) for the
// predecessors' prefixes and returns this block's exclusive prefix. One thread per block.
__device__ __forceinline__ unsigned long long chained_prefix(unsigned long long* status, unsigned bid, unsigned long long agg,
                                             int* err) {
  constexpr unsigned long long kA = 1ull << 62, kP = 2ull << 62, kMask = (1ull << 62) - 1;
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> me(status[bid]);
  if (bid == 0) {
    me.store(kP | agg, cuda::memory_order_relaxed);
    return 0;
  }
  me.store(kA | agg, cuda::memory_order_relaxed);
  unsigned long long excl = 0;
  long long j = static_cast<long long>(bid) - 1;
  unsigned spins = 0, ns = 32;
  while (j >= 0) {
    cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> st(status[j]);
    const unsigned long long s = st.load(cuda::memory_order_relaxed);
    const unsigned long long f = s >> 62;
    if (f == 0) {
      if (++spins > kSpinLimit) {
        atomicOr(err, kErrTimeout);
        break;
      }
      __nanosleep(ns);
      if (ns < 1024) ns <<= 1;
      continue;
    }
    excl += s & kMask;
    if (f == 2) break;
    --j;
  }
  me.store(kP | (excl + agg), cuda::memory_order_relaxed);
  return excl;
}

}  // namespace gsr
