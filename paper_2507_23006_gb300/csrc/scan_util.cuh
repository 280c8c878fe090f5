// Block-level scan helpers and the decoupled look-back of the chained-scan kernels.
//
// Status words are 64 bits: [63:34] epoch, [33:32] flag (1 = aggregate, 2 = inclusive prefix),
// [31:0] value. A word whose epoch differs from the launch's is "not ready", so the status
// arrays never need clearing between launches: the host hands every launch a new epoch.
#pragma once

#include <cuda/atomic>

#include "gsr_internal.cuh"

namespace gsr {

constexpr uint32_t kStatusAgg = 1u;
constexpr uint32_t kStatusPrefix = 2u;

__device__ __forceinline__ unsigned long long pack_status(uint32_t epoch, uint32_t flag, uint32_t value) {
  return (static_cast<unsigned long long>(epoch) << 34) | (static_cast<unsigned long long>(flag) << 32) | value;
}

__device__ __forceinline__ void store_status(unsigned long long* p, unsigned long long v) {
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>(*p).store(v, cuda::memory_order_relaxed);
}

__device__ __forceinline__ unsigned long long load_status(unsigned long long* p) {
  return cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>(*p).load(cuda::memory_order_relaxed);
}

// Flag of a status word for this epoch (0 = not ready).
__device__ __forceinline__ uint32_t status_flag(unsigned long long s, uint32_t epoch) {
  return (static_cast<uint32_t>(s >> 34) == epoch) ? static_cast<uint32_t>((s >> 32) & 3u) : 0u;
}

// Exclusive scan of one value per thread over the whole block (any multiple of 32 threads up
// to 1024; every thread must call it); returns the block total through *total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* total) {
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t block_total;
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
    if (lane == nw - 1) block_total = si;
  }
  __syncthreads();
  const uint32_t r = warp_sums[wid] + inc - x;
  *total = block_total;
  __syncthreads();
  return r;
}

// Exclusive scan of one 64-bit value per thread over the whole block (used with four
// independent 16-bit lanes packed in one word: no lane's total may exceed 65535). Returns the
// block total too.
__device__ __forceinline__ unsigned long long block_excl_scan64(unsigned long long x, unsigned long long* total) {
  __shared__ unsigned long long warp_sums64[32];
  __shared__ unsigned long long block_total64;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_sums64[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    const unsigned long long s = lane < nw ? warp_sums64[lane] : 0ull;
    unsigned long long si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += y;
    }
    if (lane < nw) warp_sums64[lane] = si - s;
    if (lane == nw - 1) block_total64 = si;
  }
  __syncthreads();
  const unsigned long long r = warp_sums64[wid] + inc - x;
  *total = block_total64;
  __syncthreads();
  return r;
}

// Publishes tile `bid`'s aggregate (tile 0: its inclusive prefix) for the decoupled look-back.
// One thread calls it.
__device__ __forceinline__ void publish_aggregate(unsigned long long* status, uint32_t bid, uint32_t agg,
                                                  uint32_t epoch) {
  store_status(status + bid, pack_status(epoch, bid == 0 ? kStatusPrefix : kStatusAgg, agg));
}

// Decoupled look-back for tile `bid` whose aggregate `agg` is already published, run by all 32
// lanes of one warp: reads 32 predecessors at a time, waiting (bounded) until every one of them
// up to the nearest inclusive prefix is ready, and sums them. Returns this tile's exclusive
// prefix in every lane and publishes its inclusive prefix. Values are 32-bit; the running total
// is 64-bit and the caller checks it for overflow.
__device__ __forceinline__ unsigned long long warp_lookback(unsigned long long* status, uint32_t bid, uint32_t agg,
                                                            uint32_t epoch, int* err, WaitCfg wait) {
  const int lane = threadIdx.x & 31;
  if (bid == 0) return 0;
  unsigned long long excl = 0;
  long long end = static_cast<long long>(bid) - 1;
  unsigned spins = 0, ns = 32;
  for (;;) {
    const long long j = end - lane;
    uint32_t flag = kStatusPrefix, val = 0;  // before tile 0: an inclusive prefix of 0
    if (j >= 0) {
      const unsigned long long s = load_status(status + j);
      flag = wait.never_ready ? 0u : status_flag(s, epoch);
      val = static_cast<uint32_t>(s);
    }
    const uint32_t pm = __ballot_sync(0xffffffffu, flag == kStatusPrefix);
    const uint32_t xm = __ballot_sync(0xffffffffu, flag == 0u);
    const uint32_t upto = pm ? (((pm & (0u - pm)) << 1) - 1u) : 0xffffffffu;
    if (xm & upto) {
      if (++spins > wait.limit) {
        if (lane == 0) atomicOr(err, kErrTimeout);
        break;
      }
      __nanosleep(ns);
      if (ns < 256) ns <<= 1;
      continue;
    }
    unsigned long long v = ((upto >> lane) & 1u) ? val : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (pm) break;
    end -= 32;
  }
  if (lane == 0)
    store_status(status + bid, pack_status(epoch, kStatusPrefix, static_cast<uint32_t>(excl + agg)));
  return excl;
}

// Publish and look back in one call (all 32 lanes of one warp).
__device__ __forceinline__ unsigned long long warp_chained_prefix(unsigned long long* status, uint32_t bid,
                                                                  uint32_t agg, uint32_t epoch, int* err,
                                                                  WaitCfg wait) {
  if ((threadIdx.x & 31) == 0) publish_aggregate(status, bid, agg, epoch);
  __syncwarp();
  return warp_lookback(status, bid, agg, epoch, err, wait);
}

}  // namespace gsr
