// Onesweep LSD radix sort (Adinets & Merrill 2022) of uint32 (key, value) pairs: the library's
// general sort building block (gsr_sort_pairs_u32 and its allocation-free variant) and the sort
// of the global-sort binning (gsr_opts.global_sort: the visible records by depth, then the pairs
// stably by tile), with the chained scan that turns per-record tile counts into pair offsets
// there. Each pass reads every key once: a block
// ranks its 4096 keys by the pass's 8-bit digit (stable: one warp ballot per digit bit finds
// the lanes with equal digits), publishes its per-digit counts, and takes its global digit offsets from its predecessors by a decoupled
// look-back whose waits are bounded (a wait that runs out sets an error bit and the block
// carries on, so the kernel always finishes). Blocks take their tile index from an atomic
// counter at start, so a block only ever waits for blocks that are already running. The digit
// counts of all passes come from one histogram kernel, or from the kernel that produced the
// keys (count_digits / flush_digit_counts), before the first pass.
#include <algorithm>

#include "gsr_internal.cuh"
#include "scan_util.cuh"

namespace gsr {
namespace {

__device__ __forceinline__ long long device_n(const uint32_t* d_n, long long max_n) {
  if (!d_n) return max_n;
  const long long n = static_cast<long long>(*d_n);
  return n < max_n ? n : max_n;
}

// Digit counts of every pass: each block counts its keys in shared memory, then adds its
// nonzero bins to hist[pass][256] (zeroed beforehand) with one atomic each.
__global__ void __launch_bounds__(256) hist_kernel(const uint32_t* __restrict__ keys, const uint32_t* d_n,
                                                   long long max_n, int begin_bit, int end_bit, int passes,
                                                   uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[4 * 256];
  for (int k = threadIdx.x; k < 4 * 256; k += blockDim.x) sh[k] = 0;
  __syncthreads();
  const long long n = device_n(d_n, max_n);
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    count_digits(keys[i], begin_bit, end_bit, passes, sh);
  __syncthreads();
  flush_digit_counts(sh, passes, hist);
}

// Per-digit decoupled look-back of tile `bid` (one thread per digit): publishes the tile's
// count, then sums predecessors' counts back to the nearest inclusive prefix, reading eight
// predecessors per round (the loads are independent; the walk is latency-bound otherwise).
// Waits are bounded: past wait.limit rounds the error flag is set and the partial sum is used.
__device__ __forceinline__ uint32_t lookback_digit(unsigned long long* status, uint32_t bid, int d, uint32_t agg,
                                                   uint32_t epoch, int* err, WaitCfg wait) {
  constexpr int kAhead = 8;
  unsigned long long* me = status + static_cast<size_t>(bid) * 256 + d;
  if (bid == 0) {
    store_status(me, pack_status(epoch, kStatusPrefix, agg));
    return 0;
  }
  store_status(me, pack_status(epoch, kStatusAgg, agg));
  uint32_t excl = 0;
  long long j = static_cast<long long>(bid) - 1;
  unsigned spins = 0, ns = 32;
  bool done = false;
  while (!done) {
    unsigned long long w[kAhead];
#pragma unroll
    for (int k = 0; k < kAhead; ++k)
      w[k] = (j - k >= 0) ? load_status(status + static_cast<size_t>(j - k) * 256 + d)
                          : pack_status(epoch, kStatusPrefix, 0u);  // before tile 0: a prefix of 0
    bool stalled = false;
#pragma unroll
    for (int k = 0; k < kAhead; ++k) {
      if (done || stalled) continue;
      const uint32_t f = (wait.never_ready && j - k >= 0) ? 0u : status_flag(w[k], epoch);
      if (f == 0) {
        stalled = true;
      } else {
        excl += static_cast<uint32_t>(w[k]);
        --j;
        done = f == kStatusPrefix;
      }
    }
    if (stalled && !done) {
      if (++spins > wait.limit) {
        atomicOr(err, kErrTimeout);
        break;
      }
      __nanosleep(ns);
      if (ns < 1024) ns <<= 1;
    }
  }
  store_status(me, pack_status(epoch, kStatusPrefix, excl + agg));
  return excl;
}

// One LSD pass. Resident blocks loop: each takes the next 4096-key tile from `counter` (so a
// tile only ever waits on tiles already taken by running blocks) until the keys run out.
//   rank: each of the 16 warps ranks its 256 keys item by item; lanes with equal digits are
//         found with one ballot per digit bit, and the lowest such lane adds the group to the
//         warp's counter of that digit (shared atomics, ordered by __syncwarp so that earlier
//         items rank first);
//   offsets: per digit, the warps' counts are scanned, the tile's count is published and the
//         digit's offset taken from the predecessors (look-back);
//   scatter: keys, then values, are placed in shared memory in tile-local digit order and
//         written out in runs of equal digits (consecutive threads, consecutive addresses).
__global__ void __launch_bounds__(kSortThreads) onesweep_kernel(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, const uint32_t* d_n, long long max_n, int shift, int width,
    const uint32_t* __restrict__ counts, unsigned long long* status, uint32_t* counter, uint32_t epoch,
    int* err, WaitCfg wait) {
  constexpr int kWarps = kSortThreads / 32;
  constexpr int kOut = kSortTile / kSortThreads;  // tile positions each thread writes out
  __shared__ uint32_t s_hist[kWarps][256];
  __shared__ uint32_t s_local[256];  // first tile-local position of each digit
  __shared__ uint32_t s_base[256];   // output position of tile-local position 0 of each digit
  __shared__ uint32_t s_digit[256];  // first output position of each digit (all keys)
  __shared__ uint32_t s_buf[kSortTile];
  __shared__ uint32_t s_bid;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long n = device_n(d_n, max_n);
  const uint32_t dmask = (1u << width) - 1;
  const uint32_t lt = (1u << lane) - 1;
  {  // the pass's digit counts, scanned by every block for itself
    uint32_t all;
    const uint32_t first = block_excl_scan(tid < 256 ? counts[tid] : 0u, &all);
    if (tid < 256) s_digit[tid] = first;
  }
  for (;;) {
    for (int k = tid; k < kWarps * 256; k += kSortThreads) (&s_hist[0][0])[k] = 0;
    if (tid == 0) s_bid = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t bid = s_bid;
    const long long start = static_cast<long long>(bid) * kSortTile;
    if (start >= n) break;
    const int tile_n = static_cast<int>(n - start < kSortTile ? n - start : kSortTile);
    const long long wbase = start + static_cast<long long>(w) * (32 * kSortItems);
    uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      const long long idx = wbase + j * 32 + lane;
      const bool ok = idx < n;
      key[j] = ok ? kin[idx] : 0u;
      val[j] = ok ? vin[idx] : 0u;
    }
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      const bool ok = wbase + j * 32 + lane < n;
      const uint32_t d = (key[j] >> shift) & dmask;
      uint32_t peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
      for (int bit = 0; bit < 8; ++bit) {
        if (bit < width) {
          const uint32_t ones = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
          peers &= ((d >> bit) & 1u) ? ones : ~ones;
        }
      }
      const int leader = ok ? __ffs(peers) - 1 : lane;
      uint32_t old = 0;
      if (ok && lane == leader) old = atomicAdd(&s_hist[w][d], static_cast<uint32_t>(__popc(peers)));
      old = __shfl_sync(0xffffffffu, old, leader);
      rank[j] = old + __popc(peers & lt);
      __syncwarp();
    }
    __syncthreads();
    uint32_t sum = 0;
    if (tid < 256) {  // one thread per digit
      const int d = tid;
#pragma unroll
      for (int k = 0; k < kWarps; ++k) {
        const uint32_t c = s_hist[k][d];
        s_hist[k][d] = sum;
        sum += c;
      }
    }
    uint32_t excl = 0;
    if (tid < 256) excl = lookback_digit(status, bid, tid, sum, epoch, err, wait);
    uint32_t tile_total;
    const uint32_t local = block_excl_scan(sum, &tile_total);  // every thread; digits are the first 256
    if (tid < 256) {
      s_local[tid] = local;
      s_base[tid] = s_digit[tid] + excl - local;
    }
    __syncthreads();
    uint32_t lp[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      lp[j] = 0xffffffffu;
      if (wbase + j * 32 + lane < n) {
        const uint32_t d = (key[j] >> shift) & dmask;
        lp[j] = s_local[d] + s_hist[w][d] + rank[j];
        s_buf[lp[j]] = key[j];
      }
    }
    __syncthreads();
    uint32_t pos[kOut];
#pragma unroll
    for (int k = 0; k < kOut; ++k) {
      const int t = tid + k * kSortThreads;
      if (t < tile_n) {
        const uint32_t kk = s_buf[t];
        pos[k] = s_base[(kk >> shift) & dmask] + static_cast<uint32_t>(t);
        kout[pos[k]] = kk;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSortItems; ++j)
      if (lp[j] != 0xffffffffu) s_buf[lp[j]] = val[j];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kOut; ++k) {
      const int t = tid + k * kSortThreads;
      if (t < tile_n) vout[pos[k]] = s_buf[t];
    }
    __syncthreads();
  }
}

// Exclusive scan of per-record tile counts in depth order (the global-sort binning):
// counts[i] = touched[order[i]] (or cnt_sorted[i] when given), offsets[i] out, *p_total = sum.
__global__ void __launch_bounds__(kScanThreads) pair_scan_kernel(
    const uint32_t* __restrict__ touched, const uint32_t* __restrict__ order, const uint32_t* __restrict__ cnt_sorted,
    uint32_t* __restrict__ offsets, const uint32_t* d_n, long long max_n, unsigned long long* status,
    uint32_t* counter, unsigned long long* p_total, uint32_t epoch, int* err, WaitCfg wait) {
  __shared__ uint32_t s_bid;
  __shared__ unsigned long long s_base;
  const long long n = device_n(d_n, max_n);
  for (;;) {
    if (threadIdx.x == 0) s_bid = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t bid = s_bid;
    const long long start = static_cast<long long>(bid) * (kScanThreads * kScanItems);
    if (start >= n) break;
    uint32_t x[kScanItems];
    uint32_t sum = 0;
    const long long first = start + static_cast<long long>(threadIdx.x) * kScanItems;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const long long idx = first + k;
      x[k] = 0;
      if (idx < n) x[k] = cnt_sorted ? cnt_sorted[idx] : touched[order[idx]];
      sum += x[k];
    }
    uint32_t total;
    const uint32_t excl = block_excl_scan(sum, &total);
    if (threadIdx.x < 32) {
      const unsigned long long ex = warp_chained_prefix(status, bid, total, epoch, err, wait);
      if (threadIdx.x == 0) s_base = ex;
    }
    __syncthreads();
    unsigned long long run = s_base + excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const long long idx = first + k;
      if (idx < n) {
        if (run > 0xffffffffull) atomicOr(err, kErrOverflow);
        offsets[idx] = static_cast<uint32_t>(run);
        if (idx == n - 1) *p_total = run + x[k];
      }
      run += x[k];
    }
    __syncthreads();
  }
}

}  // namespace

void sort_clear_counts(const SortScratch& sc, cudaStream_t s) {
  cudaMemsetAsync(sc.hist, 0, sizeof(uint32_t) * kSortCountWords, s);
}

size_t sort_status_words(long long max_n) {
  const long long tiles = (max_n + kSortTile - 1) / kSortTile;
  return static_cast<size_t>(std::max<long long>(tiles, 1)) * 256;
}

void radix_sort_u32(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
                    const uint32_t* d_n, long long max_n, int begin_bit, int end_bit, const SortScratch& sc,
                    uint32_t epoch, bool clear_status, bool counts_ready, int* err, cudaStream_t s) {
  if (max_n <= 0 || end_bit <= begin_bit) return;
  const int passes = (end_bit - begin_bit + 7) / 8;
  const long long tiles = (max_n + kSortTile - 1) / kSortTile;
  const size_t words = sort_status_words(max_n);
  const int grid = static_cast<int>(std::max<long long>(1, std::min<long long>(tiles, sc.grid_cap)));
  if (clear_status) cudaMemsetAsync(sc.status, 0, sizeof(unsigned long long) * words * passes, s);
  if (!counts_ready) {  // else the producer of the keys has counted their digits
    sort_clear_counts(sc, s);
    const int hblocks = std::max(1, static_cast<int>(std::min<long long>(sc.grid_cap, (max_n + 4095) / 4096)));
    hist_kernel<<<hblocks, 256, 0, s>>>(keys_in, d_n, max_n, begin_bit, end_bit, passes, sc.hist);
  }
  // ping-pong so that the last pass lands in keys_out; the inputs are never written
  const uint32_t* ksrc = keys_in;
  const uint32_t* vsrc = vals_in;
  for (int p = 0; p < passes; ++p) {
    const bool to_out = ((passes - 1 - p) % 2) == 0;
    uint32_t* kdst = to_out ? keys_out : sc.keys_tmp;
    uint32_t* vdst = to_out ? vals_out : sc.vals_tmp;
    const int shift = begin_bit + 8 * p;
    const int width = std::min(8, end_bit - shift);
    onesweep_kernel<<<grid, kSortThreads, 0, s>>>(ksrc, vsrc, kdst, vdst, d_n, max_n, shift, width, sc.hist + 256 * p,
                                                  sc.status + words * p, sc.hist + 4 * 256 + p, epoch, err,
                                                  sc.wait);
    ksrc = kdst;
    vsrc = vdst;
  }
}

void pair_offsets_scan(const uint32_t* touched, const uint32_t* order, const uint32_t* cnt_sorted,
                       uint32_t* offsets, const uint32_t* d_n, long long max_n, unsigned long long* status,
                       uint32_t* counter, unsigned long long* p_total, int* err, uint32_t epoch, int grid_cap,
                       WaitCfg wait, cudaStream_t s) {
  const long long per = kScanThreads * kScanItems;
  const int grid = static_cast<int>(std::max<long long>(1, std::min<long long>((max_n + per - 1) / per, grid_cap)));
  cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
  cudaMemsetAsync(p_total, 0, sizeof(unsigned long long), s);
  pair_scan_kernel<<<grid, kScanThreads, 0, s>>>(touched, order, cnt_sorted, offsets, d_n, max_n, status, counter,
                                                 p_total, epoch, err, wait);
}

}  // namespace gsr
