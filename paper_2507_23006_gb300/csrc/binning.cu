// Tile binning of Sec. 3.1 (with the StopThePop tile culling of Sec. 3.4.2): every visible
// record has one (tile, record) pair per tile of its 3-sigma rectangle, minus the tiles the
// culling drops. Per-tile path: the pairs are counted per tile, the counts scanned into each
// tile's [start, end), the pairs placed in their tile's range, and each tile's list sorted by
// (depth, index) (the lists of at most kTileSortSmall pairs by the forward blend itself).
// Global path: records sorted by depth, pairs emitted in that order and sorted stably by tile.
#include <algorithm>
#include <atomic>

#include "gsr_internal.cuh"
#include "scan_util.cuh"
#include "tile_util.cuh"

namespace gsr {
namespace {

// Places the (tile, record) pairs of the visible records in their tiles' ranges, 32 records per
// warp (warp_bin_pairs; launched with kPlace = true). The counting pass that sized the ranges is
// the same function, run by the preprocess's record pass as it makes the records. The order
// inside a tile is then fixed by sorting the placed keys.
template <bool kCull, bool kPlace>
__global__ void __launch_bounds__(256) bin_pairs_kernel(const Rec* __restrict__ rec, const uint32_t* d_n, long long max_n,
                                                        CamBatch cams, uint32_t* __restrict__ tile_ctr,
                                                        const uint2* __restrict__ ranges,
                                                        unsigned long long* __restrict__ keys, int* err) {
  const int lane = threadIdx.x & 31;
  long long n = static_cast<long long>(*d_n);
  if (n > max_n) n = max_n;
  // warps stride over the records 32 at a time (the grid is sized for the resident blocks)
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long base_i = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) & ~31ll; base_i < n;
       base_i += stride) {
    const long long i = base_i + lane;
    Rec r{};
    if (i < n) r = rec[i];
    warp_bin_pairs<kCull, kPlace>(lane, i < n, r, static_cast<uint32_t>(base_i), cams, tile_ctr, ranges, keys, err);
  }
}

// Exclusive scan of the per-tile pair counts (chained scan, decoupled look-back): ranges[t] =
// [start, start + count); the counter becomes the tile's cursor (start) for the placing pass;
// *p_total = P; *max_count = the largest tile's count; the tiles with more than kTileSortSmall
// pairs are listed in big[0, *n_big) (any order) for the large-list sort.
__global__ void __launch_bounds__(kScanThreads) tile_scan_kernel(uint32_t* __restrict__ ctr, uint2* __restrict__ ranges,
                                                                 int n_tiles, unsigned long long* status,
                                                                 uint32_t* counter, unsigned long long* p_total,
                                                                 uint32_t* max_count, uint32_t* big, uint32_t* n_big,
                                                                 uint32_t epoch, int* err, WaitCfg wait) {
  __shared__ uint32_t s_bid;
  __shared__ unsigned long long s_base;
  __shared__ uint32_t s_max[kScanThreads / 32];
  for (;;) {
    if (threadIdx.x == 0) s_bid = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t bid = s_bid;
    const long long start = static_cast<long long>(bid) * (kScanThreads * kScanItems);
    if (start >= n_tiles) break;
    uint32_t x[kScanItems];
    uint32_t sum = 0, mx = 0;
    const long long first = start + static_cast<long long>(threadIdx.x) * kScanItems;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const long long idx = first + k;
      x[k] = idx < n_tiles ? ctr[idx] : 0u;
      sum += x[k];
      mx = max(mx, x[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
    uint32_t tot;
    const uint32_t excl = block_excl_scan(sum, &tot);
    if (threadIdx.x < 32) {
      const unsigned long long ex = warp_chained_prefix(status, bid, tot, epoch, err, wait);
      if (threadIdx.x == 0) {
        s_base = ex;
        uint32_t m = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) m = max(m, s_max[w]);
        atomicMax(max_count, m);
      }
    }
    __syncthreads();
    unsigned long long run = s_base + excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const long long idx = first + k;
      if (idx < n_tiles) {
        if (run + x[k] > 0xffffffffull) atomicOr(err, kErrOverflow);
        ranges[idx] = make_uint2(static_cast<uint32_t>(run), static_cast<uint32_t>(run + x[k]));
        ctr[idx] = static_cast<uint32_t>(run);
        if (x[k] > static_cast<uint32_t>(kTileSortSmall)) big[atomicAdd(n_big, 1u)] = static_cast<uint32_t>(idx);
        if (idx == n_tiles - 1) *p_total = run + x[k];
      }
      run += x[k];
    }
    __syncthreads();
  }
}

// Merges the sorted runs a[0, na) and b[0, nb) (distinct keys) into out[0, na + nb) with the
// whole block: each thread finds where its share of the output starts on the merge path (a
// binary search along a diagonal) and merges that share sequentially.
__device__ void block_merge(const unsigned long long* a, int na, const unsigned long long* b, int nb,
                            unsigned long long* out) {
  const int total = na + nb;
  const int per = (total + blockDim.x - 1) / blockDim.x;
  const int d0 = min(static_cast<int>(threadIdx.x) * per, total);
  const int d1 = min(d0 + per, total);
  int lo = max(0, d0 - nb), hi = min(d0, na);
  while (lo < hi) {  // i = number of a's among the first d0 outputs
    const int mid = (lo + hi) >> 1;
    if (a[mid] < b[d0 - mid - 1]) lo = mid + 1; else hi = mid;
  }
  int i = lo, j = d0 - lo;
  for (int d = d0; d < d1; ++d) {
    const bool take_a = j >= nb || (i < na && a[i] < b[j]);
    out[d] = take_a ? a[i++] : b[j++];
  }
}

// Per-tile sort: tiles of at most kTileSortSmall pairs get a block of kSortSmallThreads each; the
// larger ones blocks of kSortBigThreads that sort up to kTileSortCap keys in shared memory.
constexpr int kSortSmallThreads = 128;
constexpr int kSortBigThreads = 1024;

// Sorts one tile's keys (depth bits << 32 | record index), i.e. its pairs by depth with ties to
// the lower record (so the lower Gaussian index, C7), and writes the records in that order (whole
// block). A list of at most `cap` keys (a power of two; s_keys holds cap keys) is sorted in shared
// memory; a longer one in runs of cap, merged pairwise in global memory through `scratch` (same
// offsets as the keys).
__device__ void sort_tile(unsigned long long* __restrict__ keys, uint2 r, uint32_t* __restrict__ vals,
                          unsigned long long* __restrict__ scratch, int cap, unsigned long long* s_keys) {
  const int n = static_cast<int>(r.y - r.x);
  unsigned long long* k = keys + r.x;
  if (n <= cap) {
    int m = 1;
    while (m < n) m <<= 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s_keys[i] = i < n ? k[i] : ~0ull;
    __syncthreads();
    block_bitonic_sort(s_keys, m);
    for (int i = threadIdx.x; i < n; i += blockDim.x) vals[r.x + i] = static_cast<uint32_t>(s_keys[i]);
    __syncthreads();
    return;
  }
  // runs of cap keys sorted in place
  for (int base = 0; base < n; base += cap) {
    const int len = min(cap, n - base);
    for (int i = threadIdx.x; i < cap; i += blockDim.x) s_keys[i] = i < len ? k[base + i] : ~0ull;
    __syncthreads();
    block_bitonic_sort(s_keys, cap);
    for (int i = threadIdx.x; i < len; i += blockDim.x) k[base + i] = s_keys[i];
    __syncthreads();
  }
  // pairwise merges, ping-ponging between the keys and the scratch
  unsigned long long* src = k;
  unsigned long long* dst = scratch + r.x;
  for (int width = cap; width < n; width <<= 1) {
    for (int lo = 0; lo < n; lo += 2 * width) {
      const int na = min(width, n - lo);
      const int nb = max(0, min(width, n - lo - width));
      block_merge(src + lo, na, src + lo + na, nb, dst + lo);
    }
    __syncthreads();
    unsigned long long* t = src;
    src = dst;
    dst = t;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) vals[r.x + i] = static_cast<uint32_t>(src[i]);
  __syncthreads();
}

// One small block per tile of at most kTileSortSmall pairs (larger tiles are left to the list sort).
__global__ void __launch_bounds__(kSortSmallThreads) tile_sort_kernel(unsigned long long* __restrict__ keys,
                                                                      const uint2* __restrict__ ranges,
                                                                      uint32_t* __restrict__ vals, int cap) {
  extern __shared__ unsigned long long s_keys[];
  const uint2 r = ranges[blockIdx.x];
  const uint32_t n = r.y - r.x;
  if (n == 0 || n > static_cast<uint32_t>(kTileSortSmall)) return;
  sort_tile(keys, r, vals, nullptr, cap, s_keys);
}

// Large blocks over the listed tiles with more than kTileSortSmall pairs.
__global__ void __launch_bounds__(kSortBigThreads) tile_sort_big_kernel(unsigned long long* __restrict__ keys,
                                                                        const uint2* __restrict__ ranges,
                                                                        uint32_t* __restrict__ vals,
                                                                        unsigned long long* __restrict__ scratch,
                                                                        const uint32_t* __restrict__ big,
                                                                        const uint32_t* __restrict__ n_big, int cap) {
  extern __shared__ unsigned long long s_keys[];
  const uint32_t nb = *n_big;
  for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) sort_tile(keys, ranges[big[b]], vals, scratch, cap, s_keys);
}

// The global-sort binning (gsr_opts.global_sort): every visible record, in depth order, emits
// its (tile, record) pairs at its offset from the pair scan, with the tile id as the key (and, in
// count_only mode, only counts the pairs StopThePop keeps); the pairs are then sorted stably by
// tile with the onesweep radix sort, and each tile's range found by binary search.
template <bool kCull, bool kCount>
__global__ void __launch_bounds__(256) duplicate_kernel(const Rec* __restrict__ rec, const uint32_t* __restrict__ order,
                                                        const uint32_t* __restrict__ offsets, const uint32_t* d_n,
                                                        long long max_n, CamBatch cams, uint32_t* __restrict__ cnt_sorted,
                                                        uint32_t* __restrict__ pkeys, uint32_t* __restrict__ pvals,
                                                        uint32_t* __restrict__ key_counts, int key_bits) {
  __shared__ uint32_t s_cnt[8][32];
  __shared__ uint32_t s_digits[4 * 256];  // digit counts of the emitted tile keys (for their sort)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int passes = (key_bits + 7) / 8;
  if (key_counts) {
    for (int k = threadIdx.x; k < 4 * 256; k += blockDim.x) s_digits[k] = 0;
    __syncthreads();
  }
  long long n = static_cast<long long>(*d_n);
  if (n > max_n) n = max_n;
  // warps stride over the records 32 at a time (the grid is sized for the resident blocks, not
  // for the capacity, so no block starts only to find nothing to do)
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long base_i = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) & ~31ll; base_i < n;
       base_i += stride) {
  const long long i = base_i + lane;
  const bool valid = i < n;
  uint32_t v = 0, off = 0, area = 0, lo = 0, hi = 0;
  float4 ra = make_float4(0, 0, 0, 0), rb = ra;
  if (valid) {
    v = order[i];
    const Rec r = rec[v];
    ra = r.a;
    rb = r.b;
    lo = __float_as_uint(r.c.z);
    hi = __float_as_uint(r.c.w);
    area = ((lo >> 16) - (lo & 0xffffu)) * (((hi >> 16) & 0x7ffu) - (hi & 0xffffu));
    if (!kCount) off = offsets[i];
  }
  uint32_t incl = area;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  s_cnt[w][lane] = 0;
  __syncwarp();
  for (uint32_t r0 = 0; r0 < total; r0 += 32) {
    const uint32_t k = r0 + lane;
    const bool active = k < total;
    int owner = 0;
#pragma unroll
    for (int b = 16; b > 0; b >>= 1) {
      const uint32_t probe = __shfl_sync(0xffffffffu, incl, owner + b - 1);
      if (probe <= k) owner += b;
    }
    owner = min(owner, 31);
    const uint32_t o_incl = __shfl_sync(0xffffffffu, incl, owner);
    const uint32_t o_area = __shfl_sync(0xffffffffu, area, owner);
    const uint32_t o_lo = __shfl_sync(0xffffffffu, lo, owner);
    const uint32_t o_hi = __shfl_sync(0xffffffffu, hi, owner);
    const uint32_t o_v = __shfl_sync(0xffffffffu, v, owner);
    const uint32_t o_off = __shfl_sync(0xffffffffu, off, owner);
    const uint32_t q = k - (o_incl - o_area);
    const uint32_t x0 = o_lo & 0xffffu, wdt = (o_lo >> 16) - x0;
    const uint32_t y0 = o_hi & 0xffffu;
    const int c = static_cast<int>(o_hi >> 27);
    const uint32_t tx = active ? x0 + q % max(wdt, 1u) : 0;
    const uint32_t ty = active ? y0 + q / max(wdt, 1u) : 0;
    bool keep = active;
    if (kCull) {
      const float mx = __shfl_sync(0xffffffffu, ra.x, owner), my = __shfl_sync(0xffffffffu, ra.y, owner);
      const float op = __shfl_sync(0xffffffffu, ra.z, owner);
      const float ca = __shfl_sync(0xffffffffu, rb.x, owner), cb = __shfl_sync(0xffffffffu, rb.y, owner);
      const float cc = __shfl_sync(0xffffffffu, rb.z, owner);
      if (active) {
        const DevCam& cam = cams.cam[c];
        const float xlo = tx * kTile + 0.5f, xhi = fminf(static_cast<float>((tx + 1) * kTile), cam.W) - 0.5f;
        const float ylo = ty * kTile + 0.5f, yhi = fminf(static_cast<float>((ty + 1) * kTile), cam.H) - 0.5f;
        const float d2 = tile_min_maha(mx, my, ca, cb, cc, xlo, xhi, ylo, yhi);
        keep = op > 0.f && __fmul_rn(0.5f, d2) <= logf(__fmul_rn(op, 255.f));
      }
      const uint32_t kb = __ballot_sync(0xffffffffu, keep);
      const uint32_t group = __match_any_sync(0xffffffffu, active ? static_cast<uint32_t>(owner) : 64u);
      const uint32_t before = __popc(kb & group & ((1u << lane) - 1));
      const uint32_t base_cnt = s_cnt[w][owner];
      __syncwarp();
      if (!kCount && keep) {
        const uint32_t pos = o_off + base_cnt + before;
        const DevCam& cam = cams.cam[c];
        const uint32_t key = static_cast<uint32_t>(cam.tile_off) + ty * cam.tiles_x + tx;
        pkeys[pos] = key;
        pvals[pos] = o_v;
        if (key_counts) count_digits(key, 0, key_bits, passes, s_digits);
      }
      if (active && lane == 31 - __clz(group)) s_cnt[w][owner] = base_cnt + __popc(kb & group);
      __syncwarp();
    } else if (active) {
      const DevCam& cam = cams.cam[c];
      const uint32_t pos = o_off + q;
      const uint32_t key = static_cast<uint32_t>(cam.tile_off) + ty * cam.tiles_x + tx;
      pkeys[pos] = key;
      pvals[pos] = o_v;
      if (key_counts) count_digits(key, 0, key_bits, passes, s_digits);
    }
  }
  if (kCount && valid) cnt_sorted[i] = s_cnt[w][lane];
  __syncwarp();  // the next round clears s_cnt
  }
  if (key_counts) {
    __syncthreads();
    flush_digit_counts(s_digits, passes, key_counts);
  }
}

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* __restrict__ a, uint32_t n, uint32_t key) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// One thread per tile: [first pair with key >= t, first pair with key >= t + 1) of the sorted
// keys; every tile is written, so nothing needs clearing first.
__global__ void ranges_kernel(const uint32_t* __restrict__ keys, uint32_t P, int n_tiles, uint2* __restrict__ ranges) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  ranges[t] = make_uint2(lower_bound_u32(keys, P, static_cast<uint32_t>(t)),
                         lower_bound_u32(keys, P, static_cast<uint32_t>(t) + 1u));
}

}  // namespace

void launch_bin_pairs(const Rec* rec, const uint32_t* d_n, long long max_n, const CamBatch& cams, int tile_cull,
                      uint32_t* tile_ctr, const uint2* ranges, unsigned long long* keys, int* err, int max_blocks,
                      cudaStream_t s) {
  if (max_n <= 0) return;
  const int blocks = static_cast<int>(std::min<long long>((max_n + 255) / 256, std::max(max_blocks, 1)));
#define GSR_BIN(C) bin_pairs_kernel<C, true><<<blocks, 256, 0, s>>>(rec, d_n, max_n, cams, tile_ctr, ranges, keys, err)
  if (tile_cull) GSR_BIN(true); else GSR_BIN(false);
#undef GSR_BIN
}

void launch_tile_scan(uint32_t* tile_ctr, uint2* ranges, int n_tiles, unsigned long long* status, uint32_t* counter,
                      unsigned long long* p_total, uint32_t* max_count, uint32_t* big, uint32_t* n_big, uint32_t epoch,
                      int* err, WaitCfg wait, int grid_cap, cudaStream_t s) {
  if (n_tiles <= 0) return;
  const long long per = kScanThreads * kScanItems;
  const int grid = static_cast<int>(std::max<long long>(1, std::min<long long>((n_tiles + per - 1) / per, grid_cap)));
  tile_scan_kernel<<<grid, kScanThreads, 0, s>>>(tile_ctr, ranges, n_tiles, status, counter, p_total, max_count, big,
                                                 n_big, epoch, err, wait);
}

void launch_tile_sort(unsigned long long* keys, const uint2* ranges, int n_tiles, uint32_t* vals,
                      unsigned long long* scratch, uint32_t max_count, const uint32_t* big, const uint32_t* n_big,
                      bool small, int grid_cap, cudaStream_t s) {
  if (n_tiles <= 0 || max_count == 0) return;
  int cap = 1;
  while (cap < static_cast<long long>(max_count) && cap < kTileSortSmall) cap <<= 1;
  if (small)
    tile_sort_kernel<<<n_tiles, kSortSmallThreads, sizeof(unsigned long long) * cap, s>>>(keys, ranges, vals, cap);
  if (max_count > static_cast<uint32_t>(kTileSortSmall)) {
    int big_cap = 1;
    while (big_cap < static_cast<long long>(max_count) && big_cap < kTileSortCap) big_cap <<= 1;
    // the large dynamic shared memory needs an opt-in in each device's context: one bit per
    // device (contexts on several host threads may get here at once; setting it twice is harmless)
    static std::atomic<uint64_t> attr_set{0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 64 || !((attr_set.load(std::memory_order_relaxed) >> dev) & 1u)) {
      if (cudaFuncSetAttribute(tile_sort_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(sizeof(unsigned long long) * kTileSortCap)) == cudaSuccess &&
          dev < 64)
        attr_set.fetch_or(1ull << dev, std::memory_order_relaxed);
    }
    tile_sort_big_kernel<<<std::max(1, grid_cap / 2), kSortBigThreads, sizeof(unsigned long long) * big_cap, s>>>(
        keys, ranges, vals, scratch, big, n_big, big_cap);
  }
}

void launch_duplicate(const Rec* rec, const uint32_t* order, const uint32_t* offsets, const uint32_t* d_n,
                      long long max_n, const CamBatch& cams, int tile_cull, uint32_t* cnt_sorted,
                      uint32_t* pair_keys, uint32_t* pair_vals, uint32_t* key_counts, int key_bits, int max_blocks,
                      cudaStream_t s) {
  if (max_n <= 0) return;
  const int blocks = static_cast<int>(std::min<long long>((max_n + 255) / 256, std::max(max_blocks, 1)));
  if (cnt_sorted) {
    duplicate_kernel<true, true><<<blocks, 256, 0, s>>>(rec, order, offsets, d_n, max_n, cams, cnt_sorted, nullptr,
                                                        nullptr, nullptr, 0);
  } else if (tile_cull) {
    duplicate_kernel<true, false><<<blocks, 256, 0, s>>>(rec, order, offsets, d_n, max_n, cams, nullptr, pair_keys,
                                                         pair_vals, key_counts, key_bits);
  } else {
    duplicate_kernel<false, false><<<blocks, 256, 0, s>>>(rec, order, offsets, d_n, max_n, cams, nullptr, pair_keys,
                                                          pair_vals, key_counts, key_bits);
  }
}

void launch_ranges(const uint32_t* sorted_keys, long long P, int n_tiles, uint2* ranges, cudaStream_t s) {
  if (n_tiles <= 0) return;
  ranges_kernel<<<(n_tiles + 255) / 256, 256, 0, s>>>(sorted_keys, static_cast<uint32_t>(P), n_tiles, ranges);
}

}  // namespace gsr
