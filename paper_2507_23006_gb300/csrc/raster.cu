// Tile binning and the per-tile alpha blending of Sec. 3.1, Eq. 2, forward and backward.
//
//   binning:    every visible record has one (tile, record) pair per tile of its 3-sigma
//               rectangle, minus the tiles StopThePop culling drops (Sec. 3.4.2): the pairs are
//               counted per tile, the counts scanned into each tile's [start, end), the pairs
//               placed in their tile's range, and each tile's list sorted by (depth, index).
//   blend fwd:  one 16x16 CTA per tile; records are staged in shared memory 256 at a time;
//               each pixel blends front to back and stops at T < 1e-4; the CTA stops loading
//               once every pixel is done.
//   blend bwd:  same tiling, contributors walked back to front recovering T_i = T_{i+1}/(1-a_i);
//               per-Gaussian gradients are summed over the warp with shuffles, over the CTA in
//               shared memory, and added to global memory once per (tile, Gaussian).
#include <algorithm>
#include <atomic>

#include "gsr_internal.cuh"
#include "scan_util.cuh"

namespace gsr {
namespace {

__device__ __forceinline__ int find_cam(const CamBatch& cams, int t) {
  int c = 0;
  while (c + 1 < cams.C && t >= cams.cam[c + 1].tile_off) ++c;
  return c;
}

// Smallest Mahalanobis distance (p - m)^T Q (p - m) over the rectangle of pixel centres of a tile.
// Every operation is explicitly rounded (no contraction left to the compiler), so the counting and
// the placing pass of the binning, two separately compiled kernels, take the same decisions.
__device__ __forceinline__ float quad_form(float a, float b, float c, float dx, float dy) {
  return __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(a, dx), dx), __fmul_rn(__fmul_rn(2.f, b), __fmul_rn(dx, dy))),
                   __fmul_rn(__fmul_rn(c, dy), dy));
}
__device__ __forceinline__ float tile_min_maha(float mx, float my, float a, float b, float c, float xlo,
                                               float xhi, float ylo, float yhi) {
  if (mx >= xlo && mx <= xhi && my >= ylo && my <= yhi) return 0.f;
  float best = INFINITY;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const float dx = __fsub_rn(e ? xhi : xlo, mx);
    const float dy = fminf(fmaxf(__fdiv_rn(__fmul_rn(-b, dx), c), __fsub_rn(ylo, my)), __fsub_rn(yhi, my));
    best = fminf(best, quad_form(a, b, c, dx, dy));
  }
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const float dy = __fsub_rn(e ? yhi : ylo, my);
    const float dx = fminf(fmaxf(__fdiv_rn(__fmul_rn(-b, dy), a), __fsub_rn(xlo, mx)), __fsub_rn(xhi, mx));
    best = fminf(best, quad_form(a, b, c, dx, dy));
  }
  return best;
}

// The blend kernels run 128 threads per 16x16 tile (four warps of 8x8 pixels, below). Records
// are staged 256 at a time.
constexpr int kBlendThreads = 128;
constexpr int kBlendWarps = kBlendThreads / 32;
constexpr int kBatch = 256;

// Each warp of a blend block covers one 8x8 quarter of the 16x16 tile (warp w: columns
// 8 (w & 1) .. +7, rows 8 (w >> 1) .. +7; lane l: column l & 7, rows 2 (l >> 3) and +1).
// Bit w is set when the Gaussian's alpha >= 1/255 box (record field d) meets the pixel centres
// of warp w; (x0, y0) is the tile's first pixel centre, (x_max, y_max) the image's last.
__device__ __forceinline__ uint32_t warp_block_mask(const float4 d, float x0, float y0, float x_max, float y_max) {
  uint32_t m = 0;
#pragma unroll
  for (int w = 0; w < kBlendWarps; ++w) {
    const float xl = x0 + 8.f * (w & 1), yl = y0 + 8.f * (w >> 1);
    const float xh = fminf(xl + 7.f, x_max), yh = fminf(yl + 7.f, y_max);
    if (d.y >= xl && d.x <= xh && d.w >= yl && d.z <= yh) m |= 1u << w;
  }
  return m;
}

// Counts (kPlace = false) or places (kPlace = true) the (tile, record) pairs of the visible
// records: one per tile of a record's rectangle, minus the tiles StopThePop culling drops (kCull;
// the same FP32 test in both passes, so they agree pair for pair). A warp takes 32 records and
// shares their tiles out over its lanes, so one huge ground splat does not stall its neighbours.
// Counting adds one to the tile's counter per kept pair; placing takes the pair's slot from the
// tile's cursor (set to the tile's first slot by the scan) and writes the key (depth bits << 32 |
// record index) there. The order inside a tile is then fixed by sorting those keys.
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
    uint32_t area = 0, lo = 0, hi = 0;
    float4 ra = make_float4(0, 0, 0, 0), rb = ra;
    if (i < n) {
      const Rec r = rec[i];
      ra = r.a;
      rb = r.b;
      lo = __float_as_uint(r.c.z);
      hi = __float_as_uint(r.c.w);
      area = ((lo >> 16) - (lo & 0xffffu)) * (((hi >> 16) & 0x7ffu) - (hi & 0xffffu));
    }
    uint32_t incl = area;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    for (uint32_t r0 = 0; r0 < total; r0 += 32) {
      const uint32_t k = r0 + lane;
      const bool active = k < total;
      int owner = 0;  // the record of pair slot k: the first lane whose inclusive count exceeds k
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
      const float mx = __shfl_sync(0xffffffffu, ra.x, owner), my = __shfl_sync(0xffffffffu, ra.y, owner);
      const float op = __shfl_sync(0xffffffffu, ra.z, owner), oz = __shfl_sync(0xffffffffu, ra.w, owner);
      const float ca = __shfl_sync(0xffffffffu, rb.x, owner), cb = __shfl_sync(0xffffffffu, rb.y, owner);
      const float cc = __shfl_sync(0xffffffffu, rb.z, owner);
      if (!active) continue;
      const uint32_t q = k - (o_incl - o_area);
      const uint32_t x0 = o_lo & 0xffffu, wdt = (o_lo >> 16) - x0;
      const uint32_t y0 = o_hi & 0xffffu;
      const int c = static_cast<int>(o_hi >> 27);
      const uint32_t tx = x0 + q % max(wdt, 1u);
      const uint32_t ty = y0 + q / max(wdt, 1u);
      const DevCam& cam = cams.cam[c];
      if (kCull) {
        const float xlo = tx * kTile + 0.5f, xhi = fminf(static_cast<float>((tx + 1) * kTile), cam.W) - 0.5f;
        const float ylo = ty * kTile + 0.5f, yhi = fminf(static_cast<float>((ty + 1) * kTile), cam.H) - 0.5f;
        const float d2 = tile_min_maha(mx, my, ca, cb, cc, xlo, xhi, ylo, yhi);
        if (!(op > 0.f && __fmul_rn(0.5f, d2) <= logf(__fmul_rn(op, 255.f)))) continue;
      }
      const uint32_t t = static_cast<uint32_t>(cam.tile_off) + ty * cam.tiles_x + tx;
      const uint32_t slot = atomicAdd(tile_ctr + t, 1u);
      if (kPlace) {
        // the counting pass made room for exactly this many pairs; a pair beyond the tile's range
        // (which identical decisions rule out) is reported, never written
        if (slot < ranges[t].y) {
          const uint32_t v = static_cast<uint32_t>(base_i) + static_cast<uint32_t>(owner);
          keys[slot] = (static_cast<unsigned long long>(__float_as_uint(oz)) << 32) | v;
        } else {
          atomicOr(err, kErrOverflow);
        }
      }
    }
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

// Sorts m keys (a power of two, at most 2 blockDim.x per round of the loop) in shared memory,
// ascending: Batcher's bitonic network, one comparator per thread and stage.
__device__ __forceinline__ void block_bitonic_sort(unsigned long long* s, int m) {
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int c = threadIdx.x; c < (m >> 1); c += blockDim.x) {
        const int i = 2 * c - (c & (j - 1));  // bit j of i is clear; its partner is i + j
        const unsigned long long a = s[i], b = s[i + j];
        if ((a > b) == ((i & k) == 0)) {
          s[i] = b;
          s[i + j] = a;
        }
      }
      __syncthreads();
    }
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

template <bool kCount>
__global__ void __launch_bounds__(kBlendThreads) blend_fwd_kernel(const Rec* __restrict__ rec,
                                                                  const uint32_t* __restrict__ pvals,
                                                                  const uint2* __restrict__ ranges, CamBatch cams,
                                                                  float3 bg, BlendFwdOut out,
                                                                  unsigned long long* counters) {
  __shared__ float4 sA[kBatch];
  __shared__ float4 sB[kBatch];
  __shared__ float2 sC[kBatch];
  __shared__ uint32_t sM[kBatch];
  const int t = blockIdx.x;
  const int c = find_cam(cams, t);
  const DevCam& cam = cams.cam[c];
  const int lt = t - cam.tile_off;
  const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
  const int tid = threadIdx.x, wid = tid >> 5;
  const int px = tx * kTile + 8 * (wid & 1) + (tid & 7);
  const int py0 = ty * kTile + 8 * (wid >> 1) + 2 * ((tid & 31) >> 3);
  const float fx = px + 0.5f;
  const float fy[2] = {py0 + 0.5f, py0 + 1.5f};
  const bool inside[2] = {px < cam.W && py0 < cam.H, px < cam.W && py0 + 1 < cam.H};
  const float x0 = tx * kTile + 0.5f, y0 = ty * kTile + 0.5f;
  const float x_max = cam.W - 0.5f, y_max = cam.H - 0.5f;
  const uint2 range = ranges[t];
  const int n = static_cast<int>(range.y - range.x);
  // Depth is accumulated relative to the pixel's first contributor (Zf): D = sum (z - Zf) w stays
  // small, so the expected depth Zf + D / (1 - T), and the backward's z_i - (expected depth), keep
  // their absolute precision at any distance (a plain sum of z w at z ~ 1000 carries 1e-4 of rounding).
  float T[2] = {1.f, 1.f}, C0[2] = {0.f, 0.f}, C1[2] = {0.f, 0.f}, C2[2] = {0.f, 0.f}, D[2] = {0.f, 0.f};
  float Zf[2] = {0.f, 0.f};
  uint32_t last[2] = {0, 0};
  bool done[2] = {!inside[0], !inside[1]};
  uint32_t n_eval = 0, n_blend = 0;
  for (int base = 0; base < n; base += kBatch) {
    if (__syncthreads_count(done[0] && done[1]) == kBlendThreads) break;
    for (int k = tid; k < kBatch; k += kBlendThreads) {
      const int idx = base + k;
      if (idx < n) {
        const Rec r = rec[pvals[range.x + idx]];
        sA[k] = r.a;
        sB[k] = r.b;
        sC[k] = make_float2(r.c.x, r.c.y);
        sM[k] = warp_block_mask(r.d, x0, y0, x_max, y_max);
      }
    }
    __syncthreads();
    const int cnt = min(kBatch, n - base);
    // Branch-free over the two pixels of a lane: every test is a predicate, so the warp runs
    // one instruction stream per Gaussian; it leaves once all of its pixels are done.
    for (int j = 0; j < cnt; ++j) {
      if (!((sM[j] >> wid) & 1u)) continue;  // no pixel of this warp can reach alpha 1/255
      if (__all_sync(0xffffffffu, done[0] && done[1])) break;
      const float4 a = sA[j];
      const float4 b = sB[j];
      const float2 cc = sC[j];
      const float dx = a.x - fx;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (kCount) n_eval += !done[q];
        const float dy = a.y - fy[q];
        const float sigma = 0.5f * (b.x * dx * dx + b.z * dy * dy) + b.y * dx * dy;
        const float alpha = fminf(kAlphaMax, a.z * __expf(-sigma));
        const bool ok = !done[q] && sigma >= 0.f && alpha >= kAlphaMin;
        const float Tn = T[q] * (1.f - alpha);
        const bool term = ok && Tn < kTMin;  // stop before T drops below 1e-4
        const bool use = ok && !term;
        const float wgt = use ? alpha * T[q] : 0.f;
        C0[q] = fmaf(b.w, wgt, C0[q]);
        C1[q] = fmaf(cc.x, wgt, C1[q]);
        C2[q] = fmaf(cc.y, wgt, C2[q]);
        Zf[q] = (use && T[q] == 1.f) ? a.w : Zf[q];  // T < 1 after the first contributor
        D[q] = fmaf(a.w - Zf[q], wgt, D[q]);
        T[q] = use ? Tn : T[q];
        last[q] = use ? static_cast<uint32_t>(base + j + 1) : last[q];
        done[q] = done[q] || term;
        if (kCount) n_blend += use;
      }
    }
  }
  if (kCount) {
    unsigned long long e = n_eval, b = n_blend;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((tid & 31) == 0) {
      atomicAdd(counters + 0, e);
      atomicAdd(counters + 1, b);
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (!inside[q]) continue;
    const long long pix = cam.pix_off + static_cast<long long>(py0 + q) * cam.W + px;
    float r0, r1, r2;
    const float o = 1.f - T[q];
    if (cam.aff) {
      const float* A = cam.aff;
      r0 = A[0] * C0[q] + A[1] * C1[q] + A[2] * C2[q] + A[3] * o;
      r1 = A[4] * C0[q] + A[5] * C1[q] + A[6] * C2[q] + A[7] * o;
      r2 = A[8] * C0[q] + A[9] * C1[q] + A[10] * C2[q] + A[11] * o;
    } else {
      r0 = C0[q]; r1 = C1[q]; r2 = C2[q];
    }
    out.rgb[3 * pix + 0] = r0 + T[q] * bg.x;
    out.rgb[3 * pix + 1] = r1 + T[q] * bg.y;
    out.rgb[3 * pix + 2] = r2 + T[q] * bg.z;
    // o is 0 (no contributor) or at least 1/255
    if (out.depth_acc) out.depth_acc[pix] = fmaf(Zf[q], o, D[q]);
    if (out.depth_exp) out.depth_exp[pix] = o > 0.f ? Zf[q] + D[q] / o : 0.f;
    if (out.alpha) out.alpha[pix] = o;
    if (out.T_final) out.T_final[pix] = T[q];
    if (out.n_contrib) out.n_contrib[pix] = last[q];
    if (out.D_state) out.D_state[pix] = make_float2(Zf[q], D[q]);
  }
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

constexpr int kGradVals = 12;

// Sums N (<= 16) per-lane values over the warp with about N + 2 shuffles instead of 5 N. Each
// round halves the vector: a lane sends the half it gives up to its partner across `kBit` and
// keeps the sum of the other half (an odd length is padded with a zero). Once one value is
// left, the remaining lane bits are summed directly. index() gives the value each lane ends up
// holding (-1: padding).
template <int N, int kBit>
struct TransposeSum {
  static __device__ __forceinline__ float run(const float* v, int lane) {
    constexpr int H = (N + 1) / 2;
    const bool up = lane & kBit;
    float w[H];
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const float lo = v[k];
      const float hi = (k + H < N) ? v[k + H] : 0.f;
      const float send = up ? lo : hi;
      const float keep = up ? hi : lo;
      w[k] = keep + __shfl_xor_sync(0xffffffffu, send, kBit);
    }
    return TransposeSum<H, kBit / 2>::run(w, lane);
  }
  static __device__ __forceinline__ int index(int lane) {
    constexpr int H = (N + 1) / 2;
    const int r = TransposeSum<H, kBit / 2>::index(lane);
    if (r < 0) return -1;
    if (lane & kBit) return r < N - H ? H + r : -1;  // the upper half holds N - H values
    return r;
  }
};
template <int kBit>
struct TransposeSum<1, kBit> {
  static __device__ __forceinline__ float run(const float* v, int) {
    float x = v[0];
#pragma unroll
    for (int b = kBit; b > 0; b >>= 1) x += __shfl_xor_sync(0xffffffffu, x, b);
    return x;
  }
  static __device__ __forceinline__ int index(int) { return 0; }
};

// Lane bits still summed directly after the halving rounds of an N-value transpose sum: lanes
// that differ only in these bits hold the same total.
template <int N>
__host__ __device__ constexpr int transpose_shared_bits() {
  int n = N, bit = 16;
  while (n > 1 && bit > 0) { n = (n + 1) / 2; bit >>= 1; }
  return 2 * bit - 1;
}

// kAbs: also accumulate |dL/dmean2D| per pixel (AbsGS densification statistics).
template <bool kCount, bool kAbs>
__global__ void __launch_bounds__(kBlendThreads, 6) blend_bwd_kernel(const Rec* __restrict__ rec,
                                                                  const uint32_t* __restrict__ pvals,
                                                                  const uint2* __restrict__ ranges, CamBatch cams,
                                                                  float3 bg, BlendBwdIn in, Grad2D* __restrict__ g2d,
                                                                  float* __restrict__ g_aff,
                                                                  unsigned long long* counters) {
  constexpr int kVals = kAbs ? kGradVals : kGradVals - 2;  // gradient values summed per Gaussian
  __shared__ float4 sA[kBatch];
  __shared__ float4 sB[kBatch];
  __shared__ float2 sC[kBatch];
  __shared__ uint32_t sV[kBatch];
  __shared__ uint32_t sM[kBatch];
  __shared__ float sAcc[kBatch][kGradVals + 1];
  __shared__ uint32_t s_max;
  __shared__ float s_aff[kBlendWarps][12];
  const int t = blockIdx.x;
  const int c = find_cam(cams, t);
  const DevCam& cam = cams.cam[c];
  const int lt = t - cam.tile_off;
  const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int t_idx = TransposeSum<kVals, 16>::index(lane);  // the gradient value this lane sums
  const bool t_keep = t_idx >= 0 && (lane & transpose_shared_bits<kVals>()) == 0;
  const int px = tx * kTile + 8 * (wid & 1) + (tid & 7);
  const int py0 = ty * kTile + 8 * (wid >> 1) + 2 * ((tid & 31) >> 3);
  const float fx = px + 0.5f;
  const float fy[2] = {py0 + 0.5f, py0 + 1.5f};
  const bool inside[2] = {px < cam.W && py0 < cam.H, px < cam.W && py0 + 1 < cam.H};
  const float x0 = tx * kTile + 0.5f, y0 = ty * kTile + 0.5f;
  const float x_max = cam.W - 0.5f, y_max = cam.H - 0.5f;
  const uint2 range = ranges[t];
  if (tid == 0) s_max = 0;
  __syncthreads();
  const float* A = cam.aff;
  const float bb0 = A ? A[3] : 0.f, bb1 = A ? A[7] : 0.f, bb2 = A ? A[11] : 0.f;
  // per pixel: upstream gradients of C = sum c a T, of the depth part and of T_final
  float Tf[2], T[2], g0[2], g1[2], g2[2], aout[2], GC0[2], GC1[2], GC2[2], GD[2], GTz[2], zr[2], zrl[2];
  float S0[2] = {0.f, 0.f}, S1[2] = {0.f, 0.f}, S2[2] = {0.f, 0.f}, SD[2] = {0.f, 0.f};
  uint32_t last[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    float zf = 0.f, D = 0.f, gda = 0.f, gde = 0.f, gal = 0.f;
    Tf[q] = 1.f;
    last[q] = 0;
    g0[q] = g1[q] = g2[q] = 0.f;
    if (inside[q]) {
      const long long pix = cam.pix_off + static_cast<long long>(py0 + q) * cam.W + px;
      Tf[q] = in.T_final[pix];
      last[q] = in.n_contrib[pix];
      const float2 ds = in.D_state[pix];  // first contributor's depth, sum of (z - it) w
      zf = ds.x;
      D = ds.y;
      if (in.d_rgb) { g0[q] = in.d_rgb[3 * pix]; g1[q] = in.d_rgb[3 * pix + 1]; g2[q] = in.d_rgb[3 * pix + 2]; }
      if (in.d_depth_acc) gda = in.d_depth_acc[pix];
      if (in.d_depth_exp) gde = in.d_depth_exp[pix];
      if (in.d_alpha) gal = in.d_alpha[pix];
      atomicMax(&s_max, last[q]);
    }
    GC0[q] = g0[q]; GC1[q] = g1[q]; GC2[q] = g2[q];
    if (A) {
      GC0[q] = A[0] * g0[q] + A[4] * g1[q] + A[8] * g2[q];
      GC1[q] = A[1] * g0[q] + A[5] * g1[q] + A[9] * g2[q];
      GC2[q] = A[2] * g0[q] + A[6] * g1[q] + A[10] * g2[q];
    }
    aout[q] = 1.f - Tf[q];
    GD[q] = gda + gde / fmaxf(aout[q], 1e-10f);
    // Depths are carried relative to the pixel's expected depth zr: with z_i = zr + d_i the depth
    // part of dL/dalpha_i, T_i z_i - S_D / (1 - a_i), equals T_i d_i - S_d / (1 - a_i)
    // + zr T_final / (1 - a_i) (the weights behind i sum to T_{i+1} - T_final); this avoids the
    // FP32 cancellation of two large, nearly equal terms when the contributors lie at similar depth.
    // d_i = (z_i - zf) - D / aout is formed from differences of nearby depths only. The T_final
    // term, (dL/dD) zr - dL/dT_final, loses its expected-depth parts, which cancel exactly:
    // it is (dL/ddepth_acc) zr + dL/dalpha - dL/drgb . (bg - b).
    const float zrel = aout[q] > 0.f ? D / aout[q] : 0.f;
    zr[q] = zf;     // d_i = (z_i - zf) - zrel
    zrl[q] = zrel;
    GTz[q] = gda * (zf + zrel) + gal - (g0[q] * (bg.x - bb0) + g1[q] * (bg.y - bb1) + g2[q] * (bg.z - bb2));
    T[q] = Tf[q];
  }
  __syncthreads();
  const int n = static_cast<int>(s_max);
  // the deepest list position any pixel of this warp walks back from: positions past it are
  // skipped without evaluating them
  const uint32_t warp_last = __reduce_max_sync(0xffffffffu, max(last[0], last[1]));
  uint32_t n_visit = 0, n_contrib = 0, n_iter = 0, n_iter_c = 0;
  for (int base = 0; base < n; base += kBatch) {
    __syncthreads();
    for (int k = tid; k < kBatch; k += kBlendThreads) {
      if (base + k < n) {
        const uint32_t pos = range.x + static_cast<uint32_t>(n - 1 - base - k);
        const uint32_t v = pvals[pos];
        const Rec r = rec[v];
        sA[k] = r.a;
        sB[k] = r.b;
        sC[k] = make_float2(r.c.x, r.c.y);
        sV[k] = v;
        sM[k] = warp_block_mask(r.d, x0, y0, x_max, y_max);
      }
#pragma unroll
      for (int m = 0; m < kGradVals; ++m) sAcc[k][m] = 0.f;
    }
    __syncthreads();
    const int cnt = min(kBatch, n - base);
    for (int j = 0; j < cnt; ++j) {
      const uint32_t pos = static_cast<uint32_t>(n - 1 - base - j);
      if (pos >= warp_last || !((sM[j] >> wid) & 1u)) continue;  // warp-uniform: nothing of this warp
      const float4 a = sA[j];
      const float4 b = sB[j];
      const float2 cc = sC[j];
      const float dx = a.x - fx;
      float dyq[2], Gq[2], arawq[2], alphaq[2];
      bool cq[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const bool vis = inside[q] && pos < last[q];
        if (kCount) n_visit += vis;
        dyq[q] = a.y - fy[q];
        const float sigma = 0.5f * (b.x * dx * dx + b.z * dyq[q] * dyq[q]) + b.y * dx * dyq[q];
        Gq[q] = __expf(-sigma);
        arawq[q] = a.z * Gq[q];
        alphaq[q] = fminf(kAlphaMax, arawq[q]);
        cq[q] = vis && sigma >= 0.f && alphaq[q] >= kAlphaMin;
        if (kCount) n_contrib += cq[q];
      }
      // warp-uniform: where no pixel of the warp takes the Gaussian, nothing below changes
      // warp-uniform: which of the lanes' two pixel rows any pixel of the warp takes the Gaussian in
      const bool any0 = __any_sync(0xffffffffu, cq[0]);
      const bool any1 = __any_sync(0xffffffffu, cq[1]);
      if (kCount) {
        n_iter += 1;
        n_iter_c += any0 || any1;
      }
      if (!(any0 || any1)) continue;  // nothing below changes
      float gv[kGradVals];
#pragma unroll
      for (int m = 0; m < kGradVals; ++m) gv[m] = 0.f;
#pragma unroll
      for (int q = 0; q < 2; ++q) {  // branch-free within a row: contributions are masked
        if (!(q ? any1 : any0)) continue;  // warp-uniform: no pixel of this row takes it
        const float dy = dyq[q];
        const float G = Gq[q];
        const float araw = arawq[q];
        const float alpha = alphaq[q];
        const bool c = cq[q];
        const float rom = __fdividef(1.f, 1.f - alpha);  // 1 / (1 - alpha) to 2 ulp (1 - alpha >= 0.01)
        const float Ti = T[q] * rom;
        const float wgt = c ? alpha * Ti : 0.f;
        const float dz = (a.w - zr[q]) - zrl[q];
        const float dal = Ti * (GC0[q] * b.w + GC1[q] * cc.x + GC2[q] * cc.y + GD[q] * dz) +
                          (GTz[q] * Tf[q] - (GC0[q] * S0[q] + GC1[q] * S1[q] + GC2[q] * S2[q] + GD[q] * SD[q])) * rom;
        S0[q] = fmaf(b.w, wgt, S0[q]);
        S1[q] = fmaf(cc.x, wgt, S1[q]);
        S2[q] = fmaf(cc.y, wgt, S2[q]);
        SD[q] = fmaf(dz, wgt, SD[q]);
        T[q] = c ? Ti : T[q];
        const float draw = (c && araw <= kAlphaMax) ? dal : 0.f;  // the clamp at 0.99 passes no gradient
        const float dsig = -draw * araw;
        const float dmx = (b.x * dx + b.y * dy) * dsig;
        const float dmy = (b.y * dx + b.z * dy) * dsig;
        gv[0] += dmx;
        gv[1] += dmy;
        gv[2] += draw * G;
        gv[3] += GD[q] * wgt;
        gv[4] += 0.5f * dx * dx * dsig;
        gv[5] += dx * dy * dsig;
        gv[6] += 0.5f * dy * dy * dsig;
        gv[7] += GC0[q] * wgt;
        gv[8] += GC1[q] * wgt;
        gv[9] += GC2[q] * wgt;
        if (kAbs) {
          gv[10] += fabsf(dmx);
          gv[11] += fabsf(dmy);
        }
      }
      const float tot = TransposeSum<kVals, 16>::run(gv, lane);
      if (t_keep) atomicAdd(&sAcc[j][t_idx], tot);
    }
    __syncthreads();
    for (int k = tid; k < cnt; k += kBlendThreads) {
      float* f = reinterpret_cast<float*>(g2d + sV[k]);
#pragma unroll
      for (int m = 0; m < kVals; ++m) {
        const float val = sAcc[k][m];
        if (val != 0.f) atomicAdd(f + m, val);
      }
    }
  }
  if (kCount) {
    unsigned long long e = n_visit, b = n_contrib;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      atomicAdd(counters + 2, e);
      atomicAdd(counters + 3, b);
      atomicAdd(counters + 4, static_cast<unsigned long long>(n_iter));  // warp-uniform counts
      atomicAdd(counters + 5, static_cast<unsigned long long>(n_iter_c));
    }
  }
  if (g_aff) {
    // dA = g C^T, db = g (1 - T_final), per pixel, summed over the tile
    float a12[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) a12[k] = 0.f;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!inside[q]) continue;
      a12[0] += g0[q] * S0[q]; a12[1] += g0[q] * S1[q]; a12[2] += g0[q] * S2[q]; a12[3] += g0[q] * aout[q];
      a12[4] += g1[q] * S0[q]; a12[5] += g1[q] * S1[q]; a12[6] += g1[q] * S2[q]; a12[7] += g1[q] * aout[q];
      a12[8] += g2[q] * S0[q]; a12[9] += g2[q] * S1[q]; a12[10] += g2[q] * S2[q]; a12[11] += g2[q] * aout[q];
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float sum = warp_sum(a12[k]);
      if (lane == 0) s_aff[wid][k] = sum;
    }
    __syncthreads();
    if (tid < 12) {
      float sum = 0.f;
      for (int k = 0; k < kBlendWarps; ++k) sum += s_aff[k][tid];
      if (sum != 0.f) atomicAdd(g_aff + 12 * c + tid, sum);
    }
  }
}

}  // namespace

void launch_bin_pairs(const Rec* rec, const uint32_t* d_n, long long max_n, const CamBatch& cams, int tile_cull,
                      uint32_t* tile_ctr, const uint2* ranges, unsigned long long* keys, int* err, int max_blocks,
                      cudaStream_t s) {
  if (max_n <= 0) return;
  const int blocks = static_cast<int>(std::min<long long>((max_n + 255) / 256, std::max(max_blocks, 1)));
#define GSR_BIN(C, P) bin_pairs_kernel<C, P><<<blocks, 256, 0, s>>>(rec, d_n, max_n, cams, tile_ctr, ranges, keys, err)
  if (keys) {
    if (tile_cull) GSR_BIN(true, true); else GSR_BIN(false, true);
  } else {
    if (tile_cull) GSR_BIN(true, false); else GSR_BIN(false, false);
  }
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
                      int grid_cap, cudaStream_t s) {
  if (n_tiles <= 0 || max_count == 0) return;
  int cap = 1;
  while (cap < static_cast<long long>(max_count) && cap < kTileSortSmall) cap <<= 1;
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

void launch_blend_fwd(const Rec* rec, const uint32_t* pair_vals, const uint2* ranges, const CamBatch& cams,
                      const float* bg, const BlendFwdOut& out, unsigned long long* counters, cudaStream_t s) {
  if (cams.total_tiles <= 0) return;
  const float3 b3 = make_float3(bg[0], bg[1], bg[2]);
  if (counters)
    blend_fwd_kernel<true><<<cams.total_tiles, kBlendThreads, 0, s>>>(rec, pair_vals, ranges, cams, b3, out, counters);
  else
    blend_fwd_kernel<false><<<cams.total_tiles, kBlendThreads, 0, s>>>(rec, pair_vals, ranges, cams, b3, out, nullptr);
}

void launch_blend_bwd(const Rec* rec, const uint32_t* pair_vals, const uint2* ranges, const CamBatch& cams,
                      const float* bg, const BlendBwdIn& in, Grad2D* g2d, float* g_aff, int absgrad,
                      unsigned long long* counters, cudaStream_t s) {
  if (cams.total_tiles <= 0) return;
  const float3 b3 = make_float3(bg[0], bg[1], bg[2]);
#define GSR_BWD(C, A)                                                                                  \
  blend_bwd_kernel<C, A><<<cams.total_tiles, kBlendThreads, 0, s>>>(rec, pair_vals, ranges, cams, b3, in, g2d, \
                                                                    g_aff, counters)
  if (counters) {
    if (absgrad) GSR_BWD(true, true); else GSR_BWD(true, false);
  } else {
    if (absgrad) GSR_BWD(false, true); else GSR_BWD(false, false);
  }
#undef GSR_BWD
}

}  // namespace gsr
