// Device helpers shared by the binning and the blend kernels (Sec. 3.1, Eq. 2): the tile
// geometry of a camera batch, the StopThePop tile test, the blend blocks' warp layout, and the
// shared-memory bitonic sort of short key lists.
#pragma once

#include "gsr_internal.cuh"

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

// The (tile, record) pairs of the 32 records v_base + lane held by a warp's lanes (`has` false
// for a lane without one; every lane of the warp calls this): one per tile of a record's
// rectangle, minus the tiles StopThePop culling drops (kCull; explicitly rounded, so every pass
// that calls this takes the same decisions). The lanes share the warp's pairs out evenly, so one
// huge ground splat does not stall its neighbours. Counting (kPlace = false) adds one to the
// tile's counter per kept pair; placing takes the pair's slot from the tile's cursor and writes
// the key (depth bits << 32 | record index) there, a slot past the tile's range (which identical
// decisions rule out) being reported in *err, never written.
template <bool kCull, bool kPlace>
__device__ __forceinline__ void warp_bin_pairs(int lane, bool has, const Rec& r, uint32_t v_base, const CamBatch& cams,
                                               uint32_t* __restrict__ tile_ctr, const uint2* __restrict__ ranges,
                                               unsigned long long* __restrict__ keys, int* err) {
  uint32_t area = 0, lo = 0, hi = 0;
  float4 ra = make_float4(0, 0, 0, 0), rb = ra;
  if (has) {
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
        const uint32_t v = v_base + static_cast<uint32_t>(owner);
        keys[slot] = (static_cast<unsigned long long>(__float_as_uint(oz)) << 32) | v;
      } else {
        atomicOr(err, kErrOverflow);
      }
    }
  }
}

// Sorts the block's keys when there are at most blockDim.x of them, ascending: thread i holds key
// i (~0 past the list) and runs Batcher's bitonic network on m (a power of two, at most
// blockDim.x) keys, exchanging with partner i ^ j by warp shuffle when j < 32 and through s_x
// (blockDim.x keys) otherwise; returns thread i's key after sorting. Every thread of the block
// calls it.
__device__ __forceinline__ unsigned long long block_bitonic_sort_regs(unsigned long long x, int m,
                                                                      unsigned long long* s_x) {
  const int i = threadIdx.x;
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      unsigned long long y;
      if (j >= 32) {  // block-uniform
        s_x[i] = x;
        __syncthreads();
        y = s_x[i ^ j];
        __syncthreads();
      } else {
        y = __shfl_xor_sync(0xffffffffu, x, j);
      }
      // the lower of the two positions keeps the smaller key where this run ascends
      const bool keep_min = ((i & j) == 0) == ((i & k) == 0);
      x = keep_min ? (x < y ? x : y) : (x < y ? y : x);
    }
  }
  return x;
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

}  // namespace
}  // namespace gsr
