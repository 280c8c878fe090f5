// Forward alpha blending of Sec. 3.1, Eq. 2: one 16x16 CTA per tile; records are staged in
// shared memory 256 at a time; each pixel blends front to back and stops at T < 1e-4; the CTA
// stops loading once every pixel is done. Short tile lists are sorted here first.
#include "gsr_internal.cuh"
#include "tile_util.cuh"

namespace gsr {
namespace {

// tile_keys (nullable): the tiles' unsorted keys (depth bits << 32 | record index) as placed by
// the binning. A tile of at most kTileSortSmall pairs is then sorted here, in shared memory (the
// dynamic shared memory holds the next power of two of the longest such list), and its record
// order written to pvals for the backward; the longer lists arrive sorted in pvals. Without
// tile_keys every list arrives sorted in pvals.
template <bool kCount>
__global__ void __launch_bounds__(kBlendThreads) blend_fwd_kernel(const Rec* __restrict__ rec, uint32_t* pvals,
                                                                  const unsigned long long* __restrict__ tile_keys,
                                                                  const uint2* __restrict__ ranges, CamBatch cams,
                                                                  float3 bg, BlendFwdOut out,
                                                                  unsigned long long* counters) {
  extern __shared__ unsigned long long s_keys[];
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
  const bool sorted_here = tile_keys != nullptr && n <= kTileSortSmall;  // block-uniform
  if (sorted_here && n > 0) {
    int m = 1;
    while (m < n) m <<= 1;
    if (m <= kBlendThreads) {  // one key per thread: mostly warp shuffles, a few block exchanges
      const unsigned long long x =
          block_bitonic_sort_regs(tid < n ? tile_keys[range.x + tid] : ~0ull, m, s_keys);
      __syncthreads();  // s_keys was the exchange buffer
      if (tid < n) {
        s_keys[tid] = x;
        pvals[range.x + tid] = static_cast<uint32_t>(x);
      }
    } else {
      for (int i = tid; i < m; i += kBlendThreads) s_keys[i] = i < n ? tile_keys[range.x + i] : ~0ull;
      __syncthreads();
      block_bitonic_sort(s_keys, m);
      for (int i = tid; i < n; i += kBlendThreads) pvals[range.x + i] = static_cast<uint32_t>(s_keys[i]);
    }
  }
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
        const Rec r = rec[sorted_here ? static_cast<uint32_t>(s_keys[idx]) : pvals[range.x + idx]];
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

}  // namespace

void launch_blend_fwd(const Rec* rec, uint32_t* pair_vals, const unsigned long long* tile_keys, uint32_t max_count,
                      const uint2* ranges, const CamBatch& cams, const float* bg, const BlendFwdOut& out,
                      unsigned long long* counters, cudaStream_t s) {
  if (cams.total_tiles <= 0) return;
  const float3 b3 = make_float3(bg[0], bg[1], bg[2]);
  size_t smem = 0;
  if (tile_keys) {  // the longest list sorted here, and at least one key per thread
    int cap = kBlendThreads;
    while (cap < static_cast<long long>(max_count) && cap < kTileSortSmall) cap <<= 1;
    smem = sizeof(unsigned long long) * cap;
  }
  if (counters)
    blend_fwd_kernel<true><<<cams.total_tiles, kBlendThreads, smem, s>>>(rec, pair_vals, tile_keys, ranges, cams, b3,
                                                                         out, counters);
  else
    blend_fwd_kernel<false><<<cams.total_tiles, kBlendThreads, smem, s>>>(rec, pair_vals, tile_keys, ranges, cams, b3,
                                                                          out, nullptr);
}

}  // namespace gsr
