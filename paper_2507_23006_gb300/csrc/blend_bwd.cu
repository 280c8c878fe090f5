// Backward pass of the alpha blending of Sec. 3.1, Eq. 2: the forward's tiling, contributors
// walked back to front recovering T_i = T_{i+1} / (1 - a_i); per-Gaussian gradients are summed
// over the warp through a row exchange in shared memory, over the CTA with shared atomics, and
// added to global memory once per (tile, Gaussian).
#include "gsr_internal.cuh"
#include "tile_util.cuh"

namespace gsr {
namespace {

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

constexpr int kGradVals = 12;

// Each lane of a warp holds two pixels of the warp's 8x8 block (column lane & 7; row lane >> 3 of
// the upper half and the row four below it in the lower half). Bit 2w + h is set when the
// Gaussian's alpha >= 1/255 box (record field d) meets the pixel centres of half h of warp w's
// block; (x0, y0) is the tile's first pixel centre, (x_max, y_max) the image's last.
__device__ __forceinline__ uint32_t warp_half_mask(const float4 d, float x0, float y0, float x_max, float y_max) {
  uint32_t m = 0;
#pragma unroll
  for (int w = 0; w < kBlendWarps; ++w) {
    const float xl = x0 + 8.f * (w & 1), xh = fminf(xl + 7.f, x_max);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float yl = y0 + 8.f * (w >> 1) + 4.f * h, yh = fminf(yl + 3.f, y_max);
      if (d.y >= xl && d.x <= xh && d.w >= yl && d.z <= yh) m |= 1u << (2 * w + h);
    }
  }
  return m;
}

// kAbs: also accumulate |dL/dmean2D| per pixel (AbsGS densification statistics). kAff: the
// gradient of the per-image 3x4 colour transform is wanted (the colour sums are then kept).
template <bool kCount, bool kAbs, bool kAff>
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
  // per-Gaussian sums of a warp: each lane writes its kVals values as one row, then lane
  // (m, part) adds value m over every kParts-th row from row `part` (row stride kVals + 1, an odd
  // number of words, so that neither the row writes nor the column reads meet a bank twice)
  constexpr int kStride = kVals + 1;
  constexpr int kParts = kVals <= 10 ? 3 : 2;
  __shared__ float sRed[kBlendWarps][32 * kStride];
  __shared__ uint32_t s_max;
  __shared__ float s_aff[kBlendWarps][12];
  const int t = blockIdx.x;
  const int c = find_cam(cams, t);
  const DevCam& cam = cams.cam[c];
  const int lt = t - cam.tile_off;
  const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  float* const red_row = &sRed[wid][lane * kStride];
  const int red_m = lane % kVals, red_part = lane / kVals;  // the value and the rows this lane sums
  const float* const red_col = &sRed[wid][red_part * kStride + red_m];
  // the lane's pixels: the upper and the lower half of the warp's 8x8 block (warp_half_mask)
  const int px = tx * kTile + 8 * (wid & 1) + (tid & 7);
  const int py0 = ty * kTile + 8 * (wid >> 1) + ((tid & 31) >> 3);
  const float fx = px + 0.5f;
  const float fy[2] = {py0 + 0.5f, py0 + 4.5f};
  const bool inside[2] = {px < cam.W && py0 < cam.H, px < cam.W && py0 + 4 < cam.H};
  const float x0 = tx * kTile + 0.5f, y0 = ty * kTile + 0.5f;
  const float x_max = cam.W - 0.5f, y_max = cam.H - 0.5f;
  const uint2 range = ranges[t];
  if (tid == 0) s_max = 0;
  __syncthreads();
  const float* A = cam.aff;
  const float bb0 = A ? A[3] : 0.f, bb1 = A ? A[7] : 0.f, bb2 = A ? A[11] : 0.f;
  // per pixel: upstream gradients of C = sum c a T, of the depth part and of T_final
  float Tf[2], T[2], g0[2], g1[2], g2[2], aout[2], GC0[2], GC1[2], GC2[2], GD[2], GTz[2], zr[2], zrl[2];
  // R = dL/dT_final-like remainder: GTz T_final minus the sum, over the contributors behind the
  // current one, of X_k w_k with X_k = GC . c_k + GD dz_k (w_k = alpha_k T_k); S: the colour sums
  // behind it (only for the transform's gradient)
  float R[2], S0[2] = {0.f, 0.f}, S1[2] = {0.f, 0.f}, S2[2] = {0.f, 0.f};
  uint32_t last[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    float zf = 0.f, D = 0.f, gda = 0.f, gde = 0.f, gal = 0.f;
    Tf[q] = 1.f;
    last[q] = 0;
    g0[q] = g1[q] = g2[q] = 0.f;
    if (inside[q]) {
      const long long pix = cam.pix_off + static_cast<long long>(py0 + 4 * q) * cam.W + px;
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
    R[q] = GTz[q] * Tf[q];
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
        sM[k] = warp_half_mask(r.d, x0, y0, x_max, y_max);
#pragma unroll
        for (int m = 0; m < kGradVals; ++m) sAcc[k][m] = 0.f;
      }
    }
    __syncthreads();
    const int cnt = min(kBatch, n - base);
    for (int j = 0; j < cnt; ++j) {
      const uint32_t pos = static_cast<uint32_t>(n - 1 - base - j);
      const uint32_t halves = (sM[j] >> (2 * wid)) & 3u;  // halves of the warp's block the box meets
      if (pos >= warp_last || halves == 0u) continue;     // warp-uniform: nothing of this warp
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
        Gq[q] = arawq[q] = alphaq[q] = 0.f;
        cq[q] = false;
        if ((halves >> q) & 1u) {  // warp-uniform: no pixel of a half outside the box takes it
          const float sigma = 0.5f * (b.x * dx * dx + b.z * dyq[q] * dyq[q]) + b.y * dx * dyq[q];
          Gq[q] = __expf(-sigma);
          arawq[q] = a.z * Gq[q];
          alphaq[q] = fminf(kAlphaMax, arawq[q]);
          cq[q] = vis && sigma >= 0.f && alphaq[q] >= kAlphaMin;
        }
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
      const float dx2 = dx * dx;
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
        const float X = GC0[q] * b.w + GC1[q] * cc.x + GC2[q] * cc.y + GD[q] * dz;
        const float dal = Ti * X + R[q] * rom;
        R[q] = fmaf(-X, wgt, R[q]);
        if (kAff) {
          S0[q] = fmaf(b.w, wgt, S0[q]);
          S1[q] = fmaf(cc.x, wgt, S1[q]);
          S2[q] = fmaf(cc.y, wgt, S2[q]);
        }
        T[q] = c ? Ti : T[q];
        const float draw = (c && araw <= kAlphaMax) ? dal : 0.f;  // the clamp at 0.99 passes no gradient
        const float dsig = -draw * araw;
        // the pixel offsets weighted by dL/dsigma: the mean's gradient is (a, b; b, c) times the
        // first moments and the conic's is (1/2, 1, 1/2) times the second moments, applied once
        // per (tile, Gaussian) when the sums are flushed
        gv[0] = fmaf(dsig, dx, gv[0]);
        gv[1] = fmaf(dsig, dy, gv[1]);
        gv[2] += draw * G;
        gv[3] += GD[q] * wgt;
        gv[4] = fmaf(dsig, dx2, gv[4]);
        gv[5] = fmaf(dsig, dx * dy, gv[5]);
        gv[6] = fmaf(dsig, dy * dy, gv[6]);
        gv[7] += GC0[q] * wgt;
        gv[8] += GC1[q] * wgt;
        gv[9] += GC2[q] * wgt;
        if (kAbs) {  // AbsGS sums |dL/dmean2D| per pixel
          gv[10] += fabsf((b.x * dx + b.y * dy) * dsig);
          gv[11] += fabsf((b.y * dx + b.z * dy) * dsig);
        }
      }
#pragma unroll
      for (int m = 0; m < kVals; ++m) red_row[m] = gv[m];
      __syncwarp();
      float tot = 0.f;
      if (red_part < kParts) {
#pragma unroll
        for (int i = 0; i < (32 + kParts - 1) / kParts; ++i)
          if (red_part + kParts * i < 32) tot += red_col[kParts * kStride * i];
      }
      // the parts of value m are in lanes m, m + kVals (and m + 2 kVals); each lane's reads are
      // complete once its sum enters the shuffles, before any lane writes the next row
      const float t1 = __shfl_down_sync(0xffffffffu, tot, kVals);
      if (kParts == 3) tot += __shfl_down_sync(0xffffffffu, tot, 2 * kVals);
      tot += t1;
      if (lane < kVals) atomicAdd(&sAcc[j][lane], tot);
    }
    __syncthreads();
    for (int k = tid; k < cnt; k += kBlendThreads) {
      float* f = reinterpret_cast<float*>(g2d + sV[k]);
      float v[kVals];
#pragma unroll
      for (int m = 0; m < kVals; ++m) v[m] = sAcc[k][m];
      const float4 cb = sB[k];  // the Gaussian's conic (a, b, c)
      const float mx = v[0], my = v[1];
      v[0] = cb.x * mx + cb.y * my;
      v[1] = cb.y * mx + cb.z * my;
      v[4] *= 0.5f;
      v[6] *= 0.5f;
#pragma unroll
      for (int m = 0; m < kVals; ++m)
        if (v[m] != 0.f) atomicAdd(f + m, v[m]);
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
  if (kAff) {
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

void launch_blend_bwd(const Rec* rec, const uint32_t* pair_vals, const uint2* ranges, const CamBatch& cams,
                      const float* bg, const BlendBwdIn& in, Grad2D* g2d, float* g_aff, int absgrad,
                      unsigned long long* counters, cudaStream_t s) {
  if (cams.total_tiles <= 0) return;
  const float3 b3 = make_float3(bg[0], bg[1], bg[2]);
#define GSR_BWD(C, A, F)                                                                                  \
  blend_bwd_kernel<C, A, F><<<cams.total_tiles, kBlendThreads, 0, s>>>(rec, pair_vals, ranges, cams, b3, in, g2d, \
                                                                       g_aff, counters)
#define GSR_BWD_AFF(C, A) \
  if (g_aff) GSR_BWD(C, A, true); else GSR_BWD(C, A, false)
  if (counters) {
    if (absgrad) { GSR_BWD_AFF(true, true); } else { GSR_BWD_AFF(true, false); }
  } else {
    if (absgrad) { GSR_BWD_AFF(false, true); } else { GSR_BWD_AFF(false, false); }
  }
#undef GSR_BWD_AFF
#undef GSR_BWD
}

}  // namespace gsr
