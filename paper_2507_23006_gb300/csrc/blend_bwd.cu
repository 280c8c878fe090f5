// Backward pass of the alpha blending of Sec. 3.1, Eq. 2: the forward's tiling, contributors
// walked back to front recovering T_i = T_{i+1} / (1 - a_i); per-Gaussian gradients are summed
// over the warp with shuffles, over the CTA in shared memory, and added to global memory once per
// (tile, Gaussian).
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
      const float tot = TransposeSum<kVals, 16>::run(gv, lane);
      if (t_keep) atomicAdd(&sAcc[j][t_idx], tot);
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
