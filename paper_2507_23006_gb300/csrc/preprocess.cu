// Per-Gaussian preprocessing (projection, colour, culling) and its backward pass.
//
// Forward (Sec. 3.1, the projection of each 3D Gaussian to a 2D one before blending):
//   Sigma = R S S^T R^T (Eq. 1) from the quaternion and scale, then for every camera of the
//   launch t = W mu + t_cam, T = J W with J the perspective Jacobian at the clamped direction,
//   Sigma2D = T Sigma T^T + eps I, the Mip-Splatting opacity compensation (Sec. 3.5.4), the
//   conic Sigma2D^-1, the 3-sigma tile rectangle, and the colour from degree <= 3 spherical
//   harmonics. Culled: z outside (near, far), a zero or non-finite quaternion, det <= 0, an
//   empty rectangle, any non-finite output.
//
// The cull pass: one thread owns one Gaussian and loops over the cameras, so the means and
// scales are read from HBM once per launch. Visible (Gaussian, camera) records are numbered
// compacted, in (Gaussian, camera) order, from the scanned per-block counts (three passes, no
// block waits on another); within one camera the compacted index grows with the Gaussian index,
// which gives the depth sort its tie-break. The record pass (preprocess_rec.cu) then makes each
// numbered record with a thread of its own.
#include <algorithm>
#include <atomic>

#include "preprocess_fwd.cuh"

namespace gsr {
namespace {

// Backward of the projection and colour. One thread per visible record; the thread holding a
// Gaussian's first record walks all of that Gaussian's cameras (its records are consecutive),
// accumulates the parameter gradients in registers and writes the Gaussian's rows once.
template <typename AT, typename ST>
// Budgeted for three resident blocks per SM (168 registers, some spills): more warps in flight
// hide more of its scattered loads and stores than the spills cost.
__global__ void __launch_bounds__(kBwdThreads, 3) preprocess_bwd_kernel(
    GaussArgs A, CamBatch cams, float eps, int aa, long long V, const Rec* __restrict__ rec,
    const uint32_t* __restrict__ owner, const Grad2D* __restrict__ g2d, ParamGrads out) {
  const long long v0 = static_cast<long long>(blockIdx.x) * kBwdThreads + threadIdx.x;
  if (v0 >= V) return;
  const uint32_t i = owner[v0];
  if (v0 > 0 && owner[v0 - 1] == i) return;  // not the Gaussian's first record
  const long long g = seg_map(A.segs, i);
  float shv[48];
  load_sh_row<ST>(A, g, shv);
  Geo G;
  if (!load_geo<AT>(A, g, G)) return;  // cannot happen for a Gaussian with a record
  float dm[3] = {0, 0, 0}, ds[3] = {0, 0, 0}, dopac = 0.f, dabs[2] = {0, 0};
  float dsh[48];
#pragma unroll
  for (int k = 0; k < 48; ++k) dsh[k] = 0.f;
  float dR[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int KC = A.K * 3;
  const int nb = (A.deg + 1) * (A.deg + 1);
  for (long long v = v0; v < V && owner[v] == i; ++v) {
    const DevCam& cam = cams.cam[rec_cam(rec[v])];
    Proj P;
    project(G, cam, eps, aa, P);
    const Grad2D gd = g2d[v];
    const float dmx = gd.a.x, dmy = gd.a.y, dop = gd.a.z, ddepth = gd.a.w;
    const float dca = gd.b.x, dcb = gd.b.y, dcc = gd.b.z;
    float drgb[3] = {gd.b.w, gd.c.x, gd.c.y};
    dabs[0] += gd.c.z;
    dabs[1] += gd.c.w;
    // colour: rgb = max(0, sum_k sh_k Y_k(dir) + 0.5)
    float rgb[3], dir[3], dn, Y[16];
    bool cl[3];
    eval_color_regs(A.deg, G, cam, shv, rgb, dir, dn, Y, cl);
    for (int ch = 0; ch < 3; ++ch)
      if (cl[ch]) drgb[ch] = 0.f;
    float wY[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      wY[k] = 0.f;
      if (k < nb) {
        dsh[3 * k + 0] += Y[k] * drgb[0];
        dsh[3 * k + 1] += Y[k] * drgb[1];
        dsh[3 * k + 2] += Y[k] * drgb[2];
        wY[k] = shv[3 * k] * drgb[0] + shv[3 * k + 1] * drgb[1] + shv[3 * k + 2] * drgb[2];
      }
    }
    float gx, gy, gz;
    sh_basis_grad(A.deg, dir[0], dir[1], dir[2], wY, gx, gy, gz);
    const float proj = gx * dir[0] + gy * dir[1] + gz * dir[2];
    const float idn = 1.f / dn;
    dm[0] += (gx - dir[0] * proj) * idn;
    dm[1] += (gy - dir[1] * proj) * idn;
    dm[2] += (gz - dir[2] * proj) * idn;
    // conic = inverse of the dilated Sigma2D: dSigma2D = -M G M
    const float g00 = dca, g01 = 0.5f * dcb, g11 = dcc;
    const float mg00 = P.ca * g00 + P.cb * g01, mg01 = P.ca * g01 + P.cb * g11;
    const float mg10 = P.cb * g00 + P.cc * g01, mg11 = P.cb * g01 + P.cc * g11;
    float da = -(mg00 * P.ca + mg01 * P.cb);
    float db = -2.f * (mg00 * P.cb + mg01 * P.cc);
    float dc = -(mg10 * P.cb + mg11 * P.cc);
    // opacity' = opacity * sqrt(det_raw / det)
    dopac += dop * P.comp;
    if (aa && P.comp > 0.f) {
      const float ratio = P.comp * P.comp;
      const float dratio = dop * G.opac * 0.5f / P.comp;
      const float ddr = dratio * P.idet;           // d det_raw
      const float ddt = -dratio * ratio * P.idet;  // d det
      const float a = P.ar + eps, cc = P.cr + eps;
      da += ddr * P.cr + ddt * cc;
      dc += ddr * P.ar + ddt * a;
      db += -2.f * P.br * (ddr + ddt);
    }
    // Sigma2D_raw = T Sigma T^T with T = J W
    float dT0[3], dT1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dT0[k] = 2.f * da * P.ST0[k] + db * P.ST1[k];
      dT1[k] = db * P.ST0[k] + 2.f * dc * P.ST1[k];
    }
    // dSigma (symmetrised) = 2 da T0 T0^T + db (T0 T1^T + T1 T0^T) + 2 dc T1 T1^T; Sigma = M M^T
    float dS[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = 0; q < 3; ++q)
        dS[r * 3 + q] = 2.f * da * P.T0[r] * P.T0[q] + db * (P.T0[r] * P.T1[q] + P.T1[r] * P.T0[q]) +
                        2.f * dc * P.T1[r] * P.T1[q];
    float Mx[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = 0; q < 3; ++q) Mx[r * 3 + q] = G.R[r * 3 + q] * G.s[q];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float dM = dS[r * 3 + 0] * Mx[0 * 3 + q] + dS[r * 3 + 1] * Mx[1 * 3 + q] + dS[r * 3 + 2] * Mx[2 * 3 + q];
        dR[r * 3 + q] += dM * G.s[q];
        ds[q] += dM * G.R[r * 3 + q];
      }
    // T = J W: dJ
    const float* W = cam.R;
    const float dJ00 = dT0[0] * W[0] + dT0[1] * W[1] + dT0[2] * W[2];
    const float dJ02 = dT0[0] * W[6] + dT0[1] * W[7] + dT0[2] * W[8];
    const float dJ11 = dT1[0] * W[3] + dT1[1] * W[4] + dT1[2] * W[5];
    const float dJ12 = dT1[0] * W[6] + dT1[1] * W[7] + dT1[2] * W[8];
    const float uc = fminf(fmaxf(P.u, -cam.limx), cam.limx);
    const float wc = fminf(fmaxf(P.w, -cam.limy), cam.limy);
    const float iz2 = P.iz * P.iz;
    float dt[3] = {0.f, 0.f, 0.f};
    dt[2] += -cam.fx * iz2 * dJ00 + cam.fx * uc * iz2 * dJ02 - cam.fy * iz2 * dJ11 + cam.fy * wc * iz2 * dJ12;
    const float duc = -cam.fx * P.iz * dJ02, dwc = -cam.fy * P.iz * dJ12;
    if (!P.clx) { dt[0] += duc * P.iz; dt[2] -= duc * P.u * P.iz; }
    if (!P.cly) { dt[1] += dwc * P.iz; dt[2] -= dwc * P.w * P.iz; }
    // mean2d = (fx X/Z + cx, fy Y/Z + cy); depth = Z
    dt[0] += cam.fx * P.iz * dmx;
    dt[1] += cam.fy * P.iz * dmy;
    dt[2] += -cam.fx * P.t[0] * iz2 * dmx - cam.fy * P.t[1] * iz2 * dmy + ddepth;
    // t = W mu + t_cam
    dm[0] += W[0] * dt[0] + W[3] * dt[1] + W[6] * dt[2];
    dm[1] += W[1] * dt[0] + W[4] * dt[1] + W[7] * dt[2];
    dm[2] += W[2] * dt[0] + W[5] * dt[1] + W[8] * dt[2];
  }
  // rotation from the normalised quaternion, then through the normalisation
  const float w = G.q[0], x = G.q[1], y = G.q[2], z = G.q[3];
  float dqn[4];
  dqn[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
  dqn[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] -
                  2.f * x * dR[8]);
  dqn[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] -
                  2.f * y * dR[8]);
  dqn[3] = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] +
                  x * dR[6] + y * dR[7]);
  const float qd = w * dqn[0] + x * dqn[1] + y * dqn[2] + z * dqn[3];
  float dq[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) dq[k] = (dqn[k] - G.q[k] * qd) * G.qinv;
  out.means[3 * g + 0] = dm[0];
  out.means[3 * g + 1] = dm[1];
  out.means[3 * g + 2] = dm[2];
  out.scales[3 * g + 0] = ds[0];
  out.scales[3 * g + 1] = ds[1];
  out.scales[3 * g + 2] = ds[2];
  out.opac[g] = dopac;
  if (out.vec4) {
    reinterpret_cast<float4*>(out.quats)[g] = make_float4(dq[0], dq[1], dq[2], dq[3]);
    float4* row = reinterpret_cast<float4*>(out.sh + g * KC);
#pragma unroll
    for (int k = 0; k < 12; ++k)
      if (4 * k < KC) row[k] = make_float4(dsh[4 * k], dsh[4 * k + 1], dsh[4 * k + 2], dsh[4 * k + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) out.quats[4 * g + k] = dq[k];
    float* row = out.sh + g * KC;
#pragma unroll
    for (int k = 0; k < 48; ++k)
      if (k < KC) row[k] = dsh[k];
  }
  if (out.absgrad) {
    out.absgrad[2 * g] = dabs[0];
    out.absgrad[2 * g + 1] = dabs[1];
  }
}

// Backward of the appearance transform, one thread per visible record, blocks looping over
// chunks of kBwdThreads records. With out = sigmoid(z): rgb' = 2 out[0..2] rgb and
// op' = (1 - out[3]) op, so dz_c = rgb'_c d rgb'_c (1 - out_c) and dz_3 = -op' d op' out_3 (no
// division by the outputs); the record's gradients are replaced by those of rgb and op
// (d rgb = 2 out d rgb', d op = (1 - out[3]) d op'), which the projection backward then uses.
// The weight gradients are sums of outer products over the records: each chunk's embeddings,
// hidden activations and pre-activation gradients are staged in shared memory and summed there
// by register tiles; the image part of w1, b1 and the image embeddings depend on a record only
// through its camera, so they are formed once per block from per-camera sums of the
// pre-activation gradients. Each block adds its totals with one atomic per parameter.
struct MlpBwdSmem {
  MlpSmem M;
  float4 lg[kBwdThreads][kEmbG / 4];   // l_G per record; float4 q of row t at q ^ ((t >> 1) & 3)
  float hid[kBwdThreads][kHid + 1];    // ReLU outputs
  float dpre[kBwdThreads][kHid + 1];   // gradients of the hidden pre-activations
  float4 dz[kBwdThreads];              // gradients of the output pre-activations
  int cam[kBwdThreads];
  float sum[kMaxCams][kHid];           // per camera: sum of dpre over the block's records
};

__global__ void __launch_bounds__(kBwdThreads) mlp_bwd_kernel(GaussArgs A, CamBatch cams, long long V,
                                                              const Rec* __restrict__ rec,
                                                              const uint32_t* __restrict__ owner, Grad2D* g2d,
                                                              float* __restrict__ g_gemb, float* __restrict__ g_iemb,
                                                              float* __restrict__ g_params) {
  constexpr int R = kBwdThreads;
  static_assert(R == 128 && kHid == 32 && kEmbG == 16 && kMlpOut == 4, "register tiles assume these sizes");
  extern __shared__ __align__(16) unsigned char mlp_bwd_raw[];
  MlpBwdSmem& S = *reinterpret_cast<MlpBwdSmem*>(mlp_bwd_raw);
  const int t = threadIdx.x;
  mlp_load_smem(A, cams.C, S.M);
  for (int e = t; e < kMaxCams * kHid; e += R) (&S.sum[0][0])[e] = 0.f;
  // register tiles: w1_G[k1][j1..j1+3]; w2[0..3][k2] and b2 over the records of quarter q2;
  // the per-camera sums of dpre[k2] over the same quarter
  const int k1 = t >> 2, j1 = (t & 3) * 4;
  const int k2 = t & 31, q2 = t >> 5;
  float a1[4] = {0.f, 0.f, 0.f, 0.f}, a2[4] = {0.f, 0.f, 0.f, 0.f}, ab2[4] = {0.f, 0.f, 0.f, 0.f};
  float cam_acc = 0.f;
  int cam_cur = -1;
  __syncthreads();
  // The thread's record of the next chunk is loaded one chunk ahead (its loads are in flight
  // during the current chunk's parameter sums): camera, opacity', rgb', the four upstream
  // gradients the transform changes, the Gaussian and its embedding.
  const long long stride = static_cast<long long>(gridDim.x) * R;
  bool f_ok = false;
  int f_cam = -1;
  long long f_g = 0;
  float f_op = 0.f, f_rgb[3] = {0.f, 0.f, 0.f}, f_d[4] = {0.f, 0.f, 0.f, 0.f}, f_lg[kEmbG];
  auto fetch = [&](long long v) {
    f_ok = v < V;
    f_cam = -1;
#pragma unroll
    for (int j = 0; j < kEmbG; ++j) f_lg[j] = 0.f;
    if (!f_ok) return;
    const float4* rp = reinterpret_cast<const float4*>(rec + v);
    const float4 ra = rp[0], rb = rp[1], rc = rp[2];
    f_op = ra.z;
    f_rgb[0] = rb.w;
    f_rgb[1] = rc.x;
    f_rgb[2] = rc.y;
    f_cam = static_cast<int>(__float_as_uint(rc.w) >> 27);
    const float* gp = reinterpret_cast<const float*>(g2d + v);
    f_d[0] = gp[2];  // opacity'
    f_d[1] = gp[7];  // red
    f_d[2] = gp[8];  // green
    f_d[3] = gp[9];  // blue
    f_g = seg_map(A.segs, owner[v]);
    load_gemb(A, f_g, f_lg);
  };
  fetch(static_cast<long long>(blockIdx.x) * R + t);
  for (long long base = static_cast<long long>(blockIdx.x) * R; base < V; base += stride) {
    const long long v = base + t;
    const int c = f_cam;
    const long long g = f_g;
    float lg[kEmbG];
#pragma unroll
    for (int j = 0; j < kEmbG; ++j) lg[j] = f_lg[j];
    float dz[kMlpOut] = {0.f, 0.f, 0.f, 0.f};
    if (f_ok) {
      uint32_t on = 0;  // ReLU active
      float out[kMlpOut];
      mlp_eval_f(S.M, lg, c, out, [&](int k, float a, float h) {
        on |= (a > 0.f ? 1u : 0u) << k;
        S.hid[t][k] = h;
      });
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) dz[ch] = f_rgb[ch] * f_d[1 + ch] * (1.f - out[ch]);
      dz[3] = -f_op * f_d[0] * out[3];
      float* gw = reinterpret_cast<float*>(g2d + v);
      gw[2] = f_d[0] * (1.f - out[3]);
      gw[7] = 2.f * out[0] * f_d[1];
      gw[8] = 2.f * out[1] * f_d[2];
      gw[9] = 2.f * out[2] * f_d[3];
      float dlg[kEmbG];
#pragma unroll
      for (int j = 0; j < kEmbG; ++j) dlg[j] = 0.f;
#pragma unroll 4
      for (int k = 0; k < kHid; ++k) {
        float dh = 0.f;
#pragma unroll
        for (int o = 0; o < kMlpOut; ++o) dh = fmaf(S.M.w2[o][k], dz[o], dh);
        const float dp = (on >> k) & 1u ? dh : 0.f;
        S.dpre[t][k] = dp;
#pragma unroll
        for (int j = 0; j < kEmbG; ++j) dlg[j] = fmaf(S.M.w1g[k][j], dp, dlg[j]);
      }
      float* dst = g_gemb + g * kEmbG;
#pragma unroll
      for (int j = 0; j < kEmbG; ++j) atomicAdd(dst + j, dlg[j]);
    } else {
#pragma unroll
      for (int k = 0; k < kHid; ++k) S.hid[t][k] = S.dpre[t][k] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < kEmbG; j += 4)  // swizzled: the eight lanes of one store phase hit distinct banks
      S.lg[t][(j >> 2) ^ ((t >> 1) & 3)] = make_float4(lg[j], lg[j + 1], lg[j + 2], lg[j + 3]);
    S.dz[t] = make_float4(dz[0], dz[1], dz[2], dz[3]);
    S.cam[t] = c;
    __syncthreads();
    fetch(base + stride + t);
    for (int u = 0; u < R; ++u) {
      const float dp = S.dpre[u][k1];
      const float4 l = S.lg[u][(j1 >> 2) ^ ((u >> 1) & 3)];
      a1[0] = fmaf(dp, l.x, a1[0]);
      a1[1] = fmaf(dp, l.y, a1[1]);
      a1[2] = fmaf(dp, l.z, a1[2]);
      a1[3] = fmaf(dp, l.w, a1[3]);
    }
    for (int u = q2 * 32; u < q2 * 32 + 32; ++u) {
      const float h = S.hid[u][k2];
      const float4 d = S.dz[u];
      a2[0] = fmaf(d.x, h, a2[0]);
      a2[1] = fmaf(d.y, h, a2[1]);
      a2[2] = fmaf(d.z, h, a2[2]);
      a2[3] = fmaf(d.w, h, a2[3]);
      ab2[0] += d.x;
      ab2[1] += d.y;
      ab2[2] += d.z;
      ab2[3] += d.w;
      const int cu = S.cam[u];  // the same for the whole warp
      if (cu != cam_cur) {
        if (cam_cur >= 0) atomicAdd(&S.sum[cam_cur][k2], cam_acc);
        cam_cur = cu;
        cam_acc = 0.f;
      }
      cam_acc += S.dpre[u][k2];
    }
    __syncthreads();
  }
  if (cam_cur >= 0) atomicAdd(&S.sum[cam_cur][k2], cam_acc);
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (a1[q] != 0.f) atomicAdd(g_params + k1 * kMlpIn + j1 + q, a1[q]);
#pragma unroll
  for (int o = 0; o < kMlpOut; ++o) {
    if (a2[o] != 0.f) atomicAdd(g_params + kMlpW2 + o * kHid + k2, a2[o]);
    if (k2 == 0 && ab2[o] != 0.f) atomicAdd(g_params + kMlpB2 + o, ab2[o]);
  }
  // the chunk arrays are free now: stage the image part of w1 (in hid) and the image
  // embeddings (in dpre) for the per-camera terms
  for (int e = t; e < kHid * kEmbI; e += R) S.hid[e / kEmbI][e % kEmbI] = __ldg(A.mlp + (e / kEmbI) * kMlpIn + kEmbG + e % kEmbI);
  for (int e = t; e < cams.C * kEmbI; e += R) S.dpre[e / kEmbI][e % kEmbI] = __ldg(A.iemb + e);
  __syncthreads();
  // image part of w1 and b1: sums over the cameras of sum[c][k] l_I(c)[j] and sum[c][k]
  for (int e = t; e < kHid * (kEmbI + 1); e += R) {
    const int k = e / (kEmbI + 1), j = e % (kEmbI + 1);
    float a = 0.f;
    if (j < kEmbI) {
      for (int c = 0; c < cams.C; ++c) a = fmaf(S.sum[c][k], S.dpre[c][j], a);
      if (a != 0.f) atomicAdd(g_params + k * kMlpIn + kEmbG + j, a);
    } else {
      for (int c = 0; c < cams.C; ++c) a += S.sum[c][k];
      if (a != 0.f) atomicAdd(g_params + kMlpB1 + k, a);
    }
  }
  // image embeddings: d l_I(c) = w1_I^T sum[c]
  for (int e = t; e < cams.C * kEmbI; e += R) {
    const int c = e / kEmbI, j = e % kEmbI;
    float a = 0.f;
#pragma unroll 8
    for (int k = 0; k < kHid; ++k) a = fmaf(S.hid[k][j], S.sum[c][k], a);
    if (a != 0.f) atomicAdd(g_iemb + e, a);
  }
}

// The transform of Gaussians [0, n) for one image embedding (A.iemb points at its row).
__global__ void __launch_bounds__(256) mlp_cache_kernel(GaussArgs A, long long n, float4* __restrict__ out) {
  __shared__ MlpSmem M;
  mlp_load_smem(A, 1, M);
  __syncthreads();
  for (long long g = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; g < n;
       g += static_cast<long long>(gridDim.x) * blockDim.x) {
    float lg[kEmbG], mo[kMlpOut];
    load_gemb(A, g, lg);
    mlp_eval(M, lg, 0, mo);
    out[g] = make_float4(mo[0], mo[1], mo[2], mo[3]);
  }
}

template <typename AT>
void launch_cull_t(const GaussArgs& g, const CamBatch& cams, float eps, int aa, const PreOut& out, int blocks,
                   cudaStream_t s) {
  preprocess_cull_kernel<AT, 5><<<blocks, kPreThreads, 0, s>>>(g, cams, eps, aa, out);
}

template <typename AT, typename ST>
void launch_bwd_t(const GaussArgs& g, const CamBatch& cams, float eps, int aa, long long V, const Rec* rec,
                  const uint32_t* owner, const Grad2D* g2d, const ParamGrads& out, cudaStream_t s) {
  const int blocks = static_cast<int>((V + kBwdThreads - 1) / kBwdThreads);
  if (blocks > 0)
    preprocess_bwd_kernel<AT, ST><<<blocks, kBwdThreads, 0, s>>>(g, cams, eps, aa, V, rec, owner, g2d, out);
}

}  // namespace

void launch_preprocess_fwd(const GaussArgs& g, const CamBatch& cams, float eps2d, int antialiased,
                           const PreOut& out, int blocks, int rec_blocks, cudaStream_t s) {
  if (blocks <= 0) return;
  if (g.attr_dtype == 0) launch_cull_t<float>(g, cams, eps2d, antialiased, out, blocks, s);
  else if (g.attr_dtype == 1) launch_cull_t<__half>(g, cams, eps2d, antialiased, out, blocks, s);
  else launch_cull_t<__nv_bfloat16>(g, cams, eps2d, antialiased, out, blocks, s);
  preprocess_offsets_kernel<<<1, kOffsetsThreads, 0, s>>>(out.counts, blocks, out.v_total, out.err);
  preprocess_compact_kernel<<<blocks, kPreThreads, 0, s>>>(g.n_render, out.vis, out.counts, out.v_total, out.owner,
                                                           out.rcam);
  launch_preprocess_rec(g, cams, eps2d, antialiased, out, rec_blocks, s);
}

// Zero fill of up to kFillSpans float arrays in one launch: each block writes 16 KB chunks (16-byte
// stores over each array's aligned body, scalar stores for the under-16-byte ends), the chunks
// dealt out to the blocks in turn. With ns_per_chunk > 0 a block starts its k-th chunk no earlier
// than k ns_per_chunk after it started (read on the GPU's nanosecond timer): the fill then runs at
// a set rate beside the kernels of the main stream instead of taking the memory bandwidth from
// them in one burst. Every wait is bounded, so a timer that stalls only speeds the fill up.
constexpr int kFillThreads = 256;
constexpr int kFillChunk = kFillThreads * 4;  // float4 per chunk (16 KB)

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(kFillThreads) zero_fill_kernel(FillSpans f, unsigned ns_per_chunk) {
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  __shared__ unsigned long long s_t0;
  if (threadIdx.x == 0) s_t0 = global_ns();
  __syncthreads();
  unsigned long long k_done = 0;  // chunks this block has written
  for (int k = 0; k < f.count; ++k) {
    float* p = f.ptr[k];
    const size_t n = f.len[k];
    const size_t mis = (reinterpret_cast<uintptr_t>(p) >> 2) & 3u;
    const size_t head = mis ? (4u - mis < n ? 4u - mis : n) : 0u;
    const size_t n4 = (n - head) >> 2;
    float4* body = reinterpret_cast<float4*>(p + head);
    const size_t chunks = (n4 + kFillChunk - 1) / kFillChunk;
    for (size_t c = blockIdx.x; c < chunks; c += gridDim.x, ++k_done) {
      if (ns_per_chunk) {
        if (threadIdx.x == 0) {
          const unsigned long long due = s_t0 + k_done * ns_per_chunk;
          for (int w = 0; w < 100000; ++w) {  // bounded: at most 100000 short sleeps
            const unsigned long long now = global_ns();
            if (now >= due) break;
            __nanosleep(static_cast<unsigned>(min(due - now, 4096ull)));
          }
        }
        __syncthreads();
      }
      const size_t i0 = c * kFillChunk;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const size_t i = i0 + e * kFillThreads + threadIdx.x;
        if (i < n4) body[i] = z;
      }
    }
    if (blockIdx.x == 0) {
      const size_t done = head + 4 * n4;
      if (threadIdx.x < head) p[threadIdx.x] = 0.f;
      if (threadIdx.x < n - done) p[done + threadIdx.x] = 0.f;
    }
  }
}

void launch_zero_fill(const FillSpans& f, int blocks, float gb_per_s, cudaStream_t s) {
  if (f.count <= 0 || blocks <= 0) return;
  // a block's chunk every (chunk bytes x blocks / rate) ns
  const double ns = gb_per_s > 0.f ? (16.0 * kFillChunk) * blocks / gb_per_s : 0.0;
  zero_fill_kernel<<<blocks, kFillThreads, 0, s>>>(f, static_cast<unsigned>(std::min(ns, 1e9)));
}

void launch_mlp_cache(const GaussArgs& A, long long n, float* out, int blocks, cudaStream_t s) {
  if (n <= 0) return;
  const long long need = (n + 255) / 256;
  mlp_cache_kernel<<<static_cast<int>(need < blocks ? need : blocks), 256, 0, s>>>(A, n, reinterpret_cast<float4*>(out));
}

void launch_mlp_bwd(const GaussArgs& g, const CamBatch& cams, long long V, const Rec* rec, const uint32_t* owner,
                    Grad2D* g2d, float* g_gemb, float* g_iemb, float* g_params, int blocks, cudaStream_t s) {
  if (V <= 0 || !g.mlp) return;
  // one bit per device: the attribute is set in each device's context (contexts on several host
  // threads may get here at once; setting it twice is harmless)
  static std::atomic<uint64_t> attr_set{0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 64 || !((attr_set.load(std::memory_order_relaxed) >> dev) & 1u)) {
    if (cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sizeof(MlpBwdSmem))) == cudaSuccess &&
        dev < 64)
      attr_set.fetch_or(1ull << dev, std::memory_order_relaxed);
  }
  const long long need = (V + kBwdThreads - 1) / kBwdThreads;
  const int grid = static_cast<int>(need < blocks ? need : blocks);
  mlp_bwd_kernel<<<grid, kBwdThreads, sizeof(MlpBwdSmem), s>>>(g, cams, V, rec, owner, g2d, g_gemb, g_iemb,
                                                               g_params);
}

void launch_preprocess_bwd(const GaussArgs& g, const CamBatch& cams, float eps2d, int antialiased, long long V,
                           const Rec* rec, const uint32_t* owner, const Grad2D* g2d, const ParamGrads& out,
                           cudaStream_t s) {
#define GSR_PREB(AT, ST) launch_bwd_t<AT, ST>(g, cams, eps2d, antialiased, V, rec, owner, g2d, out, s)
  if (g.attr_dtype == 0 && g.sh_dtype == 0) GSR_PREB(float, float);
  else if (g.attr_dtype == 0 && g.sh_dtype == 1) GSR_PREB(float, __half);
  else if (g.attr_dtype == 0 && g.sh_dtype == 2) GSR_PREB(float, __nv_bfloat16);
  else if (g.attr_dtype == 1 && g.sh_dtype == 1) GSR_PREB(__half, __half);
  else if (g.attr_dtype == 2 && g.sh_dtype == 2) GSR_PREB(__nv_bfloat16, __nv_bfloat16);
  else if (g.attr_dtype == 1 && g.sh_dtype == 0) GSR_PREB(__half, float);
  else if (g.attr_dtype == 2 && g.sh_dtype == 0) GSR_PREB(__nv_bfloat16, float);
  else if (g.attr_dtype == 1 && g.sh_dtype == 2) GSR_PREB(__half, __nv_bfloat16);
  else GSR_PREB(__nv_bfloat16, __half);
#undef GSR_PREB
}

}  // namespace gsr
