// Device code shared by the preprocess kernels: spherical harmonics, attribute loads, the
// projection (Sec. 3.1, Eq. 1) and its culls, the record layout, the appearance transform
// (Sec. 3.5.1) and the two forward preprocess kernel templates. Included by the translation units
// that instantiate the forward kernels and by the backward kernels.
#pragma once
#include <type_traits>

#include "gsr_internal.cuh"
#include "scan_util.cuh"
#include "tile_util.cuh"

namespace gsr {
namespace {

// Real spherical-harmonic constants (Condon-Shortley phase), each the normalisation
// sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the Legendre and sqrt(2) factors of its term,
// written as closed forms of pi.
constexpr float kSH0 = 0.28209479177387814f;   // 1 / (2 sqrt(pi))
constexpr float kSH1 = 0.48860251190291992f;   // sqrt(3 / (4 pi))
constexpr float kSH2a = 1.0925484305920792f;   // sqrt(15 / pi) / 2
constexpr float kSH2b = 0.31539156525252005f;  // sqrt(5 / pi) / 4
constexpr float kSH2c = 0.54627421529603959f;  // sqrt(15 / pi) / 4
constexpr float kSH3a = 0.59004358992664352f;  // sqrt(35 / (2 pi)) / 4
constexpr float kSH3b = 2.8906114426405538f;   // sqrt(105 / pi) / 2
constexpr float kSH3c = 0.45704579946446572f;  // sqrt(21 / (2 pi)) / 4
constexpr float kSH3d = 0.37317633259011540f;  // sqrt(7 / pi) / 4
constexpr float kSH3e = 1.4453057213202769f;   // sqrt(105 / pi) / 4

// Basis at a unit direction, as homogeneous polynomials of (x, y, z).
__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y) {
  Y[0] = kSH0;
  if (deg < 1) return;
  Y[1] = -kSH1 * y;
  Y[2] = kSH1 * z;
  Y[3] = -kSH1 * x;
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kSH2a * x * y;
  Y[5] = -kSH2a * y * z;
  Y[6] = kSH2b * (2.f * zz - xx - yy);
  Y[7] = -kSH2a * x * z;
  Y[8] = kSH2c * (xx - yy);
  if (deg < 3) return;
  Y[9] = -kSH3a * y * (3.f * xx - yy);
  Y[10] = kSH3b * x * y * z;
  Y[11] = -kSH3c * y * (4.f * zz - xx - yy);
  Y[12] = kSH3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -kSH3c * x * (4.f * zz - xx - yy);
  Y[14] = kSH3e * z * (xx - yy);
  Y[15] = -kSH3a * x * (xx - 3.f * yy);
}

// Accumulates sum_k w_k grad Y_k into (gx, gy, gz).
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, const float* w, float& gx,
                                              float& gy, float& gz) {
  gx = gy = gz = 0.f;
  if (deg < 1) return;
  gy -= kSH1 * w[1];
  gz += kSH1 * w[2];
  gx -= kSH1 * w[3];
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  gx += kSH2a * y * w[4];
  gy += kSH2a * x * w[4];
  gy -= kSH2a * z * w[5];
  gz -= kSH2a * y * w[5];
  gx -= 2.f * kSH2b * x * w[6];
  gy -= 2.f * kSH2b * y * w[6];
  gz += 4.f * kSH2b * z * w[6];
  gx -= kSH2a * z * w[7];
  gz -= kSH2a * x * w[7];
  gx += 2.f * kSH2c * x * w[8];
  gy -= 2.f * kSH2c * y * w[8];
  if (deg < 3) return;
  gx -= 6.f * kSH3a * x * y * w[9];
  gy -= 3.f * kSH3a * (xx - yy) * w[9];
  gx += kSH3b * y * z * w[10];
  gy += kSH3b * x * z * w[10];
  gz += kSH3b * x * y * w[10];
  gx += 2.f * kSH3c * x * y * w[11];
  gy -= kSH3c * (4.f * zz - xx - 3.f * yy) * w[11];
  gz -= 8.f * kSH3c * y * z * w[11];
  gx -= 6.f * kSH3d * x * z * w[12];
  gy -= 6.f * kSH3d * y * z * w[12];
  gz += kSH3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
  gx -= kSH3c * (4.f * zz - 3.f * xx - yy) * w[13];
  gy += 2.f * kSH3c * x * y * w[13];
  gz -= 8.f * kSH3c * x * z * w[13];
  gx += 2.f * kSH3e * x * z * w[14];
  gy -= 2.f * kSH3e * y * z * w[14];
  gz += kSH3e * (xx - yy) * w[14];
  gx -= 3.f * kSH3a * (xx - yy) * w[15];
  gy += 6.f * kSH3a * x * y * w[15];
}

constexpr int kBwdThreads = 128;

// Starts moving the 32-byte sectors of [p, p + bytes) into L2 without waiting for them (no
// registers are held): a later load of the same bytes then waits for L2 instead of DRAM.
__device__ __forceinline__ void prefetch_l2(const void* p, int bytes) {
  const char* c = static_cast<const char*>(p);
  for (int o = 0; o < bytes; o += 64) asm volatile("prefetch.global.L2 [%0];" ::"l"(c + o));
}

// Camera-independent part of a Gaussian.
struct Geo {
  float m[3];
  float s[3];
  float q[4];     // normalised (w, x, y, z)
  float qinv;     // 1 / |q| of the stored quaternion
  float R[9];
  float S[6];     // Sigma: xx, xy, xz, yy, yz, zz
  float opac;
};

template <typename AT>
__device__ __forceinline__ void load_mean_scale(const GaussArgs& A, long long g, Geo& G) {
  const AT* sc = static_cast<const AT*>(A.scales);
  G.m[0] = __ldg(A.means + 3 * g + 0);
  G.m[1] = __ldg(A.means + 3 * g + 1);
  G.m[2] = __ldg(A.means + 3 * g + 2);
  G.s[0] = ldf(sc, 3 * g + 0);
  G.s[1] = ldf(sc, 3 * g + 1);
  G.s[2] = ldf(sc, 3 * g + 2);
}

// The rest of the Gaussian (quaternion, opacity, Sigma) after load_mean_scale.
template <typename AT>
__device__ __forceinline__ bool finish_geo(const GaussArgs& A, long long g, Geo& G) {
  const AT* qt = static_cast<const AT*>(A.quats);
  const AT* op = static_cast<const AT*>(A.opac);
  float qw, qx, qy, qz;
  if (std::is_same<AT, float>::value && A.quat_vec4) {
    const float4 q4 = __ldg(reinterpret_cast<const float4*>(A.quats) + g);
    qw = q4.x; qx = q4.y; qy = q4.z; qz = q4.w;
  } else {
    qw = ldf(qt, 4 * g + 0); qx = ldf(qt, 4 * g + 1); qy = ldf(qt, 4 * g + 2); qz = ldf(qt, 4 * g + 3);
  }
  G.opac = ldf(op, g);
  const float n2 = qw * qw + qx * qx + qy * qy + qz * qz;
  if (!(n2 > 0.f) || !isfinite(n2)) return false;
  G.qinv = 1.f / sqrtf(n2);
  qw *= G.qinv; qx *= G.qinv; qy *= G.qinv; qz *= G.qinv;
  G.q[0] = qw; G.q[1] = qx; G.q[2] = qy; G.q[3] = qz;
  float* R = G.R;
  R[0] = 1.f - 2.f * (qy * qy + qz * qz); R[1] = 2.f * (qx * qy - qw * qz); R[2] = 2.f * (qx * qz + qw * qy);
  R[3] = 2.f * (qx * qy + qw * qz); R[4] = 1.f - 2.f * (qx * qx + qz * qz); R[5] = 2.f * (qy * qz - qw * qx);
  R[6] = 2.f * (qx * qz - qw * qy); R[7] = 2.f * (qy * qz + qw * qx); R[8] = 1.f - 2.f * (qx * qx + qy * qy);
  float M[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[i * 3 + j] = R[i * 3 + j] * G.s[j];
  G.S[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
  G.S[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
  G.S[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
  G.S[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
  G.S[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
  G.S[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
  return isfinite(G.S[0] + G.S[3] + G.S[5] + G.m[0] + G.m[1] + G.m[2]);
}

template <typename AT>
__device__ __forceinline__ bool load_geo(const GaussArgs& A, long long g, Geo& G) {
  load_mean_scale<AT>(A, g, G);
  return finish_geo<AT>(A, g, G);
}

// Projection of one Gaussian into one camera, with the intermediates the backward needs.
struct Proj {
  float t[3], iz, u, w;
  bool clx, cly;
  float T0[3], T1[3];    // rows of J W
  float ST0[3], ST1[3];  // Sigma T0, Sigma T1
  float ar, br, cr;      // J W Sigma W^T J^T
  float det, idet;
  float comp;            // opacity compensation (1 when not anti-aliased)
  float mx, my, ca, cb, cc, op;
  int r, x0, x1, y0, y1;
};

__device__ __forceinline__ int clamp_tile(float v, int hi) {
  const float f = floorf(v);
  return (f > 0.f) ? static_cast<int>(fminf(f, static_cast<float>(hi))) : 0;
}

__device__ __forceinline__ bool project(const Geo& G, const DevCam& c, float eps, int aa, Proj& P) {
  const float* W = c.R;
  P.t[0] = fmaf(W[0], G.m[0], fmaf(W[1], G.m[1], fmaf(W[2], G.m[2], c.t[0])));
  P.t[1] = fmaf(W[3], G.m[0], fmaf(W[4], G.m[1], fmaf(W[5], G.m[2], c.t[1])));
  P.t[2] = fmaf(W[6], G.m[0], fmaf(W[7], G.m[1], fmaf(W[8], G.m[2], c.t[2])));
  if (!(P.t[2] > c.znear && P.t[2] < c.zfar)) return false;
  P.iz = 1.f / P.t[2];
  P.u = P.t[0] * P.iz;
  P.w = P.t[1] * P.iz;
  const float uc = fminf(fmaxf(P.u, -c.limx), c.limx);
  const float wc = fminf(fmaxf(P.w, -c.limy), c.limy);
  P.clx = (P.u < -c.limx) || (P.u > c.limx);
  P.cly = (P.w < -c.limy) || (P.w > c.limy);
  const float j00 = c.fx * P.iz, j02 = -c.fx * uc * P.iz;
  const float j11 = c.fy * P.iz, j12 = -c.fy * wc * P.iz;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    P.T0[k] = j00 * W[k] + j02 * W[6 + k];
    P.T1[k] = j11 * W[3 + k] + j12 * W[6 + k];
  }
  const float* S = G.S;
  P.ST0[0] = S[0] * P.T0[0] + S[1] * P.T0[1] + S[2] * P.T0[2];
  P.ST0[1] = S[1] * P.T0[0] + S[3] * P.T0[1] + S[4] * P.T0[2];
  P.ST0[2] = S[2] * P.T0[0] + S[4] * P.T0[1] + S[5] * P.T0[2];
  P.ST1[0] = S[0] * P.T1[0] + S[1] * P.T1[1] + S[2] * P.T1[2];
  P.ST1[1] = S[1] * P.T1[0] + S[3] * P.T1[1] + S[4] * P.T1[2];
  P.ST1[2] = S[2] * P.T1[0] + S[4] * P.T1[1] + S[5] * P.T1[2];
  P.ar = P.T0[0] * P.ST0[0] + P.T0[1] * P.ST0[1] + P.T0[2] * P.ST0[2];
  P.br = P.T0[0] * P.ST1[0] + P.T0[1] * P.ST1[1] + P.T0[2] * P.ST1[2];
  P.cr = P.T1[0] * P.ST1[0] + P.T1[1] * P.ST1[1] + P.T1[2] * P.ST1[2];
  const float a = P.ar + eps, b = P.br, cc = P.cr + eps;
  P.det = a * cc - b * b;
  if (!(P.det > 0.f)) return false;
  P.idet = 1.f / P.det;
  P.comp = 1.f;
  if (aa) {
    const float ratio = (P.ar * P.cr - P.br * P.br) * P.idet;
    P.comp = ratio > 0.f ? sqrtf(ratio) : 0.f;
  }
  P.op = G.opac * P.comp;
  P.ca = cc * P.idet;
  P.cb = -b * P.idet;
  P.cc = a * P.idet;
  const float mid = 0.5f * (a + cc);
  const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - P.det));
  P.r = static_cast<int>(ceilf(3.f * sqrtf(lam)));
  P.mx = c.fx * P.t[0] * P.iz + c.cx;
  P.my = c.fy * P.t[1] * P.iz + c.cy;
  const float r = static_cast<float>(P.r);
  P.x0 = clamp_tile((P.mx - r) * (1.f / kTile), c.tiles_x);
  P.x1 = clamp_tile((P.mx + r + (kTile - 1)) * (1.f / kTile), c.tiles_x);
  P.y0 = clamp_tile((P.my - r) * (1.f / kTile), c.tiles_y);
  P.y1 = clamp_tile((P.my + r + (kTile - 1)) * (1.f / kTile), c.tiles_y);
  if ((P.x1 - P.x0) * (P.y1 - P.y0) <= 0) return false;
  return isfinite(P.mx) && isfinite(P.my) && isfinite(P.ca) && isfinite(P.cb) && isfinite(P.cc) &&
         isfinite(P.op);
}

// A cheap test that is true only when project() is certain to cull: depth outside (near, far)
// (the same decision), or a tile rectangle that is empty even for an upper bound of the radius.
// Bound: lambda_max of J W Sigma W^T J^T <= ||J||_F^2 max(scale)^2, the dilation adds eps and
// the max(0.1, .) of the radius rule at most sqrt(0.1); 1% and 2 px of slack cover FP32 rounding.
__device__ __forceinline__ bool surely_culled(const Geo& G, const DevCam& c, float eps) {
  const float* W = c.R;
  const float tz = fmaf(W[6], G.m[0], fmaf(W[7], G.m[1], fmaf(W[8], G.m[2], c.t[2])));
  if (!(tz > c.znear && tz < c.zfar)) return true;
  const float tx = fmaf(W[0], G.m[0], fmaf(W[1], G.m[1], fmaf(W[2], G.m[2], c.t[0])));
  const float ty = fmaf(W[3], G.m[0], fmaf(W[4], G.m[1], fmaf(W[5], G.m[2], c.t[1])));
  // approximate reciprocal and square root (a few ulp): far inside the bound's 1% slack
  const float iz = __fdividef(1.f, tz);
  const float uc = fminf(fmaxf(tx * iz, -c.limx), c.limx);
  const float wc = fminf(fmaxf(ty * iz, -c.limy), c.limy);
  const float smax = fmaxf(G.s[0], fmaxf(G.s[1], G.s[2]));
  const float jf2 = (c.fx * c.fx * (1.f + uc * uc) + c.fy * c.fy * (1.f + wc * wc)) * iz * iz;
  const float r2 = jf2 * smax * smax + eps + 0.31623f;  // > 0
  const float rb = 3.f * (r2 * rsqrtf(r2)) * 1.01f + 2.f;
  const float mx = c.fx * tx * iz + c.cx;
  const float my = c.fy * ty * iz + c.cy;
  return (mx + rb < 1.f) || (mx - rb >= static_cast<float>(kTile * c.tiles_x)) || (my + rb < 1.f) ||
         (my - rb >= static_cast<float>(kTile * c.tiles_y));
}

template <typename ST>
__device__ __forceinline__ void eval_color(const GaussArgs& A, long long g, const Geo& G, const DevCam& c,
                                           float rgb[3], float dir[3], float& dnorm, float Y[16],
                                           bool clamped[3]) {
  const float dx = G.m[0] - c.center[0], dy = G.m[1] - c.center[1], dz = G.m[2] - c.center[2];
  dnorm = sqrtf(dx * dx + dy * dy + dz * dz);
  const float inv = 1.f / dnorm;
  dir[0] = dx * inv; dir[1] = dy * inv; dir[2] = dz * inv;
  sh_basis(A.deg, dir[0], dir[1], dir[2], Y);
  const int nb = (A.deg + 1) * (A.deg + 1);
  const ST* sh = static_cast<const ST*>(A.sh) + g * A.K * 3;
  float v0 = 0.5f, v1 = 0.5f, v2 = 0.5f;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (k < nb) {
      v0 = fmaf(ldf(sh, 3 * k + 0), Y[k], v0);
      v1 = fmaf(ldf(sh, 3 * k + 1), Y[k], v1);
      v2 = fmaf(ldf(sh, 3 * k + 2), Y[k], v2);
    }
  }
  clamped[0] = v0 < 0.f; clamped[1] = v1 < 0.f; clamped[2] = v2 < 0.f;
  rgb[0] = fmaxf(v0, 0.f); rgb[1] = fmaxf(v1, 0.f); rgb[2] = fmaxf(v2, 0.f);
}

// eval_color with the SH row read as twelve 16-byte loads when it is FP32 and 16-byte aligned
// (A.sh_vec4); each channel sums its terms in the same order as eval_color, so the bits agree.
template <typename ST>
__device__ __forceinline__ void eval_color_vec(const GaussArgs& A, long long g, const Geo& G, const DevCam& c,
                                               float rgb[3], float dir[3], float& dnorm, float Y[16],
                                               bool clamped[3]) {
  if (!(std::is_same<ST, float>::value && A.sh_vec4)) {
    eval_color<ST>(A, g, G, c, rgb, dir, dnorm, Y, clamped);
    return;
  }
  const float dx = G.m[0] - c.center[0], dy = G.m[1] - c.center[1], dz = G.m[2] - c.center[2];
  dnorm = sqrtf(dx * dx + dy * dy + dz * dz);
  const float inv = 1.f / dnorm;
  dir[0] = dx * inv; dir[1] = dy * inv; dir[2] = dz * inv;
  sh_basis(A.deg, dir[0], dir[1], dir[2], Y);
  const int n3 = (A.deg + 1) * (A.deg + 1) * 3;
  const float4* row = reinterpret_cast<const float4*>(static_cast<const float*>(A.sh) + g * A.K * 3);
  float v[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
  for (int q = 0; q < 12; ++q) {
    if (4 * q < n3) {
      const float4 w = __ldg(row + q);
      const float e[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int el = 4 * q + r;  // coefficient el / 3, channel el % 3
        if (el < n3) v[el % 3] = fmaf(e[r], Y[el / 3], v[el % 3]);
      }
    }
  }
  clamped[0] = v[0] < 0.f; clamped[1] = v[1] < 0.f; clamped[2] = v[2] < 0.f;
  rgb[0] = fmaxf(v[0], 0.f); rgb[1] = fmaxf(v[1], 0.f); rgb[2] = fmaxf(v[2], 0.f);
}

// The Gaussian's SH coefficients of degree <= deg, in registers (zero beyond them).
template <typename ST>
__device__ __forceinline__ void load_sh_row(const GaussArgs& A, long long g, float shv[48]) {
  const int n3 = (A.deg + 1) * (A.deg + 1) * 3;
  const ST* sh = static_cast<const ST*>(A.sh) + g * A.K * 3;
  if (std::is_same<ST, float>::value && A.sh_vec4) {
    const float4* row = reinterpret_cast<const float4*>(sh);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float4 v = 4 * k < n3 ? __ldg(row + k) : make_float4(0.f, 0.f, 0.f, 0.f);
      shv[4 * k] = v.x; shv[4 * k + 1] = v.y; shv[4 * k + 2] = v.z; shv[4 * k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 48; ++k) shv[k] = k < n3 ? ldf(sh, k) : 0.f;
  }
#pragma unroll
  for (int k = 0; k < 48; ++k)
    if (k >= n3) shv[k] = 0.f;
}

// eval_color with the coefficients already in registers.
__device__ __forceinline__ void eval_color_regs(int deg, const Geo& G, const DevCam& c, const float shv[48],
                                                float rgb[3], float dir[3], float& dnorm, float Y[16],
                                                bool clamped[3]) {
  const float dx = G.m[0] - c.center[0], dy = G.m[1] - c.center[1], dz = G.m[2] - c.center[2];
  dnorm = sqrtf(dx * dx + dy * dy + dz * dz);
  const float inv = 1.f / dnorm;
  dir[0] = dx * inv; dir[1] = dy * inv; dir[2] = dz * inv;
#pragma unroll
  for (int k = 0; k < 16; ++k) Y[k] = 0.f;
  sh_basis(deg, dir[0], dir[1], dir[2], Y);
  float v0 = 0.5f, v1 = 0.5f, v2 = 0.5f;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    v0 = fmaf(shv[3 * k + 0], Y[k], v0);
    v1 = fmaf(shv[3 * k + 1], Y[k], v1);
    v2 = fmaf(shv[3 * k + 2], Y[k], v2);
  }
  clamped[0] = v0 < 0.f; clamped[1] = v1 < 0.f; clamped[2] = v2 < 0.f;
  rgb[0] = fmaxf(v0, 0.f); rgb[1] = fmaxf(v1, 0.f); rgb[2] = fmaxf(v2, 0.f);
}

// The 64-byte record of a visible (Gaussian, camera c) projection, colour left at zero.
// Where op' exp(-d^T Q d / 2) >= 1/255, i.e. d^T Q d <= 2 ln(255 op'): an ellipse whose
// half-extents are sqrt(2 ln(255 op') Sigma_xx) and sqrt(2 ln(255 op') Sigma_yy), Sigma the
// dilated covariance (sxx, syy its diagonal). Widened by 0.1% + 0.01 px so FP32 evaluation never
// falls outside.
__device__ __forceinline__ float4 alpha_box(float mx, float my, float op, float sxx, float syy) {
  const float L = logf(255.f * op);
  if (!(L > 0.f)) return make_float4(1.f, -1.f, 1.f, -1.f);  // empty: no pixel reaches 1/255
  const float ex = sqrtf(2.f * L * sxx) * 1.001f + 0.01f;
  const float ey = sqrtf(2.f * L * syy) * 1.001f + 0.01f;
  return make_float4(mx - ex, mx + ex, my - ey, my + ey);
}

__device__ __forceinline__ Rec record_geometry(const Proj& P, int c, float eps) {
  Rec rr;
  rr.a = make_float4(P.mx, P.my, P.op, P.t[2]);
  rr.b = make_float4(P.ca, P.cb, P.cc, 0.f);
  const uint32_t lo = static_cast<uint32_t>(P.x0) | (static_cast<uint32_t>(P.x1) << 16);
  const uint32_t hi = static_cast<uint32_t>(P.y0) | (static_cast<uint32_t>(P.y1) << 16) | (static_cast<uint32_t>(c) << 27);
  rr.c = make_float4(0.f, 0.f, __uint_as_float(lo), __uint_as_float(hi));
  rr.d = alpha_box(P.mx, P.my, P.op, P.ar + eps, P.cr + eps);
  return rr;
}

// The record (its owner was written by the cull pass) and the global-sort inputs.
__device__ __forceinline__ void write_record(const PreOut& out, long long v, const Rec& rr) {
  out.rec[v] = rr;
  if (out.depth_keys) {  // the global-sort binning's inputs
    const uint32_t lo = __float_as_uint(rr.c.z), hi = __float_as_uint(rr.c.w);
    out.depth_keys[v] = __float_as_uint(rr.a.w);
    out.depth_vals[v] = static_cast<uint32_t>(v);
    out.touched[v] = (((lo >> 16) & 0xffffu) - (lo & 0xffffu)) * (((hi >> 16) & 0x7ffu) - (hi & 0xffffu));
  }
}

// Appearance transform (Sec. 3.5.1) weights in shared memory: the Gaussian-embedding part of w1,
// w2 and b2, and per camera of the launch u_c = w1[:, 16:48] l_I(c) + b1 (the image part of the
// hidden layer is the same for every Gaussian seen by that camera).
struct MlpSmem {
  float w1g[kHid][kEmbG];
  float w2[kMlpOut][kHid];
  float b2[kMlpOut];
  float u[kMaxCams][kHid];
};

// Fills M from the packed parameters and image embeddings (whole block; the caller syncs).
__device__ void mlp_load_smem(const GaussArgs& A, int C, MlpSmem& M) {
  for (int e = threadIdx.x; e < kHid * kEmbG; e += blockDim.x)
    M.w1g[e / kEmbG][e % kEmbG] = __ldg(A.mlp + (e / kEmbG) * kMlpIn + e % kEmbG);
  for (int e = threadIdx.x; e < kMlpOut * kHid; e += blockDim.x) M.w2[e / kHid][e % kHid] = __ldg(A.mlp + kMlpW2 + e);
  for (int e = threadIdx.x; e < kMlpOut; e += blockDim.x) M.b2[e] = __ldg(A.mlp + kMlpB2 + e);
  // u: four threads per (camera, hidden unit), eight terms each with every load issued at once,
  // summed over the four lanes (C * kHid * 4 is a multiple of 32: whole warps take part)
  for (int e = threadIdx.x; e < C * kHid * 4; e += blockDim.x) {
    const int c = e / (kHid * 4), k = (e >> 2) % kHid, q = e & 3;
    const float* w = A.mlp + k * kMlpIn + kEmbG + q * 8;
    const float* l = A.iemb + c * kEmbI + q * 8;
    float a = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) a = fmaf(__ldg(w + j), __ldg(l + j), a);
    a += __shfl_xor_sync(0xffffffffu, a, 1);
    a += __shfl_xor_sync(0xffffffffu, a, 2);
    if (q == 0) M.u[c][k] = a + __ldg(A.mlp + kMlpB1 + k);
  }
}

__device__ __forceinline__ void load_gemb(const GaussArgs& A, long long g, float lg[kEmbG]) {
#pragma unroll
  for (int j = 0; j < kEmbG; ++j) lg[j] = __ldg(A.gemb + g * kEmbG + j);
}

// Pre-activation of hidden unit k, in two chains of eight terms; the forward and the backward's
// recomputation share it, so both see the same bits.
__device__ __forceinline__ float mlp_pre(const MlpSmem& M, const float lg[kEmbG], int c, int k) {
  float a = M.u[c][k], a2 = 0.f;
#pragma unroll
  for (int j = 0; j < kEmbG; j += 2) {
    a = fmaf(M.w1g[k][j], lg[j], a);
    a2 = fmaf(M.w1g[k][j + 1], lg[j + 1], a2);
  }
  return a + a2;
}

// Partial output pre-activations over the hidden units of quarter q (8q .. 8q+7, in order).
// f(k, a, h) sees each unit's pre-activation a and output h.
template <typename F>
__device__ __forceinline__ void mlp_zpart(const MlpSmem& M, const float lg[kEmbG], int c, int q, float zq[kMlpOut],
                                          F&& f) {
#pragma unroll
  for (int o = 0; o < kMlpOut; ++o) zq[o] = 0.f;
#pragma unroll 2
  for (int k = 8 * q; k < 8 * q + 8; ++k) {
    const float a = mlp_pre(M, lg, c, k);
    const float h = fmaxf(a, 0.f);
    f(k, a, h);
#pragma unroll
    for (int o = 0; o < kMlpOut; ++o) zq[o] = fmaf(M.w2[o][k], h, zq[o]);
  }
}

// The transform's outputs from the four quarters' partial sums: out = sigmoid(b2 + ((z0 + z1) +
// (z2 + z3))). Every evaluation (one thread, four cooperating lanes, the backward's
// recomputation) sums in this order, so all of them see the same bits.
__device__ __forceinline__ void mlp_out(const MlpSmem& M, const float z01[kMlpOut], const float z23[kMlpOut],
                                        float out[kMlpOut]) {
#pragma unroll
  for (int o = 0; o < kMlpOut; ++o) out[o] = 1.f / (1.f + __expf(-(M.b2[o] + (z01[o] + z23[o]))));
}

// The transform's outputs for a Gaussian embedding seen by camera c: out = sigmoid(w2 ReLU(u_c +
// w1_G l_G) + b2); 2 out[0..2] is the colour gain, 1 - out[3] the opacity factor. f as in mlp_zpart.
template <typename F>
__device__ __forceinline__ void mlp_eval_f(const MlpSmem& M, const float lg[kEmbG], int c, float out[kMlpOut], F&& f) {
  float z01[kMlpOut], z23[kMlpOut], zq[kMlpOut];
  mlp_zpart(M, lg, c, 0, z01, f);
  mlp_zpart(M, lg, c, 1, zq, f);
#pragma unroll
  for (int o = 0; o < kMlpOut; ++o) z01[o] += zq[o];
  mlp_zpart(M, lg, c, 2, z23, f);
  mlp_zpart(M, lg, c, 3, zq, f);
#pragma unroll
  for (int o = 0; o < kMlpOut; ++o) z23[o] += zq[o];
  mlp_out(M, z01, z23, out);
}

__device__ __forceinline__ void mlp_eval(const MlpSmem& M, const float lg[kEmbG], int c, float out[kMlpOut]) {
  mlp_eval_f(M, lg, c, out, [](int, float, float) {});
}

// The transform's outputs for Gaussian g seen by camera c: the launch's cached outputs (one image
// embedding for every camera) when it has them, else evaluated.
__device__ __forceinline__ void mlp_outputs(const GaussArgs& A, const MlpSmem& M, long long g, int c,
                                            float out[kMlpOut]) {
  if (A.mlp_cached) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(A.mlp_cached) + g);
    out[0] = v.x;
    out[1] = v.y;
    out[2] = v.z;
    out[3] = v.w;
    return;
  }
  float lg[kEmbG];
  load_gemb(A, g, lg);
  mlp_eval(M, lg, c, out);
}

// Appends the slots of the lanes with `pred` to the block's list (order within the list is
// arbitrary); one shared atomic per warp.
__device__ __forceinline__ void list_append(bool pred, uint32_t slot, uint32_t* list, uint32_t* count, int lane) {
  const uint32_t bal = __ballot_sync(0xffffffffu, pred);
  if (!bal) return;
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(count, static_cast<uint32_t>(__popc(bal)));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (pred) list[base + __popc(bal & ((1u << lane) - 1u))] = slot;
}

// The forward preprocess runs as four kernels, none of which waits on another block.
//
// preprocess_cull_kernel: block b covers kPreTile = 1024 consecutive Gaussians, four per thread
// (thread t owns slot j * 256 + t, i = b * 1024 + slot, so each load instruction is coalesced).
//   1a: a cheap conservative test per (Gaussian, camera) on the means and scales drops what is
//       certainly outside; the survivors' slots go to a block-wide list.
//   1b: the block's threads share out the list for the exact projection test (full warps however
//       sparse the survivors are), which decides visibility per camera.
//   Each Gaussian's camera bits go to vis[i], the block's record count to counts[b].
// preprocess_offsets_kernel (one block): counts[] becomes each block's first record index, the
//   total is V.
// preprocess_compact_kernel: block b scans its Gaussians' record counts in slot order and writes
//   the (Gaussian, camera) of each of its records at the record's index, so the records are in
//   (i, camera) order.
// preprocess_rec_kernel: one thread per visible record (grid-stride) loads its Gaussian again,
//   repeats the projection (the same computation, so the same bits), evaluates the colour (and
//   the appearance transform) and writes the 64-byte record. Every thread of this pass has a
//   record to make, so its scattered loads of the attribute and SH rows overlap across the
//   whole GPU. With out.tile_ctr set it also counts the records' (tile, record) pairs per tile
//   for the per-tile binning (warp_bin_pairs).
template <typename AT, int kMinBlocks>
__global__ void __launch_bounds__(kPreThreads, kMinBlocks) preprocess_cull_kernel(GaussArgs A, CamBatch cams,
                                                                                  float eps, int aa, PreOut out) {
  __shared__ uint32_t s_count;
  __shared__ uint32_t s_list[kPreTile];  // slots of the survivors of the cheap test
  __shared__ uint32_t s_aux[kPreTile];   // cameras surviving the cheap test
  __shared__ uint32_t s_mask[kPreTile];  // exact visibility bits per slot
  __shared__ uint32_t s_warp[kPreThreads / 32];
  if (threadIdx.x == 0) s_count = 0;
  __syncthreads();
  const long long base_i = static_cast<long long>(blockIdx.x) * kPreTile;
  const int lane = threadIdx.x & 31;
  {
    Geo G[kPreItems];
    bool ok[kPreItems];
    uint32_t seg_cams[kPreItems];  // cameras that render the Gaussian's segment
#pragma unroll
    for (int j = 0; j < kPreItems; ++j) {  // every load first
      const long long i = base_i + j * kPreThreads + threadIdx.x;
      ok[j] = i < A.n_render;
      seg_cams[j] = 0;
      if (ok[j]) load_mean_scale<AT>(A, seg_map_cams(A.segs, i, &seg_cams[j]), G[j]);
    }
#pragma unroll
    for (int j = 0; j < kPreItems; ++j) {
      const uint32_t slot = j * kPreThreads + threadIdx.x;
      uint32_t maybe = 0;
      if (ok[j])
        for (int c = 0; c < cams.C; ++c)
          if (((seg_cams[j] >> c) & 1u) && !surely_culled(G[j], cams.cam[c], eps)) maybe |= 1u << c;
      s_aux[slot] = maybe;
      s_mask[slot] = 0;
      if (maybe) {  // the exact test below reads the quaternion and opacity
        const long long g = seg_map(A.segs, base_i + slot);
        prefetch_l2(static_cast<const AT*>(A.quats) + 4 * g, 4 * sizeof(AT));
        prefetch_l2(static_cast<const AT*>(A.opac) + g, sizeof(AT));
      }
      list_append(maybe != 0, slot, s_list, &s_count, lane);
    }
  }
  __syncthreads();
  const uint32_t n_maybe = s_count;
  for (uint32_t k = threadIdx.x; k < n_maybe; k += kPreThreads) {
    const uint32_t slot = s_list[k];
    const uint32_t maybe = s_aux[slot];
    Geo G;
    uint32_t vis = 0;
    if (load_geo<AT>(A, seg_map(A.segs, base_i + slot), G)) {
      for (int c = 0; c < cams.C; ++c) {
        if (!(maybe & (1u << c))) continue;
        Proj P;
        if (project(G, cams.cam[c], eps, aa, P)) vis |= 1u << c;
      }
    }
    s_mask[slot] = vis;
  }
  __syncthreads();
  uint32_t n = 0;
#pragma unroll
  for (int j = 0; j < kPreItems; ++j) {
    const long long i = base_i + j * kPreThreads + threadIdx.x;
    const uint32_t m = s_mask[j * kPreThreads + threadIdx.x];
    if (i < A.n_render) out.vis[i] = m;
    n += __popc(m);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if (lane == 0) s_warp[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int w = 0; w < kPreThreads / 32; ++w) tot += s_warp[w];
    out.counts[blockIdx.x] = tot;
  }
}

// One block of kOffsetsThreads: counts[0, nb) become exclusive prefix sums (each cull block's
// first record), *v_total = V. A record index past 2^32 sets kErrOverflow.
constexpr int kOffsetsThreads = 1024;
__global__ void __launch_bounds__(kOffsetsThreads) preprocess_offsets_kernel(uint32_t* __restrict__ counts, int nb,
                                                                             uint32_t* v_total, int* err) {
  const int per = (nb + kOffsetsThreads - 1) / kOffsetsThreads;
  const int first = threadIdx.x * per;
  unsigned long long sum = 0;
#pragma unroll 4
  for (int k = first; k < min(first + per, nb); ++k) sum += counts[k];
  unsigned long long tot;
  unsigned long long run = block_excl_scan64(sum, &tot);
  for (int k = first; k < min(first + per, nb); ++k) {
    const uint32_t c = counts[k];
    counts[k] = static_cast<uint32_t>(run);
    run += c;
  }
  if (threadIdx.x == 0) {
    if (tot > 0xffffffffull) atomicOr(err, kErrOverflow);
    *v_total = static_cast<uint32_t>(tot);
  }
}

// Block b: the records of its Gaussians, numbered in (i, camera) order from offsets[b]; a block
// with none (offsets[b] equal to the next block's first record, or to V) reads nothing more.
__global__ void __launch_bounds__(kPreThreads) preprocess_compact_kernel(long long n_render,
                                                                         const uint32_t* __restrict__ vis,
                                                                         const uint32_t* __restrict__ offsets,
                                                                         const uint32_t* __restrict__ v_total,
                                                                         uint32_t* __restrict__ owner,
                                                                         uint8_t* __restrict__ rcam) {
  const uint32_t next = blockIdx.x + 1 < gridDim.x ? offsets[blockIdx.x + 1] : *v_total;
  if (next == offsets[blockIdx.x]) return;  // block-uniform
  const long long base_i = static_cast<long long>(blockIdx.x) * kPreTile;
  uint32_t mask[kPreItems];
  unsigned long long packed = 0;
#pragma unroll
  for (int j = 0; j < kPreItems; ++j) {
    const long long i = base_i + j * kPreThreads + threadIdx.x;
    mask[j] = i < n_render ? vis[i] : 0u;
    packed |= static_cast<unsigned long long>(__popc(mask[j])) << (16 * j);
  }
  unsigned long long tot_packed;
  const unsigned long long excl_packed = block_excl_scan64(packed, &tot_packed);
  long long v = offsets[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kPreItems; ++j) {
    long long r = v + static_cast<long long>((excl_packed >> (16 * j)) & 0xffffu);
    uint32_t m = mask[j];
    const uint32_t i = static_cast<uint32_t>(base_i + j * kPreThreads + threadIdx.x);
    while (m) {
      const int c = __ffs(m) - 1;
      m &= m - 1u;
      owner[r] = i;
      rcam[r] = static_cast<uint8_t>(c);
      ++r;
    }
    v += static_cast<long long>((tot_packed >> (16 * j)) & 0xffffu);
  }
}

template <typename AT, typename ST, bool kMlp>
__global__ void __launch_bounds__(kPreThreads, 3) preprocess_rec_kernel(GaussArgs A, CamBatch cams, float eps, int aa,
                                                                     PreOut out) {
  __shared__ MlpSmem s_mlp;                // appearance transform, when on
  __shared__ uint32_t s_digits[4 * 256];   // digit counts of the block's depth keys (global sort)
  if (kMlp && !A.mlp_cached) mlp_load_smem(A, cams.C, s_mlp);
  if (out.key_counts)
    for (int k = threadIdx.x; k < 4 * 256; k += kPreThreads) s_digits[k] = 0;
  if (kMlp || out.key_counts) __syncthreads();
  const long long V = static_cast<long long>(*out.v_total);
  const int lane = threadIdx.x & 31;
  const long long stride = static_cast<long long>(gridDim.x) * kPreThreads;
  // warps stride over the records 32 at a time, so the pair count below has whole warps
  for (long long base = static_cast<long long>(blockIdx.x) * kPreThreads + (threadIdx.x & ~31); base < V;
       base += stride) {
    const long long v = base + lane;
    const bool has = v < V;
    Rec rr{};
    if (has) {
      const uint32_t i = out.owner[v];
      const int c = out.rcam[v];
      const long long g = seg_map(A.segs, i);
      const DevCam& cam = cams.cam[c];
      Geo G;
      load_geo<AT>(A, g, G);
      Proj P;
      project(G, cam, eps, aa, P);  // visible: the cull pass made the same decision
      float mo[kMlpOut] = {0.5f, 0.5f, 0.5f, 0.f};
      if (kMlp) {
        mlp_outputs(A, s_mlp, g, c, mo);
        P.op *= 1.f - mo[3];
      }
      float rgb[3], dir[3], dn, Y[16];
      bool cl[3];
      eval_color_vec<ST>(A, g, G, cam, rgb, dir, dn, Y, cl);
      rr = record_geometry(P, c, eps);
      rr.b.w = 2.f * mo[0] * rgb[0];
      rr.c.x = 2.f * mo[1] * rgb[1];
      rr.c.y = 2.f * mo[2] * rgb[2];
      write_record(out, v, rr);
      if (out.key_counts) count_digits(__float_as_uint(rr.a.w), 0, 32, 4, s_digits);
    }
    if (out.tile_ctr) {  // the per-tile binning's counting pass, on the records just made
      if (out.tile_cull)
        warp_bin_pairs<true, false>(lane, has, rr, static_cast<uint32_t>(base), cams, out.tile_ctr, nullptr, nullptr,
                                    out.err);
      else
        warp_bin_pairs<false, false>(lane, has, rr, static_cast<uint32_t>(base), cams, out.tile_ctr, nullptr, nullptr,
                                     out.err);
    }
  }
  if (out.key_counts) {
    __syncthreads();
    flush_digit_counts(s_digits, 4, out.key_counts);
  }
}

}  // namespace
}  // namespace gsr
