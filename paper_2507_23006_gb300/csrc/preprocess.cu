// Per-Gaussian preprocessing (projection, colour, culling) and its backward pass.
//
// Forward (Sec. 3.1: "the 3D Gaussians are first projected onto the image plane"):
//   Sigma = R S S^T R^T (Eq. 1) from the quaternion and scale, then for every camera of the
//   launch t = W mu + t_cam, T = J W with J the perspective Jacobian at the clamped direction,
//   Sigma2D = T Sigma T^T + eps I, the Mip-Splatting opacity compensation (Sec. 3.5.4), the
//   conic Sigma2D^-1, the 3-sigma tile rectangle, and the colour from degree <= 3 spherical
//   harmonics. Culled: z outside (near, far), a zero or non-finite quaternion, det <= 0, an
//   empty rectangle, any non-finite output.
//
// One thread owns one Gaussian and loops over the cameras, so each attribute is read from HBM
// once per launch. Visible (camera, Gaussian) records are written compacted, in (block, thread,
// camera) order, with the block offsets from a single-pass chained scan (Merrill & Garland
// decoupled look-back) whose waits are bounded; within one camera the compacted index grows
// with the Gaussian index, which gives the depth sort its tie-break.
#include <type_traits>

#include "gsr_internal.cuh"
#include "scan_util.cuh"

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
  const float iz = 1.f / tz;
  const float uc = fminf(fmaxf(tx * iz, -c.limx), c.limx);
  const float wc = fminf(fmaxf(ty * iz, -c.limy), c.limy);
  const float smax = fmaxf(G.s[0], fmaxf(G.s[1], G.s[2]));
  const float jf2 = (c.fx * c.fx * (1.f + uc * uc) + c.fy * c.fy * (1.f + wc * wc)) * iz * iz;
  const float rb = 3.f * sqrtf(jf2 * smax * smax + eps + 0.31623f) * 1.01f + 2.f;
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

__device__ __forceinline__ void write_record(const PreOut& out, long long v, const Rec& rr, long long i) {
  const uint32_t lo = __float_as_uint(rr.c.z), hi = __float_as_uint(rr.c.w);
  const uint32_t w = ((lo >> 16) & 0xffffu) - (lo & 0xffffu);
  const uint32_t h = ((hi >> 16) & 0x7ffu) - (hi & 0xffffu);
  out.rec[v] = rr;
  out.depth_keys[v] = __float_as_uint(rr.a.w);
  out.depth_vals[v] = static_cast<uint32_t>(v);
  out.touched[v] = w * h;
  out.owner[v] = static_cast<uint32_t>(i);
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

constexpr int kPreStage = 256;  // records a block keeps in shared memory between its phases

// One block covers kPreTile = 1024 consecutive Gaussians, four per thread (thread t owns slot
// j * 256 + t, i = base + slot, so each load instruction is coalesced).
//   1a: a cheap conservative test per (Gaussian, camera) drops what is certainly outside; the
//       survivors' slots go to a block-wide list.
//   1b: the block's threads share out the list for the exact projection (full warps however
//       sparse the survivors are); the geometry of each visible (Gaussian, camera) record is
//       staged in shared memory.
//   The block's record counts are scanned in slot order and the block total is published for
//   its successors at once. The colour of the staged records is evaluated while the
//   predecessors finish; then one warp takes the block's offset (decoupled look-back) and the
//   staged records are written at their places, so the records are in (i, camera) order.
//   Records beyond the stage's capacity are computed again in full after the offset is known.
// kMlp: with the appearance transform (A.mlp and the embeddings are set).
template <typename AT, typename ST, bool kMlp>
__global__ void __launch_bounds__(kPreThreads, 3) preprocess_fwd_kernel(GaussArgs A, CamBatch cams, float eps, int aa,
                                                                       PreOut out) {
  __shared__ unsigned s_bid;
  __shared__ unsigned long long s_excl;
  __shared__ uint32_t s_count[2];         // survivors of the cheap test; visible records
  __shared__ uint32_t s_list[kPreTile];   // slots of the survivors
  __shared__ uint32_t s_aux[kPreTile];    // 1a: cameras surviving the cheap test; then first record per slot
  __shared__ uint32_t s_mask[kPreTile];   // exact visibility bits per slot
  __shared__ uint32_t s_unstaged[kPreTile / 32];
  __shared__ float4 s_rec[kPreStage][4];
  __shared__ uint32_t s_meta[kPreStage];  // slot | camera << 16
  __shared__ MlpSmem s_mlp;                // appearance transform, when on
  __shared__ uint32_t s_digits[4 * 256];   // digit counts of the block's depth keys
  if (threadIdx.x == 0) {
    s_bid = atomicAdd(out.counter, 1u);
    s_count[0] = 0;
    s_count[1] = 0;
  }
  if (kMlp) mlp_load_smem(A, cams.C, s_mlp);  // read after the barrier that ends phase 1a
  if (threadIdx.x < kPreTile / 32) s_unstaged[threadIdx.x] = 0;
  for (int k = threadIdx.x; k < 4 * 256; k += kPreThreads) s_digits[k] = 0;
  __syncthreads();
  const unsigned bid = s_bid;
  const long long base_i = static_cast<long long>(bid) * kPreTile;
  const int lane = threadIdx.x & 31;
  {
    Geo G[kPreItems];
    bool ok[kPreItems];
#pragma unroll
    for (int j = 0; j < kPreItems; ++j) {  // every load first
      const long long i = base_i + j * kPreThreads + threadIdx.x;
      ok[j] = i < A.n_render;
      if (ok[j]) load_mean_scale<AT>(A, seg_map(A.segs, i), G[j]);
    }
#pragma unroll
    for (int j = 0; j < kPreItems; ++j) {
      const uint32_t slot = j * kPreThreads + threadIdx.x;
      uint32_t maybe = 0;
      if (ok[j])
        for (int c = 0; c < cams.C; ++c)
          if (!surely_culled(G[j], cams.cam[c], eps)) maybe |= 1u << c;
      s_aux[slot] = maybe;
      s_mask[slot] = 0;
      list_append(maybe != 0, slot, s_list, &s_count[0], lane);
    }
  }
  __syncthreads();
  const uint32_t n_maybe = s_count[0];
  for (uint32_t k = threadIdx.x; k < n_maybe; k += kPreThreads) {
    const uint32_t slot = s_list[k];
    const uint32_t maybe = s_aux[slot];
    Geo G;
    uint32_t vis = 0;
    const long long gi = seg_map(A.segs, base_i + slot);
    if (load_geo<AT>(A, gi, G)) {
      for (int c = 0; c < cams.C; ++c) {
        if (!(maybe & (1u << c))) continue;
        Proj P;
        if (!project(G, cams.cam[c], eps, aa, P)) continue;
        vis |= 1u << c;
        const uint32_t e = atomicAdd(&s_count[1], 1u);
        if (e < kPreStage) {
          Rec rr = record_geometry(P, c, eps);
          rr.b.w = rr.c.x = rr.c.y = 1.f;  // colour gains until the colour is evaluated
          // with the appearance transform the opacity (and so the alpha box) is final only
          // after the colour phase: keep the dilated variances the box is made from
          if (kMlp) rr.d = make_float4(P.ar + eps, P.cr + eps, 0.f, 0.f);
          s_rec[e][0] = rr.a;
          s_rec[e][1] = rr.b;
          s_rec[e][2] = rr.c;
          s_rec[e][3] = rr.d;
          s_meta[e] = slot | (static_cast<uint32_t>(c) << 16);
        } else {
          atomicOr(&s_unstaged[slot >> 5], 1u << (slot & 31));
        }
      }
    }
    s_mask[slot] = vis;
  }
  __syncthreads();
  uint32_t mask[kPreItems];
  unsigned long long packed = 0;
#pragma unroll
  for (int j = 0; j < kPreItems; ++j) {
    mask[j] = s_mask[j * kPreThreads + threadIdx.x];
    packed |= static_cast<unsigned long long>(__popc(mask[j])) << (16 * j);
  }
  unsigned long long tot_packed;
  const unsigned long long excl_packed = block_excl_scan64(packed, &tot_packed);
  uint32_t total = 0;
#pragma unroll
  for (int j = 0; j < kPreItems; ++j) {
    s_aux[j * kPreThreads + threadIdx.x] = total + static_cast<uint32_t>((excl_packed >> (16 * j)) & 0xffffu);
    total += static_cast<uint32_t>((tot_packed >> (16 * j)) & 0xffffu);
  }
  if (threadIdx.x == 0) publish_aggregate(out.status, bid, total, out.epoch);
  __syncthreads();
  // colour of the staged records, while the predecessors finish
  const uint32_t n_rec = s_count[1];
  const uint32_t n_staged = n_rec < kPreStage ? n_rec : kPreStage;
  for (uint32_t e = threadIdx.x; e < n_staged; e += kPreThreads) {
    const uint32_t meta = s_meta[e];
    const long long g = seg_map(A.segs, base_i + (meta & 0xffffu));
    Geo G;
    G.m[0] = __ldg(A.means + 3 * g + 0);
    G.m[1] = __ldg(A.means + 3 * g + 1);
    G.m[2] = __ldg(A.means + 3 * g + 2);
    float mo[kMlpOut];
    if (kMlp) {  // before the colour: only the four outputs stay live through it
      float lg[kEmbG];
      load_gemb(A, g, lg);
      mlp_eval(s_mlp, lg, static_cast<int>(meta >> 16), mo);
    }
    float rgb[3], dir[3], dn, Y[16];
    bool cl[3];
    eval_color<ST>(A, g, G, cams.cam[meta >> 16], rgb, dir, dn, Y, cl);
    if (kMlp) {
      const float4 a = s_rec[e][0], d = s_rec[e][3];
      const float op = a.z * (1.f - mo[3]);
      s_rec[e][0].z = op;
      s_rec[e][3] = alpha_box(a.x, a.y, op, d.x, d.y);
      rgb[0] *= 2.f * mo[0];
      rgb[1] *= 2.f * mo[1];
      rgb[2] *= 2.f * mo[2];
    }
    s_rec[e][1].w = rgb[0];
    s_rec[e][2].x = rgb[1];
    s_rec[e][2].y = rgb[2];
  }
  if (threadIdx.x < 32) {
    const unsigned long long ex = warp_lookback(out.status, bid, total, out.epoch, out.err);
    if (threadIdx.x == 0) s_excl = ex;
  }
  __syncthreads();
  const unsigned long long block_base = s_excl;
  if (threadIdx.x == 0 && base_i <= A.n_render - 1 && A.n_render - 1 < base_i + kPreTile)
    *out.v_total = static_cast<uint32_t>(block_base + total);
  for (uint32_t e = threadIdx.x; e < n_staged; e += kPreThreads) {
    const uint32_t meta = s_meta[e];
    const uint32_t slot = meta & 0xffffu, c = meta >> 16;
    // a Gaussian with a record that did not fit the stage has all of its records written below
    if ((s_unstaged[slot >> 5] >> (slot & 31)) & 1u) continue;
    const long long v = block_base + s_aux[slot] + __popc(s_mask[slot] & ((1u << c) - 1u));
    Rec rr;
    rr.a = s_rec[e][0];
    rr.b = s_rec[e][1];
    rr.c = s_rec[e][2];
    rr.d = s_rec[e][3];
    write_record(out, v, rr, base_i + slot);
    count_digits(__float_as_uint(rr.a.w), 0, 32, 4, s_digits);
  }
  if (n_rec <= kPreStage) {  // block-uniform
    __syncthreads();
    flush_digit_counts(s_digits, 4, out.key_counts);
    return;
  }
  // records that did not fit the stage: every record of those Gaussians is computed again
  for (uint32_t k = threadIdx.x; k < n_maybe; k += kPreThreads) {
    const uint32_t slot = s_list[k];
    if (!((s_unstaged[slot >> 5] >> (slot & 31)) & 1u)) continue;
    const uint32_t vis = s_mask[slot];
    const long long i = base_i + slot;
    const long long g = seg_map(A.segs, i);
    Geo G;
    load_geo<AT>(A, g, G);
    long long v = block_base + s_aux[slot];
    for (int c = 0; c < cams.C; ++c) {
      if (!(vis & (1u << c))) continue;
      const DevCam& cam = cams.cam[c];
      Proj P;
      project(G, cam, eps, aa, P);
      float mo[kMlpOut] = {0.5f, 0.5f, 0.5f, 0.f};
      if (kMlp) {
        float lg[kEmbG];
        load_gemb(A, g, lg);
        mlp_eval(s_mlp, lg, c, mo);
        P.op *= 1.f - mo[3];
      }
      float rgb[3], dir[3], dn, Y[16];
      bool cl[3];
      eval_color<ST>(A, g, G, cam, rgb, dir, dn, Y, cl);
      Rec rr = record_geometry(P, c, eps);
      rr.b.w = 2.f * mo[0] * rgb[0];
      rr.c.x = 2.f * mo[1] * rgb[1];
      rr.c.y = 2.f * mo[2] * rgb[2];
      write_record(out, v, rr, i);
      count_digits(__float_as_uint(rr.a.w), 0, 32, 4, s_digits);
      ++v;
    }
  }
  __syncthreads();
  flush_digit_counts(s_digits, 4, out.key_counts);
}

// Backward of the projection and colour. One thread per visible record; the thread holding a
// Gaussian's first record walks all of that Gaussian's cameras (its records are consecutive),
// accumulates the parameter gradients in registers and writes the Gaussian's rows once.
template <typename AT, typename ST>
__global__ void __launch_bounds__(kBwdThreads) preprocess_bwd_kernel(
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

template <typename AT, typename ST>
void launch_fwd_t(const GaussArgs& g, const CamBatch& cams, float eps, int aa, const PreOut& out, int blocks,
                  cudaStream_t s) {
  if (g.mlp)
    preprocess_fwd_kernel<AT, ST, true><<<blocks, kPreThreads, 0, s>>>(g, cams, eps, aa, out);
  else
    preprocess_fwd_kernel<AT, ST, false><<<blocks, kPreThreads, 0, s>>>(g, cams, eps, aa, out);
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
                           const PreOut& out, int blocks, cudaStream_t s) {
  if (blocks <= 0) return;
#define GSR_PRE(AT, ST) launch_fwd_t<AT, ST>(g, cams, eps2d, antialiased, out, blocks, s)
  if (g.attr_dtype == 0 && g.sh_dtype == 0) GSR_PRE(float, float);
  else if (g.attr_dtype == 0 && g.sh_dtype == 1) GSR_PRE(float, __half);
  else if (g.attr_dtype == 0 && g.sh_dtype == 2) GSR_PRE(float, __nv_bfloat16);
  else if (g.attr_dtype == 1 && g.sh_dtype == 1) GSR_PRE(__half, __half);
  else if (g.attr_dtype == 2 && g.sh_dtype == 2) GSR_PRE(__nv_bfloat16, __nv_bfloat16);
  else if (g.attr_dtype == 1 && g.sh_dtype == 0) GSR_PRE(__half, float);
  else if (g.attr_dtype == 2 && g.sh_dtype == 0) GSR_PRE(__nv_bfloat16, float);
  else if (g.attr_dtype == 1 && g.sh_dtype == 2) GSR_PRE(__half, __nv_bfloat16);
  else GSR_PRE(__nv_bfloat16, __half);
#undef GSR_PRE
}

// Zero fill of up to kFillSpans float arrays in one launch: a grid-stride loop of 16-byte
// stores over each array's aligned body, scalar stores for the (under 16-byte) ends.
__global__ void __launch_bounds__(128) zero_fill_kernel(FillSpans f) {
  const size_t tid = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t nthr = static_cast<size_t>(gridDim.x) * blockDim.x;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int k = 0; k < f.count; ++k) {
    float* p = f.ptr[k];
    const size_t n = f.len[k];
    const size_t mis = (reinterpret_cast<uintptr_t>(p) >> 2) & 3u;
    const size_t head = mis ? (4u - mis < n ? 4u - mis : n) : 0u;
    const size_t n4 = (n - head) >> 2;
    float4* body = reinterpret_cast<float4*>(p + head);
    for (size_t i = tid; i < n4; i += nthr) body[i] = z;
    const size_t done = head + 4 * n4;
    if (tid < head) p[tid] = 0.f;
    if (tid < n - done) p[done + tid] = 0.f;
  }
}

void launch_zero_fill(const FillSpans& f, int blocks, cudaStream_t s) {
  if (f.count <= 0 || blocks <= 0) return;
  zero_fill_kernel<<<blocks, 128, 0, s>>>(f);
}

void launch_mlp_bwd(const GaussArgs& g, const CamBatch& cams, long long V, const Rec* rec, const uint32_t* owner,
                    Grad2D* g2d, float* g_gemb, float* g_iemb, float* g_params, int blocks, cudaStream_t s) {
  if (V <= 0 || !g.mlp) return;
  static uint64_t attr_set = 0;  // one bit per device: the attribute is set in each device's context
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 64 || !((attr_set >> dev) & 1u)) {
    cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(sizeof(MlpBwdSmem)));
    if (dev < 64) attr_set |= 1ull << dev;
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
