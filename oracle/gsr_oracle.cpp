// FP64 CPU oracle for the differentiable tile-based Gaussian rasterizer.
//
// TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or calls this file;
// only the tests, the package smoke check and the benchmark's CPU-baseline leg do. It shares
// no code, header, table or constant generator with the CUDA implementation.
//
// What it computes, in plain double precision and in the paper's order:
//   * Sec. 3.1, Eq. 1: each Gaussian has mean mu, covariance Sigma = R S S^T R^T (R from a
//     unit quaternion, S = diag(scale)), colour c and opacity o.
//   * Sec. 3.1 (projection onto the image plane): EWA projection Sigma2D = J W Sigma W^T J^T,
//     plus the 2D low-pass dilation; with anti-aliasing on (Sec. 3.5.4, Mip-Splatting 2D
//     filter) the opacity is scaled by sqrt(det(Sigma2D) / det(Sigma2D + eps I)).
//   * Colour from real spherical harmonics of degree <= 3, built here from the definition
//     (associated Legendre functions via Bonnet's recurrence and Re/Im of (x + i y)^m).
//   * Sec. 3.5.1 (optional): the per-Gaussian appearance transform, an MLP of the Gaussian's
//     and the image's embeddings that scales each Gaussian's colour and opacity (section
//     "Appearance transform" below).
//   * Tile binning: a Gaussian lands in every 16x16 tile of its 3-sigma rectangle; with
//     tile culling on (Sec. 3.4.2, StopThePop) a tile is dropped when the largest opacity the
//     Gaussian can reach at any pixel centre of that tile is below 1/255.
//   * Sec. 3.1, Eq. 2: front-to-back alpha blending of each pixel over its tile's list sorted
//     by depth, accumulating RGB, depth (Sec. 3.5.3 depth regulariser) and opacity.
//   * Gradients: exact reverse mode through the blending recurrence (re-walking each pixel
//     forward and keeping the prefix transmittances) and forward-mode dual numbers through
//     the projection and colour evaluation, so no chain rule of the projection is hand-written.
//   * Sec. 3.4.2: partition-level detail-level selection by camera distance, with invisible
//     partitions culled, and a Gaussian budget.
//
// Conventions the paper leaves open, and the reading taken for each:
//   alpha = min(0.99, o' G'); a Gaussian is skipped where alpha < 1/255; a pixel stops before
//   adding the Gaussian that would take its transmittance below 1e-4; pixel (x, y) samples
//   (x + 0.5, y + 0.5); eps = 0.3 px^2; the Jacobian uses x/z and y/z clamped to +-1.3 of the
//   half field of view; 3-sigma radius r = ceil(3 sqrt(lambda_max)) with
//   lambda_max = m + sqrt(max(0.1, m^2 - det)); depth = view-space z; ties in z go to the
//   lower Gaussian index; rgb = max(0, SH + 0.5); per-image appearance c' = A c + b; bg added
//   with the final transmittance.
//
// Every discrete decision that an FP32 implementation could take differently (a threshold
// within FP32 reach) is reported as a "knife-edge" mark so that tests compare only what both
// precisions must agree on.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int kTile = 16;
constexpr double kAlphaMax = 0.99;
constexpr double kAlphaMin = 1.0 / 255.0;
constexpr double kTMin = 1e-4;
constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------------------------
// Forward-mode dual numbers (value + N partial derivatives).
template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0.0; }  // NOLINT: implicit
  static Dual var(double x, int i) { Dual r(x); r.d[i] = 1.0; return r; }
};
template <int N> Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v + b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int N> Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v - b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int N> Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r; r.v = -a.v; for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r; }
template <int N> Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v * b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int N> Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v / b.v;
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r; }
template <int N> Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> Dual<N> operator*(const Dual<N>& a, double b) { return a * Dual<N>(b); }
template <int N> Dual<N> operator*(double a, const Dual<N>& b) { return Dual<N>(a) * b; }
template <int N> Dual<N> operator/(const Dual<N>& a, double b) { return a / Dual<N>(b); }
template <int N> Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> Dual<N> dsqrt(const Dual<N>& a) {
  Dual<N> r; r.v = std::sqrt(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / (2.0 * r.v);
  return r; }
inline double dsqrt(double a) { return std::sqrt(a); }
inline double val(double x) { return x; }
template <int N> double val(const Dual<N>& x) { return x.v; }

// Forward-mode magnitudes: a value and N nonnegative partials, where every operation adds up the
// absolute values of the elementary terms of its derivative (|d(ab)| <= |b| |da| + |a| |db|, and so
// on). Each partial so obtained is the sum of the magnitudes of all the products the chain rule adds
// up for it: it bounds the exact partial, and the rounding error of any evaluation of the partial
// in finite precision, in any order, scales with it rather than with the (possibly cancelling)
// exact value.
template <int N>
struct Mag {
  double v;
  double d[N];
  Mag() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
  Mag(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0.0; }  // NOLINT: implicit
  static Mag var(double x, int i) { Mag r(x); r.d[i] = 1.0; return r; }
};
template <int N> Mag<N> operator+(const Mag<N>& a, const Mag<N>& b) {
  Mag<N> r; r.v = a.v + b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int N> Mag<N> operator-(const Mag<N>& a, const Mag<N>& b) {
  Mag<N> r; r.v = a.v - b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int N> Mag<N> operator-(const Mag<N>& a) {
  Mag<N> r; r.v = -a.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i]; return r; }
template <int N> Mag<N> operator*(const Mag<N>& a, const Mag<N>& b) {
  Mag<N> r; r.v = a.v * b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * std::fabs(b.v) + std::fabs(a.v) * b.d[i];
  return r; }
template <int N> Mag<N> operator/(const Mag<N>& a, const Mag<N>& b) {
  Mag<N> r; r.v = a.v / b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / std::fabs(b.v) + std::fabs(a.v) * b.d[i] / (b.v * b.v);
  return r; }
template <int N> Mag<N> operator+(const Mag<N>& a, double b) { return a + Mag<N>(b); }
template <int N> Mag<N> operator+(double a, const Mag<N>& b) { return Mag<N>(a) + b; }
template <int N> Mag<N> operator-(const Mag<N>& a, double b) { return a - Mag<N>(b); }
template <int N> Mag<N> operator-(double a, const Mag<N>& b) { return Mag<N>(a) - b; }
template <int N> Mag<N> operator*(const Mag<N>& a, double b) { return a * Mag<N>(b); }
template <int N> Mag<N> operator*(double a, const Mag<N>& b) { return Mag<N>(a) * b; }
template <int N> Mag<N> operator/(const Mag<N>& a, double b) { return a / Mag<N>(b); }
template <int N> Mag<N> operator/(double a, const Mag<N>& b) { return Mag<N>(a) / b; }
template <int N> Mag<N> dsqrt(const Mag<N>& a) {
  Mag<N> r; r.v = std::sqrt(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / (2.0 * r.v);
  return r; }
template <int N> double val(const Mag<N>& x) { return x.v; }

// ---------------------------------------------------------------------------------------------
struct CamD {
  double R[9], t[3];
  double fx, fy, cx, cy;
  int W, H;
  double znear, zfar;
  int tiles_x, tiles_y;
  bool has_aff;
  double A[12];  // [A | b] row-major 3x4
  double center[3];
  const double* iemb = nullptr;  // image embedding [32] of the appearance transform, or NULL
};

// ---------------------------------------------------------------------------------------------
// Appearance transform (Sec. 3.5.1): a per-Gaussian embedding l_G (16) and a per-image embedding
// l_I (32) go through one hidden layer of 32 with ReLU and an output layer of 4 with a sigmoid
// (the sizes of the paper's supplementary notes). Reading of how the outputs adjust the Gaussian
// (the paper says only that they adjust colour and opacity, and pulls the opacity output toward
// zero): colour gain 2 out[0..2] on the SH colour (identity at 1/2) and opacity factor
// 1 - out[3] (identity at 0). params = w1 [32][48] | b1 [32] | w2 [4][32] | b2 [4].
constexpr int kEmbG = 16, kEmbI = 32, kHid = 32, kMlpOut = 4;
constexpr int kMlpIn = kEmbG + kEmbI;
constexpr int kMlpParams = kHid * kMlpIn + kHid + kMlpOut * kHid + kMlpOut;

void mlp_forward(const double* params, const double* lg, const double* li, double pre[kHid], double hid[kHid],
                 double out[kMlpOut]) {
  const double* w1 = params;
  const double* b1 = w1 + kHid * kMlpIn;
  const double* w2 = b1 + kHid;
  const double* b2 = w2 + kMlpOut * kHid;
  for (int k = 0; k < kHid; ++k) {
    double a = b1[k];
    for (int j = 0; j < kEmbG; ++j) a += w1[k * kMlpIn + j] * lg[j];
    for (int j = 0; j < kEmbI; ++j) a += w1[k * kMlpIn + kEmbG + j] * li[j];
    pre[k] = a;
    hid[k] = a > 0.0 ? a : 0.0;
  }
  for (int o = 0; o < kMlpOut; ++o) {
    double z = b2[o];
    for (int k = 0; k < kHid; ++k) z += w2[o * kHid + k] * hid[k];
    out[o] = 1.0 / (1.0 + std::exp(-z));
  }
}

struct OptsD {
  double eps2d;
  int antialiased;
  int tile_cull;
  double bg[3];
};

CamD load_cam(const double* row, const double* affine) {
  CamD c;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) c.R[i * 3 + j] = row[i * 4 + j];
    c.t[i] = row[i * 4 + 3];
  }
  c.fx = row[12]; c.fy = row[13]; c.cx = row[14]; c.cy = row[15];
  c.W = static_cast<int>(row[16]); c.H = static_cast<int>(row[17]);
  c.znear = row[18]; c.zfar = row[19];
  c.tiles_x = (c.W + kTile - 1) / kTile;
  c.tiles_y = (c.H + kTile - 1) / kTile;
  c.has_aff = affine != nullptr;
  for (int i = 0; i < 12; ++i) c.A[i] = affine ? affine[i] : ((i % 4 == i / 4) ? 1.0 : 0.0);
  // camera centre = -R^T t
  for (int j = 0; j < 3; ++j) {
    double s = 0.0;
    for (int i = 0; i < 3; ++i) s += c.R[i * 3 + j] * c.t[i];
    c.center[j] = -s;
  }
  return c;
}

OptsD load_opts(const double* o) {
  OptsD r;
  r.eps2d = o[0];
  r.antialiased = static_cast<int>(o[1]);
  r.tile_cull = static_cast<int>(o[2]);
  r.bg[0] = o[3]; r.bg[1] = o[4]; r.bg[2] = o[5];
  return r;
}

// ---------------------------------------------------------------------------------------------
// Real spherical harmonics from the definition.
//   Y_l^m = s_m * N_l^|m| * Q_l^|m|(z) * { sqrt2 Re((x+iy)^m) m>0 ; 1 m=0 ; sqrt2 Im((x+iy)^|m|) m<0 }
//   N_l^m = sqrt((2l+1)/(4 pi) * (l-m)!/(l+m)!), Q_l^m = d^m/dz^m P_l (Legendre polynomial),
//   s_m = (-1)^m (Condon-Shortley phase, the sign layout of common 3DGS checkpoints).
// On the unit sphere sin(theta)^m Q_l^m(cos theta) is the associated Legendre function, so this
// is the textbook real basis; the index of (l, m) is l*l + l + m.
double factorial(int k) { double r = 1.0; for (int i = 2; i <= k; ++i) r *= i; return r; }

struct LegendreTable {
  // coef[l][m][k]: coefficient of z^k in d^m/dz^m P_l(z), l, m <= 3
  double coef[4][4][4];
  LegendreTable() {
    double P[4][4] = {{0}};
    P[0][0] = 1.0;                 // P_0 = 1
    P[1][1] = 1.0;                 // P_1 = z
    for (int l = 1; l < 3; ++l) {  // Bonnet: (l+1) P_{l+1} = (2l+1) z P_l - l P_{l-1}
      for (int k = 0; k < 4; ++k) {
        double zp = (k >= 1) ? P[l][k - 1] : 0.0;
        P[l + 1][k] = ((2 * l + 1) * zp - l * P[l - 1][k]) / (l + 1);
      }
    }
    for (int l = 0; l < 4; ++l) {
      double cur[4];
      for (int k = 0; k < 4; ++k) cur[k] = P[l][k];
      for (int m = 0; m < 4; ++m) {
        for (int k = 0; k < 4; ++k) coef[l][m][k] = cur[k];
        double nxt[4] = {0, 0, 0, 0};
        for (int k = 1; k < 4; ++k) nxt[k - 1] = k * cur[k];
        for (int k = 0; k < 4; ++k) cur[k] = nxt[k];
      }
    }
  }
};
const LegendreTable& legendre() { static LegendreTable t; return t; }

template <typename T>
void sh_basis(int deg, const T& x, const T& y, const T& z, T* Y) {
  const LegendreTable& L = legendre();
  // powers of (x + i y)
  T re[4], im[4];
  re[0] = T(1.0); im[0] = T(0.0);
  for (int m = 1; m < 4; ++m) {
    re[m] = re[m - 1] * x - im[m - 1] * y;
    im[m] = re[m - 1] * y + im[m - 1] * x;
  }
  for (int l = 0; l <= deg; ++l) {
    for (int m = -l; m <= l; ++m) {
      int am = m < 0 ? -m : m;
      double N = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * factorial(l - am) / factorial(l + am));
      T q = T(0.0);
      T zk = T(1.0);
      for (int k = 0; k < 4; ++k) {
        if (L.coef[l][am][k] != 0.0) q = q + L.coef[l][am][k] * zk;
        zk = zk * z;
      }
      double sign = (am % 2) ? -1.0 : 1.0;
      T trig = (m > 0) ? std::sqrt(2.0) * re[am] : ((m < 0) ? std::sqrt(2.0) * im[am] : T(1.0));
      Y[l * l + l + m] = sign * N * q * trig;
    }
  }
}

// ---------------------------------------------------------------------------------------------
template <typename T>
void quat_to_rot(const T q[4], T R[9]) {
  const T& w = q[0]; const T& x = q[1]; const T& y = q[2]; const T& z = q[3];
  R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
  R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
  R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

struct Rect { int x0, x1, y0, y1; };

Rect rect_of(double mx, double my, double r, const CamD& c) {
  auto cl = [](double v, int hi) {
    double f = std::floor(v);
    if (!(f > 0.0)) return 0;  // also NaN -> 0
    if (f > hi) return hi;
    return static_cast<int>(f);
  };
  Rect R;
  R.x0 = cl((mx - r) / kTile, c.tiles_x);
  R.x1 = cl((mx + r + kTile - 1) / kTile, c.tiles_x);
  R.y0 = cl((my - r) / kTile, c.tiles_y);
  R.y1 = cl((my + r + kTile - 1) / kTile, c.tiles_y);
  return R;
}

template <typename T>
struct Proj {
  bool vis = false;
  T mx, my, ca, cb, cc, op, rgb[3], z;
  double rad_src = 0.0;  // 3 sqrt(lambda_max) before ceil
  int r = 0;
  Rect rect{0, 0, 0, 0};
  double Y[16];          // SH basis values at the viewing direction
  unsigned flags = 0;    // discrete decisions: bit0-2 rgb clamp, bit3/4 Jacobian clamp x/y, bit5 comp=0
  // values of intermediate decisions, for knife-edge marks
  double z_val = 0.0, det_val = 0.0, ac_val = 0.0;
  double mx_err = 0.0, my_err = 0.0;  // bound on the FP32 rounding error of mean2d (px)
  double rgb_pre[3] = {0, 0, 0}, op_pre = 0.0;  // colour and opacity before the appearance transform
};

template <typename T>
Proj<T> project(const T mean[3], const T scale[3], const T quat[4], const T& opac,
                const double* sh, int K, int deg, const CamD& cam, const OptsD& o,
                const double* mlp_out = nullptr) {
  Proj<T> P;
  // camera-space position t = W mu + t_cam
  T t[3];
  for (int i = 0; i < 3; ++i)
    t[i] = cam.R[i * 3 + 0] * mean[0] + cam.R[i * 3 + 1] * mean[1] + cam.R[i * 3 + 2] * mean[2] + cam.t[i];
  P.z_val = val(t[2]);
  if (!(val(t[2]) > cam.znear && val(t[2]) < cam.zfar)) return P;
  // unit quaternion -> rotation
  T qn2 = quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3];
  if (!(val(qn2) > 0.0) || !std::isfinite(val(qn2))) return P;
  T qn = dsqrt(qn2);
  T q[4] = {quat[0] / qn, quat[1] / qn, quat[2] / qn, quat[3] / qn};
  T Rq[9];
  quat_to_rot(q, Rq);
  // Sigma = (R S)(R S)^T
  T M[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i * 3 + j] = Rq[i * 3 + j] * scale[j];
  T S[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = T(0.0);
      for (int k = 0; k < 3; ++k) s = s + M[i * 3 + k] * M[j * 3 + k];
      S[i * 3 + j] = s;
    }
  // camera-space covariance W Sigma W^T
  T Sc[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = T(0.0);
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) s = s + cam.R[i * 3 + k] * S[k * 3 + l] * cam.R[j * 3 + l];
      Sc[i * 3 + j] = s;
    }
  // Jacobian of the perspective projection at the clamped direction
  const double limx = 1.3 * (0.5 * cam.W) / cam.fx;
  const double limy = 1.3 * (0.5 * cam.H) / cam.fy;
  T u = t[0] / t[2];
  T w = t[1] / t[2];
  if (val(u) < -limx) { u = T(-limx); P.flags |= 8u; }
  else if (val(u) > limx) { u = T(limx); P.flags |= 8u; }
  if (val(w) < -limy) { w = T(-limy); P.flags |= 16u; }
  else if (val(w) > limy) { w = T(limy); P.flags |= 16u; }
  T j0[3] = {cam.fx / t[2], T(0.0), -cam.fx * u / t[2]};
  T j1[3] = {T(0.0), cam.fy / t[2], -cam.fy * w / t[2]};
  T ar = T(0.0), br = T(0.0), cr = T(0.0);
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      ar = ar + j0[k] * Sc[k * 3 + l] * j0[l];
      br = br + j0[k] * Sc[k * 3 + l] * j1[l];
      cr = cr + j1[k] * Sc[k * 3 + l] * j1[l];
    }
  T a = ar + o.eps2d;
  T b = br;
  T c = cr + o.eps2d;
  T det = a * c - b * b;
  P.det_val = val(det);
  P.ac_val = val(a) * val(c);
  if (!(val(det) > 0.0)) return P;
  T op = opac;
  if (o.antialiased) {
    T det_r = ar * cr - br * br;
    T ratio = det_r / det;
    if (val(ratio) > 0.0) {
      op = opac * dsqrt(ratio);
    } else {
      op = T(0.0);
      P.flags |= 32u;
    }
  }
  P.op = op;
  P.ca = c / det;
  P.cb = -b / det;
  P.cc = a / det;
  double mid = 0.5 * (val(a) + val(c));
  double lam = mid + std::sqrt(std::max(0.1, mid * mid - val(det)));
  P.rad_src = 3.0 * std::sqrt(lam);
  P.r = static_cast<int>(std::ceil(P.rad_src));
  P.mx = cam.fx * t[0] / t[2] + cam.cx;
  P.my = cam.fy * t[1] / t[2] + cam.cy;
  {
    // How far an FP32 evaluation of mean2d = f t/z + c can land from the exact value: a few
    // units of rounding (2^-24) of the magnitudes summed at each step, i.e. of the terms of
    // t = W mu + t_cam and of f t/z and c, which can be far larger than the result when they
    // cancel (near the image's top-left edge, for instance).
    const double u32 = 1.0 / 16777216.0;
    double et[3];
    for (int i = 0; i < 3; ++i)
      et[i] = 4.0 * u32 * (std::fabs(cam.R[i * 3 + 0] * val(mean[0])) + std::fabs(cam.R[i * 3 + 1] * val(mean[1])) +
                           std::fabs(cam.R[i * 3 + 2] * val(mean[2])) + std::fabs(cam.t[i]));
    const double z = std::fabs(val(t[2]));
    const double u = val(t[0]) / val(t[2]), w = val(t[1]) / val(t[2]);
    const double eu = (et[0] + std::fabs(u) * et[2]) / z + 2.0 * u32 * std::fabs(u);
    const double ew = (et[1] + std::fabs(w) * et[2]) / z + 2.0 * u32 * std::fabs(w);
    P.mx_err = std::fabs(cam.fx) * eu + 4.0 * u32 * (std::fabs(cam.fx * u) + std::fabs(cam.cx));
    P.my_err = std::fabs(cam.fy) * ew + 4.0 * u32 * (std::fabs(cam.fy * w) + std::fabs(cam.cy));
  }
  P.rect = rect_of(val(P.mx), val(P.my), P.r, cam);
  if ((P.rect.x1 - P.rect.x0) * (P.rect.y1 - P.rect.y0) <= 0) return P;
  // view-dependent colour
  T d[3];
  for (int i = 0; i < 3; ++i) d[i] = mean[i] - cam.center[i];
  T dn = dsqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  T Yt[16];
  for (int k = 0; k < 16; ++k) Yt[k] = T(0.0);
  sh_basis(deg, d[0] / dn, d[1] / dn, d[2] / dn, Yt);
  const int nb = (deg + 1) * (deg + 1);
  for (int k = 0; k < 16; ++k) P.Y[k] = (k < nb) ? val(Yt[k]) : 0.0;
  for (int ch = 0; ch < 3; ++ch) {
    T v = T(0.5);
    for (int k = 0; k < nb && k < K; ++k) v = v + sh[k * 3 + ch] * Yt[k];
    if (val(v) < 0.0) { v = T(0.0); P.flags |= (1u << ch); }
    P.rgb_pre[ch] = val(v);
    if (mlp_out) v = v * (2.0 * mlp_out[ch]);
    P.rgb[ch] = v;
  }
  P.op_pre = val(op);
  if (mlp_out) op = op * (1.0 - mlp_out[3]);
  P.op = op;
  P.z = t[2];
  const double outs[] = {val(P.mx), val(P.my), val(P.ca), val(P.cb), val(P.cc), val(P.op),
                         val(P.rgb[0]), val(P.rgb[1]), val(P.rgb[2])};
  for (double v : outs)
    if (!std::isfinite(v)) return P;
  P.vis = true;
  return P;
}

// ---------------------------------------------------------------------------------------------
// Scene access (double copies of the inputs).
struct SceneD {
  int64_t n;
  const double* means;
  const double* scales;
  const double* quats;
  const double* opac;
  const double* sh;
  int K;
  int deg;
  const double* gemb = nullptr;  // [n][16] Gaussian embeddings, or NULL (no appearance transform)
  const double* mlp = nullptr;   // [kMlpParams]
};

// The appearance transform's outputs for Gaussian g seen by `cam`; false when it is off.
bool mlp_of(const SceneD& s, int64_t g, const CamD& cam, double out[kMlpOut]) {
  if (!s.mlp || !s.gemb || !cam.iemb) return false;
  double pre[kHid], hid[kHid];
  mlp_forward(s.mlp, s.gemb + kEmbG * g, cam.iemb, pre, hid, out);
  return true;
}

Proj<double> project_d(const SceneD& s, int64_t g, const CamD& cam, const OptsD& o) {
  double m[kMlpOut];
  const bool on = mlp_of(s, g, cam, m);
  return project<double>(s.means + 3 * g, s.scales + 3 * g, s.quats + 4 * g, s.opac[g],
                         s.sh + g * s.K * 3, s.K, s.deg, cam, o, on ? m : nullptr);
}

// Minimum over the tile's in-image pixel centres of the Mahalanobis distance (p-mu)^T conic (p-mu).
double tile_min_maha(const Proj<double>& p, const CamD& cam, int tx, int ty) {
  const double xlo = tx * kTile + 0.5, xhi = std::min((tx + 1) * kTile, cam.W) - 0.5;
  const double ylo = ty * kTile + 0.5, yhi = std::min((ty + 1) * kTile, cam.H) - 0.5;
  const double a = p.ca, b = p.cb, c = p.cc;
  const double mx = p.mx, my = p.my;
  if (mx >= xlo && mx <= xhi && my >= ylo && my <= yhi) return 0.0;
  auto q = [&](double dx, double dy) { return a * dx * dx + 2.0 * b * dx * dy + c * dy * dy; };
  double best = std::numeric_limits<double>::infinity();
  // vertical edges: x fixed, minimise over y
  for (double xe : {xlo, xhi}) {
    double dx = xe - mx;
    double dy = std::clamp(-b * dx / c, ylo - my, yhi - my);
    best = std::min(best, q(dx, dy));
  }
  for (double ye : {ylo, yhi}) {
    double dy = ye - my;
    double dx = std::clamp(-b * dy / a, xlo - mx, xhi - mx);
    best = std::min(best, q(dx, dy));
  }
  return best;
}

// log of (largest opacity over the tile) / (1/255); the tile is culled where this is < 0.
double tile_cull_margin(const Proj<double>& p, const CamD& cam, int tx, int ty) {
  return std::log(p.op) - 0.5 * tile_min_maha(p, cam, tx, ty) - std::log(kAlphaMin);
}

// Knife-edge check of the rectangle: do FP32-sized perturbations of the decision's inputs
// change it?  Returns the union and the intersection of the nominal and perturbed rectangles
// (the Gaussian is in every tile of the intersection whatever the precision; only the tiles of
// the union outside it are uncertain) and whether they differ.
bool rect_knife_edge(const Proj<double>& p, const CamD& cam, Rect* uni, Rect* inter) {
  const double dm_x = std::max(1e-6 * (std::fabs(p.mx) + 1.0), 4.0 * p.mx_err);
  const double dm_y = std::max(1e-6 * (std::fabs(p.my) + 1.0), 4.0 * p.my_err);
  const double dr = 1e-5 * p.rad_src;
  Rect U = p.rect, I = p.rect;
  bool differs = false;
  for (int sx = -1; sx <= 1; sx += 2)
    for (int sy = -1; sy <= 1; sy += 2)
      for (int sr = -1; sr <= 1; sr += 2) {
        int r = static_cast<int>(std::ceil(p.rad_src + sr * dr));
        Rect q = rect_of(p.mx + sx * dm_x, p.my + sy * dm_y, r, cam);
        if (q.x0 != p.rect.x0 || q.x1 != p.rect.x1 || q.y0 != p.rect.y0 || q.y1 != p.rect.y1) differs = true;
        U.x0 = std::min(U.x0, q.x0); U.x1 = std::max(U.x1, q.x1);
        U.y0 = std::min(U.y0, q.y0); U.y1 = std::max(U.y1, q.y1);
        I.x0 = std::max(I.x0, q.x0); I.x1 = std::min(I.x1, q.x1);
        I.y0 = std::max(I.y0, q.y0); I.y1 = std::min(I.y1, q.y1);
      }
  *uni = U;
  *inter = I;
  return differs;
}

struct Binned {
  std::vector<Proj<double>> proj;       // [C*n]
  std::vector<uint8_t> gmark;           // [C*n] Gaussian-level knife edge
  std::vector<int64_t> tile_off;        // [C+1]
  std::vector<int64_t> pix_off;         // [C+1]
  std::vector<std::vector<int64_t>> lists;  // per global tile: ids c*n+g in blend order
  std::vector<uint8_t> tile_mark;       // per global tile: every pixel of the tile is marked
};

void bin_all(const SceneD& s, const std::vector<CamD>& cams, const OptsD& o, Binned* B) {
  const int C = static_cast<int>(cams.size());
  const int64_t n = s.n;
  B->proj.assign(static_cast<size_t>(C) * n, Proj<double>());
  B->gmark.assign(static_cast<size_t>(C) * n, 0);
  B->tile_off.assign(C + 1, 0);
  B->pix_off.assign(C + 1, 0);
  for (int c = 0; c < C; ++c) {
    B->tile_off[c + 1] = B->tile_off[c] + static_cast<int64_t>(cams[c].tiles_x) * cams[c].tiles_y;
    B->pix_off[c + 1] = B->pix_off[c] + static_cast<int64_t>(cams[c].W) * cams[c].H;
  }
  B->lists.assign(B->tile_off[C], std::vector<int64_t>());
  B->tile_mark.assign(B->tile_off[C], 0);
  for (int c = 0; c < C; ++c) {
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t g = 0; g < n; ++g) B->proj[c * n + g] = project_d(s, g, cams[c], o);
  }
  // Gaussian-level knife edges: decided per (camera, Gaussian) in parallel; the tiles they
  // make uncertain are marked afterwards
  const int64_t CN = static_cast<int64_t>(C) * n;
  std::vector<Rect> mark_rect(CN, Rect{0, 0, 0, 0});
  std::vector<Rect> sure_rect(CN, Rect{0, 0, 0, 0});  // tiles not made uncertain inside mark_rect
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t id = 0; id < CN; ++id) {
    const int c = static_cast<int>(id / n);
    const int64_t g = id % n;
    const CamD& cam = cams[c];
    const Proj<double>& p = B->proj[id];
    const bool near_plane = std::fabs(p.z_val - cam.znear) <= 1e-6 * std::max(1.0, std::fabs(p.z_val)) ||
                            std::fabs(p.z_val - cam.zfar) <= 1e-6 * std::max(1.0, std::fabs(p.z_val));
    const bool near_det = std::isfinite(p.det_val) && std::fabs(p.det_val) <= 1e-5 * std::fabs(p.ac_val);
    if (near_plane || near_det) {
      // The Gaussian may exist in one precision and not in the other: every tile it could touch
      // is uncertain; its rectangle comes from a camera with the depth range widened a little.
      B->gmark[id] = 1;
      CamD wide = cam;
      wide.znear = cam.znear * (1.0 - 1e-5);
      wide.zfar = cam.zfar * (1.0 + 1e-5);
      Proj<double> q = project_d(s, g, wide, o);
      if (q.r > 0) mark_rect[id] = q.rect;
    }
    // visible, or culled only because its rectangle came out empty (at an image edge)
    if (!p.vis && !(p.rad_src > 0.0)) continue;
    Rect U, I;
    if (rect_knife_edge(p, cam, &U, &I)) {
      if (near_plane || near_det) {  // existence uncertain: every tile of both rectangles
        Rect& M = mark_rect[id];
        if (M.x1 > M.x0 && M.y1 > M.y0) {
          M.x0 = std::min(M.x0, U.x0); M.x1 = std::max(M.x1, U.x1);
          M.y0 = std::min(M.y0, U.y0); M.y1 = std::max(M.y1, U.y1);
        } else {
          M = U;
        }
      } else {
        mark_rect[id] = U;
        sure_rect[id] = I;
      }
      B->gmark[id] = 1;
    }
  }
  for (int64_t id = 0; id < CN; ++id) {
    const Rect& U = mark_rect[id];
    const Rect& I = sure_rect[id];
    if (!B->gmark[id]) continue;
    const int c = static_cast<int>(id / n);
    // a tile whose membership (or the Gaussian's existence) is uncertain matters only where the
    // Gaussian can reach alpha 1/255 at one of its pixel centres (checked with the nominal
    // projection when it has a conic; the margin is far above FP32 rounding)
    const Proj<double>& p = B->proj[id];
    const bool conic_ok = p.rad_src > 0.0 && p.det_val > 0.0;
    for (int ty = U.y0; ty < U.y1; ++ty)
      for (int tx = U.x0; tx < U.x1; ++tx) {
        if (tx >= I.x0 && tx < I.x1 && ty >= I.y0 && ty < I.y1) continue;
        if (conic_ok && tile_cull_margin(p, cams[c], tx, ty) < -1e-3) continue;
        B->tile_mark[B->tile_off[c] + ty * cams[c].tiles_x + tx] = 1;
      }
  }
  // binning: count kept tiles per (camera, Gaussian), then fill, both in parallel
  std::vector<int64_t> cnt(CN + 1, 0);
  std::vector<uint8_t> cull_knife(CN, 0);
  auto visit = [&](int64_t id, auto&& emit) {
    const int c = static_cast<int>(id / n);
    const CamD& cam = cams[c];
    const Proj<double>& p = B->proj[id];
    if (!p.vis) return;
    for (int ty = p.rect.y0; ty < p.rect.y1; ++ty)
      for (int tx = p.rect.x0; tx < p.rect.x1; ++tx) {
        const int64_t tile = B->tile_off[c] + ty * cam.tiles_x + tx;
        bool keep = true;
        if (o.tile_cull) {
          const double rd = tile_min_maha(p, cam, tx, ty);
          const double m = std::log(p.op) - 0.5 * rd - std::log(kAlphaMin);
          if (std::fabs(m) < 1e-4 * (1.0 + 0.5 * rd)) emit(tile, -1);
          keep = m >= 0.0;
        }
        if (keep) emit(tile, id);
      }
  };
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t id = 0; id < CN; ++id) {
    int64_t k = 0;
    visit(id, [&](int64_t, int64_t who) {
      if (who >= 0) ++k;
      else cull_knife[id] = 1;
    });
    cnt[id + 1] = k;
  }
  for (int64_t id = 0; id < CN; ++id) cnt[id + 1] += cnt[id];
  std::vector<int64_t> ptile(cnt[CN]), pid(cnt[CN]);
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t id = 0; id < CN; ++id) {
    int64_t k = cnt[id];
    visit(id, [&](int64_t tile, int64_t who) {
      if (who >= 0) { ptile[k] = tile; pid[k] = who; ++k; }
    });
  }
  // a tile-cull decision within FP32 reach marks the Gaussian and that tile
  for (int64_t id = 0; id < CN; ++id)
    if (cull_knife[id]) {
      B->gmark[id] = 1;
      visit(id, [&](int64_t tile, int64_t who) {
        if (who < 0) B->tile_mark[tile] = 1;
      });
    }
  // bucket the pairs by tile, keeping (camera, Gaussian) order inside a tile
  std::vector<int64_t> tcnt(B->lists.size(), 0);
  for (int64_t k = 0; k < cnt[CN]; ++k) ++tcnt[ptile[k]];
  for (size_t t = 0; t < B->lists.size(); ++t) B->lists[t].reserve(tcnt[t]);
  for (int64_t k = 0; k < cnt[CN]; ++k) B->lists[ptile[k]].push_back(pid[k]);
  // depth order within each tile: key (float32(z), index)
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < static_cast<int64_t>(B->lists.size()); ++t) {
    auto& L = B->lists[t];
    std::stable_sort(L.begin(), L.end(), [&](int64_t a, int64_t b) {
      float za = static_cast<float>(val(B->proj[a].z));
      float zb = static_cast<float>(val(B->proj[b].z));
      if (za != zb) return za < zb;
      return a < b;
    });
  }
}

// Test switch (oracle_set_mutation): plants one known mistake in the gradients, so that the tests
// can show that their parity bars catch it. 0, the default, computes the correct gradients.
//   1: the 0.99 clamp of alpha passes gradient (its mask is dropped)
//   2: the gradient of the degree-2 SH band has the wrong sign
//   3: the depth term of dL/dalpha is left out (the depth output's dependence on alpha and T)
//   4: the gradients of conic a and conic c are swapped (a transposed operand)
int g_mutation = 0;

// Reasons for a knife-edge mark at a pixel (bits of PixelResult::mark and of out_mark).
constexpr unsigned kMarkEdge = 1;      // the Gaussian's quadratic form is within reach of 0
constexpr unsigned kMarkAlphaMin = 2;  // alpha within reach of 1/255
constexpr unsigned kMarkAlphaMax = 4;  // alpha within reach of the 0.99 clamp
constexpr unsigned kMarkStop = 8;      // T (1 - alpha) within reach of 1e-4
constexpr unsigned kMarkTie = 16;      // two consecutive contributors at nearly equal depth
constexpr unsigned kMarkTile = 32;     // the tile's list itself is uncertain (a rectangle, a cull)
// Two consecutive contributors at nearly equal depth whose order cannot move the pixel's outputs by
// 1e-5: swapping adjacent layers i, j changes the colour by T_i alpha_i alpha_j (c_i - c_j), the
// depth by T_i alpha_i alpha_j (z_i - z_j) and leaves T unchanged, so below that bound only the
// gradients (each layer's transmittance) and the list positions depend on the order.
constexpr unsigned kMarkTieSoft = 64;

// One contributor of a pixel (for the backward re-walk).
struct Contrib {
  int64_t id;
  int64_t pos;  // position in the tile's list
  double dx, dy, sigma, araw, alpha, T;
  bool clamped;
};

struct PixelResult {
  double C[3];   // sum of c' alpha T (appearance applied per Gaussian)
  double D;      // sum of z alpha T
  double T;      // final transmittance
  int64_t last;  // list positions walked up to and including the last contributor
  unsigned mark;  // why a decision at this pixel is within FP32 reach (kMark* bits), 0 if none
  uint64_t sig;
  // The largest change the decisions within FP32 reach could make to this pixel's colour (any
  // channel), accumulated depth and alpha, if taken the other way (ties: in any order within each
  // group of near-tied consecutive contributors). Zero where nothing is marked. The tile-level
  // marks (kMarkTile: whether a Gaussian is in the tile's list at all) are not bounded.
  double bound[3];
};

inline void fnv(uint64_t* h, uint64_t v) {
  for (int i = 0; i < 8; ++i) {
    *h ^= (v >> (8 * i)) & 0xffu;
    *h *= 1099511628211ull;
  }
}

// Eq. 2, front to back, for pixel (x, y) of camera `cam` over `list`.
PixelResult composite(const Binned& B, const std::vector<int64_t>& list, const CamD& cam, int x, int y,
                      std::vector<Contrib>* trace) {
  PixelResult R{{0, 0, 0}, 0.0, 1.0, 0, 0u, 1469598103934665603ull, {0.0, 0.0, 0.0}};
  // bound bookkeeping: weights of uncertain inclusions and stops (times the largest colour and
  // depth seen, at the end), and the current group of near-tied consecutive contributors
  double incl_w = 0.0, stop_w = 0.0, cmax = 0.0, zmax = 0.0;
  double g_T = 0.0, g_keep = 1.0, g_cmin[3] = {0, 0, 0}, g_cmax[3] = {0, 0, 0}, g_zmin = 0.0, g_zmax = 0.0;
  int g_n = 0;
  auto close_group = [&]() {
    if (g_n > 1) {
      double dc = 0.0;
      for (int ch = 0; ch < 3; ++ch) dc = std::max(dc, g_cmax[ch] - g_cmin[ch]);
      const double w = g_T * (1.0 - g_keep);  // the group's total weight, the same in any order
      R.bound[0] += w * dc;
      R.bound[1] += w * (g_zmax - g_zmin);
    }
    g_n = 0;
  };
  const double px = x + 0.5, py = y + 0.5;
  double T = 1.0;
  double Terr = 0.0;  // running estimate of the FP32 relative error of T
  double prev_z = -1.0;
  double prev_T = 0.0, prev_alpha = 0.0, prev_c[3] = {0.0, 0.0, 0.0};  // the previous contributor
  for (size_t k = 0; k < list.size(); ++k) {
    const int64_t id = list[k];
    const Proj<double>& p = B.proj[id];
    const double dx = p.mx - px, dy = p.my - py;
    const double sigma = 0.5 * (p.ca * dx * dx + p.cc * dy * dy) + p.cb * dx * dy;
    const double terms = 0.5 * (std::fabs(p.ca) * dx * dx + std::fabs(p.cc) * dy * dy) + std::fabs(p.cb * dx * dy);
    const double errs = 1e-6 * terms +
                        4e-7 * (std::fabs(p.ca * dx + p.cb * dy) + std::fabs(p.cb * dx + p.cc * dy)) *
                            (std::fabs(p.mx) + std::fabs(p.my) + 1.0) + 1e-5;
    const double araw_e = p.op * std::exp(-sigma);
    if (sigma < errs && araw_e >= kAlphaMin * 0.9) {
      R.mark |= kMarkEdge;
      const double a_e = std::min(kAlphaMax, araw_e);
      incl_w += T * a_e / (1.0 - a_e);
    }
    if (sigma < 0.0) { fnv(&R.sig, static_cast<uint64_t>(id) * 8 + 1); continue; }
    const double araw = p.op * std::exp(-sigma);
    if (std::fabs(std::log(araw / kAlphaMin)) < errs) {
      R.mark |= kMarkAlphaMin;
      incl_w += T * kAlphaMin * std::exp(errs) / (1.0 - kAlphaMin);
    }
    if (std::fabs(std::log(araw / kAlphaMax)) < errs) {
      R.mark |= kMarkAlphaMax;
      incl_w += T * kAlphaMax * errs / (1.0 - kAlphaMax);  // alpha itself moves by at most that
    }
    const double alpha = std::min(kAlphaMax, araw);
    if (alpha < kAlphaMin) { fnv(&R.sig, static_cast<uint64_t>(id) * 8 + 2); continue; }
    const double Tn = T * (1.0 - alpha);
    const double terr_n = Terr + (alpha / (1.0 - alpha)) * errs + 1.2e-7;
    if (std::fabs(std::log(Tn / kTMin)) < 2.0 * terr_n + 1e-6) {
      R.mark |= kMarkStop;
      stop_w += T;  // stopping here or not moves at most the weight left, T
    }
    if (Tn < kTMin) { fnv(&R.sig, static_cast<uint64_t>(id) * 8 + 3); break; }
    double cp[3];
    for (int ch = 0; ch < 3; ++ch) {
      cp[ch] = cam.A[ch * 4 + 3];
      for (int k2 = 0; k2 < 3; ++k2) cp[ch] += cam.A[ch * 4 + k2] * p.rgb[k2];
    }
    const bool tied = prev_z >= 0.0 && std::fabs(p.z - prev_z) <= 2e-6 * std::max(p.z, prev_z);
    if (tied) {
      double dc = 0.0;
      for (int ch = 0; ch < 3; ++ch) dc = std::max(dc, std::fabs(cp[ch] - prev_c[ch]));
      const double swap = prev_T * prev_alpha * alpha * std::max(dc, std::fabs(p.z - prev_z));
      R.mark |= swap >= 1e-5 ? kMarkTie : kMarkTieSoft;
      if (g_n == 0) {  // the group starts with the previous contributor
        g_n = 1;
        g_T = prev_T;
        g_keep = 1.0 - prev_alpha;
        for (int ch = 0; ch < 3; ++ch) g_cmin[ch] = g_cmax[ch] = prev_c[ch];
        g_zmin = g_zmax = prev_z;
      }
      g_n += 1;
      g_keep *= 1.0 - alpha;
      for (int ch = 0; ch < 3; ++ch) {
        g_cmin[ch] = std::min(g_cmin[ch], cp[ch]);
        g_cmax[ch] = std::max(g_cmax[ch], cp[ch]);
      }
      g_zmin = std::min(g_zmin, p.z);
      g_zmax = std::max(g_zmax, p.z);
    } else {
      close_group();
    }
    for (int ch = 0; ch < 3; ++ch) cmax = std::max(cmax, std::fabs(cp[ch]));
    zmax = std::max(zmax, std::fabs(p.z));
    prev_z = p.z;
    prev_T = T;
    prev_alpha = alpha;
    for (int ch = 0; ch < 3; ++ch) prev_c[ch] = cp[ch];
    const bool clamped = araw > kAlphaMax;
    fnv(&R.sig, static_cast<uint64_t>(id) * 8 + (clamped ? 4 : 5));
    const double w = alpha * T;
    for (int ch = 0; ch < 3; ++ch) R.C[ch] += cp[ch] * w;
    R.D += p.z * w;
    if (trace) trace->push_back(Contrib{id, static_cast<int64_t>(k), dx, dy, sigma, araw, alpha, T, clamped});
    T = Tn;
    Terr = terr_n;
    R.last = static_cast<int64_t>(k) + 1;
  }
  close_group();
  if (incl_w > 0.0 || stop_w > 0.0) {
    // an uncertain inclusion moves the colour by at most its weight times (its colour + the
    // colour behind it), alpha by its weight; an uncertain stop moves them by at most the weight
    // left. The colour and depth bounds are those of the whole list (after the transform).
    double craw = 0.0;
    for (int64_t id : list) {
      const Proj<double>& p = B.proj[id];
      for (int ch = 0; ch < 3; ++ch) craw = std::max(craw, std::fabs(p.rgb[ch]));
      zmax = std::max(zmax, std::fabs(p.z));
    }
    for (int ch = 0; ch < 3; ++ch) {
      const double a = std::fabs(cam.A[ch * 4]) + std::fabs(cam.A[ch * 4 + 1]) + std::fabs(cam.A[ch * 4 + 2]);
      cmax = std::max(cmax, a * craw + std::fabs(cam.A[ch * 4 + 3]));
    }
    R.bound[0] += (2.0 * incl_w + stop_w) * cmax;
    R.bound[1] += (2.0 * incl_w + stop_w) * zmax;
    R.bound[2] += incl_w + stop_w;
  }
  R.T = T;
  return R;
}

bool valid_inputs(int64_t n, const double* means, const double* scales, const double* quats,
                  const double* opac, const double* sh, int K, int deg, int C, const double* cams) {
  if (n < 0 || C < 0 || deg < 0 || deg > 3 || K < (deg + 1) * (deg + 1) || K > 16) return false;
  if (n > 0 && (!means || !scales || !quats || !opac || !sh)) return false;
  if (C > 0 && !cams) return false;
  for (int c = 0; c < C; ++c) {
    const double* r = cams + 20 * c;
    if (!(r[12] > 0) || !(r[13] > 0) || r[16] < 1 || r[17] < 1 || r[16] > 16384 || r[17] > 16384) return false;
    if (!(r[18] > 0) || !(r[19] > r[18])) return false;
  }
  return true;
}

std::vector<CamD> load_cams(int C, const double* cams, const double* affines, const double* iemb = nullptr) {
  std::vector<CamD> v;
  for (int c = 0; c < C; ++c) {
    v.push_back(load_cam(cams + 20 * c, affines ? affines + 12 * c : nullptr));
    v.back().iemb = iemb ? iemb + kEmbI * c : nullptr;
  }
  return v;
}

}  // namespace

extern "C" {

// Projection of every Gaussian for one camera (Sec. 3.1 projection; Sec. 3.5.4 filter; SH colour).
// out_rec[n][16] = mx, my, conic a, b, c, opacity', r, g, b, depth, radius, x0, x1, y0, y1,
//                  tiles kept after the optional tile cull.
// out_flags[n]: bit0 visible, bit1 knife-edge, bits 2-7 the discrete decisions
//               (rgb clamp r/g/b, Jacobian clamp x/y, zero compensation).
int oracle_project(int64_t n, const double* means, const double* scales, const double* quats,
                   const double* opac, const double* sh, int K, int deg, const double* cam_row,
                   const double* opts, double* out_rec, int32_t* out_flags, const double* gemb,
                   const double* iemb, const double* mlp) {
  if (!valid_inputs(n, means, scales, quats, opac, sh, K, deg, 1, cam_row)) return -1;
  SceneD s{n, means, scales, quats, opac, sh, K, deg, gemb, mlp};
  std::vector<CamD> cams = load_cams(1, cam_row, nullptr, iemb);
  OptsD o = load_opts(opts);
  Binned B;
  bin_all(s, cams, o, &B);
  std::vector<int64_t> kept(n, 0);
  for (const auto& L : B.lists)
    for (int64_t id : L) kept[id] += 1;
  for (int64_t g = 0; g < n; ++g) {
    const Proj<double>& p = B.proj[g];
    double* r = out_rec + 16 * g;
    std::fill(r, r + 16, 0.0);
    int32_t f = 0;
    if (p.vis) {
      f |= 1;
      r[0] = p.mx; r[1] = p.my; r[2] = p.ca; r[3] = p.cb; r[4] = p.cc; r[5] = p.op;
      r[6] = p.rgb[0]; r[7] = p.rgb[1]; r[8] = p.rgb[2]; r[9] = p.z;
      r[10] = p.r; r[11] = p.rect.x0; r[12] = p.rect.x1; r[13] = p.rect.y0; r[14] = p.rect.y1;
      r[15] = static_cast<double>(kept[g]);
    }
    if (B.gmark[g]) f |= 2;
    f |= static_cast<int32_t>(p.flags << 2);
    out_flags[g] = f;
  }
  return 0;
}

// Forward render of C cameras (Eq. 2) with cameras packed one after another.
//   cams[C][20]: viewmat(12, world->camera, row-major), fx, fy, cx, cy, width, height, near, far
//   affines[C][12] or NULL: per-image [A | b] applied to each Gaussian colour
//   opts[6]: eps2d, antialiased, tile_cull, bg r, g, b
//   tile_subset: global tile ids to composite (NULL: all tiles); other pixels are left untouched
//   out_img[sum HW][8]: r, g, b, depth_acc, depth_exp, alpha, T_final, n_contrib
//   out_mark[sum HW]: nonzero where a discrete decision at this pixel is within FP32 reach: the
//                     reasons as kMark* bits
//   out_sig[sum HW] or NULL: hash of every per-Gaussian decision at the pixel
//   out_pairs[pair_cap][2] or NULL: (global tile, c*n+g) in blend order, tile-major
//   out_gmark[C*n] or NULL: Gaussian-level knife edges
//   out_bound[sum HW][3] or NULL: per pixel, the largest change of its colour (any channel),
//                     depth_acc and alpha that the marked decisions could make (PixelResult::bound)
// Returns the total number of (tile, Gaussian) pairs, or -1 on invalid arguments.
int64_t oracle_render(int64_t n, const double* means, const double* scales, const double* quats,
                      const double* opac, const double* sh, int K, int deg, int C, const double* cams,
                      const double* affines, const double* opts, const int64_t* tile_subset,
                      int64_t n_subset, double* out_img, uint8_t* out_mark, uint64_t* out_sig,
                      int64_t* out_pairs, int64_t pair_cap, uint8_t* out_gmark, const double* gemb,
                      const double* iemb, const double* mlp, double* out_bound) {
  if (!valid_inputs(n, means, scales, quats, opac, sh, K, deg, C, cams)) return -1;
  SceneD s{n, means, scales, quats, opac, sh, K, deg, gemb, mlp};
  std::vector<CamD> cv = load_cams(C, cams, affines, iemb);
  OptsD o = load_opts(opts);
  Binned B;
  bin_all(s, cv, o, &B);
  const int64_t ntiles = B.tile_off[C];
  int64_t P = 0;
  for (const auto& L : B.lists) P += static_cast<int64_t>(L.size());
  if (out_pairs && pair_cap >= P) {
    int64_t k = 0;
    for (int64_t t = 0; t < ntiles; ++t)
      for (int64_t id : B.lists[t]) { out_pairs[2 * k] = t; out_pairs[2 * k + 1] = id; ++k; }
  }
  if (out_gmark)
    for (int64_t i = 0; i < static_cast<int64_t>(C) * n; ++i) out_gmark[i] = B.gmark[i];
  std::vector<int64_t> tiles;
  if (tile_subset) tiles.assign(tile_subset, tile_subset + n_subset);
  else { tiles.resize(ntiles); for (int64_t t = 0; t < ntiles; ++t) tiles[t] = t; }
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t ti = 0; ti < static_cast<int64_t>(tiles.size()); ++ti) {
    const int64_t t = tiles[ti];
    if (t < 0 || t >= ntiles) continue;
    int c = 0;
    while (t >= B.tile_off[c + 1]) ++c;
    const CamD& cam = cv[c];
    const int64_t lt = t - B.tile_off[c];
    const int tx = static_cast<int>(lt % cam.tiles_x), ty = static_cast<int>(lt / cam.tiles_x);
    for (int yy = 0; yy < kTile; ++yy)
      for (int xx = 0; xx < kTile; ++xx) {
        const int x = tx * kTile + xx, y = ty * kTile + yy;
        if (x >= cam.W || y >= cam.H) continue;
        PixelResult R = composite(B, B.lists[t], cam, x, y, nullptr);
        const int64_t pix = B.pix_off[c] + static_cast<int64_t>(y) * cam.W + x;
        double* out = out_img + 8 * pix;
        const double alpha = 1.0 - R.T;
        for (int ch = 0; ch < 3; ++ch) out[ch] = R.C[ch] + R.T * o.bg[ch];
        out[3] = R.D;
        out[4] = R.D / std::max(alpha, 1e-10);
        out[5] = alpha;
        out[6] = R.T;
        out[7] = static_cast<double>(R.last);
        if (out_mark) out_mark[pix] = static_cast<uint8_t>(R.mark | (B.tile_mark[t] ? kMarkTile : 0u));
        if (out_sig) out_sig[pix] = R.sig;
        if (out_bound)
          for (int k = 0; k < 3; ++k) out_bound[3 * pix + k] = R.bound[k];
      }
  }
  return P;
}

// Analytic gradients of L = sum over pixels of <up_grads, (rgb, depth_acc, depth_exp, alpha)>.
//   up_grads[sum HW][6]: dL/d r, g, b, depth_acc, depth_exp, alpha
//   g_means[n][3], g_scales[n][3], g_quats[n][4], g_opac[n], g_sh[n][K][3]: overwritten
//   g_affine[C][12] or NULL; g_absgrad[n][2] or NULL (sum over pixels of |dL/dmean2d| per axis)
//   g2d[C*n][12] or NULL: per (camera, Gaussian) gradients of mean2d x/y, conic a/b/c,
//                         opacity', rgb, depth, |mean2d| x/y
//   tile_subset[n_subset] or NULL: only the pixels of these global tiles enter L (the result
//                         equals the full gradient when up_grads is zero on every other pixel)
//   g_mag[n][11 + 3K] or NULL: per parameter (mean 3, scale 3, quaternion 4, opacity, SH), the
//                         magnitude of the sum that gives its gradient: the same chain rule with
//                         every sum replaced by the sum of its terms' magnitudes, through the
//                         blend walk and the projection (Mag). It bounds |gradient| and sets the
//                         scale of the rounding error of any finite-precision evaluation of it.
int oracle_backward(int64_t n, const double* means, const double* scales, const double* quats,
                    const double* opac, const double* sh, int K, int deg, int C, const double* cams,
                    const double* affines, const double* opts, const double* up_grads,
                    double* g_means, double* g_scales, double* g_quats, double* g_opac, double* g_sh,
                    double* g_affine, double* g_absgrad, double* g2d_out, const int64_t* tile_subset,
                    int64_t n_subset, double* g_mag, const double* gemb, const double* iemb, const double* mlp,
                    double* g_gemb, double* g_iemb, double* g_mlp) {
  if (!valid_inputs(n, means, scales, quats, opac, sh, K, deg, C, cams)) return -1;
  SceneD s{n, means, scales, quats, opac, sh, K, deg, gemb, mlp};
  std::vector<CamD> cv = load_cams(C, cams, affines, iemb);
  const bool mlp_on = gemb && iemb && mlp;
  // per visible (camera, Gaussian): d(MLP output logits), for the serial weight reduction below
  std::vector<double> mlp_dz(mlp_on ? static_cast<size_t>(C) * n * kMlpOut : 0, 0.0);
  OptsD o = load_opts(opts);
  Binned B;
  bin_all(s, cv, o, &B);
  const int64_t ntiles = B.tile_off[C];
  std::vector<int64_t> list_off(ntiles + 1, 0);
  for (int64_t t = 0; t < ntiles; ++t) list_off[t + 1] = list_off[t] + static_cast<int64_t>(B.lists[t].size());
  const int64_t P = list_off[ntiles];
  // per (tile, Gaussian) gradient contributions, reduced serially afterwards (deterministic)
  constexpr int G2 = 12;
  std::vector<double> pairbuf(static_cast<size_t>(P) * G2, 0.0);
  // with g_mag: the same per-pixel contributions in absolute value (10 per pair)
  constexpr int GM = 10;
  std::vector<double> pairabs(g_mag ? static_cast<size_t>(P) * GM : 0, 0.0);
  std::vector<double> tile_aff(static_cast<size_t>(ntiles) * 12, 0.0);
  std::vector<uint8_t> use_tile(ntiles, tile_subset ? 0 : 1);
  if (tile_subset)
    for (int64_t k = 0; k < n_subset; ++k)
      if (tile_subset[k] >= 0 && tile_subset[k] < ntiles) use_tile[tile_subset[k]] = 1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < ntiles; ++t) {
    if (!use_tile[t]) continue;
    int c = 0;
    while (t >= B.tile_off[c + 1]) ++c;
    const CamD& cam = cv[c];
    const int64_t lt = t - B.tile_off[c];
    const int tx = static_cast<int>(lt % cam.tiles_x), ty = static_cast<int>(lt / cam.tiles_x);
    const auto& list = B.lists[t];
    std::vector<Contrib> tr;
    for (int yy = 0; yy < kTile; ++yy)
      for (int xx = 0; xx < kTile; ++xx) {
        const int x = tx * kTile + xx, y = ty * kTile + yy;
        if (x >= cam.W || y >= cam.H) continue;
        tr.clear();
        PixelResult R = composite(B, list, cam, x, y, &tr);
        const int64_t pix = B.pix_off[c] + static_cast<int64_t>(y) * cam.W + x;
        const double* up = up_grads + 6 * pix;
        const double alpha_out = 1.0 - R.T;
        // outputs: rgb = C + T bg; depth_acc = D; depth_exp = D / max(alpha, 1e-10); alpha = 1 - T
        double D_bar = up[3] + up[4] / std::max(alpha_out, 1e-10);
        double aout_bar = up[5] + ((alpha_out > 1e-10) ? -up[4] * R.D / (alpha_out * alpha_out) : 0.0);
        double T_bar = -aout_bar;
        for (int ch = 0; ch < 3; ++ch) T_bar += up[ch] * o.bg[ch];
        // with g_mag, the same quantities as sums of their terms' magnitudes (see Mag above)
        const double D_bar_abs = std::fabs(up[3]) + std::fabs(up[4]) / std::max(alpha_out, 1e-10);
        double T_bar_abs = std::fabs(up[5]) + ((alpha_out > 1e-10) ? std::fabs(up[4] * R.D) / (alpha_out * alpha_out) : 0.0);
        for (int ch = 0; ch < 3; ++ch) T_bar_abs += std::fabs(up[ch] * o.bg[ch]);
        const double* Cbar = up;  // dL/dC' per channel
        // reverse over contributors:  C += c' a T ; D += z a T ; T <- T (1 - a)
        for (int64_t i = static_cast<int64_t>(tr.size()) - 1; i >= 0; --i) {
          const Contrib& q = tr[i];
          const Proj<double>& p = B.proj[q.id];
          double cp[3];
          for (int ch = 0; ch < 3; ++ch) {
            cp[ch] = cam.A[ch * 4 + 3];
            for (int k2 = 0; k2 < 3; ++k2) cp[ch] += cam.A[ch * 4 + k2] * p.rgb[k2];
          }
          // T_{i+1} = T_i (1 - a_i)
          double a_bar = -q.T * T_bar;
          double Ti_bar = (1.0 - q.alpha) * T_bar;
          double cdot = Cbar[0] * cp[0] + Cbar[1] * cp[1] + Cbar[2] * cp[2];
          a_bar += cdot * q.T;
          Ti_bar += cdot * q.alpha;
          if (g_mutation != 3) {
            a_bar += D_bar * p.z * q.T;
            Ti_bar += D_bar * p.z * q.alpha;
          }
          double cp_bar[3];
          for (int ch = 0; ch < 3; ++ch) cp_bar[ch] = Cbar[ch] * q.alpha * q.T;
          double z_bar = D_bar * q.alpha * q.T;
          T_bar = Ti_bar;
          // a = min(0.99, araw); araw = o' exp(-sigma)
          double araw_bar = (q.clamped && g_mutation != 1) ? 0.0 : a_bar;
          double op_bar = araw_bar * std::exp(-q.sigma);
          double sig_bar = -araw_bar * q.araw;
          double ca_bar = 0.5 * q.dx * q.dx * sig_bar;
          double cb_bar = q.dx * q.dy * sig_bar;
          double cc_bar = 0.5 * q.dy * q.dy * sig_bar;
          double mx_bar = (p.ca * q.dx + p.cb * q.dy) * sig_bar;
          double my_bar = (p.cc * q.dy + p.cb * q.dx) * sig_bar;
          double rgb_bar[3];
          for (int k2 = 0; k2 < 3; ++k2) {
            rgb_bar[k2] = 0.0;
            for (int ch = 0; ch < 3; ++ch) rgb_bar[k2] += cam.A[ch * 4 + k2] * cp_bar[ch];
          }
          for (int ch = 0; ch < 3; ++ch) {
            for (int k2 = 0; k2 < 3; ++k2) tile_aff[t * 12 + ch * 4 + k2] += cp_bar[ch] * p.rgb[k2];
            tile_aff[t * 12 + ch * 4 + 3] += cp_bar[ch];
          }
          const int64_t pos = q.pos;
          double* pb = pairbuf.data() + (list_off[t] + pos) * G2;
          if (g_mutation == 4) std::swap(ca_bar, cc_bar);
          pb[0] += mx_bar; pb[1] += my_bar; pb[2] += ca_bar; pb[3] += cb_bar; pb[4] += cc_bar;
          pb[5] += op_bar; pb[6] += rgb_bar[0]; pb[7] += rgb_bar[1]; pb[8] += rgb_bar[2];
          pb[9] += z_bar; pb[10] += std::fabs(mx_bar); pb[11] += std::fabs(my_bar);
          if (g_mag) {
            // the same chain with every sum replaced by the sum of its terms' magnitudes
            double cdot_abs = 0.0;
            for (int ch = 0; ch < 3; ++ch) cdot_abs += std::fabs(Cbar[ch] * cp[ch]);
            const double dz_abs = std::fabs(D_bar_abs * p.z);
            const double a_abs = q.T * T_bar_abs + (cdot_abs + dz_abs) * q.T;
            T_bar_abs = (1.0 - q.alpha) * T_bar_abs + (cdot_abs + dz_abs) * q.alpha;
            const double raw_abs = q.clamped ? 0.0 : a_abs;
            const double sig_abs = raw_abs * q.araw;
            double rgb_abs[3];
            for (int k2 = 0; k2 < 3; ++k2) {
              rgb_abs[k2] = 0.0;
              for (int ch = 0; ch < 3; ++ch) rgb_abs[k2] += std::fabs(cam.A[ch * 4 + k2] * Cbar[ch]) * q.alpha * q.T;
            }
            double* pa = pairabs.data() + (list_off[t] + pos) * GM;
            const double v[GM] = {(std::fabs(p.ca * q.dx) + std::fabs(p.cb * q.dy)) * sig_abs,
                                  (std::fabs(p.cc * q.dy) + std::fabs(p.cb * q.dx)) * sig_abs,
                                  0.5 * q.dx * q.dx * sig_abs, std::fabs(q.dx * q.dy) * sig_abs,
                                  0.5 * q.dy * q.dy * sig_abs, raw_abs * std::exp(-q.sigma),
                                  rgb_abs[0], rgb_abs[1], rgb_abs[2], D_bar_abs * q.alpha * q.T};
            for (int j = 0; j < GM; ++j) pa[j] += v[j];
          }
        }
      }
  }
  std::vector<double> g2d(static_cast<size_t>(C) * n * G2, 0.0);
  std::vector<double> g2abs(g_mag ? static_cast<size_t>(C) * n * GM : 0, 0.0);
  for (int64_t t = 0; t < ntiles; ++t)
    for (int64_t k = 0; k < static_cast<int64_t>(B.lists[t].size()); ++k) {
      const int64_t id = B.lists[t][k];
      const double* pb = pairbuf.data() + (list_off[t] + k) * G2;
      for (int j = 0; j < G2; ++j) g2d[id * G2 + j] += pb[j];
      if (g_mag) {
        const double* pa = pairabs.data() + (list_off[t] + k) * GM;
        for (int j = 0; j < GM; ++j) g2abs[id * GM + j] += pa[j];
      }
    }
  if (g_affine) {
    std::fill(g_affine, g_affine + 12 * C, 0.0);
    for (int64_t t = 0; t < ntiles; ++t) {
      int c = 0;
      while (t >= B.tile_off[c + 1]) ++c;
      for (int j = 0; j < 12; ++j) g_affine[12 * c + j] += tile_aff[t * 12 + j];
    }
  }
  if (g2d_out) std::copy(g2d.begin(), g2d.end(), g2d_out);
  // projection and colour: forward-mode derivatives w.r.t. the 11 geometric parameters
  // (mean 3, scale 3, quaternion 4, opacity 1); SH enters linearly.
  using D11 = Dual<11>;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t g = 0; g < n; ++g) {
    double gm[3] = {0, 0, 0}, gs[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, go = 0.0;
    double gsh[48];
    std::fill(gsh, gsh + 48, 0.0);
    double gabs[2] = {0, 0};
    double gemb_acc[kEmbG];
    std::fill(gemb_acc, gemb_acc + kEmbG, 0.0);
    double mag[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, mag_sh[48];
    std::fill(mag_sh, mag_sh + 48, 0.0);
    D11 m[3], sc[3], q[4], op;
    for (int i = 0; i < 3; ++i) m[i] = D11::var(means[3 * g + i], i);
    for (int i = 0; i < 3; ++i) sc[i] = D11::var(scales[3 * g + i], 3 + i);
    for (int i = 0; i < 4; ++i) q[i] = D11::var(quats[4 * g + i], 6 + i);
    op = D11::var(opac[g], 10);
    for (int c = 0; c < C; ++c) {
      if (!B.proj[c * n + g].vis) continue;
      const double* gg = g2d.data() + (c * n + g) * G2;
      double mo[kMlpOut];
      const bool on = mlp_of(s, g, cv[c], mo);
      Proj<D11> p = project<D11>(m, sc, q, op, sh + g * K * 3, K, deg, cv[c], o, on ? mo : nullptr);
      if (!p.vis) continue;
      const D11* outs[10] = {&p.mx, &p.my, &p.ca, &p.cb, &p.cc, &p.op, &p.rgb[0], &p.rgb[1], &p.rgb[2], &p.z};
      double acc[11];
      std::fill(acc, acc + 11, 0.0);
      for (int j = 0; j < 10; ++j)
        for (int k = 0; k < 11; ++k) acc[k] += gg[j] * outs[j]->d[k];
      for (int i = 0; i < 3; ++i) gm[i] += acc[i];
      for (int i = 0; i < 3; ++i) gs[i] += acc[3 + i];
      for (int i = 0; i < 4; ++i) gq[i] += acc[6 + i];
      go += acc[10];
      const int nb = (deg + 1) * (deg + 1);
      for (int ch = 0; ch < 3; ++ch) {
        if (p.flags & (1u << ch)) continue;  // rgb clamped at 0
        const double gain = on ? 2.0 * mo[ch] : 1.0;
        for (int k = 0; k < nb && k < K; ++k) {
          const double sign = (g_mutation == 2 && k >= 4 && k < 9) ? -1.0 : 1.0;
          gsh[k * 3 + ch] += sign * p.Y[k] * gain * gg[6 + ch];
        }
      }
      if (on) {
        // appearance transform: rgb = 2 out[0..2] rgb_pre, op' = (1 - out[3]) op_pre
        double dz[kMlpOut];
        for (int ch = 0; ch < 3; ++ch) dz[ch] = 2.0 * p.rgb_pre[ch] * gg[6 + ch];
        dz[3] = -p.op_pre * gg[5];
        for (int oo = 0; oo < kMlpOut; ++oo) dz[oo] *= mo[oo] * (1.0 - mo[oo]);  // through the sigmoid
        for (int oo = 0; oo < kMlpOut; ++oo) mlp_dz[(static_cast<size_t>(c) * n + g) * kMlpOut + oo] = dz[oo];
        if (g_gemb) {
          double pre[kHid], hid[kHid], out4[kMlpOut];
          mlp_forward(mlp, gemb + kEmbG * g, cv[c].iemb, pre, hid, out4);
          const double* w1 = mlp;
          const double* w2 = mlp + kHid * kMlpIn + kHid;
          for (int k = 0; k < kHid; ++k) {
            if (!(pre[k] > 0.0)) continue;
            double dh = 0.0;
            for (int oo = 0; oo < kMlpOut; ++oo) dh += w2[oo * kHid + k] * dz[oo];
            for (int j = 0; j < kEmbG; ++j) gemb_acc[j] += w1[k * kMlpIn + j] * dh;
          }
        }
      }
      gabs[0] += gg[10];
      gabs[1] += gg[11];
      if (g_mag) {
        // magnitude: the per-pixel contributions' magnitudes through the projection's partials
        // taken as sums of magnitudes (Mag)
        using M11 = Mag<11>;
        M11 mm[3], ms[3], mq[4], mop;
        for (int i = 0; i < 3; ++i) mm[i] = M11::var(means[3 * g + i], i);
        for (int i = 0; i < 3; ++i) ms[i] = M11::var(scales[3 * g + i], 3 + i);
        for (int i = 0; i < 4; ++i) mq[i] = M11::var(quats[4 * g + i], 6 + i);
        mop = M11::var(opac[g], 10);
        Proj<M11> pm = project<M11>(mm, ms, mq, mop, sh + g * K * 3, K, deg, cv[c], o, on ? mo : nullptr);
        const M11* mouts[10] = {&pm.mx, &pm.my, &pm.ca, &pm.cb, &pm.cc, &pm.op, &pm.rgb[0], &pm.rgb[1], &pm.rgb[2],
                                &pm.z};
        const double* ga = g2abs.data() + (c * n + g) * GM;
        for (int j = 0; j < 10; ++j)
          for (int k = 0; k < 11; ++k) mag[k] += ga[j] * mouts[j]->d[k];
        for (int ch = 0; ch < 3; ++ch) {
          if (p.flags & (1u << ch)) continue;
          for (int k = 0; k < nb && k < K; ++k) mag_sh[k * 3 + ch] += std::fabs(p.Y[k]) * ga[6 + ch];
        }
      }
    }
    for (int i = 0; i < 3; ++i) g_means[3 * g + i] = gm[i];
    for (int i = 0; i < 3; ++i) g_scales[3 * g + i] = gs[i];
    for (int i = 0; i < 4; ++i) g_quats[4 * g + i] = gq[i];
    g_opac[g] = go;
    for (int k = 0; k < K * 3; ++k) g_sh[g * K * 3 + k] = (k < 48) ? gsh[k] : 0.0;
    if (g_absgrad) { g_absgrad[2 * g] = gabs[0]; g_absgrad[2 * g + 1] = gabs[1]; }
    if (g_gemb && mlp_on)
      for (int j = 0; j < kEmbG; ++j) g_gemb[kEmbG * g + j] = gemb_acc[j];
    if (g_mag) {
      double* out = g_mag + static_cast<size_t>(g) * (11 + 3 * K);
      for (int k = 0; k < 11; ++k) out[k] = mag[k];
      for (int k = 0; k < K * 3; ++k) out[11 + k] = (k < 48) ? mag_sh[k] : 0.0;
    }
  }
  if (mlp_on && (g_mlp || g_iemb)) {
    // weights and image embeddings: sums over every visible (camera, Gaussian)
    std::vector<double> gw(kMlpParams, 0.0), gi(static_cast<size_t>(C) * kEmbI, 0.0);
    const double* w1 = mlp;
    const double* w2 = mlp + kHid * kMlpIn + kHid;
    for (int c = 0; c < C; ++c)
      for (int64_t g = 0; g < n; ++g) {
        const double* dz = mlp_dz.data() + (static_cast<size_t>(c) * n + g) * kMlpOut;
        if (dz[0] == 0.0 && dz[1] == 0.0 && dz[2] == 0.0 && dz[3] == 0.0) continue;
        double pre[kHid], hid[kHid], out4[kMlpOut];
        mlp_forward(mlp, gemb + kEmbG * g, cv[c].iemb, pre, hid, out4);
        double* gw1 = gw.data();
        double* gb1 = gw1 + kHid * kMlpIn;
        double* gw2 = gb1 + kHid;
        double* gb2 = gw2 + kMlpOut * kHid;
        for (int oo = 0; oo < kMlpOut; ++oo) {
          gb2[oo] += dz[oo];
          for (int k = 0; k < kHid; ++k) gw2[oo * kHid + k] += dz[oo] * hid[k];
        }
        for (int k = 0; k < kHid; ++k) {
          if (!(pre[k] > 0.0)) continue;
          double dh = 0.0;
          for (int oo = 0; oo < kMlpOut; ++oo) dh += w2[oo * kHid + k] * dz[oo];
          gb1[k] += dh;
          for (int j = 0; j < kEmbG; ++j) gw1[k * kMlpIn + j] += dh * gemb[kEmbG * g + j];
          for (int j = 0; j < kEmbI; ++j) {
            gw1[k * kMlpIn + kEmbG + j] += dh * cv[c].iemb[j];
            gi[static_cast<size_t>(c) * kEmbI + j] += dh * w1[k * kMlpIn + kEmbG + j];
          }
        }
      }
    if (g_mlp) std::copy(gw.begin(), gw.end(), g_mlp);
    if (g_iemb) std::copy(gi.begin(), gi.end(), g_iemb);
  }
  return 0;
}

// Real SH basis at unit directions dirs[m][3] (degree <= 3): out[m][16].
int oracle_sh_basis(int64_t m, const double* dirs, int deg, double* out) {
  if (deg < 0 || deg > 3) return -1;
  for (int64_t i = 0; i < m; ++i) {
    double Y[16];
    std::fill(Y, Y + 16, 0.0);
    sh_basis<double>(deg, dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], Y);
    std::copy(Y, Y + 16, out + 16 * i);
  }
  return 0;
}

// Sec. 3.4.2: partition-level detail-level selection.
//   aabb[P][6] = xmin, ymin, zmin, xmax, ymax, zmax (world)
//   level_offsets[L][P+1]: Gaussians of partition p at level l are
//                          [level_offsets[l][p], level_offsets[l][p+1]) of the concatenated arrays
//   thresholds[L-1] ascending: distance < thresholds[0] -> level L-1 (finest) ... else level 0
//   budget <= 0: no budget. Over budget: repeatedly lower by one level the farthest partition
//   (ties: larger index) that is above level 0.
//   Outputs: level_out[P] (-1 = culled), segs_out[P][2] (begin, count), *nsegs, *n_sel.
// Returns 0, 1 when still over budget with every visible partition at level 0, -1 on bad input.
int oracle_select_lod(int P, const double* aabb, int L, const int64_t* level_offsets,
                      const double* cam_row, const double* thresholds, int64_t budget,
                      int32_t* level_out, int64_t* segs_out, int32_t* nsegs, int64_t* n_sel) {
  if (P < 0 || L < 1 || !cam_row) return -1;
  CamD cam = load_cam(cam_row, nullptr);
  std::vector<double> dist(P, 0.0);
  std::vector<int> lev(P, -1);
  for (int p = 0; p < P; ++p) {
    const double* b = aabb + 6 * p;
    // culled iff some frustum half-space has all 8 corners strictly outside
    bool culled = false;
    for (int plane = 0; plane < 6 && !culled; ++plane) {
      bool all_out = true;
      for (int corner = 0; corner < 8 && all_out; ++corner) {
        double w[3] = {b[(corner & 1) ? 3 : 0], b[(corner & 2) ? 4 : 1], b[(corner & 4) ? 5 : 2]};
        double x = cam.t[0], y = cam.t[1], z = cam.t[2];
        for (int k = 0; k < 3; ++k) {
          x += cam.R[0 * 3 + k] * w[k];
          y += cam.R[1 * 3 + k] * w[k];
          z += cam.R[2 * 3 + k] * w[k];
        }
        bool out;
        switch (plane) {
          case 0: out = z < cam.znear; break;
          case 1: out = z > cam.zfar; break;
          case 2: out = cam.fx * x + cam.cx * z < 0.0; break;            // u < 0
          case 3: out = cam.fx * x + (cam.cx - cam.W) * z > 0.0; break;  // u > W
          case 4: out = cam.fy * y + cam.cy * z < 0.0; break;            // v < 0
          default: out = cam.fy * y + (cam.cy - cam.H) * z > 0.0; break; // v > H
        }
        all_out = all_out && out;
      }
      culled = all_out;
    }
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      double q = std::clamp(cam.center[k], b[k], b[3 + k]);
      d2 += (cam.center[k] - q) * (cam.center[k] - q);
    }
    dist[p] = std::sqrt(d2);
    if (culled) continue;
    int l = 0;
    for (int k = 0; k < L - 1; ++k)
      if (dist[p] < thresholds[k]) { l = L - 1 - k; break; }
    lev[p] = l;
  }
  auto count = [&](int p, int l) { return level_offsets[static_cast<int64_t>(l) * (P + 1) + p + 1] -
                                          level_offsets[static_cast<int64_t>(l) * (P + 1) + p]; };
  int64_t total = 0;
  for (int p = 0; p < P; ++p)
    if (lev[p] >= 0) total += count(p, lev[p]);
  int status = 0;
  if (budget > 0) {
    while (total > budget) {
      int pick = -1;
      for (int p = 0; p < P; ++p) {
        if (lev[p] <= 0) continue;
        if (pick < 0 || dist[p] > dist[pick] || (dist[p] == dist[pick] && p > pick)) pick = p;
      }
      if (pick < 0) { status = 1; break; }
      total -= count(pick, lev[pick]);
      lev[pick] -= 1;
      total += count(pick, lev[pick]);
    }
  }
  int ns = 0;
  for (int p = 0; p < P; ++p) {
    level_out[p] = lev[p];
    if (lev[p] < 0) continue;
    int64_t cnt = count(p, lev[p]);
    if (cnt <= 0) continue;
    segs_out[2 * ns] = level_offsets[static_cast<int64_t>(lev[p]) * (P + 1) + p];
    segs_out[2 * ns + 1] = cnt;
    ++ns;
  }
  *nsegs = ns;
  *n_sel = total;
  return status;
}

// Sets the test switch above (0 restores the correct gradients); returns the previous value.
int oracle_set_mutation(int k) {
  const int prev = g_mutation;
  g_mutation = k;
  return prev;
}

int oracle_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_num_threads(int k) {
#ifdef _OPENMP
  if (k > 0) omp_set_num_threads(k);
#else
  (void)k;
#endif
}

}  // extern "C"
