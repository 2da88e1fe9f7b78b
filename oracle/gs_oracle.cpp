// FP64 CPU oracle of the tile-based differentiable 3D-Gaussian rasterizer.
//
// TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline leg
// of the benchmark may load this library. The product path never calls it.
// It shares no code, header or constant table with the CUDA library.
//
// What the paper fixes and what is read into it
// ---------------------------------------------
// The paper represents the map as 3D Gaussians with a mean, a covariance and an
// opacity (Sec. II-A) rendered by a GPU splatting renderer that the mapping
// optimiser differentiates (Fig. 3, renders I1 and I2; Sec. II-B "splat-wise
// back-propagation"). It never writes the renderer out. This file takes the
// standard EWA-splatting reading of it:
//   * Sigma  = Rq diag(exp(2 s)) Rq^T with Rq from the normalised (w,x,y,z) quaternion;
//   * Sigma2 = J W Sigma W^T J^T + 0.3 I with J the perspective Jacobian whose
//     x/z, y/z arguments are clamped to 1.3 * half the field of view;
//   * conic  = Sigma2^-1; opacity = sigmoid(logit); colour = stored RGB;
//   * per pixel centre (i+0.5, j+0.5), front to back over the tile's depth-sorted list:
//       power = -0.5 d^T conic d (d = mean2D - pixel), skip if power > 0;
//       alpha = min(0.99, o exp(power)), skip if alpha < 1/255;
//       stop before a Gaussian whose T (1 - alpha) < 1e-4;
//       C += c alpha T, D += z alpha T, T *= 1 - alpha.
//
// Parity structure
// ----------------
// 1. orc_project_mirror: the FP32 "discrete mirror". It evaluates, in binary32
//    with a fixed operation order, exactly the quantities that decide integers:
//    the camera depth (sort key), the culls, the pixel radius, the tile
//    rectangle and, row by row, the tiles of the rectangle that the widened
//    alpha >= 1/255 ellipse meets. Both this mirror and the CUDA projection follow one written
//    operation order (the library header documents it), so keys, order and
//    ranges can be compared bit for bit.
// 2. orc_bin: pair emission in (view, Gaussian) order, std::stable_sort by the
//    64-bit key, per-tile [start, end) ranges.
// 3. orc_render_fwd / orc_render_bwd / orc_project_bwd: every continuous quantity
//    is recomputed in FP64 from the (exactly dequantised) stored inputs, over the
//    discrete lists of step 2. The backward pass is hand-derived reverse mode.
//
// Build: g++ -O2 -std=c++17 -fopenmp -ffp-contract=off -fPIC -shared
// (-ffp-contract=off keeps the FP32 mirror's a*b+c from being fused).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- constants (method readings)
constexpr double kDilation = 0.3;          // added to the 2D covariance diagonal (px^2)
constexpr double kJacClamp = 1.3;          // J's x/z, y/z clamped to 1.3 * tan(half FoV)
constexpr double kAlphaMax = 0.99;         // opacity clamp
constexpr double kAlphaMin = 1.0 / 255.0;  // skip threshold
constexpr double kTStop = 1e-4;            // transmittance stop threshold

// ================================================================= FP32 discrete mirror
//
// Deterministic binary32 exponential: Cody & Waite (1980) additive range reduction
// x = k ln2 + r with ln2 split in a 16-bit head and a tail, then the degree-7
// Taylor polynomial of e^r by Horner's rule with fused multiply-adds, scaled by 2^k.
// It is used only so that the scale exp(s) entering the radius and rectangle is
// the same binary32 number on both sides of the parity test.
float expdet(float x) {
  if (x != x) return x;
  x = (x < -80.0f) ? -80.0f : ((x > 80.0f) ? 80.0f : x);
  const float kf = std::rint(x * 0x1.715476p+0f);  // nearest binary32 of log2(e)
  float r = std::fma(-kf, 0x1.62e4p-1f, x);         // ln2 head (exact product)
  r = std::fma(-kf, 0x1.7f7d1cp-20f, r);            // ln2 tail
  float p = 0x1.a01a02p-13f;                        // 1/7!
  p = std::fma(p, r, 0x1.6c16c2p-10f);              // 1/6!
  p = std::fma(p, r, 0x1.111112p-7f);               // 1/5!
  p = std::fma(p, r, 0x1.555556p-5f);               // 1/4!
  p = std::fma(p, r, 0x1.555556p-3f);               // 1/3!
  p = std::fma(p, r, 0x1p-1f);                      // 1/2!
  p = std::fma(p, r, 1.0f);
  p = std::fma(p, r, 1.0f);
  const int k = static_cast<int>(kf);
  const uint32_t bits = static_cast<uint32_t>(k + 127) << 23;
  float scale;
  std::memcpy(&scale, &bits, 4);
  return p * scale;
}

// Deterministic binary32 natural logarithm of a positive normal x: x = m 2^e with m in
// [sqrt(1/2), sqrt(2)), ln m = 2 atanh(s) with s = (m - 1)/(m + 1), the atanh series to
// s^9 by Horner's rule, and e ln2 added with the same head / tail split of ln2 as expdet.
float logdet(float x) {
  if (!(x > 0.0f) || !std::isfinite(x)) return x > 0.0f ? x : -INFINITY;
  uint32_t bits;
  std::memcpy(&bits, &x, 4);
  if ((bits >> 23) == 0) return -INFINITY;  // subnormal: far below any level the mirror uses
  int e = static_cast<int>(bits >> 23) - 127;
  const uint32_t mb = (bits & 0x7fffffu) | 0x3f800000u;
  float m;
  std::memcpy(&m, &mb, 4);
  if (m > 0x1.6a09e6p+0f) {  // sqrt(2)
    m = m * 0.5f;
    e += 1;
  }
  const float s = (m - 1.0f) / (m + 1.0f);
  const float s2 = s * s;
  float p = 0x1.c71c72p-4f;             // 1/9
  p = std::fma(p, s2, 0x1.24924ap-3f);  // 1/7
  p = std::fma(p, s2, 0x1.99999ap-3f);  // 1/5
  p = std::fma(p, s2, 0x1.555556p-2f);  // 1/3
  p = std::fma(p, s2, 1.0f);
  const float lm = (2.0f * s) * p;
  const float ef = static_cast<float>(e);
  return std::fma(ef, 0x1.62e4p-1f, std::fma(ef, 0x1.7f7d1cp-20f, lm));
}

// The ellipse of a projected Gaussian inside which its opacity can reach 1/255, widened by
// a safety margin, as the discrete mirror evaluates it: E = {d : d^T Sigma2^-1 d <= kap}
// with kap = 2 (ln(255 o) + 0.02 |ln(255 o)| + 1.5e-4). Stored: the mean (u, v), Sigma2's
// off-diagonal b, 1 / c (c: Sigma2's yy entry), sqrt(det Sigma2), the half-extents
// hx = sqrt(kap a), hy = sqrt(kap c), and kxy = b / a (the y offset, per unit x offset, of
// E's leftmost / rightmost points).
struct Ellipse {
  float u, v, b, inv_c, sdet, hx, hy, kxy;
};

// Tile columns [*xa, *xb] of tile row ty whose pixel centres' square, widened by
// 0.05 px + 0.2% of the half-extent, meets E; clamped to [x0, x1). *xa > *xb: none.
// E's part inside the row's (widened) strip of pixel-centre rows is convex; its x-extent
// ends at E's leftmost / rightmost point when that lies inside the strip, else where E's
// boundary crosses the strip edge on that point's side.
void row_span(const Ellipse& E, int ty, int x0, int x1, int tile, int* xa, int* xb) {
  *xa = 1;
  *xb = 0;
  const float tf = static_cast<float>(tile);
  const float mgx = std::fma(0.002f, E.hx, 0.05f);
  const float mgy = std::fma(0.002f, E.hy, 0.05f);
  const float y_lo = static_cast<float>(ty) * tf;
  const float Y0 = (y_lo + 0.5f) - mgy;
  const float Y1 = (y_lo + (tf - 0.5f)) + mgy;
  if (E.v + E.hy < Y0 || E.v - E.hy > Y1) return;
  auto cross = [&](float Ye, float sgn) {
    const float dye = Ye - E.v;
    const float ad = std::fabs(dye);
    const float w = std::sqrt(std::fmax((E.hy - ad) * (E.hy + ad), 0.0f));
    return E.u + std::fma(sgn * E.sdet, w, E.b * dye) * E.inv_c;
  };
  const float yR = std::fma(E.kxy, E.hx, E.v);
  const float yL = std::fma(-E.kxy, E.hx, E.v);
  const float xr = (yR >= Y0 && yR <= Y1) ? E.u + E.hx : (yR > Y1 ? cross(Y1, 1.0f) : cross(Y0, 1.0f));
  const float xl = (yL >= Y0 && yL <= Y1) ? E.u - E.hx : (yL > Y1 ? cross(Y1, -1.0f) : cross(Y0, -1.0f));
  const float inv_t = 1.0f / tf;
  float fa = std::ceil(((xl - mgx) - (tf - 0.5f)) * inv_t);
  float fb = std::floor(((xr + mgx) - 0.5f) * inv_t);
  fa = std::fmax(fa, static_cast<float>(x0));
  fb = std::fmin(fb, static_cast<float>(x1 - 1));
  if (!(fa <= fb)) return;
  *xa = static_cast<int>(fa);
  *xb = static_cast<int>(fb);
}

struct MirrorOut {
  bool valid;
  float zc, u, v;
  int radius;
  int x0, x1, y0, y1;
  uint32_t count;  // tiles of the rectangle whose row span meets the ellipse
  Ellipse E;
};

// The FP32 operation order below is the contract shared with the CUDA projection.
MirrorOut mirror_one(const float* p, const float* ls, const float* q, float logit, const float* cam,
                     int W, int H, int tile, float near) {
  MirrorOut o{};
  o.valid = false;
  const float fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3];
  const float* R = cam + 4;
  const float* t = cam + 13;
  // 1. camera-space position
  const float xc = std::fma(R[0], p[0], std::fma(R[1], p[1], std::fma(R[2], p[2], t[0])));
  const float yc = std::fma(R[3], p[0], std::fma(R[4], p[1], std::fma(R[5], p[2], t[1])));
  const float zc = std::fma(R[6], p[0], std::fma(R[7], p[1], std::fma(R[8], p[2], t[2])));
  o.zc = zc;
  if (!(zc > near)) return o;
  // 2. normalised quaternion
  const float n2 = std::fma(q[0], q[0], std::fma(q[1], q[1], std::fma(q[2], q[2], q[3] * q[3])));
  const float nq = std::sqrt(n2);
  if (!(nq > 0.0f)) return o;
  const float w = q[0] / nq, x = q[1] / nq, y = q[2] / nq, z = q[3] / nq;
  // 3. rotation matrix
  const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
  const float wx = w * x, wy = w * y, wz = w * z;
  float Q[3][3];
  Q[0][0] = 1.0f - 2.0f * (yy + zz); Q[0][1] = 2.0f * (xy - wz); Q[0][2] = 2.0f * (xz + wy);
  Q[1][0] = 2.0f * (xy + wz); Q[1][1] = 1.0f - 2.0f * (xx + zz); Q[1][2] = 2.0f * (yz - wx);
  Q[2][0] = 2.0f * (xz - wy); Q[2][1] = 2.0f * (yz + wx); Q[2][2] = 1.0f - 2.0f * (xx + yy);
  // 4. scaled axes M = Q diag(exp(s))
  const float S[3] = {expdet(ls[0]), expdet(ls[1]), expdet(ls[2])};
  float M[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i][j] = Q[i][j] * S[j];
  // 5. rotate into the camera frame: Nm = R M
  float Nm[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      Nm[i][j] = std::fma(R[3 * i + 0], M[0][j], std::fma(R[3 * i + 1], M[1][j], R[3 * i + 2] * M[2][j]));
  // 6. clamped perspective Jacobian
  const float xz_ = xc / zc, yz_ = yc / zc;
  const float limx = 1.3f * ((0.5f * static_cast<float>(W)) / fx);
  const float limy = 1.3f * ((0.5f * static_cast<float>(H)) / fy);
  const float txz = std::fmin(std::fmax(xz_, -limx), limx);
  const float tyz = std::fmin(std::fmax(yz_, -limy), limy);
  const float j00 = fx / zc, j02 = -(j00 * txz);
  const float j11 = fy / zc, j12 = -(j11 * tyz);
  // 7. m = J Nm (2x3); Sigma2 = m m^T + 0.3 I
  float m1[3], m2[3];
  for (int j = 0; j < 3; ++j) {
    m1[j] = std::fma(j00, Nm[0][j], j02 * Nm[2][j]);
    m2[j] = std::fma(j11, Nm[1][j], j12 * Nm[2][j]);
  }
  // 8. entries and determinant (Lagrange identity: |m1|^2|m2|^2 - (m1.m2)^2 = |m1 x m2|^2)
  const float aa = std::fma(m1[0], m1[0], std::fma(m1[1], m1[1], m1[2] * m1[2]));
  const float cc = std::fma(m2[0], m2[0], std::fma(m2[1], m2[1], m2[2] * m2[2]));
  const float bb = std::fma(m1[0], m2[0], std::fma(m1[1], m2[1], m1[2] * m2[2]));
  const float a = aa + 0.3f, c = cc + 0.3f;
  const float k0 = std::fma(m1[1], m2[2], -(m1[2] * m2[1]));
  const float k1 = std::fma(m1[2], m2[0], -(m1[0] * m2[2]));
  const float k2 = std::fma(m1[0], m2[1], -(m1[1] * m2[0]));
  const float det = (std::fma(k0, k0, std::fma(k1, k1, k2 * k2)) + 0.3f * (aa + cc)) + 0.09f;
  if (!(det > 0.0f)) return o;
  // 9. largest eigenvalue and 3-sigma radius
  const float mid = 0.5f * (a + c);
  const float hd = 0.5f * (a - c);
  const float disc = std::fmax(std::fma(hd, hd, bb * bb), 0.1f);
  const float lmax = mid + std::sqrt(disc);
  const float rf = std::fmin(std::ceil(3.0f * std::sqrt(lmax)), 1048576.0f);
  if (!(rf == rf)) return o;
  // 10. projected mean
  const float u = std::fma(fx, xz_, cx);
  const float v = std::fma(fy, yz_, cy);
  if (!std::isfinite(u) || !std::isfinite(v)) return o;
  o.u = u;
  o.v = v;
  // 11. tiles whose square meets [u-r, u+r] x [v-r, v+r]
  const float inv_tile = 1.0f / static_cast<float>(tile);
  const float Tx = static_cast<float>((W + tile - 1) / tile);
  const float Ty = static_cast<float>((H + tile - 1) / tile);
  const float x0f = std::fmin(std::fmax(std::floor((u - rf) * inv_tile), 0.0f), Tx);
  const float x1f = std::fmin(std::fmax(std::floor((u + rf) * inv_tile) + 1.0f, 0.0f), Tx);
  const float y0f = std::fmin(std::fmax(std::floor((v - rf) * inv_tile), 0.0f), Ty);
  const float y1f = std::fmin(std::fmax(std::floor((v + rf) * inv_tile) + 1.0f, 0.0f), Ty);
  o.radius = static_cast<int>(rf);
  o.x0 = static_cast<int>(x0f);
  o.x1 = static_cast<int>(x1f);
  o.y0 = static_cast<int>(y0f);
  o.y1 = static_cast<int>(y1f);
  o.valid = (o.x1 - o.x0) * (o.y1 - o.y0) > 0;
  if (!o.valid) return o;
  // 12. opacity level and the widened ellipse; tiles per row of the rectangle
  const float ee = expdet(-logit);
  const float op = 1.0f / (1.0f + ee);
  const float L = logdet(255.0f * op);
  const float Lm = (L + 0.02f * std::fabs(L)) + 1.5e-4f;
  if (!(Lm >= 0.0f)) return o;  // the opacity never reaches 1/255: no pairs
  const float kap = 2.0f * Lm;
  o.E = Ellipse{u, v, bb, 1.0f / c, std::sqrt(det), std::sqrt(kap * a), std::sqrt(kap * c), bb / a};
  uint32_t cnt = 0;
  for (int ty = o.y0; ty < o.y1; ++ty) {
    int xa, xb;
    row_span(o.E, ty, o.x0, o.x1, tile, &xa, &xb);
    if (xa <= xb) cnt += static_cast<uint32_t>(xb - xa + 1);
  }
  o.count = cnt;
  return o;
}

// ================================================================= FP64 geometry
struct Proj64 {
  double pc[3];      // camera-space mean
  double u, v;       // projected mean (pixels)
  double A, B, C;    // conic = Sigma2^-1 entries (0,0), (0,1), (1,1)
  double a, b, c;    // Sigma2 entries
  double o;          // opacity
  double rgb[3];
  double J[2][3];    // clamped Jacobian
  bool clampx, clampy;
  double Rq[3][3], S[3], qhat[4], qnorm;
  double Sigma[3][3];
};

void quat_to_rot(const double q[4], double R[3][3]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}

// Plain definition of the projection (Sec. II-A reading), every step in double.
Proj64 project64(const double* p, const double* ls, const double* q, double logit, const double* rgb,
                 const double* cam, int W, int H) {
  Proj64 P{};
  const double fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3];
  const double* R = cam + 4;
  const double* t = cam + 13;
  for (int i = 0; i < 3; ++i) P.pc[i] = R[3 * i] * p[0] + R[3 * i + 1] * p[1] + R[3 * i + 2] * p[2] + t[i];
  const double x = P.pc[0], y = P.pc[1], z = P.pc[2];
  P.qnorm = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int i = 0; i < 4; ++i) P.qhat[i] = q[i] / P.qnorm;
  quat_to_rot(P.qhat, P.Rq);
  for (int j = 0; j < 3; ++j) P.S[j] = std::exp(ls[j]);
  // Sigma = Rq S S Rq^T
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += P.Rq[i][k] * P.S[k] * P.S[k] * P.Rq[j][k];
      P.Sigma[i][j] = s;
    }
  // clamped Jacobian
  const double limx = kJacClamp * (0.5 * W / fx), limy = kJacClamp * (0.5 * H / fy);
  double txz = x / z, tyz = y / z;
  P.clampx = (txz < -limx) || (txz > limx);
  P.clampy = (tyz < -limy) || (tyz > limy);
  txz = std::min(std::max(txz, -limx), limx);
  tyz = std::min(std::max(tyz, -limy), limy);
  P.J[0][0] = fx / z; P.J[0][1] = 0; P.J[0][2] = -fx * txz / z;
  P.J[1][0] = 0; P.J[1][1] = fy / z; P.J[1][2] = -fy * tyz / z;
  // T = J R (2x3); Sigma2 = T Sigma T^T + 0.3 I
  double T[2][3];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) T[i][j] = P.J[i][0] * R[j] + P.J[i][1] * R[3 + j] + P.J[i][2] * R[6 + j];
  double S2[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) s += T[i][k] * P.Sigma[k][l] * T[j][l];
      S2[i][j] = s;
    }
  P.a = S2[0][0] + kDilation;
  P.b = S2[0][1];
  P.c = S2[1][1] + kDilation;
  const double det = P.a * P.c - P.b * P.b;
  P.A = P.c / det;
  P.B = -P.b / det;
  P.C = P.a / det;
  P.u = fx * x / z + cx;
  P.v = fy * y / z + cy;
  P.o = 1.0 / (1.0 + std::exp(-logit));
  for (int i = 0; i < 3; ++i) P.rgb[i] = rgb[i];
  return P;
}


// ================================================================= per-pixel compositing
struct PixelResult {
  double rgb[3], depth, T;
  int last;        // 1 + list position of the last composited Gaussian (0 if none)
  int evals;       // list entries examined, including the one that stops the pixel
  int n_near;      // decisions taken within the guard band of a threshold
  int first_near;  // list position of the first such decision (-1 if none)
};

struct Guard {
  double alpha, T, power;  // relative half-widths of the bands around 1/255, 1e-4 and 0
};

struct Contrib {  // one composited Gaussian of a pixel, as the backward pass needs it
  uint32_t g;
  double alpha, T, G, dx, dy;
  bool clamped;
};

// Front-to-back compositing of one pixel over its tile's sorted list (Sec. II-A reading).
// view: the FP64 projections of this view, indexed by Gaussian id.
// flip_at >= 0 inverts the near-threshold decision taken at that list position.
// zmax: depth of an external surface at the pixel (+inf: none). The list is in depth order, so
// the first Gaussian at or behind it ends the pixel (it is not composited).
PixelResult walk_pixel(const Proj64* view, const uint32_t* vals, uint32_t start, uint32_t end, double px,
                       double py, const Guard& gd, int flip_at, std::vector<Contrib>* trace,
                       double zmax = INFINITY) {
  PixelResult r{};
  r.first_near = -1;
  double T = 1.0;
  auto near_decision = [&](int pos, bool& decision, bool& flip_here) {
    ++r.n_near;
    if (r.first_near < 0) r.first_near = pos;
    if (flip_here) {
      decision = !decision;
      flip_here = false;
    }
  };
  for (uint32_t i = start; i < end; ++i) {
    const int pos = static_cast<int>(i - start);
    const uint32_t g = vals[i];
    const Proj64& P = view[g];
    bool flip_here = (pos == flip_at);
    if (std::isfinite(zmax)) {
      bool behind = P.pc[2] >= zmax;  // decision 0: the external surface occludes the rest
      if (std::fabs(P.pc[2] / zmax - 1.0) <= 1e-6) near_decision(pos, behind, flip_here);
      if (behind) break;
    }
    ++r.evals;
    const double dx = P.u - px, dy = P.v - py;
    const double power = -0.5 * (P.A * dx * dx + P.C * dy * dy) - P.B * dx * dy;
    const double mag = 0.5 * (std::fabs(P.A) * dx * dx + std::fabs(P.C) * dy * dy) + std::fabs(P.B * dx * dy);
    bool skip = power > 0.0;  // decision 1
    if (std::fabs(power) <= gd.power * mag) near_decision(pos, skip, flip_here);
    if (skip) continue;
    const double G = std::exp(power);
    const bool clamped = P.o * G > kAlphaMax;
    const double alpha = clamped ? kAlphaMax : P.o * G;
    skip = alpha < kAlphaMin;  // decision 2
    if (std::fabs(alpha / kAlphaMin - 1.0) <= gd.alpha) near_decision(pos, skip, flip_here);
    if (skip) continue;
    const double Tn = T * (1.0 - alpha);
    bool stop = Tn < kTStop;  // decision 3
    if (std::fabs(Tn / kTStop - 1.0) <= gd.T) near_decision(pos, stop, flip_here);
    if (stop) break;
    const double w = alpha * T;
    for (int ch = 0; ch < 3; ++ch) r.rgb[ch] += P.rgb[ch] * w;
    r.depth += P.pc[2] * w;
    if (trace) trace->push_back(Contrib{g, alpha, T, G, dx, dy, clamped});
    T = Tn;
    r.last = pos + 1;
  }
  r.T = T;
  return r;
}

inline int tiles_x(int W, int tile) { return (W + tile - 1) / tile; }
inline int tiles_y(int H, int tile) { return (H + tile - 1) / tile; }

std::vector<Proj64> project_all(int64_t N, const double* means, const double* log_scales, const double* quats,
                                const double* logits, const double* rgb, int K, const double* cams, int W, int H) {
  std::vector<Proj64> pr(static_cast<size_t>(K) * N);
#pragma omp parallel for schedule(static)
  for (int64_t kg = 0; kg < static_cast<int64_t>(K) * N; ++kg) {
    const int64_t k = kg / N, g = kg % N;
    pr[kg] = project64(means + 3 * g, log_scales + 3 * g, quats + 4 * g, logits[g], rgb + 3 * g, cams + 16 * k, W, H);
  }
  return pr;
}

// 3x3 helpers for the backward chain
using M3 = double[3][3];

void cross3(const double a[3], const double b[3], double out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

}  // namespace

extern "C" {

// Deterministic binary32 exp used by the discrete mirror (exposed for its pin tests).
void orc_expdet_f32(const float* x, float* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = expdet(x[i]);
}

// Deterministic binary32 log used by the discrete mirror (exposed for its pin tests).
void orc_logdet_f32(const float* x, float* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = logdet(x[i]);
}

// FP32 discrete mirror over K views x N Gaussians. Outputs per (k, g), index k*N+g:
// depth_bits (binary32 bits of the camera depth), radius, rect[4] = x0,x1,y0,y1
// (tile indices, half-open), count = tiles emitted (0 = culled), uv = binary32 mean2D,
// ell[8] = the widened ellipse (u, v, b, 1/c, sqrt det, hx, hy, kxy; zeros when count = 0).
void orc_project_mirror(int64_t N, const float* means, const float* log_scales, const float* quats,
                        const float* logits, int K, const float* cams, int W, int H, int tile, float near,
                        uint32_t* depth_bits, int32_t* radius, int32_t* rect, uint32_t* count, float* uv,
                        float* ell) {
#pragma omp parallel for schedule(static)
  for (int64_t kg = 0; kg < static_cast<int64_t>(K) * N; ++kg) {
    const int64_t k = kg / N, g = kg % N;
    const MirrorOut m = mirror_one(means + 3 * g, log_scales + 3 * g, quats + 4 * g, logits[g], cams + 16 * k, W, H,
                                   tile, near);
    uint32_t bits;
    std::memcpy(&bits, &m.zc, 4);
    depth_bits[kg] = bits;
    radius[kg] = m.valid ? m.radius : 0;
    rect[4 * kg + 0] = m.valid ? m.x0 : 0;
    rect[4 * kg + 1] = m.valid ? m.x1 : 0;
    rect[4 * kg + 2] = m.valid ? m.y0 : 0;
    rect[4 * kg + 3] = m.valid ? m.y1 : 0;
    count[kg] = m.valid ? m.count : 0u;
    uv[2 * kg + 0] = m.u;
    uv[2 * kg + 1] = m.v;
    const Ellipse E = (m.valid && m.count) ? m.E : Ellipse{};
    const float e8[8] = {E.u, E.v, E.b, E.inv_c, E.sdet, E.hx, E.hy, E.kxy};
    for (int i = 0; i < 8; ++i) ell[8 * kg + i] = e8[i];
  }
}

// FP64 projection of every (view, Gaussian): out [K*N, 8] = u, v, A, B, C, z, opacity, det(Sigma2).
void orc_project64(int64_t N, const double* means, const double* log_scales, const double* quats,
                   const double* logits, const double* rgb, int K, const double* cams, int W, int H, double* out) {
  const std::vector<Proj64> pr = project_all(N, means, log_scales, quats, logits, rgb, K, cams, W, H);
  for (int64_t kg = 0; kg < static_cast<int64_t>(K) * N; ++kg) {
    const Proj64& P = pr[kg];
    double* o = out + 8 * kg;
    o[0] = P.u;
    o[1] = P.v;
    o[2] = P.A;
    o[3] = P.B;
    o[4] = P.C;
    o[5] = P.pc[2];
    o[6] = P.o;
    o[7] = P.a * P.c - P.b * P.b;
  }
}

// Pair emission in increasing (k, g) order, row by row through each rectangle, in each
// row the columns of its span (row_span); key = (global tile id << 32) | depth bits,
// value = g; std::stable_sort by key keeps equal keys in emission order.
// ranges[t] = [start, end) of global tile t (empty = [0,0)). Returns P (the number of
// pairs), or -1 if P > capacity (nothing written then).
int64_t orc_bin(int64_t N, int K, int W, int H, int tile, const uint32_t* count, const int32_t* rect,
                const float* ell, const uint32_t* depth_bits, int64_t capacity, uint64_t* keys, uint32_t* vals,
                uint32_t* ranges) {
  const int Tx = tiles_x(W, tile), Ty = tiles_y(H, tile);
  int64_t P = 0;
  for (int64_t kg = 0; kg < static_cast<int64_t>(K) * N; ++kg) P += count[kg];
  if (P > capacity) return -1;
  std::vector<uint64_t> k_emit(P);
  std::vector<uint32_t> v_emit(P);
  int64_t o = 0;
  for (int64_t kg = 0; kg < static_cast<int64_t>(K) * N; ++kg) {
    if (!count[kg]) continue;
    const int64_t k = kg / N, g = kg % N;
    const int32_t* r = rect + 4 * kg;
    const float* e = ell + 8 * kg;
    const Ellipse E{e[0], e[1], e[2], e[3], e[4], e[5], e[6], e[7]};
    for (int ty = r[2]; ty < r[3]; ++ty) {
      int xa, xb;
      row_span(E, ty, r[0], r[1], tile, &xa, &xb);
      for (int tx = xa; tx <= xb; ++tx) {
        const uint64_t tid = static_cast<uint64_t>(k) * Tx * Ty + static_cast<uint64_t>(ty) * Tx + tx;
        k_emit[o] = (tid << 32) | depth_bits[kg];
        v_emit[o] = static_cast<uint32_t>(g);
        ++o;
      }
    }
  }
  if (o != P) return -1;  // the spans disagree with the counts (cannot happen)
  std::vector<int64_t> idx(P);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return k_emit[a] < k_emit[b]; });
  for (int64_t i = 0; i < P; ++i) {
    keys[i] = k_emit[idx[i]];
    vals[i] = v_emit[idx[i]];
  }
  const int64_t nt = static_cast<int64_t>(K) * Tx * Ty;
  for (int64_t t = 0; t < 2 * nt; ++t) ranges[t] = 0;
  for (int64_t i = 0; i < P; ++i) {
    const uint64_t t = keys[i] >> 32;
    if (i == 0 || (keys[i - 1] >> 32) != t) ranges[2 * t] = static_cast<uint32_t>(i);
    if (i == P - 1 || (keys[i + 1] >> 32) != t) ranges[2 * t + 1] = static_cast<uint32_t>(i + 1);
  }
  return P;
}

// FP64 forward render of K views over the discrete lists (vals, ranges).
// Images: rgb [K,3,H,W]; depth, T, last, evals, near [K,H,W].
// alt_*: for a pixel with near-threshold decisions, the result with the first one
// inverted; elsewhere a copy of the primary result. Returns the total eval count.
int64_t orc_render_fwd(int64_t N, const double* means, const double* log_scales, const double* quats,
                       const double* logits, const double* rgb, int K, const double* cams, int W, int H, int tile,
                       const uint32_t* vals, const uint32_t* ranges, double guard_alpha, double guard_T,
                       double guard_power, double* out_rgb, double* out_depth, double* out_T, int32_t* out_last,
                       int32_t* out_evals, int32_t* out_near, double* alt_rgb, double* alt_depth, double* alt_T,
                       int32_t* alt_last) {
  const std::vector<Proj64> pr = project_all(N, means, log_scales, quats, logits, rgb, K, cams, W, H);
  const int Tx = tiles_x(W, tile), Ty = tiles_y(H, tile);
  const Guard gd{guard_alpha, guard_T, guard_power};
  const int64_t HW = static_cast<int64_t>(H) * W;
  int64_t evals = 0;
#pragma omp parallel for collapse(2) schedule(dynamic, 2) reduction(+ : evals)
  for (int k = 0; k < K; ++k)
    for (int py = 0; py < H; ++py) {
      const Proj64* view = pr.data() + static_cast<int64_t>(k) * N;
      for (int px = 0; px < W; ++px) {
        const int64_t t = static_cast<int64_t>(k) * Tx * Ty + (py / tile) * Tx + (px / tile);
        const uint32_t s = ranges[2 * t], e = ranges[2 * t + 1];
        const double cxp = px + 0.5, cyp = py + 0.5;
        const PixelResult r = walk_pixel(view, vals, s, e, cxp, cyp, gd, -1, nullptr);
        const PixelResult a = r.n_near ? walk_pixel(view, vals, s, e, cxp, cyp, gd, r.first_near, nullptr) : r;
        const int64_t pix = static_cast<int64_t>(py) * W + px;
        for (int ch = 0; ch < 3; ++ch) {
          out_rgb[(static_cast<int64_t>(k) * 3 + ch) * HW + pix] = r.rgb[ch];
          alt_rgb[(static_cast<int64_t>(k) * 3 + ch) * HW + pix] = a.rgb[ch];
        }
        const int64_t kp = static_cast<int64_t>(k) * HW + pix;
        out_depth[kp] = r.depth;
        out_T[kp] = r.T;
        out_last[kp] = r.last;
        out_evals[kp] = r.evals;
        out_near[kp] = r.n_near;
        alt_depth[kp] = a.depth;
        alt_T[kp] = a.T;
        alt_last[kp] = a.last;
        evals += r.evals;
      }
    }
  return evals;
}

// FP64 forward render with occlusion by an external surface (a digital-twin depth buffer):
// ext_depth [K,H,W] (float, > 0), ext_rgb [K,3,H,W] (may be NULL: black). Per pixel the list
// is composited front to back until the first Gaussian at or behind ext_depth; the surface then
// shows through the remaining transmittance: rgb += T ext_rgb, depth += T ext_depth.
// Outputs as orc_render_fwd (primary and alternative for near-threshold pixels).
void orc_render_occluded(int64_t N, const double* means, const double* log_scales, const double* quats,
                         const double* logits, const double* rgb, int K, const double* cams, int W, int H, int tile,
                         const uint32_t* vals, const uint32_t* ranges, const float* ext_depth, const float* ext_rgb,
                         double guard_alpha, double guard_T, double guard_power, double* out_rgb, double* out_depth,
                         double* out_T, int32_t* out_near, double* alt_rgb, double* alt_depth, double* alt_T) {
  const std::vector<Proj64> pr = project_all(N, means, log_scales, quats, logits, rgb, K, cams, W, H);
  const int Tx = tiles_x(W, tile), Ty = tiles_y(H, tile);
  const Guard gd{guard_alpha, guard_T, guard_power};
  const int64_t HW = static_cast<int64_t>(H) * W;
#pragma omp parallel for collapse(2) schedule(dynamic, 2)
  for (int k = 0; k < K; ++k)
    for (int py = 0; py < H; ++py) {
      const Proj64* view = pr.data() + static_cast<int64_t>(k) * N;
      for (int px = 0; px < W; ++px) {
        const int64_t t = static_cast<int64_t>(k) * Tx * Ty + (py / tile) * Tx + (px / tile);
        const uint32_t s = ranges[2 * t], e = ranges[2 * t + 1];
        const int64_t pix = static_cast<int64_t>(py) * W + px, kp = static_cast<int64_t>(k) * HW + pix;
        const double zmax = static_cast<double>(ext_depth[kp]);
        const PixelResult r = walk_pixel(view, vals, s, e, px + 0.5, py + 0.5, gd, -1, nullptr, zmax);
        const PixelResult a =
            r.n_near ? walk_pixel(view, vals, s, e, px + 0.5, py + 0.5, gd, r.first_near, nullptr, zmax) : r;
        for (int ch = 0; ch < 3; ++ch) {
          const double bg = ext_rgb ? static_cast<double>(ext_rgb[(static_cast<int64_t>(k) * 3 + ch) * HW + pix]) : 0.0;
          out_rgb[(static_cast<int64_t>(k) * 3 + ch) * HW + pix] = r.rgb[ch] + r.T * bg;
          alt_rgb[(static_cast<int64_t>(k) * 3 + ch) * HW + pix] = a.rgb[ch] + a.T * bg;
        }
        out_depth[kp] = r.depth + r.T * zmax;
        alt_depth[kp] = a.depth + a.T * zmax;
        out_T[kp] = r.T;
        alt_T[kp] = a.T;
        out_near[kp] = r.n_near;
      }
    }
}

// FP64 render of selected tiles only (full-size parity on sampled outputs): the same per-pixel
// compositing as orc_render_fwd, for every pixel of each listed global tile id, projecting only
// the Gaussians of that tile's list. Outputs are [n_tiles, 16*16] per pixel of the tile in
// row-major order (rgb: [n_tiles, 3, 256]); pixels outside the image get near = -1.
void orc_render_tiles(int64_t N, const double* means, const double* log_scales, const double* quats,
                      const double* logits, const double* rgb, int K, const double* cams, int W, int H, int tile,
                      const uint32_t* vals, const uint32_t* ranges, int n_tiles, const int64_t* tiles,
                      double guard_alpha, double guard_T, double guard_power, double* out_rgb, double* out_depth,
                      double* out_T, int32_t* out_last, int32_t* out_near, double* alt_rgb, double* alt_depth,
                      double* alt_T, int32_t* alt_last) {
  const int Tx = tiles_x(W, tile), Ty = tiles_y(H, tile);
  const Guard gd{guard_alpha, guard_T, guard_power};
  const int P = tile * tile;
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < n_tiles; ++i) {
    const int64_t t = tiles[i];
    const int k = static_cast<int>(t / (static_cast<int64_t>(Tx) * Ty));
    const int r = static_cast<int>(t - static_cast<int64_t>(k) * Tx * Ty);
    const int ty = r / Tx, tx = r - ty * Tx;
    const uint32_t s = ranges[2 * t], e = ranges[2 * t + 1];
    const double* cam = cams + 16 * k;
    // the tile's list, projected, indexed by list position
    std::vector<Proj64> local(e - s);
    std::vector<uint32_t> idx(e - s);
    for (uint32_t j = s; j < e; ++j) {
      const int64_t g = vals[j];
      local[j - s] = project64(means + 3 * g, log_scales + 3 * g, quats + 4 * g, logits[g], rgb + 3 * g, cam, W, H);
      idx[j - s] = j - s;
    }
    for (int q = 0; q < P; ++q) {
      const int px = tx * tile + q % tile, py = ty * tile + q / tile;
      const int64_t o = static_cast<int64_t>(i) * P + q;
      if (px >= W || py >= H) {
        out_near[o] = -1;
        continue;
      }
      const PixelResult pr = walk_pixel(local.data(), idx.data(), 0, e - s, px + 0.5, py + 0.5, gd, -1, nullptr);
      const PixelResult a =
          pr.n_near ? walk_pixel(local.data(), idx.data(), 0, e - s, px + 0.5, py + 0.5, gd, pr.first_near, nullptr)
                    : pr;
      for (int ch = 0; ch < 3; ++ch) {
        out_rgb[(static_cast<int64_t>(i) * 3 + ch) * P + q] = pr.rgb[ch];
        alt_rgb[(static_cast<int64_t>(i) * 3 + ch) * P + q] = a.rgb[ch];
      }
      out_depth[o] = pr.depth;
      out_T[o] = pr.T;
      out_last[o] = pr.last;
      out_near[o] = pr.n_near;
      alt_depth[o] = a.depth;
      alt_T[o] = a.T;
      alt_last[o] = a.last;
    }
  }
}

// Contributors of one pixel (test aid for the transmittance-product and weight pins).
// Returns the number of composited Gaussians (at most max_n are written).
int orc_pixel_trace(int64_t N, const double* means, const double* log_scales, const double* quats,
                    const double* logits, const double* rgb, const double* cam, int W, int H, int tile,
                    const uint32_t* vals, const uint32_t* ranges, int k, int px, int py, int max_n, int32_t* g_out,
                    double* alpha_out, double* T_out, double* T_final) {
  std::vector<Proj64> view(N);
  for (int64_t g = 0; g < N; ++g)
    view[g] = project64(means + 3 * g, log_scales + 3 * g, quats + 4 * g, logits[g], rgb + 3 * g, cam, W, H);
  const int Tx = tiles_x(W, tile), Ty = tiles_y(H, tile);
  const int64_t t = static_cast<int64_t>(k) * Tx * Ty + (py / tile) * Tx + (px / tile);
  std::vector<Contrib> tr;
  const Guard gd{0, 0, 0};
  const PixelResult r = walk_pixel(view.data(), vals, ranges[2 * t], ranges[2 * t + 1], px + 0.5, py + 0.5, gd, -1, &tr);
  for (int i = 0; i < static_cast<int>(tr.size()) && i < max_n; ++i) {
    g_out[i] = static_cast<int32_t>(tr[i].g);
    alpha_out[i] = tr[i].alpha;
    T_out[i] = tr[i].T;
  }
  *T_final = r.T;
  return static_cast<int>(tr.size());
}

// FP64 backward of the compositing (reverse mode of walk_pixel, primary decisions).
// Inputs: upstream dL/drgb [K,3,H,W], dL/ddepth [K,H,W], dL/dT [K,H,W] (nullable).
// Outputs (overwritten): d_uv [K*N,2], d_conic [K*N,3] = (A, B, C), d_z [K*N],
// d_opac [N] (gradient w.r.t. the opacity o), d_rgb [N,3].
// Per contributor i of a pixel with suffix S = sum_{j>i} x_j alpha_j T_j:
//   dC/dc_i = alpha_i T_i,  dC/dalpha_i = c_i T_i - S_c / (1 - alpha_i),
//   dT_final/dalpha_i = -T_final / (1 - alpha_i); the 0.99 clamp passes no gradient.
void orc_render_bwd(int64_t N, const double* means, const double* log_scales, const double* quats,
                    const double* logits, const double* rgb, int K, const double* cams, int W, int H, int tile,
                    const uint32_t* vals, const uint32_t* ranges, const double* dL_drgb, const double* dL_ddepth,
                    const double* dL_dT, double* d_uv, double* d_conic, double* d_z, double* d_opac,
                    double* d_rgb) {
  const std::vector<Proj64> pr = project_all(N, means, log_scales, quats, logits, rgb, K, cams, W, H);
  const int Tx = tiles_x(W, tile), Ty = tiles_y(H, tile);
  const int64_t HW = static_cast<int64_t>(H) * W;
  const int64_t KN = static_cast<int64_t>(K) * N;
  std::fill(d_uv, d_uv + 2 * KN, 0.0);
  std::fill(d_conic, d_conic + 3 * KN, 0.0);
  std::fill(d_z, d_z + KN, 0.0);
  std::fill(d_opac, d_opac + N, 0.0);
  std::fill(d_rgb, d_rgb + 3 * N, 0.0);
  const Guard gd{0, 0, 0};
#pragma omp parallel for collapse(2) schedule(dynamic, 2)
  for (int k = 0; k < K; ++k)
    for (int py = 0; py < H; ++py) {
      const Proj64* view = pr.data() + static_cast<int64_t>(k) * N;
      std::vector<Contrib> tr;
      std::vector<double> Sc, Sz;
      for (int px = 0; px < W; ++px) {
        const int64_t t = static_cast<int64_t>(k) * Tx * Ty + (py / tile) * Tx + (px / tile);
        tr.clear();
        const PixelResult r = walk_pixel(view, vals, ranges[2 * t], ranges[2 * t + 1], px + 0.5, py + 0.5, gd, -1, &tr);
        const int n = static_cast<int>(tr.size());
        if (!n) continue;
        const int64_t pix = static_cast<int64_t>(py) * W + px;
        double gc[3];
        for (int ch = 0; ch < 3; ++ch) gc[ch] = dL_drgb[(static_cast<int64_t>(k) * 3 + ch) * HW + pix];
        const double gD = dL_ddepth[static_cast<int64_t>(k) * HW + pix];
        const double gT = dL_dT ? dL_dT[static_cast<int64_t>(k) * HW + pix] : 0.0;
        // suffix sums S_i = sum_{j>i} x_j alpha_j T_j, for x = colour channels and depth
        Sc.assign(3 * (n + 1), 0.0);
        Sz.assign(n + 1, 0.0);
        for (int i = n - 1; i >= 0; --i) {
          const Proj64& P = view[tr[i].g];
          const double w = tr[i].alpha * tr[i].T;
          for (int ch = 0; ch < 3; ++ch) Sc[3 * i + ch] = Sc[3 * (i + 1) + ch] + P.rgb[ch] * w;
          Sz[i] = Sz[i + 1] + P.pc[2] * w;
        }
        for (int i = 0; i < n; ++i) {
          const Contrib& c = tr[i];
          const Proj64& P = view[c.g];
          const double w = c.alpha * c.T;
          const double inv1m = 1.0 / (1.0 - c.alpha);
          double dalpha = 0.0;
          for (int ch = 0; ch < 3; ++ch) dalpha += gc[ch] * (P.rgb[ch] * c.T - Sc[3 * (i + 1) + ch] * inv1m);
          dalpha += gD * (P.pc[2] * c.T - Sz[i + 1] * inv1m);
          dalpha += -gT * r.T * inv1m;
          const int64_t kg = static_cast<int64_t>(k) * N + c.g;
          for (int ch = 0; ch < 3; ++ch) {
#pragma omp atomic
            d_rgb[3 * c.g + ch] += w * gc[ch];
          }
#pragma omp atomic
          d_z[kg] += w * gD;
          if (c.clamped) continue;
          // alpha = o G, G = exp(power)
#pragma omp atomic
          d_opac[c.g] += c.G * dalpha;
          const double dpow = c.alpha * dalpha;
          // power = -0.5 (A dx^2 + C dy^2) - B dx dy with (dx, dy) = mean2D - pixel
#pragma omp atomic
          d_conic[3 * kg + 0] += -0.5 * c.dx * c.dx * dpow;
#pragma omp atomic
          d_conic[3 * kg + 1] += -c.dx * c.dy * dpow;
#pragma omp atomic
          d_conic[3 * kg + 2] += -0.5 * c.dy * c.dy * dpow;
#pragma omp atomic
          d_uv[2 * kg + 0] += -(P.A * c.dx + P.B * c.dy) * dpow;
#pragma omp atomic
          d_uv[2 * kg + 1] += -(P.C * c.dy + P.B * c.dx) * dpow;
        }
      }
    }
}

// FP64 backward of the projection: screen-space gradients -> parameter and pose gradients.
// Inputs as produced by orc_render_bwd. Outputs (overwritten): g_means [N,3], g_log_scales [N,3],
// g_quats [N,4] (w.r.t. the raw, unnormalised quaternion), g_logits [N], g_rgb [N,3],
// g_pose [K,6] = (rho, phi) for the left perturbation T <- Exp(xi) T at xi = 0.
void orc_project_bwd(int64_t N, const double* means, const double* log_scales, const double* quats,
                     const double* logits, const double* rgb, int K, const double* cams, int W, int H,
                     const double* d_uv, const double* d_conic, const double* d_z, const double* d_opac,
                     const double* d_rgb, double* g_means, double* g_log_scales, double* g_quats, double* g_logits,
                     double* g_rgb, double* g_pose) {
  std::fill(g_means, g_means + 3 * N, 0.0);
  std::fill(g_log_scales, g_log_scales + 3 * N, 0.0);
  std::fill(g_quats, g_quats + 4 * N, 0.0);
  std::fill(g_pose, g_pose + 6 * K, 0.0);
  for (int64_t g = 0; g < N; ++g) {
    const double o = 1.0 / (1.0 + std::exp(-logits[g]));
    g_logits[g] = d_opac[g] * o * (1.0 - o);
    for (int ch = 0; ch < 3; ++ch) g_rgb[3 * g + ch] = d_rgb[3 * g + ch];
  }
  for (int k = 0; k < K; ++k) {
    const double* cam = cams + 16 * k;
    const double fx = cam[0], fy = cam[1];
    const double* R = cam + 4;
    double pose[6] = {0, 0, 0, 0, 0, 0};
#pragma omp parallel
    {
      double pose_l[6] = {0, 0, 0, 0, 0, 0};
#pragma omp for schedule(static)
      for (int64_t g = 0; g < N; ++g) {
        const int64_t kg = static_cast<int64_t>(k) * N + g;
        const double gu = d_uv[2 * kg], gv = d_uv[2 * kg + 1];
        const double gA = d_conic[3 * kg], gB = d_conic[3 * kg + 1], gC = d_conic[3 * kg + 2];
        const double gz = d_z[kg];
        if (gu == 0 && gv == 0 && gA == 0 && gB == 0 && gC == 0 && gz == 0) continue;
        const Proj64 P = project64(means + 3 * g, log_scales + 3 * g, quats + 4 * g, logits[g], rgb + 3 * g, cam, W, H);
        const double x = P.pc[0], y = P.pc[1], z = P.pc[2];
        // conic X = Sigma2^-1; dL/dSigma2 = -X Gbar X with Gbar the symmetric gradient of X
        const double X[2][2] = {{P.A, P.B}, {P.B, P.C}};
        const double Gb[2][2] = {{gA, 0.5 * gB}, {0.5 * gB, gC}};
        double XG[2][2], G2[2][2];
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 2; ++j) XG[i][j] = X[i][0] * Gb[0][j] + X[i][1] * Gb[1][j];
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 2; ++j) G2[i][j] = -(XG[i][0] * X[0][j] + XG[i][1] * X[1][j]);
        // T = J R; Sigma2 = T Sigma T^T + 0.3 I
        double T[2][3];
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 3; ++j) T[i][j] = P.J[i][0] * R[j] + P.J[i][1] * R[3 + j] + P.J[i][2] * R[6 + j];
        // dL/dT = 2 G2 T Sigma ; dL/dSigma = T^T G2 T
        double TS[2][3], dT[2][3], dSig[3][3];
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 3; ++j) TS[i][j] = T[i][0] * P.Sigma[0][j] + T[i][1] * P.Sigma[1][j] + T[i][2] * P.Sigma[2][j];
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 3; ++j) dT[i][j] = 2.0 * (G2[i][0] * TS[0][j] + G2[i][1] * TS[1][j]);
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int a = 0; a < 2; ++a)
              for (int b = 0; b < 2; ++b) s += T[a][i] * G2[a][b] * T[b][j];
            dSig[i][j] = s;
          }
        // T = J R: dL/dJ = dT R^T ; dL/dR (covariance part) = J^T dT
        double dJ[2][3], dRc[3][3];
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 3; ++j) dJ[i][j] = dT[i][0] * R[3 * j] + dT[i][1] * R[3 * j + 1] + dT[i][2] * R[3 * j + 2];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) dRc[i][j] = P.J[0][i] * dT[0][j] + P.J[1][i] * dT[1][j];
        // Sigma = M M^T, M = Rq S: dL/dM = 2 dSig M
        double Mm[3][3], dM[3][3];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) Mm[i][j] = P.Rq[i][j] * P.S[j];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) dM[i][j] = 2.0 * (dSig[i][0] * Mm[0][j] + dSig[i][1] * Mm[1][j] + dSig[i][2] * Mm[2][j]);
        double dRq[3][3];
        for (int j = 0; j < 3; ++j) {
          double ds = 0;
          for (int i = 0; i < 3; ++i) {
            dRq[i][j] = dM[i][j] * P.S[j];
            ds += dM[i][j] * P.Rq[i][j];
          }
          g_log_scales[3 * g + j] += ds * P.S[j];  // s = exp(log_scale)
        }
        // rotation matrix -> normalised quaternion (partials of each entry)
        const double w = P.qhat[0], qx = P.qhat[1], qy = P.qhat[2], qz = P.qhat[3];
        double dq[4];
        dq[0] = 2 * (-qz * dRq[0][1] + qy * dRq[0][2] + qz * dRq[1][0] - qx * dRq[1][2] - qy * dRq[2][0] + qx * dRq[2][1]);
        dq[1] = 2 * (qy * dRq[0][1] + qz * dRq[0][2] + qy * dRq[1][0] - 2 * qx * dRq[1][1] - w * dRq[1][2] +
                     qz * dRq[2][0] + w * dRq[2][1] - 2 * qx * dRq[2][2]);
        dq[2] = 2 * (-2 * qy * dRq[0][0] + qx * dRq[0][1] + w * dRq[0][2] + qx * dRq[1][0] + qz * dRq[1][2] -
                     w * dRq[2][0] + qz * dRq[2][1] - 2 * qy * dRq[2][2]);
        dq[3] = 2 * (-2 * qz * dRq[0][0] - w * dRq[0][1] + qx * dRq[0][2] + w * dRq[1][0] - 2 * qz * dRq[1][1] +
                     qy * dRq[1][2] + qx * dRq[2][0] + qy * dRq[2][1]);
        // normalisation q_hat = q / |q|
        const double dot = w * dq[0] + qx * dq[1] + qy * dq[2] + qz * dq[3];
        for (int i = 0; i < 4; ++i) g_quats[4 * g + i] += (dq[i] - P.qhat[i] * dot) / P.qnorm;
        // Jacobian entries -> camera-space mean
        const double txz = P.clampx ? (x / z < 0 ? -1 : 1) * kJacClamp * (0.5 * W / fx) : x / z;
        const double tyz = P.clampy ? (y / z < 0 ? -1 : 1) * kJacClamp * (0.5 * H / fy) : y / z;
        double dpc[3] = {0, 0, 0};
        // J00 = fx/z, J02 = -fx txz / z, J11 = fy/z, J12 = -fy tyz / z
        dpc[2] += dJ[0][0] * (-fx / (z * z)) + dJ[1][1] * (-fy / (z * z));
        dpc[2] += dJ[0][2] * (fx * txz / (z * z)) + dJ[1][2] * (fy * tyz / (z * z));
        if (!P.clampx) {
          dpc[0] += dJ[0][2] * (-fx / (z * z));
          dpc[2] += dJ[0][2] * (fx * x / (z * z * z));
        }
        if (!P.clampy) {
          dpc[1] += dJ[1][2] * (-fy / (z * z));
          dpc[2] += dJ[1][2] * (fy * y / (z * z * z));
        }
        // mean2D u = fx x/z + cx, v = fy y/z + cy; depth output z
        dpc[0] += gu * fx / z;
        dpc[1] += gv * fy / z;
        dpc[2] += -gu * fx * x / (z * z) - gv * fy * y / (z * z) + gz;
        // p_c = R p + t
        for (int j = 0; j < 3; ++j) g_means[3 * g + j] += R[j] * dpc[0] + R[3 + j] * dpc[1] + R[6 + j] * dpc[2];
        // pose (rho, phi): d p_c = rho + phi x p_c ; d R = [phi]x R
        double pxg[3];
        cross3(P.pc, dpc, pxg);
        double A[3][3];  // A = R dRc^T
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) A[i][j] = R[3 * i] * dRc[j][0] + R[3 * i + 1] * dRc[j][1] + R[3 * i + 2] * dRc[j][2];
        pose_l[0] += dpc[0];
        pose_l[1] += dpc[1];
        pose_l[2] += dpc[2];
        pose_l[3] += pxg[0] + A[1][2] - A[2][1];
        pose_l[4] += pxg[1] + A[2][0] - A[0][2];
        pose_l[5] += pxg[2] + A[0][1] - A[1][0];
      }
#pragma omp critical
      for (int i = 0; i < 6; ++i) pose[i] += pose_l[i];
    }
    for (int i = 0; i < 6; ++i) g_pose[6 * k + i] = pose[i];
  }
}

// Photometric loss of the mapping step: per view, mean |R - R*| over 3HW values plus
// lambda * mean |D - D*| over HW values, summed over views; sign(0) = 0.
// Writes dL/drgb and dL/ddepth; returns L.
double orc_loss_l1(const double* rgb, const double* depth, const double* rgb_t, const double* depth_t, int K, int H,
                   int W, double lambda_depth, double* dL_drgb, double* dL_ddepth) {
  const int64_t HW = static_cast<int64_t>(H) * W;
  double L = 0.0;
  const double inv3 = 1.0 / (3.0 * HW), inv1 = 1.0 / static_cast<double>(HW);
  for (int64_t i = 0; i < K * 3 * HW; ++i) {
    const double d = rgb[i] - rgb_t[i];
    L += std::fabs(d) * inv3;
    dL_drgb[i] = (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) * inv3;
  }
  for (int64_t i = 0; i < K * HW; ++i) {
    const double d = depth[i] - depth_t[i];
    L += lambda_depth * std::fabs(d) * inv1;
    dL_ddepth[i] = lambda_depth * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) * inv1;
  }
  return L;
}

}  // extern "C"
