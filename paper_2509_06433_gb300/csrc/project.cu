// Projection of 3D Gaussians (Sec. II-A scene model) for K views: 2D mean, conic,
// depth, pixel radius, tile rectangle and the tiles of that rectangle which the widened
// alpha >= 1/255 ellipse meets (counted row by row) of every (view, Gaussian) item.
//
// Two arithmetic regimes live here:
//  * the DISCRETE path (camera depth used as the sort key, the culls, the radius, the
//    tile rectangle and the emitted tiles) runs in binary32 in one fixed operation order,
//    with explicit round-to-nearest intrinsics so the compiler cannot fuse or reorder anything;
//  * the CONTINUOUS path carries the camera-space mean and the 2D mean as unevaluated
//    float pairs (hi + lo, Dot2-style compensated arithmetic), so the 2D mean that the
//    compositing uses is accurate to ~1e-12 px instead of ~4e-5 px at 640 px.
#include "gs_internal.cuh"
#include "sh.cuh"

namespace gs {
namespace {

// Deterministic binary32 exponential: Cody & Waite additive range reduction x = k ln2 + r
// with a 16-bit head of ln2 (so k * head is exact) and a tail, then the degree-7 Taylor
// polynomial of e^r by Horner's rule, scaled by 2^k. Max error 1 ulp on [-80, 80].
__device__ __forceinline__ float exp_det(float x) {
  if (x != x) return x;
  x = (x < -80.0f) ? -80.0f : ((x > 80.0f) ? 80.0f : x);
  const float kf = rintf(__fmul_rn(x, 0x1.715476p+0f));
  float r = __fmaf_rn(-kf, 0x1.62e4p-1f, x);
  r = __fmaf_rn(-kf, 0x1.7f7d1cp-20f, r);
  float p = 0x1.a01a02p-13f;
  p = __fmaf_rn(p, r, 0x1.6c16c2p-10f);
  p = __fmaf_rn(p, r, 0x1.111112p-7f);
  p = __fmaf_rn(p, r, 0x1.555556p-5f);
  p = __fmaf_rn(p, r, 0x1.555556p-3f);
  p = __fmaf_rn(p, r, 0x1p-1f);
  p = __fmaf_rn(p, r, 1.0f);
  p = __fmaf_rn(p, r, 1.0f);
  const int k = static_cast<int>(kf);
  return __fmul_rn(p, __int_as_float((k + 127) << 23));
}

// Deterministic binary32 natural logarithm of a positive normal x: x = m 2^e with m in
// [sqrt(1/2), sqrt(2)), ln m = 2 atanh(s), s = (m - 1)/(m + 1), by the atanh series to s^9
// (Horner), plus e ln2 with the head / tail split of ln2 used by exp_det. Within 4 ulp.
__device__ __forceinline__ float log_det(float x) {
  if (!(x > 0.0f) || !isfinite(x)) return x > 0.0f ? x : -INFINITY;
  const uint32_t bits = __float_as_uint(x);
  if ((bits >> 23) == 0) return -INFINITY;
  int e = static_cast<int>(bits >> 23) - 127;
  float m = __uint_as_float((bits & 0x7fffffu) | 0x3f800000u);
  if (m > 0x1.6a09e6p+0f) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float s2 = __fmul_rn(s, s);
  float p = 0x1.c71c72p-4f;
  p = __fmaf_rn(p, s2, 0x1.24924ap-3f);
  p = __fmaf_rn(p, s2, 0x1.99999ap-3f);
  p = __fmaf_rn(p, s2, 0x1.555556p-2f);
  p = __fmaf_rn(p, s2, 1.0f);
  const float lm = __fmul_rn(__fmul_rn(2.0f, s), p);
  const float ef = static_cast<float>(e);
  return __fmaf_rn(ef, 0x1.62e4p-1f, __fmaf_rn(ef, 0x1.7f7d1cp-20f, lm));
}

struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF renorm(float s, float e) {
  const float hi = __fadd_rn(s, e);
  return {hi, __fsub_rn(e, __fsub_rn(hi, s))};
}
// r0 p0 + r1 p1 + r2 p2 + t as hi + lo
__device__ __forceinline__ FF dot3_plus(float r0, float r1, float r2, float p0, float p1, float p2, float t) {
  const FF a = two_prod(r0, p0);
  const FF b = two_prod(r1, p1);
  const FF c = two_sum(a.hi, b.hi);
  float err = __fadd_rn(a.lo, __fadd_rn(b.lo, c.lo));
  const FF d = two_prod(r2, p2);
  const FF e = two_sum(c.hi, d.hi);
  err = __fadd_rn(err, __fadd_rn(d.lo, e.lo));
  const FF f = two_sum(e.hi, t);
  err = __fadd_rn(err, f.lo);
  return renorm(f.hi, err);
}
// f * (x / z) + c with x, z given as hi + lo
__device__ __forceinline__ FF proj_coord(float f, float c, FF x, FF z) {
  const float q = __fdiv_rn(x.hi, z.hi);
  float r = __fmaf_rn(-q, z.hi, x.hi);  // exact remainder
  r = __fadd_rn(r, __fmaf_rn(-q, z.lo, x.lo));
  const float ql = __fdiv_rn(r, z.hi);
  const FF p = two_prod(f, q);
  const float pl = __fmaf_rn(f, ql, p.lo);
  const FF s = two_sum(p.hi, c);
  return renorm(s.hi, __fadd_rn(pl, s.lo));
}

// Row spans a projection warp keeps from its first row pass for its second (per round of 32
// items; rows beyond are computed again).
constexpr int kSpanCache = 128;

__device__ __forceinline__ uint32_t pack16(int lo, int hi) {
  return static_cast<uint32_t>(lo) | (static_cast<uint32_t>(hi) << 16);
}

// Whether an item in front of the near plane certainly has an empty tile rectangle, from a
// bound on its radius that needs no covariance: each row of R Q S (R, Q rotations, S the
// scales) has length <= max S, so |m1| <= (fx / z)(1 + |tx|) max S (m1, m2: the rows of J R Q S
// whose squares sum, with the dilation, to the trace a + c), and lambda_max <= a + c +
// sqrt(0.1). The bound carries a 1% + 2 px margin and the 2D mean a 1e-4 relative + 1 px one,
// so the exact computation would cull such an item too; the margins also cover the few-ulp
// errors of the approximate exp, reciprocal, quotient and square root the bound is computed
// with (it runs for every item, the exact projection only for the survivors). NaN anywhere
// keeps the item (the exact path culls it itself).
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ bool off_screen(const Layout& L, const gs_camera_t& cam, float xc, float yc, float zc,
                                           const float (&ls)[3]) {
  const float smax = __expf(fmaxf(ls[0], fmaxf(ls[1], ls[2]))) * 1.002f;
  const float iz = __fdividef(1.0f, zc);
  const float xz = xc * iz, yz = yc * iz;
  const float limx = 1.3f * __fdividef(0.5f * static_cast<float>(L.W), cam.fx);
  const float limy = 1.3f * __fdividef(0.5f * static_cast<float>(L.H), cam.fy);
  const float m1 = fabsf(cam.fx) * iz * (1.0f + fminf(fabsf(xz), limx)) * smax;
  const float m2 = fabsf(cam.fy) * iz * (1.0f + fminf(fabsf(yz), limy)) * smax;
  const float rb = 3.0f * sqrt_approx(m1 * m1 + m2 * m2 + 1.0f) * 1.01f + 2.0f;
  const float u = cam.fx * xz + cam.cx, v = cam.fy * yz + cam.cy;
  const float mu = 1e-4f * fabsf(u) + 1.0f, mv = 1e-4f * fabsf(v) + 1.0f;
  const float xhi = static_cast<float>(kTile * (L.Tx + 1)), yhi = static_cast<float>(kTile * (L.Ty + 1));
  return (u - rb - mu > xhi) || (u + rb + mu < -2.0f * kTile) || (v - rb - mv > yhi) || (v + rb + mv < -2.0f * kTile);
}

// The projection of one item that survived the cull: the discrete path in binary32 (culls,
// radius, tile rectangle, the widened alpha >= 1/255 ellipse) and, for an item with an ellipse,
// the continuous path (compensated 2D mean, conic, depth), whose records it writes.
struct Projected {
  Ellipse E;
  int x0, x1, y0, y1, radius;
  float z;
  bool live;  // has an ellipse and a non-empty rectangle: its rows are examined next
};

__device__ __forceinline__ Projected project_item(const Layout& L, const GaussPtrs& G, const gs_camera_t& cam,
                                                  int64_t idx, int64_t g, uint8_t* __restrict__ ws) {
  Projected P{};
  const float p0 = load_attr(G.means, 3 * g + 0, G.means_dtype);
  const float p1 = load_attr(G.means, 3 * g + 1, G.means_dtype);
  const float p2 = load_attr(G.means, 3 * g + 2, G.means_dtype);
  float ls[3], q[4];
  for (int j = 0; j < 3; ++j) ls[j] = load_attr(G.log_scales, 3 * g + j, G.dtype);
  for (int j = 0; j < 4; ++j) q[j] = load_attr(G.quats, 4 * g + j, G.dtype);
  const float lg = load_attr(G.logits, g, G.dtype);
  const float* R = cam.R;
  const float* t = cam.t;
  // ---------------- discrete path: fixed binary32 operation order -----------------
  bool valid = true;
  const float xc = __fmaf_rn(R[0], p0, __fmaf_rn(R[1], p1, __fmaf_rn(R[2], p2, t[0])));
  const float yc = __fmaf_rn(R[3], p0, __fmaf_rn(R[4], p1, __fmaf_rn(R[5], p2, t[1])));
  const float zc = __fmaf_rn(R[6], p0, __fmaf_rn(R[7], p1, __fmaf_rn(R[8], p2, t[2])));
  valid = zc > L.near_plane;
  const float n2 = __fmaf_rn(q[0], q[0], __fmaf_rn(q[1], q[1], __fmaf_rn(q[2], q[2], __fmul_rn(q[3], q[3]))));
  const float nq = __fsqrt_rn(n2);
  valid = valid && (nq > 0.0f);
  const float qw = __fdiv_rn(q[0], nq), qx = __fdiv_rn(q[1], nq), qy = __fdiv_rn(q[2], nq), qz = __fdiv_rn(q[3], nq);
  const float xx = __fmul_rn(qx, qx), yy = __fmul_rn(qy, qy), zz = __fmul_rn(qz, qz);
  const float xy = __fmul_rn(qx, qy), xz = __fmul_rn(qx, qz), yz = __fmul_rn(qy, qz);
  const float wx = __fmul_rn(qw, qx), wy = __fmul_rn(qw, qy), wz = __fmul_rn(qw, qz);
  float Q[3][3];
  Q[0][0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(yy, zz)));
  Q[0][1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
  Q[0][2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
  Q[1][0] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
  Q[1][1] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, zz)));
  Q[1][2] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
  Q[2][0] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
  Q[2][1] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
  Q[2][2] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, yy)));
  const float S0 = exp_det(ls[0]), S1 = exp_det(ls[1]), S2 = exp_det(ls[2]);
  float M[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    M[i][0] = __fmul_rn(Q[i][0], S0);
    M[i][1] = __fmul_rn(Q[i][1], S1);
    M[i][2] = __fmul_rn(Q[i][2], S2);
  }
  float Nm[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Nm[i][j] = __fmaf_rn(R[3 * i + 0], M[0][j], __fmaf_rn(R[3 * i + 1], M[1][j], __fmul_rn(R[3 * i + 2], M[2][j])));
  const float xz_ = __fdiv_rn(xc, zc), yz_ = __fdiv_rn(yc, zc);
  const float limx = __fmul_rn(1.3f, __fdiv_rn(__fmul_rn(0.5f, static_cast<float>(L.W)), cam.fx));
  const float limy = __fmul_rn(1.3f, __fdiv_rn(__fmul_rn(0.5f, static_cast<float>(L.H)), cam.fy));
  const float txz = fminf(fmaxf(xz_, -limx), limx);
  const float tyz = fminf(fmaxf(yz_, -limy), limy);
  const float j00 = __fdiv_rn(cam.fx, zc), j02 = -__fmul_rn(j00, txz);
  const float j11 = __fdiv_rn(cam.fy, zc), j12 = -__fmul_rn(j11, tyz);
  float m1[3], m2[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    m1[j] = __fmaf_rn(j00, Nm[0][j], __fmul_rn(j02, Nm[2][j]));
    m2[j] = __fmaf_rn(j11, Nm[1][j], __fmul_rn(j12, Nm[2][j]));
  }
  const float aa = __fmaf_rn(m1[0], m1[0], __fmaf_rn(m1[1], m1[1], __fmul_rn(m1[2], m1[2])));
  const float cc = __fmaf_rn(m2[0], m2[0], __fmaf_rn(m2[1], m2[1], __fmul_rn(m2[2], m2[2])));
  const float bb = __fmaf_rn(m1[0], m2[0], __fmaf_rn(m1[1], m2[1], __fmul_rn(m1[2], m2[2])));
  const float a = __fadd_rn(aa, 0.3f), c = __fadd_rn(cc, 0.3f);
  const float k0 = __fmaf_rn(m1[1], m2[2], -__fmul_rn(m1[2], m2[1]));
  const float k1 = __fmaf_rn(m1[2], m2[0], -__fmul_rn(m1[0], m2[2]));
  const float k2 = __fmaf_rn(m1[0], m2[1], -__fmul_rn(m1[1], m2[0]));
  const float det = __fadd_rn(__fadd_rn(__fmaf_rn(k0, k0, __fmaf_rn(k1, k1, __fmul_rn(k2, k2))),
                                        __fmul_rn(0.3f, __fadd_rn(aa, cc))),
                              0.09f);
  valid = valid && (det > 0.0f);
  const float mid = __fmul_rn(0.5f, __fadd_rn(a, c));
  const float hd = __fmul_rn(0.5f, __fsub_rn(a, c));
  const float disc = fmaxf(__fmaf_rn(hd, hd, __fmul_rn(bb, bb)), 0.1f);
  const float lmax = __fadd_rn(mid, __fsqrt_rn(disc));
  const float rf = fminf(ceilf(__fmul_rn(3.0f, __fsqrt_rn(lmax))), 1048576.0f);
  valid = valid && (rf == rf);
  const float u = __fmaf_rn(cam.fx, xz_, cam.cx);
  const float v = __fmaf_rn(cam.fy, yz_, cam.cy);
  valid = valid && isfinite(u) && isfinite(v);
  const float inv_tile = 1.0f / static_cast<float>(kTile);
  const float Txf = static_cast<float>(L.Tx), Tyf = static_cast<float>(L.Ty);
  const float x0f = fminf(fmaxf(floorf(__fmul_rn(__fsub_rn(u, rf), inv_tile)), 0.0f), Txf);
  const float x1f = fminf(fmaxf(__fadd_rn(floorf(__fmul_rn(__fadd_rn(u, rf), inv_tile)), 1.0f), 0.0f), Txf);
  const float y0f = fminf(fmaxf(floorf(__fmul_rn(__fsub_rn(v, rf), inv_tile)), 0.0f), Tyf);
  const float y1f = fminf(fmaxf(__fadd_rn(floorf(__fmul_rn(__fadd_rn(v, rf), inv_tile)), 1.0f), 0.0f), Tyf);
  P.z = zc;
  if (valid) {
    P.x0 = static_cast<int>(x0f);
    P.x1 = static_cast<int>(x1f);
    P.y0 = static_cast<int>(y0f);
    P.y1 = static_cast<int>(y1f);
    P.radius = static_cast<int>(rf);
    if ((P.x1 - P.x0) * (P.y1 - P.y0) == 0) {
      P.x0 = P.x1 = P.y0 = P.y1 = P.radius = 0;
    } else {
      // the widened alpha >= 1/255 ellipse; its rows are examined by the warp
      const float op = __fdiv_rn(1.0f, __fadd_rn(1.0f, exp_det(-lg)));
      const float Lg = log_det(__fmul_rn(255.0f, op));
      const float Lm = __fadd_rn(__fadd_rn(Lg, __fmul_rn(0.02f, fabsf(Lg))), 1.5e-4f);
      if (Lm >= 0.0f) {
        const float kap = __fmul_rn(2.0f, Lm);
        P.E = Ellipse{u, v, bb, __fdiv_rn(1.0f, c), __fsqrt_rn(det), __fsqrt_rn(__fmul_rn(kap, a)),
                      __fsqrt_rn(__fmul_rn(kap, c)), __fdiv_rn(bb, a)};
        P.live = true;
      }
    }
  }
  // ---------------- continuous path ----------------------------------------------
  if (P.live) {  // (the records of an item that emits nothing are never read)
    const FF X = dot3_plus(R[0], R[1], R[2], p0, p1, p2, t[0]);
    const FF Y = dot3_plus(R[3], R[4], R[5], p0, p1, p2, t[1]);
    const FF Z = dot3_plus(R[6], R[7], R[8], p0, p1, p2, t[2]);
    const FF U = proj_coord(cam.fx, cam.cx, X, Z);
    const FF V = proj_coord(cam.fy, cam.cy, Y, Z);
    at<float4>(ws, L.proj_uv)[idx] = make_float4(U.hi, U.lo, V.hi, V.lo);
    // conic = Sigma2^-1 = [[c, -b], [-b, a]] / det with det from the Lagrange identity
    const float inv_det = 1.0f / det;
    at<float4>(ws, L.proj_conic)[idx] = make_float4(c * inv_det, -bb * inv_det, a * inv_det, Z.hi);
  }
  return P;
}

// Projection of L.proj_items consecutive (view, Gaussian) items per block (256 to 2048, a power
// of two chosen from K N), in two phases.
// Phase 1 (every item, every lane busy): the colour and opacity of view 0's items (the NaN
// check of every Gaussian), the camera-space depth and the off-screen bound; the survivors are
// marked in a shared bit mask. Phase 2: the survivors, densely packed onto the block's
// threads in increasing item order, go through the whole projection (project_item), then
// their rectangles' rows are examined warp-cooperatively: pass 1 counts each item's emitted
// tiles and finds its first and last non-empty rows (adding the spans to the span grid), pass
// 2 writes its row-span table entries. An item that emits pairs is live: its bit goes to
// live_mask, its binning record (depth key, tiles emitted, item id, row-span entries) to the
// block's segment of the staging arrays in item order (compacted by k_live_copy), its depth
// key's digits to the item-sort histograms. The last block to finish scans the blocks' live
// counts into their first positions among the live items.
// The block of items (in item order) that launched block b takes. The n blocks of items are seen
// as rows of Bv = ceil(n / K) blocks, one row per view (rows cut at block boundaries, so a row
// is about one view's items; the last row may be shorter), and the launch order walks this
// grid column by column: the blocks in flight at any time read about the same Gaussians for
// every view, which then come from L2 for all but the first view. A bijection of [0, n).
__device__ __forceinline__ int64_t proj_block(const Layout& L, int64_t b) {
  const int64_t n = L.n_proj_groups;
  if (L.K <= 1) return b;
  const int64_t bv = (n + L.K - 1) / L.K;
  const int64_t rows = (n + bv - 1) / bv;  // non-empty rows (at most K)
  if (rows <= 1) return b;
  const int64_t rem = n - (rows - 1) * bv;  // blocks in the last row, 1 .. bv
  int64_t r, k;
  if (b < rem * rows) {  // columns that every row has
    r = b / rows;
    k = b % rows;
  } else {  // the remaining columns, which the last row lacks
    const int64_t c = b - rem * rows;
    r = rem + c / (rows - 1);
    k = c % (rows - 1);
  }
  return k * bv + r;
}

// (Compiled for 4 resident blocks per SM, 64 registers: the kernel is latency-bound, and 32
// warps per SM hide more of it than 24; 12% faster at aerial2m than at 3 blocks.)
__global__ void __launch_bounds__(kProjThreads, 4) k_project(Layout L, GaussPtrs G, const gs_camera_t* __restrict__ cams,
                                                         uint8_t* __restrict__ ws) {
  pdl_wait();
  constexpr int kWords = kProjItemsMax / 32;
  static_assert(kWords == 64, "the survivor scan below gives each lane of warp 0 two mask words");
  static_assert(kWords % (kProjThreads / 32) == 0, "phase 1 covers the mask words in whole rounds");
  const int words = L.proj_items / 32;
  const int64_t blk = proj_block(L, blockIdx.x);
  const int64_t first = blk * L.proj_items;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  __shared__ uint32_t s_hist[4 * 256];
  // the block's rectangles are first added into a shared copy of its first view's difference
  // grid (when it fits), then flushed with one global atomic per non-zero cell
  __shared__ int32_t s_grid[kProjGridCells];
  __shared__ uint32_t s_surv[kWords], s_spre[kWords + 1], s_live[kWords];
  __shared__ uint32_t s_wcnt[kProjThreads / 32];
  __shared__ uint32_t s_seg;
  __shared__ int s_acc[kProjThreads / 32][3][32];  // per warp and lane: tiles, first row, last row
  __shared__ int s_carry[kProjThreads / 32][32];   // tiles of an item's rows already written
  // the first kSpanCache row spans of each warp's round (pass 1), read again by pass 2
  __shared__ int2 s_span[kProjThreads / 32][kSpanCache];
  const int gstride = L.Tx + 1;
  const int gcells = gstride * (L.Ty + 1);
  const bool use_sgrid = gcells <= kProjGridCells;
  const int k_block = static_cast<int>(first / (L.N > 0 ? L.N : 1));
  for (int i = threadIdx.x; i < 4 * 256; i += kProjThreads) s_hist[i] = 0;
  if (threadIdx.x < kWords) s_live[threadIdx.x] = 0;
  if (threadIdx.x == 0) s_seg = 0;

  // ---------------- phase 1: every item --------------------------------------------
  for (int r = 0; r < kWords / (kProjThreads / 32); ++r) {
    if (r * kProjThreads >= L.proj_items) {  // (block-uniform) the block's mask words end here
      if (lane == 0) s_surv[r * (kProjThreads / 32) + wib] = 0u;
      continue;
    }
    const int64_t idx = first + r * kProjThreads + threadIdx.x;
    bool surv = false;
    if (idx < L.KN) {
      const int k = static_cast<int>(idx / L.N);
      const int64_t g = idx - static_cast<int64_t>(k) * L.N;
      const gs_camera_t& cam = cams[k];
      const float p0 = load_attr(G.means, 3 * g + 0, G.means_dtype);
      const float p1 = load_attr(G.means, 3 * g + 1, G.means_dtype);
      const float p2 = load_attr(G.means, 3 * g + 2, G.means_dtype);
      float ls[3];
      for (int j = 0; j < 3; ++j) ls[j] = load_attr(G.log_scales, 3 * g + j, G.dtype);
      // colour and opacity: once per Gaussian, or per item when the colour depends on the view
      if (k == 0 || L.color_stride != 0) {
        float q[4];
        for (int j = 0; j < 4; ++j) q[j] = load_attr(G.quats, 4 * g + j, G.dtype);
        const float lg = load_attr(G.logits, g, G.dtype);
        float c0, c1, c2;
        bool finite_c = true;
        if (L.color_mode == GS_COLOR_SH) {
          const ShDir u = sh_dir(p0, p1, p2, cam);
          float Y[kShMaxCoeffs];
          sh_basis(u.x, u.y, u.z, Y);
          const float3 raw = sh_raw(G.rgb, G.dtype, g, L.sh_coeffs, Y, finite_c);
          c0 = fmaxf(raw.x, 0.0f), c1 = fmaxf(raw.y, 0.0f), c2 = fmaxf(raw.z, 0.0f);
        } else {
          c0 = load_attr(G.rgb, 3 * g + 0, G.dtype);
          c1 = load_attr(G.rgb, 3 * g + 1, G.dtype);
          c2 = load_attr(G.rgb, 3 * g + 2, G.dtype);
          finite_c = isfinite(c0) && isfinite(c1) && isfinite(c2);
        }
        const float o = 1.0f / (1.0f + expf(-lg));
        at<float4>(ws, L.color_opacity)[k * L.color_stride + g] = make_float4(c0, c1, c2, o);
        const bool finite = isfinite(p0) && isfinite(p1) && isfinite(p2) && isfinite(ls[0]) && isfinite(ls[1]) &&
                            isfinite(ls[2]) && isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) && isfinite(q[3]) &&
                            isfinite(lg) && finite_c;
        if (k == 0 && !finite) atomicOr(&at<Status>(ws, L.status)->err, GS_DEVERR_NONFINITE);
      }
      const float* R = cam.R;
      const float* t = cam.t;
      // the depth exactly as project_item computes it; behind the near plane or certainly off
      // screen: culled without the rest of the projection
      const float xc = __fmaf_rn(R[0], p0, __fmaf_rn(R[1], p1, __fmaf_rn(R[2], p2, t[0])));
      const float yc = __fmaf_rn(R[3], p0, __fmaf_rn(R[4], p1, __fmaf_rn(R[5], p2, t[1])));
      const float zc = __fmaf_rn(R[6], p0, __fmaf_rn(R[7], p1, __fmaf_rn(R[8], p2, t[2])));
      surv = zc > L.near_plane && !off_screen(L, cam, xc, yc, zc, ls);
    }
    const uint32_t ballot = __ballot_sync(0xffffffffu, surv);
    if (lane == 0) s_surv[r * (kProjThreads / 32) + wib] = ballot;
  }
  __syncthreads();
  // exclusive prefix of the survivors over the mask words (warp 0; kWords = 2 per lane)
  if (wib == 0) {
    const uint32_t c0 = __popc(s_surv[2 * lane]), c1 = __popc(s_surv[2 * lane + 1]);
    uint32_t incl = c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    s_spre[2 * lane] = incl - c0 - c1;
    s_spre[2 * lane + 1] = incl - c1;
    if (lane == 31) s_spre[kWords] = incl;
  }
  __syncthreads();
  const int n_surv = static_cast<int>(s_spre[kWords]);
  if (use_sgrid && n_surv > 0) {
    for (int i = threadIdx.x; i < gcells; i += kProjThreads) s_grid[i] = 0;
  }
  __syncthreads();

  // ---------------- phase 2: the survivors, kProjThreads per round ---------------------
  auto owner = [&](int st, int r) {  // the last lane whose first row number is <= r
    int o = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int cand = o + step;
      const int sc = __shfl_sync(0xffffffffu, st, cand & 31);
      if (cand < 32 && sc <= r) o = cand;
    }
    return o;
  };
  auto owner_ellipse = [&](const Ellipse& E, int o) {
    Ellipse e;
    e.u = __shfl_sync(0xffffffffu, E.u, o);
    e.v = __shfl_sync(0xffffffffu, E.v, o);
    e.b = __shfl_sync(0xffffffffu, E.b, o);
    e.inv_c = __shfl_sync(0xffffffffu, E.inv_c, o);
    e.sdet = __shfl_sync(0xffffffffu, E.sdet, o);
    e.hx = __shfl_sync(0xffffffffu, E.hx, o);
    e.hy = __shfl_sync(0xffffffffu, E.hy, o);
    e.kxy = __shfl_sync(0xffffffffu, E.kxy, o);
    return e;
  };
  auto warp_excl_scan = [&](int x, int& total) {
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    total = __shfl_sync(0xffffffffu, incl, 31);
    return incl - x;
  };
  uint32_t lm;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lm));
  for (int base = 0; base < n_surv; base += kProjThreads) {
    const int j = base + threadIdx.x;
    int64_t idx = -1;
    int kv = 0;
    Projected P{};
    if (j < n_surv) {
      // the j-th survivor: its mask word (binary search over the prefix), then its bit
      int lo = 0, hi = kWords;  // s_spre[lo] <= j < s_spre[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_spre[mid] <= static_cast<uint32_t>(j)) lo = mid; else hi = mid;
      }
      const int bit = __fns(s_surv[lo], 0, j - static_cast<int>(s_spre[lo]) + 1);
      idx = first + 32 * lo + bit;
      kv = static_cast<int>(idx / L.N);
      P = project_item(L, G, cams[kv], idx, idx - static_cast<int64_t>(kv) * L.N, ws);
    }
    // the rectangles' rows, shared out over the warp: the warp's items' rows are numbered
    // consecutively (item by item) and examined 32 at a time, one row per lane, so a warp
    // holding one tall rectangle does not idle the other lanes
    s_acc[wib][0][lane] = 0;
    s_acc[wib][1][lane] = 0x7fffffff;
    s_acc[wib][2][lane] = -1;
    __syncwarp();
    int st1 = 0;  // this lane's item's first row number in pass 1
    {
      int total = 0;
      st1 = warp_excl_scan(P.live ? P.y1 - P.y0 : 0, total);
      const int st = st1;
      for (int rb = 0; rb < total; rb += 32) {
        const int r = rb + lane;
        const int o = owner(st, r);
        const Ellipse eo = owner_ellipse(P.E, o);
        const int ox0 = __shfl_sync(0xffffffffu, P.x0, o), ox1 = __shfl_sync(0xffffffffu, P.x1, o);
        const int oy0 = __shfl_sync(0xffffffffu, P.y0, o), ok = __shfl_sync(0xffffffffu, kv, o);
        const int ost = __shfl_sync(0xffffffffu, st, o);
        if (r < total) {
          const int ty = oy0 + (r - ost);
          const int2 sp = row_span(eo, ty, ox0, ox1);
          if (r < kSpanCache) s_span[wib][r] = sp;
          if (sp.x <= sp.y) {
            atomicAdd(&s_acc[wib][0][o], sp.y - sp.x + 1);
            atomicMin(&s_acc[wib][1][o], ty);
            atomicMax(&s_acc[wib][2][o], ty);
            int32_t* dg = (use_sgrid && ok == k_block)
                              ? s_grid
                              : at<int32_t>(ws, L.tile_diff) + static_cast<int64_t>(ok) * gcells;
            atomicAdd(&dg[ty * gstride + sp.x], 1);  // row-wise prefix sum: pairs per tile
            atomicAdd(&dg[ty * gstride + sp.y + 1], -1);
          }
        }
      }
      __syncwarp();
    }
    const uint32_t count = static_cast<uint32_t>(s_acc[wib][0][lane]);
    const int row_first = s_acc[wib][1][lane];
    const uint32_t nrows = count ? static_cast<uint32_t>(s_acc[wib][2][lane] - row_first + 1) : 0u;
    const bool is_live = idx >= 0 && count > 0;  // emits at least one pair
    const uint32_t item_key = __float_as_uint(P.z);
    if (is_live) {
      at<int4>(ws, L.proj_tiles)[idx] = make_int4(0, static_cast<int>(pack16(P.x0, P.x1)),
                                                  static_cast<int>(pack16(P.y0, P.y1)), static_cast<int>(count));
      at<uint32_t>(ws, L.proj_depth_key)[idx] = item_key;
      at<int32_t>(ws, L.proj_radius)[idx] = P.radius;
    }
    // row-span table entries for the item's rows first..last (one counter atomic per warp)
    uint2 rows_out = make_uint2(0, 0);
    {
      uint32_t incl = nrows;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      uint32_t rbase = 0;
      if (lane == 31 && incl) rbase = atomicAdd(&at<Status>(ws, L.status)->row_ctr, incl);
      rbase = __shfl_sync(0xffffffffu, rbase, 31) + (incl - nrows);
      const bool fits = nrows && static_cast<uint64_t>(rbase) + nrows <= static_cast<uint64_t>(L.cap);
      if (nrows && !fits) atomicOr(&at<Status>(ws, L.status)->err, GS_DEVERR_PAIR_OVERFLOW);
      if (is_live) rows_out = fits ? make_uint2(rbase, nrows) : make_uint2(0, 0);
      int total = 0;
      const int st = warp_excl_scan(fits ? static_cast<int>(nrows) : 0, total);
      int2* tab = at<int2>(ws, L.row_table);
      s_carry[wib][lane] = 0;
      __syncwarp();
      for (int b2 = 0; b2 < total; b2 += 32) {
        const int r = b2 + lane;
        const int o = owner(st, r);
        const int ofirst = __shfl_sync(0xffffffffu, row_first, o);
        const uint32_t obase = __shfl_sync(0xffffffffu, rbase, o);
        const int ost = __shfl_sync(0xffffffffu, st, o);
        // the row's index in pass 1 (the owner's rows from its rectangle's first row on)
        const int r1 = __shfl_sync(0xffffffffu, st1, o) + (ofirst - __shfl_sync(0xffffffffu, P.y0, o)) + (r - ost);
        const bool cached = r < total && r1 < kSpanCache;
        int2 sp = make_int2(1, 0);
        int ty = 0, len = 0;
        if (__all_sync(0xffffffffu, cached || r >= total)) {
          if (r < total) {
            ty = ofirst + (r - ost);
            sp = s_span[wib][r1];
          }
        } else {
          const Ellipse eo = owner_ellipse(P.E, o);
          const int ox0 = __shfl_sync(0xffffffffu, P.x0, o), ox1 = __shfl_sync(0xffffffffu, P.x1, o);
          if (r < total) {
            ty = ofirst + (r - ost);
            sp = cached ? s_span[wib][r1] : row_span(eo, ty, ox0, ox1);
          }
        }
        len = sp.x <= sp.y ? sp.y - sp.x + 1 : 0;
        // inclusive sum of len over this round's rows of the same item (they are adjacent lanes)
        int inc = len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, inc, d);
          const int od = __shfl_up_sync(0xffffffffu, o, d);
          if (lane >= d && od == o) inc += y;
        }
        const int carry = s_carry[wib][o];
        if (r < total)
          tab[obase + static_cast<uint32_t>(ty - ofirst)] = make_int2(carry + inc - len, (sp.x & 0xffff) | (ty << 16));
        const int onext = __shfl_down_sync(0xffffffffu, o, 1);
        __syncwarp();
        if (lane == 31 || onext != o) s_carry[wib][o] = carry + inc;
        __syncwarp();
      }
    }
    // the live items of this round, in item order: their bits, and their binning records at
    // the end of the block's segment
    const uint32_t ballot = __ballot_sync(0xffffffffu, is_live);
    if (lane == 0) s_wcnt[wib] = __popc(ballot);
    __syncthreads();
    uint32_t before = s_seg;
    for (int w = 0; w < wib; ++w) before += s_wcnt[w];
    if (is_live) {
      atomicOr(&s_live[(idx - first) >> 5], 1u << (idx & 31));
      const int64_t pos = first + before + __popc(ballot & lm);
      at<uint32_t>(ws, L.item_keys[1])[pos] = item_key;        // staging: depth-sort key
      at<uint32_t>(ws, L.item_vals[1])[pos] = static_cast<uint32_t>(idx);  // staging: item id
      at<uint32_t>(ws, L.sorted_counts)[pos] = count;          // staging: tiles emitted
      at<uint2>(ws, L.item_rect)[pos] = rows_out;              // staging: row-span entries (as uint2)
#pragma unroll
      for (int p = 0; p < 4; ++p) atomicAdd(&s_hist[p * 256 + ((item_key >> (8 * p)) & 0xffu)], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t tot = 0;
      for (int w = 0; w < kProjThreads / 32; ++w) tot += s_wcnt[w];
      s_seg += tot;
    }
  }
  __syncthreads();
  // the block's live mask words, its live count, its span grid and its histograms
  if (threadIdx.x < words) {
    const int64_t w = first / 32 + threadIdx.x;
    if (w < (L.KN + 31) / 32) at<uint32_t>(ws, L.live_mask)[w] = s_live[threadIdx.x];
  }
  if (threadIdx.x == 0) at<uint32_t>(ws, L.live_blocks)[blk] = s_seg;
  if (use_sgrid && n_surv > 0 && k_block < L.K) {
    int32_t* dg = at<int32_t>(ws, L.tile_diff) + static_cast<int64_t>(k_block) * gcells;
    for (int i = threadIdx.x; i < gcells; i += kProjThreads)
      if (s_grid[i]) atomicAdd(&dg[i], s_grid[i]);
  }
  uint32_t* hist = at<uint32_t>(ws, L.item_hist);
  for (int i = threadIdx.x; i < 4 * 256; i += kProjThreads)
    if (s_hist[i]) atomicAdd(&hist[i], s_hist[i]);
  // clear the look-back status of the item sort
  const uint64_t used = static_cast<uint64_t>(L.max_item_tiles) * 256;
  const uint64_t gsize = static_cast<uint64_t>(gridDim.x) * kProjThreads;
  uint32_t* sst = at<uint32_t>(ws, L.item_status);
  for (int p = 0; p < 4; ++p)
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * kProjThreads + threadIdx.x; i < used; i += gsize)
      sst[static_cast<uint64_t>(p) * used + i] = 0;
  // the last block to finish scans the blocks' live counts: each block's first position among
  // the live items (live_bases), and the number of live items
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  Status* st = at<Status>(ws, L.status);
  if (threadIdx.x == 0) s_last = atomicAdd(&st->proj_done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last) {
    __threadfence();
    const uint32_t* cnt = at<uint32_t>(ws, L.live_blocks);
    uint32_t* bases = at<uint32_t>(ws, L.live_bases);
    uint32_t carry = 0;
    for (int64_t b0 = 0; b0 < L.n_proj_groups; b0 += kProjThreads) {
      const int64_t b = b0 + threadIdx.x;
      const uint32_t x = b < L.n_proj_groups ? __ldcg(&cnt[b]) : 0u;
      uint32_t incl = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (lane == 31) s_wcnt[wib] = incl;
      __syncthreads();
      uint32_t before = 0, total = 0;
      for (int w = 0; w < kProjThreads / 32; ++w) {
        before += w < wib ? s_wcnt[w] : 0u;
        total += s_wcnt[w];
      }
      if (b < L.n_proj_groups) bases[b] = carry + before + incl - x;
      carry += total;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      st->n_live = carry;
      st->proj_done = 0;
    }
  }
  pdl_trigger();
}

// Compaction of the live items, in increasing item order k N + g: each projection block's
// segment of staged binning records goes to the block's first position among the live items,
// as the depth-sort keys (the item sort's input, with values = positions), the items' ids,
// tiles emitted and row-span entries; and each live-mask word's rank base (live_wpre).
__global__ void __launch_bounds__(kProjThreads) k_live_copy(Layout L, uint8_t* __restrict__ ws) {
  pdl_begin();
  constexpr int kWords = kProjItemsMax / 32;
  const int64_t b = blockIdx.x, first = b * L.proj_items;
  const uint32_t cnt = at<uint32_t>(ws, L.live_blocks)[b], base = at<uint32_t>(ws, L.live_bases)[b];
  for (uint32_t i = threadIdx.x; i < cnt; i += kProjThreads) {
    const uint32_t pos = base + i;
    at<uint32_t>(ws, L.item_keys[0])[pos] = at<uint32_t>(ws, L.item_keys[1])[first + i];
    at<uint32_t>(ws, L.item_vals[0])[pos] = pos;
    at<uint32_t>(ws, L.live_kg)[pos] = at<uint32_t>(ws, L.item_vals[1])[first + i];
    at<uint32_t>(ws, L.live_count)[pos] = at<uint32_t>(ws, L.sorted_counts)[first + i];
    at<uint2>(ws, L.live_rows)[pos] = at<uint2>(ws, L.item_rect)[first + i];
  }
  // rank bases of the block's mask words (warps 0-1: up to 64 words)
  if (threadIdx.x < kWords) {
    const int64_t w = first / 32 + threadIdx.x;
    const bool in = threadIdx.x < L.proj_items / 32 && w < (L.KN + 31) / 32;
    const uint32_t c = in ? __popc(at<uint32_t>(ws, L.live_mask)[w]) : 0u;
    uint32_t incl = c;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    __shared__ uint32_t s_w0;
    if (threadIdx.x == 31) s_w0 = incl;
    __syncwarp();
    asm volatile("bar.sync 1, 64;");  // the two warps of the mask words
    const uint32_t off = threadIdx.x >= 32 ? s_w0 : 0u;
    if (in) at<uint32_t>(ws, L.live_wpre)[w] = base + off + incl - c;
  }
}

}  // namespace

cudaError_t launch_project(const Layout& L, const GaussPtrs& g, const gs_camera_t* cams, void* ws, cudaStream_t s) {
  auto* w = static_cast<uint8_t*>(ws);
  const unsigned groups = static_cast<unsigned>(L.n_proj_groups);
  launch(k_project, groups, kProjThreads, 0, s, L, g, cams, w);
  launch(k_live_copy, groups, kProjThreads, 0, s, L, w);
  return cudaGetLastError();
}

}  // namespace gs
