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

__device__ __forceinline__ uint32_t pack16(int lo, int hi) {
  return static_cast<uint32_t>(lo) | (static_cast<uint32_t>(hi) << 16);
}

__global__ void __launch_bounds__(kProjBlock, 3) k_project(Layout L, GaussPtrs G, const gs_camera_t* __restrict__ cams,
                                                       uint8_t* __restrict__ ws) {
  pdl_wait();
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * kProjBlock + threadIdx.x;
  __shared__ uint32_t s_hist[4 * 256];
  // the block's rectangles are first added into a shared copy of its first view's difference
  // grid (when it fits), then flushed with one global atomic per non-zero cell
  __shared__ int32_t s_grid[kProjGridCells];
  const int gstride = L.Tx + 1;
  const int gcells = gstride * (L.Ty + 1);
  const bool use_sgrid = gcells <= kProjGridCells;
  const int k_block = static_cast<int>((static_cast<int64_t>(blockIdx.x) * kProjBlock) / (L.N > 0 ? L.N : 1));
  for (int i = threadIdx.x; i < 4 * 256; i += kProjBlock) s_hist[i] = 0;
  if (use_sgrid)
    for (int i = threadIdx.x; i < gcells; i += kProjBlock) s_grid[i] = 0;
  __syncthreads();
  uint32_t count = 0, item_key = 0xffffffffu;
  // the item's widened ellipse and tile rectangle, for the warp's row passes below
  Ellipse E{};
  int x0 = 0, x1 = 0, y0 = 0, y1 = 0, kv = 0;
  bool live = false;
  float z_item = 0.0f;
  if (idx < L.KN) {
    const int k = static_cast<int>(idx / L.N);
    const int64_t g = idx - static_cast<int64_t>(k) * L.N;
    const gs_camera_t cam = cams[k];
    const float p0 = load_attr(G.means, 3 * g + 0, G.means_dtype);
    const float p1 = load_attr(G.means, 3 * g + 1, G.means_dtype);
    const float p2 = load_attr(G.means, 3 * g + 2, G.means_dtype);
    float ls[3], q[4];
    for (int j = 0; j < 3; ++j) ls[j] = load_attr(G.log_scales, 3 * g + j, G.dtype);
    for (int j = 0; j < 4; ++j) q[j] = load_attr(G.quats, 4 * g + j, G.dtype);
    const float* R = cam.R;
    const float* t = cam.t;
    const float lg = load_attr(G.logits, g, G.dtype);
    // colour and opacity: once per Gaussian, or per item when the colour depends on the view
    if (k == 0 || L.color_stride != 0) {
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

    // ---------------- discrete path: fixed binary32 operation order -----------------
    bool valid = true;
    const float xc = __fmaf_rn(R[0], p0, __fmaf_rn(R[1], p1, __fmaf_rn(R[2], p2, t[0])));
    const float yc = __fmaf_rn(R[3], p0, __fmaf_rn(R[4], p1, __fmaf_rn(R[5], p2, t[1])));
    const float zc = __fmaf_rn(R[6], p0, __fmaf_rn(R[7], p1, __fmaf_rn(R[8], p2, t[2])));
    valid = zc > L.near_plane;
    const float n2 = __fmaf_rn(q[0], q[0], __fmaf_rn(q[1], q[1], __fmaf_rn(q[2], q[2], __fmul_rn(q[3], q[3]))));
    const float nq = __fsqrt_rn(n2);
    valid = valid && (nq > 0.0f);
    const float qw = __fdiv_rn(q[0], nq), qx = __fdiv_rn(q[1], nq), qy = __fdiv_rn(q[2], nq),
                qz = __fdiv_rn(q[3], nq);
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
    int radius = 0;
    if (valid) {
      x0 = static_cast<int>(x0f);
      x1 = static_cast<int>(x1f);
      y0 = static_cast<int>(y0f);
      y1 = static_cast<int>(y1f);
      radius = static_cast<int>(rf);
      if ((x1 - x0) * (y1 - y0) == 0) {
        x0 = x1 = y0 = y1 = radius = 0;
      } else {
        // the widened alpha >= 1/255 ellipse; its rows are examined by the warp below
        const float op = __fdiv_rn(1.0f, __fadd_rn(1.0f, exp_det(-lg)));
        const float Lg = log_det(__fmul_rn(255.0f, op));
        const float Lm = __fadd_rn(__fadd_rn(Lg, __fmul_rn(0.02f, fabsf(Lg))), 1.5e-4f);
        if (Lm >= 0.0f) {
          const float kap = __fmul_rn(2.0f, Lm);
          E = Ellipse{u, v, bb, __fdiv_rn(1.0f, c), __fsqrt_rn(det), __fsqrt_rn(__fmul_rn(kap, a)),
                      __fsqrt_rn(__fmul_rn(kap, c)), __fdiv_rn(bb, a)};
          at<Ellipse>(ws, L.proj_ell)[idx] = E;
          live = true;
        }
      }
    }
    at<uint32_t>(ws, L.proj_depth_key)[idx] = __float_as_uint(zc);
    at<int32_t>(ws, L.proj_radius)[idx] = radius;
    kv = k;
    z_item = zc;

    // ---------------- continuous path ----------------------------------------------
    if (live) {  // (the records of an item that emits nothing are never read)
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
  }

  // ---------------- the rectangle's rows, shared out over the warp -------------------
  // The warp's items' rows are numbered consecutively (item by item) and examined 32 at a time,
  // one row per lane, so a warp holding one tall rectangle does not idle the other lanes. A row
  // owner's ellipse and rectangle come from its lane by shuffles. Pass 1 counts each item's
  // emitted tiles and finds its first and last non-empty rows (and adds the spans to the span
  // grid); pass 2 writes the item's row-span table entries.
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  __shared__ int s_acc[kProjBlock / 32][3][32];  // per warp and lane: tiles, first row, last row
  s_acc[wib][0][lane] = 0;
  s_acc[wib][1][lane] = 0x7fffffff;
  s_acc[wib][2][lane] = -1;
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
  auto owner_ellipse = [&](int o) {
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
  {
    int total = 0;
    const int st = warp_excl_scan(live ? y1 - y0 : 0, total);
    __syncwarp();
    for (int base = 0; base < total; base += 32) {
      const int r = base + lane;
      const int o = owner(st, r);
      const Ellipse eo = owner_ellipse(o);
      const int ox0 = __shfl_sync(0xffffffffu, x0, o), ox1 = __shfl_sync(0xffffffffu, x1, o);
      const int oy0 = __shfl_sync(0xffffffffu, y0, o), ok = __shfl_sync(0xffffffffu, kv, o);
      const int ost = __shfl_sync(0xffffffffu, st, o);
      if (r < total) {
        const int ty = oy0 + (r - ost);
        const int2 sp = row_span(eo, ty, ox0, ox1);
        if (sp.x <= sp.y) {
          atomicAdd(&s_acc[wib][0][o], sp.y - sp.x + 1);
          atomicMin(&s_acc[wib][1][o], ty);
          atomicMax(&s_acc[wib][2][o], ty);
          int32_t* dg = (use_sgrid && ok == k_block) ? s_grid
                                                      : at<int32_t>(ws, L.tile_diff) + static_cast<int64_t>(ok) * gcells;
          atomicAdd(&dg[ty * gstride + sp.x], 1);  // row-wise prefix sum: pairs per tile
          atomicAdd(&dg[ty * gstride + sp.y + 1], -1);
        }
      }
    }
    __syncwarp();
  }
  count = static_cast<uint32_t>(s_acc[wib][0][lane]);
  const int row_first = s_acc[wib][1][lane];
  const uint32_t nrows = count ? static_cast<uint32_t>(s_acc[wib][2][lane] - row_first + 1) : 0u;
  if (idx < L.KN) {
    if (count) item_key = __float_as_uint(z_item);
    at<int4>(ws, L.proj_tiles)[idx] =
        make_int4(0, static_cast<int>(pack16(x0, x1)), static_cast<int>(pack16(y0, y1)), static_cast<int>(count));
  }
  // row-span table entries for the item's rows first..last (one counter atomic per warp)
  {
    uint32_t incl = nrows;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    uint32_t base = 0;
    if (lane == 31 && incl) base = atomicAdd(&at<Status>(ws, L.status)->row_ctr, incl);
    base = __shfl_sync(0xffffffffu, base, 31) + (incl - nrows);
    const bool fits = nrows && static_cast<uint64_t>(base) + nrows <= static_cast<uint64_t>(L.cap);
    if (nrows && !fits) atomicOr(&at<Status>(ws, L.status)->err, GS_DEVERR_PAIR_OVERFLOW);
    if (idx < L.KN) at<uint2>(ws, L.proj_rows)[idx] = fits ? make_uint2(base, nrows) : make_uint2(0, 0);
    int total = 0;
    const int st = warp_excl_scan(fits ? static_cast<int>(nrows) : 0, total);
    int2* tab = at<int2>(ws, L.row_table);
    __shared__ int s_carry[kProjBlock / 32][32];  // tiles in the item's rows already written
    s_carry[wib][lane] = 0;
    __syncwarp();
    for (int b2 = 0; b2 < total; b2 += 32) {
      const int r = b2 + lane;
      const int o = owner(st, r);
      const Ellipse eo = owner_ellipse(o);
      const int ox0 = __shfl_sync(0xffffffffu, x0, o), ox1 = __shfl_sync(0xffffffffu, x1, o);
      const int ofirst = __shfl_sync(0xffffffffu, row_first, o);
      const uint32_t obase = __shfl_sync(0xffffffffu, base, o);
      const int ost = __shfl_sync(0xffffffffu, st, o);
      int2 sp = make_int2(1, 0);
      int ty = 0, len = 0;
      if (r < total) {
        ty = ofirst + (r - ost);
        sp = row_span(eo, ty, ox0, ox1);
        len = sp.x <= sp.y ? sp.y - sp.x + 1 : 0;
      }
      // inclusive sum of len over this round's rows of the same item (they are adjacent lanes)
      int inc = len;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, d);
        const int od = __shfl_up_sync(0xffffffffu, o, d);
        if (lane >= d && od == o) inc += y;
      }
      const int carry = s_carry[wib][o];
      if (r < total) tab[obase + static_cast<uint32_t>(ty - ofirst)] = make_int2(carry + inc - len, (sp.x & 0xffff) | (ty << 16));
      const int onext = __shfl_down_sync(0xffffffffu, o, 1);
      __syncwarp();
      if (lane == 31 || onext != o) s_carry[wib][o] = carry + inc;
      __syncwarp();
    }
  }
  // depth-sort key of the item (culled items sort last and emit nothing) and its digit counts
  if (idx < L.KN) {
    const uint32_t key = item_key;
    at<uint32_t>(ws, L.item_keys[0])[idx] = key;
    at<uint32_t>(ws, L.item_vals[0])[idx] = static_cast<uint32_t>(idx);
#pragma unroll
    for (int p = 0; p < 4; ++p) atomicAdd(&s_hist[p * 256 + ((key >> (8 * p)) & 0xffu)], 1u);
  }
  __syncthreads();
  if (use_sgrid && k_block < L.K) {
    int32_t* dg = at<int32_t>(ws, L.tile_diff) + static_cast<int64_t>(k_block) * gcells;
    for (int i = threadIdx.x; i < gcells; i += kProjBlock)
      if (s_grid[i]) atomicAdd(&dg[i], s_grid[i]);
  }
  uint32_t* hist = at<uint32_t>(ws, L.item_hist);
  for (int i = threadIdx.x; i < 4 * 256; i += kProjBlock)
    if (s_hist[i]) atomicAdd(&hist[i], s_hist[i]);
  // clear the look-back status of the item sort
  const uint64_t used = static_cast<uint64_t>(L.max_item_tiles) * 256;
  const uint64_t gsize = static_cast<uint64_t>(gridDim.x) * kProjBlock;
  uint32_t* st = at<uint32_t>(ws, L.item_status);
  for (int p = 0; p < 4; ++p)
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * kProjBlock + threadIdx.x; i < used; i += gsize)
      st[static_cast<uint64_t>(p) * used + i] = 0;
  pdl_trigger();
}

}  // namespace

cudaError_t launch_project(const Layout& L, const GaussPtrs& g, const gs_camera_t* cams, void* ws, cudaStream_t s) {
  launch(k_project, static_cast<unsigned>(L.n_proj_blocks), kProjBlock, 0, s, L, g, cams, static_cast<uint8_t*>(ws));
  return cudaGetLastError();
}

}  // namespace gs
