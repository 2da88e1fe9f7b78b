// Tile compositing: forward (render) and backward (splat gradients).
//
// One CTA per (view, 16x16 tile). Each thread owns PX vertically adjacent pixels of one
// column (PX = 1, 2 or 4, chosen per workload), so the horizontal offset to a splat is
// shared and every splat record loaded from shared memory serves PX pixels. The per-pixel
// update is branch-free (a masked blend with weight 0 leaves every accumulator bit for bit
// unchanged), so the PX pixel chains interleave, and pairs of them share packed FP32
// instructions (add / multiply / FMA on two pixels at once). The tile's depth-sorted list is
// walked in chunks staged in shared memory as three float4 and a row mask per splat (coalesced
// loads of the sorted keys, whose low word is the Gaussian id, one gather of the projected
// record each).
//
// Both kernels evaluate a splat's opacity with the same inline function on the same
// operands, so the backward pass takes exactly the forward pass's skip and stop decisions
// and recovers the same transmittance T_i front to back, without storing per-splat alphas.
//
// The backward pass sums each splat's 10 gradient sums over a warp's pixels (PX per lane,
// then a 12-shuffle warp reduction), writes one partial per warp into shared memory, and at
// the end of each chunk sums the warp partials in a fixed order into one record per
// (splat, tile) pair of the pair-gradient buffer, marking the pair in a bit mask; pairs
// behind every pixel's last contributor of their tile get no record (their gradient is
// zero). No floating-point atomics: the gradients are deterministic.
//
// This header holds what both compositing kernels share (raster_fwd.cu, raster_bwd.cu).
#pragma once

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTStop = 1e-4f;
// Resident blocks per SM the compiler must fit at 4 pixels per thread (64 threads): a register
// budget of 80 per thread (no spills) for the forward and backward kernels, 72 (a few spilled
// bytes) for the fused forward + backward. The packed pixel pairs leave the compositing loops
// bound by instruction latency as much as by issue, and more resident blocks hide more of it
// (the fused kernel at aerial2m: 6.68 ms at 10 blocks, 6.15 at 12, 6.00 at 14).
constexpr int kMinBlocksPx4 = 12;
constexpr int kMinBlocksFusedPx4 = 14;
constexpr int kFwdChunk = 128;  // splats staged per forward chunk (default; 64 and 256 also built)
constexpr int kBwdChunk = 64;   // splats staged per backward chunk (default; 32 and 128 also built)

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Packed FP32 (sm_100 family): one instruction applies an add, a multiply or a fused
// multiply-add to two pixels' operands, each component rounded exactly as the scalar
// __fadd_rn / __fmul_rn / __fmaf_rn would round it. A thread's PX pixels are processed in
// groups of W = 2 (PX = 2, 4) or W = 1 (PX = 1) components, so every variant still takes
// bit-identical decisions; a splat's operands are broadcast into register pairs once per splat
// (staging them duplicated in shared memory instead costs more in loads and shared memory than
// the broadcasts).
template <int W>
struct Vec;
template <>
struct Vec<1> {
  using T = float;
};
template <>
struct Vec<2> {
  using T = float2;
};
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float comp(float v, int) { return v; }
__device__ __forceinline__ float comp(float2 v, int i) { return i ? v.y : v.x; }
__device__ __forceinline__ void set_comp(float& v, int, float x) { v = x; }
__device__ __forceinline__ void set_comp(float2& v, int i, float x) {
  if (i) v.y = x;
  else v.x = x;
}
__device__ __forceinline__ float hsum(float v) { return v; }
__device__ __forceinline__ float hsum(float2 v) { return v.x + v.y; }
template <int W>
__device__ __forceinline__ typename Vec<W>::T bcast(float x) {
  if constexpr (W == 1) return x;
  else return make_float2(x, x);
}
// Staged splat: A = (x, y, qa, qb), B = (qc, opacity, depth, log2 opacity), C = (r, g, b, -) where
// (x, y) is the 2D mean relative to the tile origin and power * log2(e) = qa dx^2 + qb dx dy + qc dy^2.
// rows: bit r is set when the splat's ellipse {opacity * 2^power >= 1/255}, widened by a safety
// margin, meets the pixel-centre row y = r + 0.5 of the tile within the columns [0.5, 15.5]. A
// warp none of whose rows is set skips the splat without changing any decision.
template <int CH>
struct Stage {
  float4 A[CH], B[CH], C[CH];
  uint32_t rows[CH];
};

// Rows of the tile (bit r: pixel-centre row r) met by the ellipse Q(d) = Qa dx^2 + Qb dx dy +
// Qc dy^2 <= tau around (mx, my), inside the column strip [0.5, 15.5]. The ellipse's part
// inside the strip is convex, so its y-extent is an interval: its ends are the ellipse's
// top / bottom points when they lie inside the strip, else the ellipse's crossings of the
// strip edge on their side. Margins: 2% + 2e-4 on tau (log2 units), 0.05 px on the strip, 0.05
// px + 0.2% of the half-height on the interval; they also cover the few-ulp errors of the
// approximate logarithm, quotients and square roots used here (every staged splat computes its
// mask, in both passes). Anything that is not a proper ellipse keeps every row.
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ uint32_t splat_rows(float mx, float my, float Qa, float Qb, float Qc, float opacity) {
  const float tau0 = __log2f(255.0f * opacity);
  const float tau = tau0 + 0.02f * fabsf(tau0) + 2e-4f;
  if (!(tau >= 0.0f)) return 0u;  // opacity below 1/255 (or NaN): no pixel keeps the splat
  // determinant Qa Qc - (Qb/2)^2 with the products' rounding errors restored (no cancellation)
  const float h = 0.5f * Qb;
  const float p1 = Qa * Qc, p2 = h * h;
  const float D = (p1 - p2) + (fmaf(Qa, Qc, -p1) - fmaf(h, h, -p2));
  if (!(Qa > 0.0f) || !(Qc > 0.0f) || !(D > 0.0f)) return 0xffffu;
  const float hx = sqrt_approx(__fdividef(tau * Qc, D)), hy = sqrt_approx(__fdividef(tau * Qa, D));
  if (!(hx < 1e7f) || !(hy < 1e7f)) return 0xffffu;
  constexpr float xa = 0.5f - 0.05f, xb = 15.5f + 0.05f;
  if (mx + hx < xa || mx - hx > xb) return 0u;
  const float sl = __fdividef(h, Qa);  // the ellipse's widest chord at height dy is centred on mx - sl dy
  const float xt = mx - sl * hy, xbot = mx + sl * hy;
  // dy where the ellipse crosses x = xe (upper: sign +1)
  auto cross = [&](float xe, float sign) {
    const float dxe = xe - mx, ad = fabsf(dxe);
    const float disc = fmaxf(D * (hx - ad) * (hx + ad), 0.0f);  // Qc tau - D dxe^2
    return __fdividef(fmaf(sign, sqrt_approx(disc), -h * dxe), Qc);
  };
  const float up = xt < xa ? cross(xa, 1.0f) : (xt > xb ? cross(xb, 1.0f) : hy);
  const float dn = xbot < xa ? cross(xa, -1.0f) : (xbot > xb ? cross(xb, -1.0f) : -hy);
  const float mm = fmaf(2e-3f, hy, 0.05f);
  const float r0 = fmaxf(ceilf(my + dn - mm - 0.5f), 0.0f);
  const float r1 = fminf(floorf(my + up + mm - 0.5f), 15.0f);
  if (r0 > r1) return 0u;  // (a NaN bound leaves its side at the tile edge)
  return (2u << static_cast<int>(r1)) - (1u << static_cast<int>(r0));
}

template <int CH>
__device__ __forceinline__ uint32_t stage_splat(Stage<CH>& S, int j, const Layout& L, const uint8_t* ws,
                                                const uint64_t* keys, uint32_t i, int k, float ox, float oy) {
  uint32_t gid = static_cast<uint32_t>(keys[i]);  // sorted key = (tile << 32) | Gaussian id
  if (!GS_INDEX_OK(static_cast<int64_t>(gid) < L.N, &at<Status>(const_cast<uint8_t*>(ws), L.status)->err)) gid = 0;
  const int64_t kg = static_cast<int64_t>(k) * L.N + gid;
  const float4 uv = at<float4>(ws, L.proj_uv)[kg];
  const float4 cn = at<float4>(ws, L.proj_conic)[kg];
  const float4 co = at<float4>(ws, L.color_opacity)[k * L.color_stride + gid];
  const float x = __fadd_rn(__fsub_rn(uv.x, ox), uv.y), y = __fadd_rn(__fsub_rn(uv.z, oy), uv.w);
  const float qa = __fmul_rn(cn.x, -0.5f * kLog2e), qb = __fmul_rn(cn.y, -kLog2e), qc = __fmul_rn(cn.z, -0.5f * kLog2e);
  const float lo = __log2f(co.w);
  S.A[j] = make_float4(x, y, qa, qb);
  S.B[j] = make_float4(qc, co.w, cn.w, lo);
  S.C[j] = make_float4(co.x, co.y, co.z, 0.0f);
  S.rows[j] = splat_rows(x, y, -qa, -qb, -qc, co.w);
  return gid;
}

// Opacity of a splat at a pixel, in one form shared by every compositing kernel, so that they
// all take the same decisions. For the pixel column at offset dx = x - (column + 0.5) from the
// splat's mean, a lane forms once per splat (splat_column)
//   c1 = qb dx,   c0 = qa dx^2 + log2(opacity),
// and per pixel row at offset dy the exponent  e = (qc dy + c1) dy + c0 = power log2(e) + log2(o),
// so raw = 2^e = opacity * exp(power) costs two FMAs and one ex2. The splat is kept at the pixel
// (not skipped) when power <= 0, i.e. e <= log2(o), and alpha = min(raw, 0.99) >= 1/255.
// The offsets are formed as additions of the negated pixel centre (exact small integers + 0.5),
// which round exactly as the subtractions would.
template <int W>
struct Column {
  typename Vec<W>::T dx, c1, c0;
};
template <int W>
__device__ __forceinline__ Column<W> splat_column(const float4& A, const float4& B, typename Vec<W>::T npx) {
  Column<W> c;
  c.dx = vadd(bcast<W>(A.x), npx);
  c.c1 = vmul(bcast<W>(A.w), c.dx);
  c.c0 = vfma(vmul(bcast<W>(A.z), c.dx), c.dx, bcast<W>(B.w));
  return c;
}
template <int W>
__device__ __forceinline__ typename Vec<W>::T splat_exponent(const float4& B, const Column<W>& c,
                                                             typename Vec<W>::T dy) {
  return vfma(vfma(bcast<W>(B.x), dy, c.c1), dy, c.c0);
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct TileCoord {
  int k, tx, ty;
};
__device__ __forceinline__ TileCoord tile_coord(const Layout& L, int64_t tile_g) {
  const int64_t per_view = static_cast<int64_t>(L.Tx) * L.Ty;
  TileCoord c;
  c.k = static_cast<int>(tile_g / per_view);
  const int tt = static_cast<int>(tile_g - c.k * per_view);
  c.ty = tt / L.Tx;
  c.tx = tt - c.ty * L.Tx;
  return c;
}

int pick_px(int requested, int fallback) { return (requested == 1 || requested == 2 || requested == 4) ? requested : fallback; }
// chunk depth: a power of two in [lo, hi], else the default
int pick_chunk(int requested, int lo, int hi, int fallback) {
  return (requested >= lo && requested <= hi && (requested & (requested - 1)) == 0) ? requested : fallback;
}


}  // namespace
}  // namespace gs
