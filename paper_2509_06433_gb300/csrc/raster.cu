// Tile compositing: forward (render) and backward (splat gradients).
//
// One CTA per (view, 16x16 tile). Each thread owns PX vertically adjacent pixels of one
// column (PX = 1, 2 or 4, chosen per workload), so the horizontal offset to a splat is
// shared and every splat record loaded from shared memory serves PX pixels. The per-pixel
// update is branch-free (a masked blend with weight 0 leaves every accumulator bit for bit
// unchanged), so the PX pixel chains interleave. The tile's depth-sorted list is walked in
// chunks staged in shared memory as three float4 and a row mask per splat (coalesced loads
// of the sorted keys, whose low word is the Gaussian id, one gather of the projected record each).
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
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTStop = 1e-4f;
constexpr int kFwdChunk = 128;  // splats staged per forward chunk
constexpr int kBwdChunk = 64;   // splats staged per backward chunk

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Staged splat: A = (x, y, qa, qb), B = (qc, opacity, depth, -), C = (r, g, b, -) where
// (x, y) is the 2D mean relative to the tile origin and power * log2(e) = qa dx^2 + qb dx dy + qc dy^2.
// rows: bit r is set when the splat's ellipse {opacity * 2^power >= 1/255}, widened by a safety
// margin, meets the pixel-centre row y = r + 0.5 of the tile within the columns [0.5, 15.5].
// A warp none of whose rows is set skips the splat without changing any decision.
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
// px + 0.2% of the half-height on the interval. Anything that is not a proper ellipse keeps
// every row.
__device__ __forceinline__ uint32_t splat_rows(float mx, float my, float Qa, float Qb, float Qc, float opacity) {
  const float tau0 = log2f(255.0f * opacity);
  const float tau = tau0 + 0.02f * fabsf(tau0) + 2e-4f;
  if (!(tau >= 0.0f)) return 0u;  // opacity below 1/255 (or NaN): no pixel keeps the splat
  // determinant Qa Qc - (Qb/2)^2 with the products' rounding errors restored (no cancellation)
  const float h = 0.5f * Qb;
  const float p1 = Qa * Qc, p2 = h * h;
  const float D = (p1 - p2) + (fmaf(Qa, Qc, -p1) - fmaf(h, h, -p2));
  if (!(Qa > 0.0f) || !(Qc > 0.0f) || !(D > 0.0f)) return 0xffffu;
  const float hx = sqrtf(tau * Qc / D), hy = sqrtf(tau * Qa / D);
  if (!(hx < 1e7f) || !(hy < 1e7f)) return 0xffffu;
  constexpr float xa = 0.5f - 0.05f, xb = 15.5f + 0.05f;
  if (mx + hx < xa || mx - hx > xb) return 0u;
  const float sl = h / Qa;  // the ellipse's widest chord at height dy is centred on mx - sl dy
  const float xt = mx - sl * hy, xbot = mx + sl * hy;
  // dy where the ellipse crosses x = xe (upper: sign +1)
  auto cross = [&](float xe, float sign) {
    const float dxe = xe - mx, ad = fabsf(dxe);
    const float disc = fmaxf(D * (hx - ad) * (hx + ad), 0.0f);  // Qc tau - D dxe^2
    return (fmaf(sign, sqrtf(disc), -h * dxe)) / Qc;
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
  const uint32_t gid = static_cast<uint32_t>(keys[i]);  // sorted key = (tile << 32) | Gaussian id
  const int64_t kg = static_cast<int64_t>(k) * L.N + gid;
  const float4 uv = at<float4>(ws, L.proj_uv)[kg];
  const float4 cn = at<float4>(ws, L.proj_conic)[kg];
  const float4 co = at<float4>(ws, L.color_opacity)[gid];
  const float x = __fadd_rn(__fsub_rn(uv.x, ox), uv.y), y = __fadd_rn(__fsub_rn(uv.z, oy), uv.w);
  const float qa = __fmul_rn(cn.x, -0.5f * kLog2e), qb = __fmul_rn(cn.y, -kLog2e), qc = __fmul_rn(cn.z, -0.5f * kLog2e);
  S.A[j] = make_float4(x, y, qa, qb);
  S.B[j] = make_float4(qc, co.w, cn.w, 0.0f);
  S.C[j] = make_float4(co.x, co.y, co.z, 0.0f);
  S.rows[j] = splat_rows(x, y, -qa, -qb, -qc, co.w);
  return gid;
}

// Opacity of a splat at pixel offset (dx, dy) with qadx = qa * dx. keep: the splat is not
// skipped (power <= 0 and alpha >= 1/255). G = exp(power); raw = opacity * G before the clamp.
struct Alpha {
  float alpha, G, raw;
  bool keep;
};
__device__ __forceinline__ Alpha splat_alpha(const float4& A, const float4& B, float qadx, float dx, float dy) {
  Alpha r;
  const float p = __fmaf_rn(dx, __fmaf_rn(A.w, dy, qadx), __fmul_rn(__fmul_rn(B.x, dy), dy));
  r.G = ex2_approx(p);
  r.raw = __fmul_rn(B.y, r.G);
  r.alpha = fminf(r.raw, kAlphaMax);
  r.keep = (p <= 0.0f) && (r.alpha >= kAlphaMin);
  return r;
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

// ============================================================================ forward
// Per pixel, amin is the opacity a splat must reach to be kept: 1/255 while the pixel is
// open, +inf once it has stopped (or lies outside the image), so a stopped pixel skips every
// later splat without a separate flag. A kept splat that does not stop the pixel is blended
// through ae = alpha (else ae = 0): w = ae T and T <- T - ae T leave every accumulator bit for
// bit unchanged when ae = 0, so the blend needs no selects. STATS = true also counts the
// evaluations (list entries examined, including the one that stops a pixel) and the blended
// ones; the decisions and outputs are the same.
// L1 loss fused into the forward pass (LOSS = true): the targets, the gradient images it
// writes, per-tile partial sums and the block counter that elects the last block to finish,
// which sums the partials in tile order into *d_loss.
struct FusedLoss {
  const float* rgb_t;
  const float* depth_t;
  float* g_rgb;
  float* g_depth;
  float* partials;
  uint32_t* counter;
  float* d_loss;
};

__device__ __forceinline__ float sgn(float d) { return d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f); }

template <int PX, bool STATS, bool LOSS>
__global__ void __launch_bounds__(kTilePixels / PX) k_raster_fwd(Layout L, const uint8_t* __restrict__ ws,
                                                                 float* __restrict__ out_rgb,
                                                                 float* __restrict__ out_depth,
                                                                 float* __restrict__ out_T,
                                                                 int32_t* __restrict__ out_last,
                                                                 uint64_t* __restrict__ evals_out,
                                                                 uint64_t* __restrict__ blended_out, FusedLoss F) {
  pdl_wait();
  constexpr int kThreads = kTilePixels / PX;
  constexpr int kWarps = kThreads / 32;
  const float kInf = __int_as_float(0x7f800000);
  __shared__ Stage<kFwdChunk> S;
  __shared__ uint32_t s_red[2][kWarps];
  const TileCoord tc = tile_coord(L, blockIdx.x);
  const int lx = threadIdx.x & (kTile - 1), ly = (threadIdx.x / kTile) * PX;
  const int px = tc.tx * kTile + lx, py = tc.ty * kTile + ly;
  const uint64_t* keys = at<uint64_t>(ws, (L.passes & 1) ? L.keys[1] : L.keys[0]);
  const uint2 rg = at<uint2>(ws, L.ranges)[blockIdx.x];
  const float ox = static_cast<float>(tc.tx * kTile), oy = static_cast<float>(tc.ty * kTile);
  const float pxc = static_cast<float>(lx) + 0.5f, pyc = static_cast<float>(ly) + 0.5f;
  // this warp's pixel rows: (2 * warp) * PX .. (2 * warp + 2) * PX - 1
  const uint32_t wrows = ((1u << (2 * PX)) - 1u) << ((threadIdx.x >> 5) * 2 * PX);
  float T[PX], cr[PX], cg[PX], cb[PX], cd[PX], amin[PX];
  int32_t last[PX], stop_at[PX];
  uint32_t blended = 0;
  bool all_done = true;
#pragma unroll
  for (int q = 0; q < PX; ++q) {
    T[q] = 1.0f;
    cr[q] = cg[q] = cb[q] = cd[q] = 0.0f;
    last[q] = 0;
    stop_at[q] = -1;
    const bool outside = !(px < L.W && py + q < L.H);
    amin[q] = outside ? kInf : kAlphaMin;
    all_done = all_done && outside;
  }
  for (uint32_t base = rg.x; base < rg.y; base += kFwdChunk) {
    if (__syncthreads_count(!all_done) == 0) break;
    for (int jj = threadIdx.x; jj < kFwdChunk; jj += kThreads) {
      const uint32_t i = base + jj;
      if (i < rg.y) stage_splat(S, jj, L, ws, keys, i, tc.k, ox, oy);
    }
    __syncthreads();
    const int n = min(kFwdChunk, static_cast<int>(rg.y - base));
    const int pos0 = static_cast<int>(base - rg.x);
    for (int j = 0; j < n; ++j) {
      if ((j & 7) == 0) {  // warp-uniform early exit, checked every 8 splats (extra ones are no-ops)
        all_done = true;
#pragma unroll
        for (int q = 0; q < PX; ++q) all_done = all_done && (amin[q] == kInf);
        if (__all_sync(0xffffffffu, all_done)) break;
      }
      if (!(S.rows[j] & wrows)) continue;
      const float4 A = S.A[j], B = S.B[j], C = S.C[j];
      const float dx = __fsub_rn(A.x, pxc);
      const float qadx = __fmul_rn(A.z, dx);
      const int pos = pos0 + j;
#pragma unroll
      for (int q = 0; q < PX; ++q) {
        // pixel-centre offsets are formed the same way whatever PX is, so every variant
        // takes bit-identical decisions
        const float dy = __fsub_rn(A.y, pyc + static_cast<float>(q));
        const float p = __fmaf_rn(dx, __fmaf_rn(A.w, dy, qadx), __fmul_rn(__fmul_rn(B.x, dy), dy));
        const float alpha = fminf(__fmul_rn(B.y, ex2_approx(p)), kAlphaMax);
        const bool keep = (p <= 0.0f) && (alpha >= amin[q]);
        const float Tn = __fmaf_rn(-T[q], alpha, T[q]);
        const bool stop = keep && (Tn < kTStop);
        const bool blend = keep && !stop;
        const float ae = blend ? alpha : 0.0f;
        const float w = __fmul_rn(ae, T[q]);
        cr[q] = __fmaf_rn(C.x, w, cr[q]);
        cg[q] = __fmaf_rn(C.y, w, cg[q]);
        cb[q] = __fmaf_rn(C.z, w, cb[q]);
        cd[q] = __fmaf_rn(B.z, w, cd[q]);
        T[q] = __fmaf_rn(-T[q], ae, T[q]);
        last[q] = blend ? pos + 1 : last[q];
        amin[q] = stop ? kInf : amin[q];
        if (STATS) {
          stop_at[q] = stop ? pos : stop_at[q];
          blended += blend ? 1u : 0u;
        }
      }
    }
  }
  pdl_trigger();
  const int64_t HW = static_cast<int64_t>(L.H) * L.W;
  const int len = static_cast<int>(rg.y - rg.x);
  uint32_t evals = 0;
  float loss = 0.0f;
  const float inv3 = 1.0f / (3.0f * static_cast<float>(HW));
  const float invd = L.lambda_depth / static_cast<float>(HW);
#pragma unroll
  for (int q = 0; q < PX; ++q) {
    const int y = py + q;
    if (px < L.W && y < L.H) {
      if (STATS) evals += static_cast<uint32_t>(stop_at[q] >= 0 ? stop_at[q] + 1 : len);
      const int64_t pix = static_cast<int64_t>(y) * L.W + px;
      const int64_t c0 = static_cast<int64_t>(tc.k) * 3 * HW + pix;
      if (out_rgb) {
        out_rgb[c0] = cr[q];
        out_rgb[c0 + HW] = cg[q];
        out_rgb[c0 + 2 * HW] = cb[q];
      }
      if (out_depth) out_depth[tc.k * HW + pix] = cd[q];
      if (out_T) out_T[tc.k * HW + pix] = T[q];
      if (out_last) out_last[tc.k * HW + pix] = last[q];
      if (LOSS) {
        // L = sum_k [ mean_{3HW} |R - R*| + lambda mean_{HW} |D - D*| ], sign(0) = 0
        const float c[3] = {cr[q], cg[q], cb[q]};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          const float d = c[ch] - F.rgb_t[c0 + ch * HW];
          loss += fabsf(d) * inv3;
          F.g_rgb[c0 + ch * HW] = sgn(d) * inv3;
        }
        const float d = cd[q] - F.depth_t[tc.k * HW + pix];
        loss += fabsf(d) * invd;
        F.g_depth[tc.k * HW + pix] = sgn(d) * invd;
      }
    }
  }
  if (LOSS) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    __shared__ float s_loss[kWarps];
    __shared__ bool s_last;
    if ((threadIdx.x & 31) == 0) s_loss[threadIdx.x >> 5] = loss;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.0f;
      for (int w = 0; w < kWarps; ++w) t += s_loss[w];
      F.partials[blockIdx.x] = t;
      __threadfence();
      s_last = atomicAdd(F.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
      // the last block sums every tile's partial in a fixed order
      __threadfence();
      float v = 0.0f;
      for (uint32_t i = threadIdx.x; i < gridDim.x; i += kThreads) v += __ldcg(&F.partials[i]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      __syncthreads();
      if ((threadIdx.x & 31) == 0) s_loss[threadIdx.x >> 5] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < kWarps; ++w) t += s_loss[w];
        F.d_loss[0] = t;
        *F.counter = 0;
      }
    }
  }
  if (STATS) {
    uint32_t e = evals, c = blended;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
      s_red[0][threadIdx.x >> 5] = e;
      s_red[1][threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t te = 0, tcn = 0;
      for (int w = 0; w < kWarps; ++w) {
        te += s_red[0][w];
        tcn += s_red[1][w];
      }
      if (te) atomicAdd(reinterpret_cast<unsigned long long*>(evals_out), static_cast<unsigned long long>(te));
      if (tcn) atomicAdd(reinterpret_cast<unsigned long long*>(blended_out), static_cast<unsigned long long>(tcn));
    }
  }
}

// ============================================================================ backward

// Sum of 10 values over a warp, leaving each value in some lane (12 shuffles): halves of
// the value set are exchanged across lane bit 4 (5 pairs), then bit 3 (2 pairs + 1 plain),
// bit 2 (1 pair + 1 plain), bit 1 (1 pair), bit 0 (plain). On return, lane l with l & 1 == 0
// holds value reduce10_index(l) when (l & 2) == 0 or (l & 12) == 0.
__device__ __forceinline__ float warp_reduce10(const float (&x)[10], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  float y[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const float send = b4 ? x[i] : x[i + 5];
    const float keep = b4 ? x[i + 5] : x[i];
    y[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float z[3];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = b3 ? y[2 * i] : y[2 * i + 1];
    const float keep = b3 ? y[2 * i + 1] : y[2 * i];
    z[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  z[2] = y[4] + __shfl_xor_sync(0xffffffffu, y[4], 8);
  float w[2];
  {
    const float send = b2 ? z[0] : z[1];
    const float keep = b2 ? z[1] : z[0];
    w[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  w[1] = z[2] + __shfl_xor_sync(0xffffffffu, z[2], 4);
  float u;
  {
    const float send = b1 ? w[0] : w[1];
    const float keep = b1 ? w[1] : w[0];
    u = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  return u + __shfl_xor_sync(0xffffffffu, u, 1);
}
__device__ __forceinline__ int reduce10_index(int lane) {
  const int half = (lane & 16) ? 5 : 0;
  return (lane & 2) ? half + 4 : half + ((lane >> 3) & 1) + 2 * ((lane >> 2) & 1);
}
__device__ __forceinline__ bool reduce10_writer(int lane) { return !(lane & 1) && (!(lane & 2) || !(lane & 12)); }

// Gradient record layout (floats): 0 du, 1 dv, 2 dA, 3 dB, 4 dC, 5 dz, 6 do, 7 dr, 8 dg, 9 db.
//
// Per pixel, with dpow = dL/dpower / ln 2 (zero where the splat is skipped or clamped) and
// (dx, dy) the offset mean - pixel centre, the geometric terms are sums over the pixels of
//   du = ln2 (2 qa dx + qb dy) dpow,  dv = ln2 (qb dx + 2 qc dy) dpow,
//   dA = -dx^2 dpow / 2,  dB = -dx dy dpow,  dC = -dy^2 dpow / 2,  do = dpow / opacity.
// A lane's pixels share dx, so it keeps only P0 = sum dpow, P1 = sum dy dpow, P2 = sum dy^2 dpow
// and the warp reduces R = (dx P0, P1, dx^2 P0, dx P1, P2, P0); the splat's coefficients
// qa, qb, qc, opacity are applied once per pair when the warp partials are summed.
template <int PX>
__global__ void __launch_bounds__(kTilePixels / PX) k_raster_bwd(Layout L, uint8_t* __restrict__ ws,
                                                                 const float* __restrict__ rgb,
                                                                 const float* __restrict__ depth,
                                                                 const float* __restrict__ T_final,
                                                                 const int32_t* __restrict__ last_in,
                                                                 const float* __restrict__ g_rgb,
                                                                 const float* __restrict__ g_depth,
                                                                 const float* __restrict__ g_T) {
  pdl_wait();
  constexpr int kThreads = kTilePixels / PX;
  constexpr int kWarps = kThreads / 32;
  __shared__ Stage<kBwdChunk> S;
  __shared__ uint32_t s_slot[kBwdChunk];
  __shared__ float s_part[kWarps][kBwdChunk][10];
  __shared__ int s_maxlast[kWarps];
  const TileCoord tc = tile_coord(L, blockIdx.x);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = threadIdx.x & (kTile - 1), ly = (threadIdx.x / kTile) * PX;
  const int px = tc.tx * kTile + lx, py = tc.ty * kTile + ly;
  const uint64_t* keys = at<uint64_t>(ws, (L.passes & 1) ? L.keys[1] : L.keys[0]);
  const uint32_t* slots = at<uint32_t>(ws, (L.passes & 1) ? L.vals[1] : L.vals[0]);  // emission index = record slot
  const uint2 rg = at<uint2>(ws, L.ranges)[blockIdx.x];
  const float ox = static_cast<float>(tc.tx * kTile), oy = static_cast<float>(tc.ty * kTile);
  const float pxc = static_cast<float>(lx) + 0.5f, pyc = static_cast<float>(ly) + 0.5f;
  const uint32_t wrows = ((1u << (2 * PX)) - 1u) << ((threadIdx.x >> 5) * 2 * PX);
  float* pair_grads = at<float>(ws, L.pair_grads);
  uint32_t* pair_valid = at<uint32_t>(ws, L.pair_valid);
  const int64_t HW = static_cast<int64_t>(L.H) * L.W;

  float T[PX], Sg[PX], hT[PX], gr[PX], gg[PX], gb[PX], gd[PX];
  int last[PX];
  int wl = 0;
#pragma unroll
  for (int q = 0; q < PX; ++q) {
    T[q] = 1.0f;
    Sg[q] = hT[q] = gr[q] = gg[q] = gb[q] = gd[q] = 0.0f;
    last[q] = 0;
    const int y = py + q;
    if (px < L.W && y < L.H) {
      const int64_t pix = static_cast<int64_t>(y) * L.W + px;
      const int64_t c0 = static_cast<int64_t>(tc.k) * 3 * HW + pix;
      gr[q] = g_rgb[c0];
      gg[q] = g_rgb[c0 + HW];
      gb[q] = g_rgb[c0 + 2 * HW];
      gd[q] = g_depth[tc.k * HW + pix];
      Sg[q] = gr[q] * rgb[c0] + gg[q] * rgb[c0 + HW] + gb[q] * rgb[c0 + 2 * HW] + gd[q] * depth[tc.k * HW + pix];
      if (g_T) hT[q] = g_T[tc.k * HW + pix] * T_final[tc.k * HW + pix];
      last[q] = last_in[tc.k * HW + pix];
      wl = max(wl, last[q]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, o));
  const int warp_last = wl;  // this warp's pixels need list positions [0, warp_last)
  if (lane == 0) s_maxlast[warp] = wl;
  __syncthreads();
  int max_last = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) max_last = max(max_last, s_maxlast[w]);
  const uint32_t stop = min(rg.y, rg.x + static_cast<uint32_t>(max_last));
  const int idx = reduce10_index(lane);
  const bool writer = reduce10_writer(lane);
  constexpr float kLn2 = 0.6931471805599453f;

  for (uint32_t base = rg.x; base < stop; base += kBwdChunk) {
    for (int jj = threadIdx.x; jj < kBwdChunk; jj += kThreads) {
      const uint32_t i = base + jj;
      if (i < stop) {
        stage_splat(S, jj, L, ws, keys, i, tc.k, ox, oy);
        s_slot[jj] = slots[i];
      }
    }
    for (int e = threadIdx.x; e < kWarps * kBwdChunk * 10; e += kThreads) (&s_part[0][0][0])[e] = 0.0f;
    __syncthreads();
    const int n = min(kBwdChunk, static_cast<int>(stop - base));
    const int pos0 = static_cast<int>(base - rg.x);
    const int nw = min(n, warp_last - pos0);  // splats of this chunk this warp must visit
    for (int j = 0; j < nw; ++j) {
      if (!(S.rows[j] & wrows)) continue;
      const float4 A = S.A[j], B = S.B[j];
      const float dx = __fsub_rn(A.x, pxc);
      const float qadx = __fmul_rn(A.z, dx);
      const int pos = pos0 + j;
      // phase 1: opacity and keep/skip decision for the thread's pixels
      Alpha a[PX];
      float dy[PX];
      bool okq[PX];
      bool contrib = false;
#pragma unroll
      for (int q = 0; q < PX; ++q) {
        dy[q] = __fsub_rn(A.y, pyc + static_cast<float>(q));
        a[q] = splat_alpha(A, B, qadx, dx, dy[q]);
        okq[q] = a[q].keep && (pos < last[q]);
        contrib = contrib || okq[q];
      }
      // phase 2 (skipped when no pixel of the warp keeps the splat): gradient terms
      if (!__any_sync(0xffffffffu, contrib)) continue;
      const float4 C = S.C[j];
      float P0 = 0.0f, P1 = 0.0f, P2 = 0.0f, cz = 0.0f, cr = 0.0f, cgr = 0.0f, cb = 0.0f;
#pragma unroll
      for (int q = 0; q < PX; ++q) {
        // aok = alpha for a kept splat, else 0: then w = 0 and Sg, T stay bit for bit unchanged
        const bool ok = okq[q];
        const bool open = ok && !(a[q].raw > kAlphaMax);  // the 0.99 clamp passes no gradient
        const float Tq = T[q];
        const float aok = ok ? a[q].alpha : 0.0f;
        const float w = __fmul_rn(aok, Tq);
        const float cgz = C.x * gr[q] + C.y * gg[q] + C.z * gb[q] + B.z * gd[q];
        const float sg = __fmaf_rn(-cgz, w, Sg[q]);  // colour/depth behind this splat, weighted by dL/dpixel
        const float dalpha = Tq * cgz - __fdividef(sg + hT[q], 1.0f - a[q].alpha);
        const float dpow = (open ? a[q].alpha : 0.0f) * dalpha;
        const float ydp = dy[q] * dpow;
        P0 += dpow;
        P1 += ydp;
        P2 = fmaf(dy[q], ydp, P2);
        cz = fmaf(w, gd[q], cz);
        cr = fmaf(w, gr[q], cr);
        cgr = fmaf(w, gg[q], cgr);
        cb = fmaf(w, gb[q], cb);
        Sg[q] = sg;
        T[q] = __fmaf_rn(-Tq, aok, Tq);
      }
      const float dxP0 = dx * P0;
      const float v[10] = {dxP0, P1, dx * dxP0, dx * P1, P2, cz, P0, cr, cgr, cb};
      const float r = warp_reduce10(v, lane);
      if (writer) s_part[warp][j][idx] = r;
    }
    __syncthreads();
    for (int jj = threadIdx.x; jj < n; jj += kThreads) {
      float R[10];
#pragma unroll
      for (int q = 0; q < 10; ++q) {
        float acc = 0.0f;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) acc += s_part[w][jj][q];
        R[q] = acc;
      }
      // R = (sum dx P0, sum P1, sum dx^2 P0, sum dx P1, sum P2, dz, sum P0, dr, dg, db)
      const float4 A = S.A[jj], B = S.B[jj];
      const float du = kLn2 * (2.0f * A.z * R[0] + A.w * R[1]);
      const float dv = kLn2 * (2.0f * B.x * R[1] + A.w * R[0]);
      const float dop = R[6] != 0.0f ? R[6] / B.y : 0.0f;
      const uint32_t slot = s_slot[jj];
      float4* dst = reinterpret_cast<float4*>(pair_grads + static_cast<size_t>(slot) * kPairGradStride);
      dst[0] = make_float4(du, dv, -0.5f * R[2], -R[3]);
      dst[1] = make_float4(-0.5f * R[4], R[5], dop, R[7]);
      dst[2] = make_float4(R[8], R[9], 0.0f, 0.0f);
      atomicOr(&pair_valid[slot >> 5], 1u << (slot & 31));
    }
    __syncthreads();
  }
  // pairs behind every pixel's last contributor get no record: their bit stays clear
  pdl_trigger();
}

int pick_px(int requested, int fallback) { return (requested == 1 || requested == 2 || requested == 4) ? requested : fallback; }

}  // namespace

cudaError_t launch_raster_fwd(const Layout& L, void* ws, float* rgb, float* depth, float* T_final, int32_t* last,
                              bool stats, const FusedLossArgs* loss, cudaStream_t s) {
  Status* st = at<Status>(ws, L.status);
  if (stats) {
    cudaMemsetAsync(&st->evals, 0, sizeof(uint64_t), s);
    cudaMemsetAsync(&st->composited, 0, sizeof(uint64_t), s);
  }
  if (L.n_tiles == 0) {
    if (loss) cudaMemsetAsync(loss->d_loss, 0, sizeof(float), s);
    return cudaGetLastError();
  }
  const unsigned grid = static_cast<unsigned>(L.n_tiles);
  const uint8_t* w = static_cast<const uint8_t*>(ws);
  uint64_t *ev = &st->evals, *cp = &st->composited;
  FusedLoss F{};
  if (loss)
    F = FusedLoss{loss->rgb_t, loss->depth_t, loss->g_rgb, loss->g_depth, at<float>(ws, L.tile_loss), &st->loss_ctr,
                  loss->d_loss};
  const int px = pick_px(L.fwd_px, kDefaultFwdPx);
#define GS_FWD(P, ST, LO) \
  launch(k_raster_fwd<P, ST, LO>, grid, kTilePixels / P, 0, s, L, w, rgb, depth, T_final, last, ev, cp, F)
  if (loss) {
    switch (px) {
      case 1: GS_FWD(1, false, true); break;
      case 2: GS_FWD(2, false, true); break;
      default: GS_FWD(4, false, true); break;
    }
  } else if (stats) {
    switch (px) {
      case 1: GS_FWD(1, true, false); break;
      case 2: GS_FWD(2, true, false); break;
      default: GS_FWD(4, true, false); break;
    }
  } else {
    switch (px) {
      case 1: GS_FWD(1, false, false); break;
      case 2: GS_FWD(2, false, false); break;
      default: GS_FWD(4, false, false); break;
    }
  }
#undef GS_FWD
  return cudaGetLastError();
}

cudaError_t launch_raster_bwd(const Layout& L, void* ws, const float* rgb, const float* depth, const float* T_final,
                              const int32_t* last, const float* dL_drgb, const float* dL_ddepth, const float* dL_dT,
                              cudaStream_t s) {
  if (L.n_tiles == 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>(L.n_tiles);
  uint8_t* w = static_cast<uint8_t*>(ws);
  switch (pick_px(L.bwd_px, kDefaultBwdPx)) {
    case 1: launch(k_raster_bwd<1>, grid, kTilePixels, 0, s, L, w, rgb, depth, T_final, last, dL_drgb, dL_ddepth, dL_dT); break;
    case 2: launch(k_raster_bwd<2>, grid, kTilePixels / 2, 0, s, L, w, rgb, depth, T_final, last, dL_drgb, dL_ddepth, dL_dT); break;
    default: launch(k_raster_bwd<4>, grid, kTilePixels / 4, 0, s, L, w, rgb, depth, T_final, last, dL_drgb, dL_ddepth, dL_dT); break;
  }
  return cudaGetLastError();
}

}  // namespace gs
