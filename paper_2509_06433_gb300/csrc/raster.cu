// Tile compositing: forward (render) and backward (splat gradients).
//
// One CTA of 128 threads per (view, 16x16 tile); each thread owns two vertically adjacent
// pixels of one column, so the horizontal offset to a splat is shared and every splat
// record loaded from shared memory serves two pixels. The tile's depth-sorted list is
// walked in chunks of 128 splats staged in shared memory as three float4 per splat
// (coalesced loads of the sorted Gaussian ids, one gather of the projected record each).
//
// Both kernels evaluate a splat's opacity with the same inline function on the same
// operands, so the backward pass takes exactly the forward pass's skip and stop decisions
// and recovers the same transmittance T_i front to back, without storing per-splat alphas.
//
// The backward pass sums each splat's 10 gradient terms over a warp's 64 pixels (two per
// lane, then a transpose-reduce: 16 shuffles for 16 padded values), writes one partial per
// warp into shared memory, and at the end of each chunk sums the 4 warp partials in a
// fixed order into one record per (splat, tile) pair of the pair-gradient buffer. No global
// atomics: the gradients are deterministic.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kRasterThreads = kTilePixels / 2;  // two pixels per thread
constexpr int kWarps = kRasterThreads / 32;
constexpr int kChunk = kRasterThreads;           // splats staged per chunk
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTStop = 1e-4f;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Staged splat: A = (x, y, qa, qb), B = (qc, opacity, depth, -), C = (r, g, b, -) where
// (x, y) is the 2D mean relative to the tile origin and power * log2(e) = qa dx^2 + qb dx dy + qc dy^2.
struct Stage {
  float4 A[kChunk], B[kChunk], C[kChunk];
};

__device__ __forceinline__ uint32_t stage_splat(Stage& S, int j, const Layout& L, const uint8_t* ws,
                                                const uint32_t* vals, uint32_t i, int k, float ox, float oy) {
  const uint32_t gid = vals[i];
  const int64_t kg = static_cast<int64_t>(k) * L.N + gid;
  const float4 uv = at<float4>(ws, L.proj_uv)[kg];
  const float4 cn = at<float4>(ws, L.proj_conic)[kg];
  const float4 co = at<float4>(ws, L.color_opacity)[gid];
  S.A[j] = make_float4(__fadd_rn(__fsub_rn(uv.x, ox), uv.y), __fadd_rn(__fsub_rn(uv.z, oy), uv.w),
                       __fmul_rn(cn.x, -0.5f * kLog2e), __fmul_rn(cn.y, -kLog2e));
  S.B[j] = make_float4(__fmul_rn(cn.z, -0.5f * kLog2e), co.w, cn.w, 0.0f);
  S.C[j] = make_float4(co.x, co.y, co.z, 0.0f);
  return gid;
}

// Opacity of a splat at pixel offset (dx, dy). Returns false when the splat is skipped
// (power > 0 or alpha < 1/255). G = exp(power); clamped: alpha hit 0.99.
__device__ __forceinline__ bool splat_alpha(const float4& A, const float4& B, float dx, float dy, float& alpha,
                                            float& G, bool& clamped) {
  const float p = __fmaf_rn(dx, __fmaf_rn(A.z, dx, __fmul_rn(A.w, dy)), __fmul_rn(__fmul_rn(B.x, dy), dy));
  if (p > 0.0f) return false;
  G = ex2_approx(p);
  const float a = __fmul_rn(B.y, G);
  clamped = a > kAlphaMax;
  alpha = clamped ? kAlphaMax : a;
  return alpha >= kAlphaMin;
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
struct FwdPixel {
  float T, r, g, b, d;
  int32_t last;
  uint32_t evals, blended;
  bool done;
};

__device__ __forceinline__ void fwd_step(FwdPixel& P, const float4& A, const float4& B, const float4& C, float dx,
                                         float dy, int pos) {
  ++P.evals;
  float alpha, G;
  bool clamped;
  if (!splat_alpha(A, B, dx, dy, alpha, G, clamped)) return;
  const float Tn = __fmaf_rn(-P.T, alpha, P.T);
  if (Tn < kTStop) {
    P.done = true;
    return;
  }
  const float w = __fmul_rn(alpha, P.T);
  P.r = __fmaf_rn(C.x, w, P.r);
  P.g = __fmaf_rn(C.y, w, P.g);
  P.b = __fmaf_rn(C.z, w, P.b);
  P.d = __fmaf_rn(B.z, w, P.d);
  P.T = Tn;
  ++P.blended;
  P.last = pos + 1;
}

__global__ void __launch_bounds__(kRasterThreads) k_raster_fwd(Layout L, const uint8_t* __restrict__ ws,
                                                               float* __restrict__ out_rgb,
                                                               float* __restrict__ out_depth,
                                                               float* __restrict__ out_T,
                                                               int32_t* __restrict__ out_last,
                                                               uint64_t* __restrict__ evals_out,
                                                               uint64_t* __restrict__ blended_out) {
  __shared__ Stage S;
  __shared__ uint32_t s_red[2][kWarps];
  const TileCoord tc = tile_coord(L, blockIdx.x);
  const int lx = threadIdx.x & (kTile - 1), ly = (threadIdx.x / kTile) * 2;
  const int px = tc.tx * kTile + lx, py = tc.ty * kTile + ly;
  const uint32_t* vals = at<uint32_t>(ws, (L.passes & 1) ? L.vals[1] : L.vals[0]);
  const uint2 rg = at<uint2>(ws, L.ranges)[blockIdx.x];
  const float ox = static_cast<float>(tc.tx * kTile), oy = static_cast<float>(tc.ty * kTile);
  const float pxc = static_cast<float>(lx) + 0.5f, pyc0 = static_cast<float>(ly) + 0.5f,
              pyc1 = static_cast<float>(ly + 1) + 0.5f;
  FwdPixel p0{1.0f, 0.f, 0.f, 0.f, 0.f, 0, 0u, 0u, !(px < L.W && py < L.H)};
  FwdPixel p1{1.0f, 0.f, 0.f, 0.f, 0.f, 0, 0u, 0u, !(px < L.W && py + 1 < L.H)};
  for (uint32_t base = rg.x; base < rg.y; base += kChunk) {
    if (__syncthreads_count(!(p0.done && p1.done)) == 0) break;
    const uint32_t i = base + threadIdx.x;
    if (i < rg.y) stage_splat(S, threadIdx.x, L, ws, vals, i, tc.k, ox, oy);
    __syncthreads();
    const int n = min(kChunk, static_cast<int>(rg.y - base));
    const int pos0 = static_cast<int>(base - rg.x);
    for (int j = 0; j < n && !(p0.done && p1.done); ++j) {
      const float4 A = S.A[j], B = S.B[j], C = S.C[j];
      const float dx = __fsub_rn(A.x, pxc);
      if (!p0.done) fwd_step(p0, A, B, C, dx, __fsub_rn(A.y, pyc0), pos0 + j);
      if (!p1.done) fwd_step(p1, A, B, C, dx, __fsub_rn(A.y, pyc1), pos0 + j);
    }
  }
  const int64_t HW = static_cast<int64_t>(L.H) * L.W;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const FwdPixel& P = q ? p1 : p0;
    const int y = py + q;
    if (px < L.W && y < L.H) {
      const int64_t pix = static_cast<int64_t>(y) * L.W + px;
      if (out_rgb) {
        out_rgb[(static_cast<int64_t>(tc.k) * 3 + 0) * HW + pix] = P.r;
        out_rgb[(static_cast<int64_t>(tc.k) * 3 + 1) * HW + pix] = P.g;
        out_rgb[(static_cast<int64_t>(tc.k) * 3 + 2) * HW + pix] = P.b;
      }
      if (out_depth) out_depth[tc.k * HW + pix] = P.d;
      if (out_T) out_T[tc.k * HW + pix] = P.T;
      if (out_last) out_last[tc.k * HW + pix] = P.last;
    }
  }
  uint32_t e = p0.evals + p1.evals, c = p0.blended + p1.blended;
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

// ============================================================================ backward

// 16 values per lane -> each value summed over the warp. On return v[0] of lane l holds
// the sum of value index ((l>>4)&1)*8 + ((l>>3)&1)*4 + ((l>>2)&1)*2 + ((l>>1)&1)
// (lanes l and l^1 hold the same sum).
__device__ __forceinline__ void warp_transpose_reduce16(float (&v)[16], int lane) {
  {
    const bool hi = lane & 16;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float send = hi ? v[i] : v[i + 8];
      const float keep = hi ? v[i + 8] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
  }
  {
    const bool hi = lane & 8;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float send = hi ? v[i] : v[i + 4];
      const float keep = hi ? v[i + 4] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
  }
  {
    const bool hi = lane & 4;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float send = hi ? v[i] : v[i + 2];
      const float keep = hi ? v[i + 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
  }
  {
    const bool hi = lane & 2;
    const float send = hi ? v[0] : v[1];
    const float keep = hi ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

struct BwdPixel {
  float T, Sg, hT, gr, gg, gb, gd;
  int last;
};

// Gradient record layout (floats): 0 du, 1 dv, 2 dA, 3 dB, 4 dC, 5 dz, 6 do, 7 dr, 8 dg, 9 db.
// Adds this pixel's terms for splat (A, B, C) at list position pos into v; returns true if it blended.
__device__ __forceinline__ bool bwd_step(BwdPixel& P, const float4& A, const float4& B, const float4& C, float dx,
                                         float dy, int pos, float (&v)[16]) {
  if (pos >= P.last) return false;
  float alpha, G;
  bool clamped;
  if (!splat_alpha(A, B, dx, dy, alpha, G, clamped)) return false;
  const float T = P.T;
  const float w = __fmul_rn(alpha, T);
  const float cgz = C.x * P.gr + C.y * P.gg + C.z * P.gb + B.z * P.gd;
  P.Sg -= cgz * w;  // now: colour/depth behind this splat, weighted by dL/dpixel
  const float dalpha = T * cgz - (P.Sg + P.hT) / (1.0f - alpha);
  v[5] += w * P.gd;
  v[7] += w * P.gr;
  v[8] += w * P.gg;
  v[9] += w * P.gb;
  if (!clamped) {
    // power = -0.5 (A dx^2 + C dy^2) - B dx dy with qa = -0.5 A log2e, qb = -B log2e, qc = -0.5 C log2e
    constexpr float kLn2 = 0.6931471805599453f;
    const float dpow = alpha * dalpha;
    const float dpl = dpow * kLn2;
    v[6] += G * dalpha;
    v[2] += -0.5f * dx * dx * dpow;
    v[3] += -dx * dy * dpow;
    v[4] += -0.5f * dy * dy * dpow;
    v[0] += (2.0f * A.z * dx + A.w * dy) * dpl;
    v[1] += (2.0f * B.x * dy + A.w * dx) * dpl;
  }
  P.T = __fmaf_rn(-T, alpha, T);
  return true;
}

__device__ __forceinline__ uint32_t pair_slot(const int4& tl, int tx, int ty) {
  const uint32_t x0 = static_cast<uint32_t>(tl.y) & 0xffffu, x1 = static_cast<uint32_t>(tl.y) >> 16;
  const uint32_t y0 = static_cast<uint32_t>(tl.z) & 0xffffu;
  return static_cast<uint32_t>(tl.x) + (static_cast<uint32_t>(ty) - y0) * (x1 - x0) + (static_cast<uint32_t>(tx) - x0);
}

__global__ void __launch_bounds__(kRasterThreads) k_raster_bwd(Layout L, uint8_t* __restrict__ ws,
                                                               const float* __restrict__ rgb,
                                                               const float* __restrict__ depth,
                                                               const float* __restrict__ T_final,
                                                               const int32_t* __restrict__ last_in,
                                                               const float* __restrict__ g_rgb,
                                                               const float* __restrict__ g_depth,
                                                               const float* __restrict__ g_T) {
  __shared__ Stage S;
  __shared__ uint32_t s_slot[kChunk];
  __shared__ float s_part[kWarps][kChunk][10];
  __shared__ int s_maxlast[kWarps];
  const TileCoord tc = tile_coord(L, blockIdx.x);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = threadIdx.x & (kTile - 1), ly = (threadIdx.x / kTile) * 2;
  const int px = tc.tx * kTile + lx, py = tc.ty * kTile + ly;
  const uint32_t* vals = at<uint32_t>(ws, (L.passes & 1) ? L.vals[1] : L.vals[0]);
  const uint2 rg = at<uint2>(ws, L.ranges)[blockIdx.x];
  const float ox = static_cast<float>(tc.tx * kTile), oy = static_cast<float>(tc.ty * kTile);
  const float pxc = static_cast<float>(lx) + 0.5f, pyc0 = static_cast<float>(ly) + 0.5f,
              pyc1 = static_cast<float>(ly + 1) + 0.5f;
  const int4* tiles = at<int4>(ws, L.proj_tiles);
  float* pair_grads = at<float>(ws, L.pair_grads);
  const int64_t HW = static_cast<int64_t>(L.H) * L.W;

  BwdPixel pp[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    BwdPixel& P = pp[q];
    P = BwdPixel{1.0f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0};
    const int y = py + q;
    if (px < L.W && y < L.H) {
      const int64_t pix = static_cast<int64_t>(y) * L.W + px;
      const int64_t c0 = static_cast<int64_t>(tc.k) * 3 * HW + pix;
      P.gr = g_rgb[c0];
      P.gg = g_rgb[c0 + HW];
      P.gb = g_rgb[c0 + 2 * HW];
      P.gd = g_depth[tc.k * HW + pix];
      P.Sg = P.gr * rgb[c0] + P.gg * rgb[c0 + HW] + P.gb * rgb[c0 + 2 * HW] + P.gd * depth[tc.k * HW + pix];
      if (g_T) P.hT = g_T[tc.k * HW + pix] * T_final[tc.k * HW + pix];
      P.last = last_in[tc.k * HW + pix];
    }
  }
  int wl = max(pp[0].last, pp[1].last);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, o));
  const int warp_last = wl;  // this warp's pixels need list positions [0, warp_last)
  if (lane == 0) s_maxlast[warp] = wl;
  __syncthreads();
  int max_last = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) max_last = max(max_last, s_maxlast[w]);
  const uint32_t stop = min(rg.y, rg.x + static_cast<uint32_t>(max_last));
  const int idx = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);

  for (uint32_t base = rg.x; base < stop; base += kChunk) {
    const uint32_t i = base + threadIdx.x;
    if (i < stop) {
      const uint32_t gid = stage_splat(S, threadIdx.x, L, ws, vals, i, tc.k, ox, oy);
      s_slot[threadIdx.x] = pair_slot(tiles[static_cast<int64_t>(tc.k) * L.N + gid], tc.tx, tc.ty);
    }
    for (int e = threadIdx.x; e < kWarps * kChunk * 10; e += kRasterThreads) (&s_part[0][0][0])[e] = 0.0f;
    __syncthreads();
    const int n = min(kChunk, static_cast<int>(stop - base));
    const int pos0 = static_cast<int>(base - rg.x);
    const int nw = min(n, warp_last - pos0);  // splats of this chunk this warp must visit
    for (int j = 0; j < nw; ++j) {
      const float4 A = S.A[j], B = S.B[j], C = S.C[j];
      float v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = 0.0f;
      const float dx = __fsub_rn(A.x, pxc);
      bool contrib = bwd_step(pp[0], A, B, C, dx, __fsub_rn(A.y, pyc0), pos0 + j, v);
      contrib |= bwd_step(pp[1], A, B, C, dx, __fsub_rn(A.y, pyc1), pos0 + j, v);
      if (__any_sync(0xffffffffu, contrib)) {
        warp_transpose_reduce16(v, lane);
        if (!(lane & 1) && idx < 10) s_part[warp][j][idx] = v[0];
      }
    }
    __syncthreads();
    if (threadIdx.x < n) {
      float a[10];
#pragma unroll
      for (int q = 0; q < 10; ++q) {
        float acc = 0.0f;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) acc += s_part[w][threadIdx.x][q];
        a[q] = acc;
      }
      float4* dst = reinterpret_cast<float4*>(pair_grads + static_cast<size_t>(s_slot[threadIdx.x]) * kPairGradStride);
      dst[0] = make_float4(a[0], a[1], a[2], a[3]);
      dst[1] = make_float4(a[4], a[5], a[6], a[7]);
      dst[2] = make_float4(a[8], a[9], 0.0f, 0.0f);
    }
    __syncthreads();
  }
  // pairs behind every pixel's last contributor receive zero records
  for (uint32_t i = stop + threadIdx.x; i < rg.y; i += kRasterThreads) {
    const uint32_t gid = vals[i];
    const uint32_t slot = pair_slot(tiles[static_cast<int64_t>(tc.k) * L.N + gid], tc.tx, tc.ty);
    float4* dst = reinterpret_cast<float4*>(pair_grads + static_cast<size_t>(slot) * kPairGradStride);
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    dst[0] = zero;
    dst[1] = zero;
    dst[2] = zero;
  }
}

}  // namespace

cudaError_t launch_raster_fwd(const Layout& L, void* ws, float* rgb, float* depth, float* T_final, int32_t* last,
                              cudaStream_t s) {
  Status* st = at<Status>(ws, L.status);
  cudaMemsetAsync(&st->evals, 0, sizeof(uint64_t), s);
  cudaMemsetAsync(&st->composited, 0, sizeof(uint64_t), s);
  if (L.n_tiles == 0) return cudaGetLastError();
  k_raster_fwd<<<static_cast<unsigned>(L.n_tiles), kRasterThreads, 0, s>>>(
      L, static_cast<const uint8_t*>(ws), rgb, depth, T_final, last, &st->evals, &st->composited);
  return cudaGetLastError();
}

cudaError_t launch_raster_bwd(const Layout& L, void* ws, const float* rgb, const float* depth, const float* T_final,
                              const int32_t* last, const float* dL_drgb, const float* dL_ddepth, const float* dL_dT,
                              cudaStream_t s) {
  if (L.n_tiles == 0) return cudaSuccess;
  k_raster_bwd<<<static_cast<unsigned>(L.n_tiles), kRasterThreads, 0, s>>>(L, static_cast<uint8_t*>(ws), rgb, depth,
                                                                           T_final, last, dL_drgb, dL_ddepth, dL_dT);
  return cudaGetLastError();
}

}  // namespace gs
