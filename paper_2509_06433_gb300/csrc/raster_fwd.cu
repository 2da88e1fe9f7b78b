// Forward compositing (gs_raster_fwd, gs_raster_fwd_stats, gs_raster_fwd_l1, and with the
// backward pass fused, gs_raster_fwd_l1_bwd); see raster_common.cuh for the staging and the
// opacity test both compositing kernels share.
#include <type_traits>

#include "raster_sweep.cuh"

namespace gs {
namespace {

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

// Occlusion by an external surface (OCC = true): per pixel its depth and, optionally, colour
// ([K,H,W], [K,3,H,W]). The list is in depth order, so the first splat at or behind the surface
// ends the pixel (it is not composited); the surface then shows through the remaining
// transmittance: rgb += T ext_rgb, depth += T ext_depth.
struct Occlusion {
  const float* depth;
  const float* rgb;
};

// CHB > 0 (with LOSS only): the block continues into the backward pass of its tile (the sweep
// of gs_raster_bwd, staging CHB splats per chunk) as soon as its forward is done, from the loss
// gradient, colour, depth and last contributor of its pixels still in registers; the results
// equal gs_raster_fwd_l1 followed by gs_raster_bwd (dL_dT = NULL) with PX pixels per thread.
// The workspace is read-only to the forward; the variant with the fused backward also writes
// its gradient records, record bits and error word there, so it takes a mutable pointer.
template <int CHB>
using RasterWs = typename std::conditional<(CHB > 0), uint8_t*, const uint8_t*>::type;

// Shared memory of the forward: its staged chunk; with the fused backward, the backward sweep's
// shared memory in the same bytes (the forward's chunks are dead once every thread has passed
// the loss reduction's barriers, before the sweep starts).
template <int PX, int CH, int CHB>
union FusedSmem {
  Stage<CH> S;
  BwdSmem<PX, CHB> M;
};
template <int PX, int CH, int CHB>
struct FwdSmemOf {
  using T = FusedSmem<PX, CH, CHB>;
};
template <int PX, int CH>
struct FwdSmemOf<PX, CH, 0> {
  struct T {
    Stage<CH> S;
  };
};

// MANY = false (the fused variant only): compiled without the blocks-per-SM register budget, for
// grids that fit on the GPU in one wave anyway, where each block's own latency sets the time.
template <int PX, int CH, bool STATS, bool LOSS, bool OCC = false, int CHB = 0, bool MANY = true>
__global__ void __launch_bounds__(kTilePixels / PX,
                                  (PX == 4 && MANY) ? (CHB > 0 ? kMinBlocksFusedPx4 : kMinBlocksPx4) : 1)
    k_raster_fwd(Layout L, RasterWs<CHB> __restrict__ ws, float* __restrict__ out_rgb, float* __restrict__ out_depth,
                 float* __restrict__ out_T, int32_t* __restrict__ out_last, uint64_t* __restrict__ evals_out,
                 uint64_t* __restrict__ blended_out, FusedLoss F, Occlusion O) {
  static_assert(CHB == 0 || (LOSS && !STATS && !OCC), "the fused backward follows the loss-fused forward");
  pdl_wait();
  constexpr int kThreads = kTilePixels / PX;
  constexpr int kWarps = kThreads / 32;
  const float kInf = __int_as_float(0x7f800000);
  __shared__ typename FwdSmemOf<PX, CH, CHB>::T sm;
  Stage<CH>& S = sm.S;
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
  constexpr int W = PX >= 2 ? 2 : 1, G = PX / W;  // pixel q is component q % W of group q / W
  using V = typename Vec<W>::T;
  V T[G], cr[G], cg[G], cb[G], cd[G], npy[G];
  float amin[PX];
  int32_t last[PX], stop_at[PX];
  float zmax[PX];
  uint32_t blended = 0;
  bool all_done = true;
  const V npx = bcast<W>(-pxc), one = bcast<W>(1.0f), zero = bcast<W>(0.0f), minus1 = bcast<W>(-1.0f);
#pragma unroll
  for (int g = 0; g < G; ++g) {
    T[g] = one;
    cr[g] = cg[g] = cb[g] = cd[g] = zero;
#pragma unroll
    for (int i = 0; i < W; ++i) set_comp(npy[g], i, -(pyc + static_cast<float>(g * W + i)));
  }
#pragma unroll
  for (int q = 0; q < PX; ++q) {
    last[q] = 0;
    stop_at[q] = -1;
    const bool outside = !(px < L.W && py + q < L.H);
    amin[q] = outside ? kInf : kAlphaMin;
    zmax[q] = kInf;
    if (OCC && !outside) zmax[q] = O.depth[tc.k * static_cast<int64_t>(L.H) * L.W + static_cast<int64_t>(py + q) * L.W + px];
    all_done = all_done && outside;
  }
  // the loss targets of the thread's pixels, loaded now so that the loads overlap the compositing
  float tgt[LOSS ? PX : 1][4];
  if (LOSS) {
    const int64_t HW = static_cast<int64_t>(L.H) * L.W;
#pragma unroll
    for (int q = 0; q < PX; ++q) {
      tgt[q][0] = tgt[q][1] = tgt[q][2] = tgt[q][3] = 0.0f;
      if (px < L.W && py + q < L.H) {
        const int64_t pix = static_cast<int64_t>(py + q) * L.W + px;
        const int64_t c0 = static_cast<int64_t>(tc.k) * 3 * HW + pix;
        tgt[q][0] = __ldg(F.rgb_t + c0);
        tgt[q][1] = __ldg(F.rgb_t + c0 + HW);
        tgt[q][2] = __ldg(F.rgb_t + c0 + 2 * HW);
        tgt[q][3] = __ldg(F.depth_t + tc.k * HW + pix);
      }
    }
  }
  for (uint32_t base = rg.x; base < rg.y; base += CH) {
    if (__syncthreads_count(!all_done) == 0) break;
    for (int jj = threadIdx.x; jj < CH; jj += kThreads) {
      const uint32_t i = base + jj;
      if (i < rg.y) stage_splat(S, jj, L, ws, keys, i, tc.k, ox, oy);
    }
    __syncthreads();
    const int n = min(CH, static_cast<int>(rg.y - base));
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
      const Column<W> col = splat_column<W>(A, B, npx);
      const V cR = bcast<W>(C.x), cG = bcast<W>(C.y), cB = bcast<W>(C.z), cZ = bcast<W>(B.z), Ay = bcast<W>(A.y);
      const int pos = pos0 + j;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const V e = splat_exponent<W>(B, col, vadd(Ay, npy[g]));
        const V nT = vmul(T[g], minus1);
        V alpha;
        bool keep[W];
#pragma unroll
        for (int i = 0; i < W; ++i) {
          const int q = g * W + i;
          const float a = fminf(ex2_approx(comp(e, i)), kAlphaMax);
          set_comp(alpha, i, a);
          keep[i] = (comp(e, i) <= B.w) && (a >= amin[q]);
        }
        const V Tn = vfma(nT, alpha, T[g]);  // T (1 - alpha)
        V ae;  // alpha for a blended splat, else 0 (then w = 0 and T, the sums stay bit for bit)
#pragma unroll
        for (int i = 0; i < W; ++i) {
          const int q = g * W + i;
          bool kp = keep[i], behind = false;
          if (OCC) {
            behind = B.z >= zmax[q];  // the splat's camera depth at or behind the surface
            kp = kp && !behind;
          }
          const bool stop = kp && (comp(Tn, i) < kTStop);
          const bool blend = kp && !stop;
          set_comp(ae, i, blend ? comp(alpha, i) : 0.0f);
          last[q] = blend ? pos + 1 : last[q];
          amin[q] = (stop || behind) ? kInf : amin[q];
          if (STATS) {
            stop_at[q] = stop ? pos : stop_at[q];
            blended += blend ? 1u : 0u;
          }
        }
        const V w = vmul(ae, T[g]);
        cr[g] = vfma(cR, w, cr[g]);
        cg[g] = vfma(cG, w, cg[g]);
        cb[g] = vfma(cB, w, cb[g]);
        cd[g] = vfma(cZ, w, cd[g]);
        T[g] = vfma(nT, ae, T[g]);
      }
    }
  }
  if (CHB == 0) pdl_trigger();  // (the fused backward lets the next grid launch only at its end)
  const int64_t HW = static_cast<int64_t>(L.H) * L.W;
  const int len = static_cast<int>(rg.y - rg.x);
  float bg[CHB > 0 ? PX : 1][4];  // the loss gradient of each pixel (fused backward)
#pragma unroll
  for (int q = 0; q < (CHB > 0 ? PX : 1); ++q) bg[q][0] = bg[q][1] = bg[q][2] = bg[q][3] = 0.0f;
  uint32_t evals = 0;
  float loss = 0.0f;
  const float inv3 = 1.0f / (3.0f * static_cast<float>(HW));
  const float invd = L.lambda_depth / static_cast<float>(HW);
#pragma unroll
  for (int q = 0; q < PX; ++q) {
    const int y = py + q;
    float vr = comp(cr[q / W], q % W), vg = comp(cg[q / W], q % W), vb = comp(cb[q / W], q % W);
    float vd = comp(cd[q / W], q % W);
    const float vT = comp(T[q / W], q % W);
    if (px < L.W && y < L.H) {
      if (STATS) evals += static_cast<uint32_t>(stop_at[q] >= 0 ? stop_at[q] + 1 : len);
      const int64_t pix = static_cast<int64_t>(y) * L.W + px;
      const int64_t c0 = static_cast<int64_t>(tc.k) * 3 * HW + pix;
      if (OCC) {  // the external surface through the remaining transmittance
        if (O.rgb) {
          vr = __fmaf_rn(vT, O.rgb[c0], vr);
          vg = __fmaf_rn(vT, O.rgb[c0 + HW], vg);
          vb = __fmaf_rn(vT, O.rgb[c0 + 2 * HW], vb);
        }
        vd = __fmaf_rn(vT, zmax[q], vd);
      }
      if (out_rgb) {
        out_rgb[c0] = vr;
        out_rgb[c0 + HW] = vg;
        out_rgb[c0 + 2 * HW] = vb;
      }
      if (out_depth) out_depth[tc.k * HW + pix] = vd;
      if (out_T) out_T[tc.k * HW + pix] = vT;
      if (out_last) out_last[tc.k * HW + pix] = last[q];
      if (LOSS) {
        // L = sum_k [ mean_{3HW} |R - R*| + lambda mean_{HW} |D - D*| ], sign(0) = 0
        const float c[3] = {vr, vg, vb};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          const float d = c[ch] - tgt[LOSS ? q : 0][ch];
          loss += fabsf(d) * inv3;
          const float gv = sgn(d) * inv3;
          F.g_rgb[c0 + ch * HW] = gv;
          if (CHB > 0) bg[CHB > 0 ? q : 0][ch] = gv;
        }
        const float d = vd - tgt[LOSS ? q : 0][3];
        loss += fabsf(d) * invd;
        const float gv = sgn(d) * invd;
        F.g_depth[tc.k * HW + pix] = gv;
        if (CHB > 0) bg[CHB > 0 ? q : 0][3] = gv;
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
  if constexpr (CHB > 0) {
    // the backward pass of this tile, from registers: the weighted colour behind the first
    // splat is the loss gradient applied to the pixel's output (no dL/dT_final term)
    BwdSmem<PX, CHB>& M = sm.M;
    float Sg[PX], hT[PX], gr[PX], gg[PX], gb[PX], gd[PX];
    int lst[PX];
#pragma unroll
    for (int q = 0; q < PX; ++q) {
      gr[q] = bg[q][0];
      gg[q] = bg[q][1];
      gb[q] = bg[q][2];
      gd[q] = bg[q][3];
      const bool in = px < L.W && py + q < L.H;
      Sg[q] = in ? weighted_colour(gr[q], gg[q], gb[q], gd[q], comp(cr[q / W], q % W), comp(cg[q / W], q % W),
                                   comp(cb[q / W], q % W), comp(cd[q / W], q % W))
                 : 0.0f;
      hT[q] = 0.0f;
      lst[q] = in ? last[q] : 0;
    }
    bwd_sweep<PX, CHB, false>(M, L, ws, tc, rg, Sg, hT, gr, gg, gb, gd, lst);
    pdl_trigger();
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

}  // namespace

cudaError_t launch_raster_fwd_l1_bwd(const Layout& L, void* ws, float* rgb, float* depth, float* T_final, int32_t* last,
                                     const FusedLossArgs& loss, cudaStream_t s) {
  Status* st = at<Status>(ws, L.status);
  if (L.n_tiles == 0) {
    cudaMemsetAsync(loss.d_loss, 0, sizeof(float), s);
    return cudaGetLastError();
  }
  const unsigned grid = static_cast<unsigned>(L.n_tiles);
  uint8_t* w = static_cast<uint8_t*>(ws);
  uint64_t *ev = &st->evals, *cp = &st->composited;
  const FusedLoss F{loss.rgb_t, loss.depth_t, loss.g_rgb, loss.g_depth, at<float>(ws, L.tile_loss), &st->loss_ctr,
                    loss.d_loss};
  const int px = pick_px(L.fwd_px, kDefaultFwdPx);
  const int ch = pick_chunk(L.fwd_chunk, 64, 256, kFwdChunk);
  // the backward phase stages kBwdChunk splats per chunk (the chunk depth changes no result); at 4
  // pixels per thread, a grid that the variant without the blocks-per-SM register budget runs in
  // one wave (its resident blocks per SM, from the occupancy calculator, times the SMs) takes it
  static int uncapped_blocks[64] = {};  // per device: resident blocks per SM of the uncapped variant
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (!uncapped_blocks[dev]) {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_raster_fwd<4, 128, false, true, false, kBwdChunk, false>,
                                                  kTilePixels / 4, 0);
    uncapped_blocks[dev] = b > 0 ? b : 1;
  }
  const bool one_wave = L.n_tiles <= static_cast<int64_t>(device_sms()) * uncapped_blocks[dev];
#define GS_FB_M(P, C, M)                                                                                             \
  launch(k_raster_fwd<P, C, false, true, false, kBwdChunk, M>, grid, kTilePixels / P,                                 \
         cap_smem(k_raster_fwd<P, C, false, true, false, kBwdChunk, M>, L.raster_bps), s, L, w, rgb, depth, T_final, \
         last, ev, cp, F, Occlusion{})
#define GS_FB(P, C)                       \
  if (one_wave) {                         \
    GS_FB_M(P, C, (P != 4));              \
  } else {                                \
    GS_FB_M(P, C, true);                  \
  }
#define GS_FB_CH(P)                  \
  switch (ch) {                      \
    case 64: GS_FB(P, 64); break;    \
    case 256: GS_FB(P, 256); break;  \
    default: GS_FB(P, 128); break;   \
  }
  switch (px) {
    case 1: GS_FB_CH(1); break;
    case 2: GS_FB_CH(2); break;
    default: GS_FB_CH(4); break;
  }
#undef GS_FB_CH
#undef GS_FB
#undef GS_FB_M
  return cudaGetLastError();
}

cudaError_t launch_raster_fwd(const Layout& L, void* ws, float* rgb, float* depth, float* T_final, int32_t* last,
                              bool stats, const FusedLossArgs* loss, cudaStream_t s, const float* ext_depth,
                              const float* ext_rgb) {
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
  const int ch = pick_chunk(L.fwd_chunk, 64, 256, kFwdChunk);
#define GS_FWD(P, C, ST, LO)                                                                                  \
  launch(k_raster_fwd<P, C, ST, LO>, grid, kTilePixels / P, cap_smem(k_raster_fwd<P, C, ST, LO>, L.raster_bps), s, \
         L, w, rgb, depth, T_final, last, ev, cp, F, Occlusion{})
#define GS_FWD_CH(P, ST, LO)              \
  switch (ch) {                           \
    case 64: GS_FWD(P, 64, ST, LO); break;   \
    case 256: GS_FWD(P, 256, ST, LO); break; \
    default: GS_FWD(P, 128, ST, LO); break;  \
  }
  if (ext_depth) {  // occlusion by an external surface: one chunk depth
    const Occlusion O{ext_depth, ext_rgb};
    switch (px) {
      case 1: launch(k_raster_fwd<1, kFwdChunk, false, false, true>, grid, kTilePixels, 0, s, L, w, rgb, depth, T_final,
                     last, ev, cp, F, O); break;
      case 2: launch(k_raster_fwd<2, kFwdChunk, false, false, true>, grid, kTilePixels / 2, 0, s, L, w, rgb, depth,
                     T_final, last, ev, cp, F, O); break;
      default: launch(k_raster_fwd<4, kFwdChunk, false, false, true>, grid, kTilePixels / 4, 0, s, L, w, rgb, depth,
                      T_final, last, ev, cp, F, O); break;
    }
  } else if (stats) {  // the counting variant: one chunk depth (the chunking changes no decision)
    switch (px) {
      case 1: GS_FWD(1, kFwdChunk, true, false); break;
      case 2: GS_FWD(2, kFwdChunk, true, false); break;
      default: GS_FWD(4, kFwdChunk, true, false); break;
    }
  } else if (loss) {
    switch (px) {
      case 1: GS_FWD_CH(1, false, true); break;
      case 2: GS_FWD_CH(2, false, true); break;
      default: GS_FWD_CH(4, false, true); break;
    }
  } else {
    switch (px) {
      case 1: GS_FWD_CH(1, false, false); break;
      case 2: GS_FWD_CH(2, false, false); break;
      default: GS_FWD_CH(4, false, false); break;
    }
  }
#undef GS_FWD_CH
#undef GS_FWD
  return cudaGetLastError();
}

}  // namespace gs
