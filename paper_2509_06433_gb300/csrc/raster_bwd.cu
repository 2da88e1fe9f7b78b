// Backward compositing (gs_raster_bwd): loads the forward outputs and the upstream gradients
// of its pixels, then runs the tile's backward sweep (raster_sweep.cuh).
#include "raster_sweep.cuh"

namespace gs {
namespace {

template <int PX, int CH>
__global__ void __launch_bounds__(kTilePixels / PX, PX == 4 ? kMinBlocksPx4 : 1) k_raster_bwd(Layout L, uint8_t* __restrict__ ws,
                                                                 const float* __restrict__ rgb,
                                                                 const float* __restrict__ depth,
                                                                 const float* __restrict__ T_final,
                                                                 const int32_t* __restrict__ last_in,
                                                                 const float* __restrict__ g_rgb,
                                                                 const float* __restrict__ g_depth,
                                                                 const float* __restrict__ g_T) {
  pdl_wait();
  __shared__ BwdSmem<PX, CH> M;
  const TileCoord tc = tile_coord(L, blockIdx.x);
  const int lx = threadIdx.x & (kTile - 1), ly = (threadIdx.x / kTile) * PX;
  const int px = tc.tx * kTile + lx, py = tc.ty * kTile + ly;
  const uint2 rg = at<uint2>(ws, L.ranges)[blockIdx.x];
  const int64_t HW = static_cast<int64_t>(L.H) * L.W;
  float Sg[PX], hT[PX], gr[PX], gg[PX], gb[PX], gd[PX];
  int last[PX];
#pragma unroll
  for (int q = 0; q < PX; ++q) {
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
      Sg[q] = weighted_colour(gr[q], gg[q], gb[q], gd[q], rgb[c0], rgb[c0 + HW], rgb[c0 + 2 * HW],
                              depth[tc.k * HW + pix]);
      if (g_T) hT[q] = g_T[tc.k * HW + pix] * T_final[tc.k * HW + pix];
      last[q] = last_in[tc.k * HW + pix];
    }
  }
  bwd_sweep<PX, CH>(M, L, ws, tc, rg, Sg, hT, gr, gg, gb, gd, last);
  pdl_trigger();
}

}  // namespace

cudaError_t launch_raster_bwd(const Layout& L, void* ws, const float* rgb, const float* depth, const float* T_final,
                              const int32_t* last, const float* dL_drgb, const float* dL_ddepth, const float* dL_dT,
                              cudaStream_t s) {
  if (L.n_tiles == 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>(L.n_tiles);
  uint8_t* w = static_cast<uint8_t*>(ws);
  const int ch = pick_chunk(L.bwd_chunk, 32, 128, kBwdChunk);
#define GS_BWD(P, C)                                                                                             \
  launch(k_raster_bwd<P, C>, grid, kTilePixels / P, cap_smem(k_raster_bwd<P, C>, L.raster_bps), s, L, w, rgb, depth, \
         T_final, last, dL_drgb, dL_ddepth, dL_dT)
#define GS_BWD_CH(P)                 \
  switch (ch) {                      \
    case 32: GS_BWD(P, 32); break;   \
    case 128: GS_BWD(P, 128); break; \
    default: GS_BWD(P, 64); break;   \
  }
  switch (pick_px(L.bwd_px, kDefaultBwdPx)) {
    case 1: GS_BWD_CH(1); break;
    case 2: GS_BWD_CH(2); break;
    default: GS_BWD_CH(4); break;
  }
#undef GS_BWD_CH
#undef GS_BWD
  return cudaGetLastError();
}

}  // namespace gs
