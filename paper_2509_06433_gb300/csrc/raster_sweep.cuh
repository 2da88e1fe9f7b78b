// The backward sweep of one tile (the body of gs_raster_bwd, also run by the loss-fused forward
// when it continues into the backward pass); see raster_common.cuh for the staging and the
// opacity test it shares with the forward.
#pragma once

#include "raster_common.cuh"

namespace gs {
namespace {

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

// Shared memory of one backward sweep: the staged chunk, the chunk's record slots, the warp
// partials of its 10 sums and the warps' largest `last`.
template <int PX, int CH>
struct BwdSmem {
  static constexpr int kWarps = kTilePixels / PX / 32;
  Stage<CH> S;
  uint32_t slot[CH];
  float part[kWarps][CH][10];
  int maxlast[kWarps];
};

// Colour and depth of a pixel weighted by its upstream gradient, in one fixed rounding order (the
// backward's starting value of the weighted colour behind each splat).
__device__ __forceinline__ float weighted_colour(float gr, float gg, float gb, float gd, float r, float g, float b,
                                                 float d) {
  return __fmaf_rn(gd, d, __fmaf_rn(gb, b, __fmaf_rn(gg, g, __fmul_rn(gr, r))));
}

// Gradient record layout (floats): 0 du, 1 dv, 2 dA, 3 dB, 4 dC, 5 dz, 6 do, 7 dr, 8 dg, 9 db.
//
// Per pixel, with dpow = dL/dpower / ln 2 (zero where the splat is skipped or clamped) and
// (dx, dy) the offset mean - pixel centre, the geometric terms are sums over the pixels of
//   du = ln2 (2 qa dx + qb dy) dpow,  dv = ln2 (qb dx + 2 qc dy) dpow,
//   dA = -dx^2 dpow / 2,  dB = -dx dy dpow,  dC = -dy^2 dpow / 2,  do = dpow / opacity.
// A lane's pixels share dx, so it keeps only P0 = sum dpow, P1 = sum dy dpow, P2 = sum dy^2 dpow
// (per packed pair of pixels, the halves added before the reduction) and the warp reduces
// R = (dx P0, P1, dx^2 P0, dx P1, P2, P0); the splat's coefficients qa, qb, qc, opacity are
// applied once per pair when the warp partials are summed.
//
// Per pixel of the calling thread (PX vertically adjacent pixels of one column): Sg = the
// weighted colour of the forward output (weighted_colour), hT = dL/dT_final * T_final, the
// upstream gradients and `last` (0 for pixels outside the image). The sweep walks the tile's
// list front to back up to the largest `last` of its pixels, recomputing T from 1, and writes
// one record per pair in front of some pixel's last contributor. All threads of the block call it.
// HT = false: every hT is zero (no dL/dT_final term) and the sweep leaves it out; the results are
// the same bit for bit (a zero addend changes at most the sign of a zero, which the sums drop).
template <int PX, int CH, bool HT = true>
__device__ __forceinline__ void bwd_sweep(BwdSmem<PX, CH>& M, const Layout& L, uint8_t* __restrict__ ws,
                                          const TileCoord& tc, uint2 rg, const float (&Sg)[PX], const float (&hT)[PX],
                                          const float (&gr)[PX], const float (&gg)[PX], const float (&gb)[PX],
                                          const float (&gd)[PX], const int (&last)[PX]) {
  constexpr int kThreads = kTilePixels / PX;
  constexpr int kWarps = kThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = threadIdx.x & (kTile - 1), ly = (threadIdx.x / kTile) * PX;
  const uint64_t* keys = at<uint64_t>(ws, (L.passes & 1) ? L.keys[1] : L.keys[0]);
  const uint32_t* slots = at<uint32_t>(ws, (L.passes & 1) ? L.vals[1] : L.vals[0]);  // emission index = record slot
  const float ox = static_cast<float>(tc.tx * kTile), oy = static_cast<float>(tc.ty * kTile);
  const float pxc = static_cast<float>(lx) + 0.5f, pyc = static_cast<float>(ly) + 0.5f;
  const uint32_t wrows = ((1u << (2 * PX)) - 1u) << ((threadIdx.x >> 5) * 2 * PX);
  float* pair_grads = at<float>(ws, L.pair_grads);
  uint32_t* pair_valid = at<uint32_t>(ws, L.pair_valid);
  constexpr int W = PX >= 2 ? 2 : 1, G = PX / W;  // pixel q is component q % W of group q / W
  using V = typename Vec<W>::T;
  const V npx = bcast<W>(-pxc), zero = bcast<W>(0.0f), minus1 = bcast<W>(-1.0f);
  V T[G], npy[G], Sgv[G], hTv[G], grv[G], ggv[G], gbv[G], gdv[G];
  int wl = 0;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    T[g] = bcast<W>(1.0f);
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const int q = g * W + i;
      set_comp(npy[g], i, -(pyc + static_cast<float>(q)));
      set_comp(Sgv[g], i, Sg[q]);
      set_comp(hTv[g], i, hT[q]);
      set_comp(grv[g], i, gr[q]);
      set_comp(ggv[g], i, gg[q]);
      set_comp(gbv[g], i, gb[q]);
      set_comp(gdv[g], i, gd[q]);
      wl = max(wl, last[q]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, o));
  const int warp_last = wl;  // this warp's pixels need list positions [0, warp_last)
  if (lane == 0) M.maxlast[warp] = wl;
  __syncthreads();
  int max_last = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) max_last = max(max_last, M.maxlast[w]);
  const uint32_t stop = min(rg.y, rg.x + static_cast<uint32_t>(max_last));
  const int idx = reduce10_index(lane);
  const bool writer = reduce10_writer(lane);
  constexpr float kLn2 = 0.6931471805599453f;

  for (uint32_t base = rg.x; base < stop; base += CH) {
    for (int jj = threadIdx.x; jj < CH; jj += kThreads) {
      const uint32_t i = base + jj;
      if (i < stop) {
        stage_splat(M.S, jj, L, ws, keys, i, tc.k, ox, oy);
        M.slot[jj] = slots[i];
      }
    }
    for (int e = threadIdx.x; e < kWarps * CH * 10; e += kThreads) (&M.part[0][0][0])[e] = 0.0f;
    __syncthreads();
    const int n = min(CH, static_cast<int>(stop - base));
    const int pos0 = static_cast<int>(base - rg.x);
    const int nw = min(n, warp_last - pos0);  // splats of this chunk this warp must visit
    for (int j = 0; j < nw; ++j) {
      if (!(M.S.rows[j] & wrows)) continue;
      const float4 A = M.S.A[j], B = M.S.B[j];
      const Column<W> col = splat_column<W>(A, B, npx);
      const V Ay = bcast<W>(A.y);
      const int pos = pos0 + j;
      // phase 1: opacity and keep/skip decision for the thread's pixels
      V dy[G], alpha[G];
      float raw[PX];
      bool okq[PX];
      bool contrib = false;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        dy[g] = vadd(Ay, npy[g]);
        const V e = splat_exponent<W>(B, col, dy[g]);
#pragma unroll
        for (int i = 0; i < W; ++i) {
          const int q = g * W + i;
          raw[q] = ex2_approx(comp(e, i));
          const float a = fminf(raw[q], kAlphaMax);
          set_comp(alpha[g], i, a);
          okq[q] = (comp(e, i) <= B.w) && (a >= kAlphaMin) && (pos < last[q]);
          contrib = contrib || okq[q];
        }
      }
      // phase 2 (skipped when no pixel of the warp keeps the splat): gradient terms, two pixels
      // per packed instruction. The colour-gradient sums are kept negated (nw = -w).
      if (!__any_sync(0xffffffffu, contrib)) continue;
      const float4 C = M.S.C[j];
      const V cR = bcast<W>(C.x), cG = bcast<W>(C.y), cB = bcast<W>(C.z), cZ = bcast<W>(B.z);
      V P0 = zero, P1 = zero, P2 = zero, ncz = zero, ncr = zero, ncg = zero, ncb = zero;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        // aok = alpha for a kept splat, else 0: then w = 0 and Sg, T stay unchanged;
        // oal = alpha where the gradient passes (kept and not clamped at 0.99), else 0
        V aok, oal, nr;
#pragma unroll
        for (int i = 0; i < W; ++i) {
          const int q = g * W + i;
          const float a = comp(alpha[g], i);
          set_comp(aok, i, okq[q] ? a : 0.0f);
          set_comp(oal, i, (okq[q] && !(raw[q] > kAlphaMax)) ? a : 0.0f);
          set_comp(nr, i, rcp_approx(a - 1.0f));  // -1 / (1 - alpha)
        }
        const V nT = vmul(T[g], minus1);
        const V nw = vmul(aok, nT);
        const V cgz = vfma(cZ, gdv[g], vfma(cB, gbv[g], vfma(cG, ggv[g], vmul(cR, grv[g]))));
        const V sg = vfma(cgz, nw, Sgv[g]);  // colour/depth behind this splat, weighted by dL/dpixel
        const V dalpha = vfma(T[g], cgz, vmul(HT ? vadd(sg, hTv[g]) : sg, nr));
        const V dpow = vmul(oal, dalpha);
        const V ydp = vmul(dy[g], dpow);
        P0 = vadd(P0, dpow);
        P1 = vadd(P1, ydp);
        P2 = vfma(dy[g], ydp, P2);
        ncz = vfma(nw, gdv[g], ncz);
        ncr = vfma(nw, grv[g], ncr);
        ncg = vfma(nw, ggv[g], ncg);
        ncb = vfma(nw, gbv[g], ncb);
        Sgv[g] = sg;
        T[g] = vfma(nT, aok, T[g]);
      }
      const float p0 = hsum(P0), p1 = hsum(P1);
      const float dx = comp(col.dx, 0);
      const float dxP0 = dx * p0;
      const float v[10] = {dxP0, p1, dx * dxP0, dx * p1, hsum(P2), hsum(ncz), p0, hsum(ncr), hsum(ncg), hsum(ncb)};
      const float r = warp_reduce10(v, lane);
      if (writer) M.part[warp][j][idx] = r;
    }
    __syncthreads();
    for (int jj = threadIdx.x; jj < n; jj += kThreads) {
      float R[10];
#pragma unroll
      for (int q = 0; q < 10; ++q) {
        float acc = 0.0f;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) acc += M.part[w][jj][q];
        R[q] = acc;
      }
      // R = (sum dx P0, sum P1, sum dx^2 P0, sum dx P1, sum P2, -dz, sum P0, -dr, -dg, -db)
      const float qa = M.S.A[jj].z, qb = M.S.A[jj].w, qc = M.S.B[jj].x, op = M.S.B[jj].y;
      const float du = kLn2 * (2.0f * qa * R[0] + qb * R[1]);
      const float dv = kLn2 * (2.0f * qc * R[1] + qb * R[0]);
      const float dop = R[6] != 0.0f ? R[6] / op : 0.0f;
      const uint32_t slot = M.slot[jj];
      if (!GS_INDEX_OK(static_cast<int64_t>(slot) < L.cap, &at<Status>(ws, L.status)->err)) continue;
      float4* dst = reinterpret_cast<float4*>(pair_grads + static_cast<size_t>(slot) * kPairGradStride);
      dst[0] = make_float4(du, dv, -0.5f * R[2], -R[3]);
      dst[1] = make_float4(-0.5f * R[4], -R[5], dop, -R[7]);
      dst[2] = make_float4(-R[8], -R[9], 0.0f, 0.0f);
      atomicOr(&pair_valid[slot >> 5], 1u << (slot & 31));
    }
    __syncthreads();
  }
  // pairs behind every pixel's last contributor get no record: their bit stays clear
}

}  // namespace
}  // namespace gs
