// Tile compositing: forward (render) and backward (splat gradients).
//
// One CTA per (view, 16x16 tile), one thread per pixel. The tile's depth-sorted list is
// walked in chunks of 256 splats staged in shared memory (coalesced loads of the sorted
// Gaussian ids, one gather of the projected record per splat). Both kernels evaluate the
// splat opacity with the same inline function and the same operand values, so the
// backward pass takes exactly the forward pass's skip and stop decisions and recovers the
// same transmittance T_i front to back, without storing per-splat alphas.
//
// The backward pass reduces each splat's 10 gradient terms over the 32 pixels of a warp
// by a transpose-reduce (16 shuffles for 16 padded values), over the 8 warps through
// shared-memory atomics, and writes one record per (splat, tile) pair into the pair
// gradient buffer: no global atomics, so the summed gradients are deterministic.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = kTilePixels;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTStop = 1e-4f;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Splat record in shared memory (structure of arrays, one chunk).
struct SplatSmem {
  float x[kThreads], y[kThreads];        // tile-relative 2D mean
  float qa[kThreads], qb[kThreads], qc[kThreads];  // power * log2(e) = qa dx^2 + qb dx dy + qc dy^2
  float o[kThreads];
  float r[kThreads], g[kThreads], b[kThreads], z[kThreads];
};

// Loads splat `i` of the sorted list into slot `j`; returns the Gaussian id.
__device__ __forceinline__ uint32_t load_splat(SplatSmem& S, int j, const Layout& L, const uint8_t* ws,
                                               const uint32_t* vals, uint32_t i, int k, float ox, float oy) {
  const uint32_t gid = vals[i];
  const int64_t kg = static_cast<int64_t>(k) * L.N + gid;
  const float4 uv = at<float4>(ws, L.proj_uv)[kg];
  const float4 cn = at<float4>(ws, L.proj_conic)[kg];
  const float4 co = at<float4>(ws, L.color_opacity)[gid];
  S.x[j] = __fadd_rn(__fsub_rn(uv.x, ox), uv.y);
  S.y[j] = __fadd_rn(__fsub_rn(uv.z, oy), uv.w);
  S.qa[j] = __fmul_rn(cn.x, -0.5f * kLog2e);
  S.qb[j] = __fmul_rn(cn.y, -kLog2e);
  S.qc[j] = __fmul_rn(cn.z, -0.5f * kLog2e);
  S.z[j] = cn.w;
  S.r[j] = co.x;
  S.g[j] = co.y;
  S.b[j] = co.z;
  S.o[j] = co.w;
  return gid;
}

// Opacity of splat j at pixel offset (dx, dy). Returns false when the splat is skipped
// (power > 0 or alpha < 1/255). G = exp(power); clamped: alpha hit 0.99.
__device__ __forceinline__ bool splat_alpha(const SplatSmem& S, int j, float dx, float dy, float& alpha, float& G,
                                            bool& clamped) {
  const float p = __fmaf_rn(dx, __fmaf_rn(S.qa[j], dx, __fmul_rn(S.qb[j], dy)), __fmul_rn(__fmul_rn(S.qc[j], dy), dy));
  if (p > 0.0f) return false;
  G = ex2_approx(p);
  const float a = __fmul_rn(S.o[j], G);
  clamped = a > kAlphaMax;
  alpha = clamped ? kAlphaMax : a;
  return alpha >= kAlphaMin;
}

__global__ void __launch_bounds__(kThreads) k_raster_fwd(Layout L, const uint8_t* __restrict__ ws,
                                                         float* __restrict__ out_rgb, float* __restrict__ out_depth,
                                                         float* __restrict__ out_T, int32_t* __restrict__ out_last,
                                                         uint64_t* __restrict__ evals_out,
                                                         uint64_t* __restrict__ composited_out) {
  __shared__ SplatSmem S;
  __shared__ uint32_t s_evals[kThreads / 32], s_blend[kThreads / 32];
  const int64_t tile_g = blockIdx.x;
  const int64_t per_view = static_cast<int64_t>(L.Tx) * L.Ty;
  const int k = static_cast<int>(tile_g / per_view);
  const int tt = static_cast<int>(tile_g - k * per_view);
  const int ty = tt / L.Tx, tx = tt - ty * L.Tx;
  const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile;
  const int px = tx * kTile + lx, py = ty * kTile + ly;
  const bool inside = px < L.W && py < L.H;
  const uint32_t* vals = at<uint32_t>(ws, (L.passes & 1) ? L.vals[1] : L.vals[0]);
  const uint2 rg = at<uint2>(ws, L.ranges)[tile_g];
  const float ox = static_cast<float>(tx * kTile), oy = static_cast<float>(ty * kTile);
  const float pxc = static_cast<float>(lx) + 0.5f, pyc = static_cast<float>(ly) + 0.5f;
  float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f, cd = 0.0f;
  int32_t last = 0;
  uint32_t evals = 0, blended = 0;
  bool done = !inside;
  for (uint32_t base = rg.x; base < rg.y; base += kThreads) {
    if (__syncthreads_count(!done) == 0) break;
    const uint32_t i = base + threadIdx.x;
    if (i < rg.y) load_splat(S, threadIdx.x, L, ws, vals, i, k, ox, oy);
    __syncthreads();
    const int n = min(kThreads, static_cast<int>(rg.y - base));
    if (!done) {
      for (int j = 0; j < n; ++j) {
        ++evals;
        float alpha, G;
        bool clamped;
        if (!splat_alpha(S, j, __fsub_rn(S.x[j], pxc), __fsub_rn(S.y[j], pyc), alpha, G, clamped)) continue;
        const float Tn = __fmaf_rn(-T, alpha, T);
        if (Tn < kTStop) {
          done = true;
          break;
        }
        const float w = __fmul_rn(alpha, T);
        cr = __fmaf_rn(S.r[j], w, cr);
        cg = __fmaf_rn(S.g[j], w, cg);
        cb = __fmaf_rn(S.b[j], w, cb);
        cd = __fmaf_rn(S.z[j], w, cd);
        T = Tn;
        ++blended;
        last = static_cast<int32_t>(base - rg.x) + j + 1;
      }
    }
  }
  if (inside) {
    const int64_t HW = static_cast<int64_t>(L.H) * L.W;
    const int64_t pix = static_cast<int64_t>(py) * L.W + px;
    if (out_rgb) {
      out_rgb[(static_cast<int64_t>(k) * 3 + 0) * HW + pix] = cr;
      out_rgb[(static_cast<int64_t>(k) * 3 + 1) * HW + pix] = cg;
      out_rgb[(static_cast<int64_t>(k) * 3 + 2) * HW + pix] = cb;
    }
    if (out_depth) out_depth[k * HW + pix] = cd;
    if (out_T) out_T[k * HW + pix] = T;
    if (out_last) out_last[k * HW + pix] = last;
  }
  uint32_t e = evals, c = blended;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_evals[threadIdx.x >> 5] = e;
    s_blend[threadIdx.x >> 5] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t tot = 0, totc = 0;
    for (int w = 0; w < kThreads / 32; ++w) {
      tot += s_evals[w];
      totc += s_blend[w];
    }
    if (tot) atomicAdd(reinterpret_cast<unsigned long long*>(evals_out), static_cast<unsigned long long>(tot));
    if (totc) atomicAdd(reinterpret_cast<unsigned long long*>(composited_out), static_cast<unsigned long long>(totc));
  }
}

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

// Gradient record layout (floats): 0 du, 1 dv, 2 dA, 3 dB, 4 dC, 5 dz, 6 do, 7 dr, 8 dg, 9 db.
__global__ void __launch_bounds__(kThreads) k_raster_bwd(Layout L, uint8_t* __restrict__ ws,
                                                         const float* __restrict__ rgb, const float* __restrict__ depth,
                                                         const float* __restrict__ T_final,
                                                         const int32_t* __restrict__ last_in,
                                                         const float* __restrict__ g_rgb,
                                                         const float* __restrict__ g_depth,
                                                         const float* __restrict__ g_T) {
  __shared__ SplatSmem S;
  __shared__ float s_acc[kThreads][kPairGradStride];
  // per-warp partial sums of a sub-chunk of kSub splats, summed over warps in a fixed order
  constexpr int kSub = 32;
  __shared__ float s_part[kThreads / 32][kSub][10];
  __shared__ uint32_t s_slot[kThreads];
  __shared__ int s_maxlast[kThreads / 32];
  const int64_t tile_g = blockIdx.x;
  const int64_t per_view = static_cast<int64_t>(L.Tx) * L.Ty;
  const int k = static_cast<int>(tile_g / per_view);
  const int tt = static_cast<int>(tile_g - k * per_view);
  const int ty = tt / L.Tx, tx = tt - ty * L.Tx;
  const int lane = threadIdx.x & 31;
  const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile;
  const int px = tx * kTile + lx, py = ty * kTile + ly;
  const bool inside = px < L.W && py < L.H;
  const uint32_t* vals = at<uint32_t>(ws, (L.passes & 1) ? L.vals[1] : L.vals[0]);
  const uint2 rg = at<uint2>(ws, L.ranges)[tile_g];
  const float ox = static_cast<float>(tx * kTile), oy = static_cast<float>(ty * kTile);
  const float pxc = static_cast<float>(lx) + 0.5f, pyc = static_cast<float>(ly) + 0.5f;
  const int4* tiles = at<int4>(ws, L.proj_tiles);
  float* pair_grads = at<float>(ws, L.pair_grads);

  float gr = 0.f, gg = 0.f, gb = 0.f, gd = 0.f, Sg = 0.f, hT = 0.f;
  int lastp = 0;
  if (inside) {
    const int64_t HW = static_cast<int64_t>(L.H) * L.W;
    const int64_t pix = static_cast<int64_t>(py) * L.W + px;
    const int64_t c0 = (static_cast<int64_t>(k) * 3) * HW + pix;
    gr = g_rgb[c0];
    gg = g_rgb[c0 + HW];
    gb = g_rgb[c0 + 2 * HW];
    gd = g_depth[k * HW + pix];
    Sg = gr * rgb[c0] + gg * rgb[c0 + HW] + gb * rgb[c0 + 2 * HW] + gd * depth[k * HW + pix];
    if (g_T) hT = g_T[k * HW + pix] * T_final[k * HW + pix];
    lastp = last_in[k * HW + pix];
  }
  int ml = lastp;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ml = max(ml, __shfl_xor_sync(0xffffffffu, ml, o));
  if (lane == 0) s_maxlast[threadIdx.x >> 5] = ml;
  __syncthreads();
  int max_last = 0;
  for (int w = 0; w < kThreads / 32; ++w) max_last = max(max_last, s_maxlast[w]);
  const uint32_t stop = min(rg.y, rg.x + static_cast<uint32_t>(max_last));
  float T = 1.0f;

  for (uint32_t base = rg.x; base < stop; base += kThreads) {
    const uint32_t i = base + threadIdx.x;
    if (i < stop) {
      const uint32_t gid = load_splat(S, threadIdx.x, L, ws, vals, i, k, ox, oy);
      const int4 tl = tiles[static_cast<int64_t>(k) * L.N + gid];
      const uint32_t x0 = static_cast<uint32_t>(tl.y) & 0xffffu, x1 = static_cast<uint32_t>(tl.y) >> 16;
      const uint32_t y0 = static_cast<uint32_t>(tl.z) & 0xffffu;
      s_slot[threadIdx.x] = static_cast<uint32_t>(tl.x) + (static_cast<uint32_t>(ty) - y0) * (x1 - x0) +
                            (static_cast<uint32_t>(tx) - x0);
    }
#pragma unroll
    for (int q = 0; q < kPairGradStride; ++q) s_acc[threadIdx.x][q] = 0.0f;
    __syncthreads();
    const int n = min(kThreads, static_cast<int>(stop - base));
    const int pos0 = static_cast<int>(base - rg.x);
    for (int j = 0; j < n; ++j) {
      float v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = 0.0f;
      bool contrib = false;
      if (pos0 + j < lastp) {
        const float dx = __fsub_rn(S.x[j], pxc), dy = __fsub_rn(S.y[j], pyc);
        float alpha, G;
        bool clamped;
        if (splat_alpha(S, j, dx, dy, alpha, G, clamped)) {
          const float Tn = __fmaf_rn(-T, alpha, T);
          const float w = __fmul_rn(alpha, T);
          const float cgz = S.r[j] * gr + S.g[j] * gg + S.b[j] * gb + S.z[j] * gd;
          Sg -= cgz * w;  // now: sum over the splats behind this one
          const float dalpha = T * cgz - (Sg + hT) / (1.0f - alpha);
          v[5] = w * gd;
          v[7] = w * gr;
          v[8] = w * gg;
          v[9] = w * gb;
          if (!clamped) {
            const float dpow = alpha * dalpha;
            // power = -0.5 (A dx^2 + C dy^2) - B dx dy; qa = -0.5 A log2e, qb = -B log2e, qc = -0.5 C log2e
            constexpr float kLn2 = 0.6931471805599453f;
            v[6] = G * dalpha;
            v[2] = -0.5f * dx * dx * dpow;
            v[3] = -dx * dy * dpow;
            v[4] = -0.5f * dy * dy * dpow;
            v[0] = (2.0f * S.qa[j] * dx + S.qb[j] * dy) * kLn2 * dpow;
            v[1] = (2.0f * S.qc[j] * dy + S.qb[j] * dx) * kLn2 * dpow;
          }
          T = Tn;
          contrib = true;
        }
      }
      const int idx = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
      float red = 0.0f;
      if (__any_sync(0xffffffffu, contrib)) {
        warp_transpose_reduce16(v, lane);
        red = v[0];
      }
      if (!(lane & 1) && idx < 10) s_part[threadIdx.x >> 5][j % kSub][idx] = red;
      if ((j % kSub) == kSub - 1 || j == n - 1) {
        __syncthreads();
        const int j0 = j - (j % kSub);
        for (int e = threadIdx.x; e < kSub * 10; e += kThreads) {
          const int jj = e / 10, q = e - jj * 10;
          if (j0 + jj <= j) {
            float acc = 0.0f;
#pragma unroll
            for (int wv = 0; wv < kThreads / 32; ++wv) acc += s_part[wv][jj][q];
            s_acc[j0 + jj][q] = acc;
          }
        }
        __syncthreads();
      }
    }
    __syncthreads();
    if (threadIdx.x < n) {
      float4* dst = reinterpret_cast<float4*>(pair_grads + static_cast<size_t>(s_slot[threadIdx.x]) * kPairGradStride);
      const float* a = s_acc[threadIdx.x];
      dst[0] = make_float4(a[0], a[1], a[2], a[3]);
      dst[1] = make_float4(a[4], a[5], a[6], a[7]);
      dst[2] = make_float4(a[8], a[9], 0.0f, 0.0f);
    }
    __syncthreads();
  }
  // pairs behind every pixel's last contributor receive zero records
  for (uint32_t i = stop + threadIdx.x; i < rg.y; i += kThreads) {
    const uint32_t gid = vals[i];
    const int4 tl = tiles[static_cast<int64_t>(k) * L.N + gid];
    const uint32_t x0 = static_cast<uint32_t>(tl.y) & 0xffffu, x1 = static_cast<uint32_t>(tl.y) >> 16;
    const uint32_t y0 = static_cast<uint32_t>(tl.z) & 0xffffu;
    const uint32_t slot =
        static_cast<uint32_t>(tl.x) + (static_cast<uint32_t>(ty) - y0) * (x1 - x0) + (static_cast<uint32_t>(tx) - x0);
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
  k_raster_fwd<<<static_cast<unsigned>(L.n_tiles), kThreads, 0, s>>>(L, static_cast<const uint8_t*>(ws), rgb, depth,
                                                                     T_final, last, &st->evals, &st->composited);
  return cudaGetLastError();
}

cudaError_t launch_raster_bwd(const Layout& L, void* ws, const float* rgb, const float* depth, const float* T_final,
                              const int32_t* last, const float* dL_drgb, const float* dL_ddepth, const float* dL_dT,
                              cudaStream_t s) {
  if (L.n_tiles == 0) return cudaSuccess;
  k_raster_bwd<<<static_cast<unsigned>(L.n_tiles), kThreads, 0, s>>>(L, static_cast<uint8_t*>(ws), rgb, depth,
                                                                     T_final, last, dL_drgb, dL_ddepth, dL_dT);
  return cudaGetLastError();
}

}  // namespace gs
