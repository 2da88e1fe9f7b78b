// Photometric loss of a mapping step and its image gradient:
//   L = sum_k [ mean_{3HW} |R - R*| + lambda mean_{HW} |D - D*| ],  sign(0) = 0.
// One thread per pixel (all K views); per-block partial sums are reduced in a fixed order
// by a second kernel, so L is deterministic.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float sgn(float d) { return d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f); }

__global__ void __launch_bounds__(kThreads) k_loss(Layout L, const float* __restrict__ rgb,
                                                  const float* __restrict__ depth, const float* __restrict__ rgb_t,
                                                  const float* __restrict__ depth_t, float* __restrict__ g_rgb,
                                                  float* __restrict__ g_depth, float* __restrict__ partials) {
  pdl_begin();
  const int64_t HW = static_cast<int64_t>(L.H) * L.W;
  const int64_t total = HW * L.K;
  const float inv3 = 1.0f / (3.0f * static_cast<float>(HW));
  const float invd = L.lambda_depth / static_cast<float>(HW);
  float acc = 0.0f;
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; p < total;
       p += static_cast<int64_t>(gridDim.x) * kThreads) {
    const int64_t k = p / HW, pix = p - k * HW;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t i = (k * 3 + c) * HW + pix;
      const float d = rgb[i] - rgb_t[i];
      acc += fabsf(d) * inv3;
      g_rgb[i] = sgn(d) * inv3;
    }
    const float d = depth[p] - depth_t[p];
    acc += fabsf(d) * invd;
    g_depth[p] = sgn(d) * invd;
  }
  __shared__ float s[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < kThreads / 32; ++w) t += s[w];
    partials[blockIdx.x] = t;
  }
}

__global__ void k_loss_final(const float* __restrict__ partials, int n, float* __restrict__ out) {
  pdl_begin();
  __shared__ float s[32];
  float acc = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) t += s[w];
    out[0] = t;
  }
}

}  // namespace

cudaError_t launch_loss(const Layout& L, const float* rgb, const float* depth, const float* rgb_t,
                        const float* depth_t, float* g_rgb, float* g_depth, float* d_loss, void* ws, cudaStream_t s) {
  float* partials = at<float>(ws, L.loss_partials);
  launch(k_loss, static_cast<unsigned>(L.n_loss_blocks), kThreads, 0, s, L, rgb, depth, rgb_t, depth_t, g_rgb, g_depth,
                                                                     partials);
  launch(k_loss_final, 1, 1024, 0, s, partials, static_cast<int>(L.n_loss_blocks), d_loss);
  return cudaGetLastError();
}

}  // namespace gs
