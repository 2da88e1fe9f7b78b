// Map-accuracy metrics (Sec. IV measures a map by the PSNR and SSIM of its rendered views
// against the key-frames): per-image PSNR and SSIM of float images [B, C, H, W].
//
// PSNR = 10 log10(R^2 / MSE) over all C*H*W values of an image. SSIM (Wang et al. 2004) uses
// an 11 x 11 separable Gaussian window (sigma 1.5, taps normalised to sum 1) over zero-padded
// planes and C1 = (0.01 R)^2, C2 = (0.03 R)^2; an image's SSIM is the mean of its map.
//
// Both are deterministic: every block writes one partial sum to the caller's scratch, and one
// block per image adds its partials in a fixed order (in FP64). SSIM stages a 26 x 26 halo tile
// of both planes in shared memory, filters the five moments (x, y, x^2, y^2, xy) along x for
// the 26 rows, then along y for the 16 x 16 outputs.
#include <math.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kMetThreads = 256;
constexpr int kPsnrChunk = 8192;  // values per PSNR block
constexpr int kSsimTile = 16;
constexpr int kSsimTaps = 11;
constexpr int kSsimRad = kSsimTaps / 2;
constexpr int kSsimIn = kSsimTile + 2 * kSsimRad;  // 26

struct Window {
  float w[kSsimTaps];
};

// sum over the block's 256 threads in a fixed order (shuffle tree, then the 8 warp sums in order)
__device__ __forceinline__ float block_sum(float v, float* s_warp) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.0f;
  if (threadIdx.x == 0)
    for (int w = 0; w < kMetThreads / 32; ++w) t += s_warp[w];
  return t;
}

__device__ __forceinline__ double block_sum_f64(double v, double* s_warp) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kMetThreads / 32; ++w) t += s_warp[w];
  return t;
}

__global__ void __launch_bounds__(kMetThreads) k_sqdiff(const float* __restrict__ x, const float* __restrict__ y,
                                                       int64_t per_image, int blocks_per_image,
                                                       float* __restrict__ partials) {
  pdl_begin();
  __shared__ float s_warp[kMetThreads / 32];
  const int64_t base = static_cast<int64_t>(blockIdx.y) * per_image;
  const int64_t lo = static_cast<int64_t>(blockIdx.x) * kPsnrChunk;
  const int64_t hi = lo + kPsnrChunk < per_image ? lo + kPsnrChunk : per_image;
  float acc = 0.0f;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kMetThreads) {
    const float d = x[base + i] - y[base + i];
    acc = fmaf(d, d, acc);
  }
  const float t = block_sum(acc, s_warp);
  if (threadIdx.x == 0) partials[static_cast<int64_t>(blockIdx.y) * blocks_per_image + blockIdx.x] = t;
}

__global__ void __launch_bounds__(kMetThreads) k_psnr_final(const float* __restrict__ partials, int blocks_per_image,
                                                           int64_t per_image, float range, float* __restrict__ out) {
  pdl_begin();
  __shared__ double s_warp[kMetThreads / 32];
  double acc = 0.0;
  for (int j = threadIdx.x; j < blocks_per_image; j += kMetThreads)
    acc += partials[static_cast<int64_t>(blockIdx.x) * blocks_per_image + j];
  const double t = block_sum_f64(acc, s_warp);
  if (threadIdx.x == 0) {
    const double mse = t / static_cast<double>(per_image);
    const double r = range;
    out[blockIdx.x] = mse > 0.0 ? static_cast<float>(10.0 * log10(r * r / mse)) : INFINITY;
  }
}

// one block per (16 x 16 tile, plane); plane = image * C + channel
__global__ void __launch_bounds__(kMetThreads) k_ssim(const float* __restrict__ x, const float* __restrict__ y, int H,
                                                     int W, int tiles_x, int tiles_per_plane, Window win, float c1,
                                                     float c2, float* __restrict__ map, float* __restrict__ partials) {
  pdl_begin();
  __shared__ float sx[kSsimIn][kSsimIn], sy[kSsimIn][kSsimIn];
  __shared__ float hm[5][kSsimIn][kSsimTile];
  __shared__ float s_warp[kMetThreads / 32];
  const int64_t plane = blockIdx.y;
  const int t = blockIdx.x;
  const int ty0 = (t / tiles_x) * kSsimTile, tx0 = (t % tiles_x) * kSsimTile;
  const int64_t HW = static_cast<int64_t>(H) * W;
  const float* xp = x + plane * HW;
  const float* yp = y + plane * HW;
  for (int i = threadIdx.x; i < kSsimIn * kSsimIn; i += kMetThreads) {
    const int r = i / kSsimIn, c = i - r * kSsimIn;
    const int gy = ty0 + r - kSsimRad, gx = tx0 + c - kSsimRad;
    const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
    const int64_t o = static_cast<int64_t>(gy) * W + gx;
    sx[r][c] = in ? xp[o] : 0.0f;
    sy[r][c] = in ? yp[o] : 0.0f;
  }
  __syncthreads();
  // along x: the 26 rows x 16 output columns
  for (int i = threadIdx.x; i < kSsimIn * kSsimTile; i += kMetThreads) {
    const int r = i / kSsimTile, c = i - r * kSsimTile;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f, a4 = 0.0f;
#pragma unroll
    for (int a = 0; a < kSsimTaps; ++a) {
      const float u = sx[r][c + a], v = sy[r][c + a], w = win.w[a];
      a0 = fmaf(w, u, a0);
      a1 = fmaf(w, v, a1);
      a2 = fmaf(w, u * u, a2);
      a3 = fmaf(w, v * v, a3);
      a4 = fmaf(w, u * v, a4);
    }
    hm[0][r][c] = a0;
    hm[1][r][c] = a1;
    hm[2][r][c] = a2;
    hm[3][r][c] = a3;
    hm[4][r][c] = a4;
  }
  __syncthreads();
  // along y: one output pixel per thread
  const int r = threadIdx.x / kSsimTile, c = threadIdx.x - r * kSsimTile;
  float mx = 0.0f, my = 0.0f, exx = 0.0f, eyy = 0.0f, exy = 0.0f;
#pragma unroll
  for (int a = 0; a < kSsimTaps; ++a) {
    const float w = win.w[a];
    mx = fmaf(w, hm[0][r + a][c], mx);
    my = fmaf(w, hm[1][r + a][c], my);
    exx = fmaf(w, hm[2][r + a][c], exx);
    eyy = fmaf(w, hm[3][r + a][c], eyy);
    exy = fmaf(w, hm[4][r + a][c], exy);
  }
  const float vx = exx - mx * mx, vy = eyy - my * my, cxy = exy - mx * my;
  const float s = ((2.0f * mx * my + c1) * (2.0f * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2));
  const int gy = ty0 + r, gx = tx0 + c;
  const bool valid = gy < H && gx < W;
  if (valid && map) map[plane * HW + static_cast<int64_t>(gy) * W + gx] = s;
  const float tot = block_sum(valid ? s : 0.0f, s_warp);
  if (threadIdx.x == 0) partials[plane * tiles_per_plane + t] = tot;
}

__global__ void __launch_bounds__(kMetThreads) k_mean_final(const float* __restrict__ partials, int64_t per_image,
                                                           double count, float* __restrict__ out) {
  pdl_begin();
  __shared__ double s_warp[kMetThreads / 32];
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < per_image; j += kMetThreads)
    acc += partials[static_cast<int64_t>(blockIdx.x) * per_image + j];
  const double t = block_sum_f64(acc, s_warp);
  if (threadIdx.x == 0) out[blockIdx.x] = static_cast<float>(t / count);
}

bool dims_ok(int32_t B, int32_t C, int32_t H, int32_t W) {
  return B >= 1 && C >= 1 && H >= 1 && W >= 1 && B <= 65535 && static_cast<int64_t>(B) * C <= 65535 && H <= 65536 &&
         W <= 65536;
}
int64_t psnr_blocks(int32_t C, int32_t H, int32_t W) {
  const int64_t n = static_cast<int64_t>(C) * H * W;
  return (n + kPsnrChunk - 1) / kPsnrChunk;
}
int64_t ssim_tiles(int32_t H, int32_t W) {
  return static_cast<int64_t>((W + kSsimTile - 1) / kSsimTile) * ((H + kSsimTile - 1) / kSsimTile);
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status_t gs_metrics_tmp_size(int32_t images, int32_t channels, int32_t height, int32_t width,
                                           size_t* bytes) {
  if (!bytes || !dims_ok(images, channels, height, width)) return GS_ERR_INVALID_ARG;
  const int64_t a = images * psnr_blocks(channels, height, width);
  const int64_t b = static_cast<int64_t>(images) * channels * ssim_tiles(height, width);
  *bytes = static_cast<size_t>(a > b ? a : b) * sizeof(float);
  return GS_OK;
}

extern "C" gs_status_t gs_psnr(const float* x, const float* y, int32_t images, int32_t channels, int32_t height,
                               int32_t width, float data_range, float* psnr, void* tmp, size_t tmp_bytes,
                               void* stream) {
  size_t need = 0;
  if (!x || !y || !psnr || !tmp || !(data_range > 0.0f)) return GS_ERR_INVALID_ARG;
  if (gs_metrics_tmp_size(images, channels, height, width, &need) != GS_OK) return GS_ERR_INVALID_ARG;
  if (tmp_bytes < need) return GS_ERR_WORKSPACE_TOO_SMALL;
  const int64_t per_image = static_cast<int64_t>(channels) * height * width;
  const int nb = static_cast<int>(psnr_blocks(channels, height, width));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* part = static_cast<float*>(tmp);
  launch(k_sqdiff, dim3(nb, images), kMetThreads, 0, s, x, y, per_image, nb, part);
  launch(k_psnr_final, images, kMetThreads, 0, s, part, nb, per_image, data_range, psnr);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

extern "C" gs_status_t gs_ssim(const float* x, const float* y, int32_t images, int32_t channels, int32_t height,
                               int32_t width, float data_range, float* ssim, float* ssim_map, void* tmp,
                               size_t tmp_bytes, void* stream) {
  size_t need = 0;
  if (!x || !y || !ssim || !tmp || !(data_range > 0.0f)) return GS_ERR_INVALID_ARG;
  if (gs_metrics_tmp_size(images, channels, height, width, &need) != GS_OK) return GS_ERR_INVALID_ARG;
  if (tmp_bytes < need) return GS_ERR_WORKSPACE_TOO_SMALL;
  // normalised Gaussian taps, computed in FP64 and rounded once
  Window win;
  double w[kSsimTaps], sum = 0.0;
  for (int a = 0; a < kSsimTaps; ++a) {
    const double r = a - kSsimRad;
    w[a] = exp(-(r * r) / (2.0 * 1.5 * 1.5));
    sum += w[a];
  }
  for (int a = 0; a < kSsimTaps; ++a) win.w[a] = static_cast<float>(w[a] / sum);
  const float c1 = static_cast<float>((0.01 * data_range) * (0.01 * data_range));
  const float c2 = static_cast<float>((0.03 * data_range) * (0.03 * data_range));
  const int tiles_x = (width + kSsimTile - 1) / kSsimTile;
  const int tiles = static_cast<int>(ssim_tiles(height, width));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* part = static_cast<float*>(tmp);
  launch(k_ssim, dim3(tiles, images * channels), kMetThreads, 0, s, x, y, height, width, tiles_x, tiles, win, c1, c2,
         ssim_map, part);
  launch(k_mean_final, images, kMetThreads, 0, s, part, static_cast<int64_t>(channels) * tiles,
         static_cast<double>(channels) * height * width, ssim);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
