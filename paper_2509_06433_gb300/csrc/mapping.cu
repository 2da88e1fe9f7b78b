// The mapping loop around the rasterizer (Sec. II-B: the mapping optimiser updates the map by
// comparing rendered images with the key-frames): an Adam step of every Gaussian parameter on
// FP32 master values, and the insertion of a key-frame's pixels as new Gaussians.
//
// Adam: one thread per scalar over the 11 + w values of every Gaussian (means 3, log-scales 3,
// quaternion 4, opacity logit 1, colour w: 3, or the spherical-harmonic coefficients), group by
// group, so every access is coalesced. The state holds m and v in the same group layout
// (2 x (11 + w) N floats) and, after them, the step
// count as a float; a one-thread kernel advances the count after the update, so the step can
// be replayed from a CUDA graph.
//
// Key-frame insertion: every stride-th pixel (x and y) whose depth is > near and, when a
// transmittance image of the current map is given, whose transmittance is > t_min becomes one
// Gaussian: its centre back-projected to the depth, isotropic log-scale
// ln(scale_factor * stride * depth / f) (f = (fx + fy) / 2), identity quaternion, opacity logit
// logit0, the pixel's colour. Candidates are counted per block, the counts scanned in one
// block, and the Gaussians written in row-major pixel order (deterministic).
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kAdamThreads = 256;
constexpr int kGroups = 5;

struct AdamArgs {
  float* p[kGroups];
  const float* g[kGroups];
  void* store[kGroups];  // optional reduced-storage copies (nullptr: none)
  int store_dtype[kGroups];
  float lr[kGroups];
  int64_t n[kGroups];    // scalars per group
  int64_t off[kGroups];  // offset of the group in the state's m and v
  float* m;
  float* v;
  const float* step;     // the step count before this update
  float beta1, beta2, eps;
  int64_t total;
};

__device__ __forceinline__ void store_attr(void* p, int64_t i, int dtype, float x) {
  if (dtype == GS_BF16) static_cast<__nv_bfloat16*>(p)[i] = __float2bfloat16_rn(x);
  else if (dtype == GS_F16) static_cast<__half*>(p)[i] = __float2half_rn(x);
  else static_cast<float*>(p)[i] = x;
}

__global__ void __launch_bounds__(kAdamThreads) k_map_adam(AdamArgs a) {
  pdl_begin();
  const float t = *a.step + 1.0f;
  const float c1 = 1.0f - powf(a.beta1, t), c2 = 1.0f - powf(a.beta2, t);
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * kAdamThreads + threadIdx.x; e < a.total;
       e += static_cast<int64_t>(gridDim.x) * kAdamThreads) {
    int k = 0;
#pragma unroll
    for (int q = 1; q < kGroups; ++q) k = e >= a.off[q] ? q : k;
    const int64_t i = e - a.off[k];
    const float g = a.g[k][i];
    const float m = a.beta1 * a.m[e] + (1.0f - a.beta1) * g;
    const float v = a.beta2 * a.v[e] + (1.0f - a.beta2) * g * g;
    a.m[e] = m;
    a.v[e] = v;
    const float p = a.p[k][i] - a.lr[k] * (m / c1) / (sqrtf(v / c2) + a.eps);
    a.p[k][i] = p;
    if (a.store[k]) store_attr(a.store[k], i, a.store_dtype[k], p);
  }
}

__global__ void k_adam_tick(float* step) {
  pdl_begin();
  *step += 1.0f;
}

// ---------------------------------------------------------------- key-frame insertion
constexpr int kKfThreads = 256;

struct KfArgs {
  const gs_camera_t* cam;  // device
  const float* rgb;    // [3, H, W]
  const float* depth;  // [H, W]
  const float* T;      // [H, W] or nullptr
  int W, H, stride, gw, gh;  // gw x gh sample grid
  float near, t_min, scale_factor, logit0;
  uint32_t* block_counts;
  uint32_t* d_count;
  float *means, *log_scales, *quats, *logits, *colours;
  int64_t first, capacity;  // write Gaussians [first, first + count) of arrays holding `capacity`
};

__device__ __forceinline__ bool kf_selected(const KfArgs& a, int s, int& x, int& y, float& d) {
  if (s >= a.gw * a.gh) return false;
  y = (s / a.gw) * a.stride;
  x = (s % a.gw) * a.stride;
  d = a.depth[static_cast<int64_t>(y) * a.W + x];
  if (!(d > a.near)) return false;
  if (a.T && !(a.T[static_cast<int64_t>(y) * a.W + x] > a.t_min)) return false;
  return true;
}

__global__ void __launch_bounds__(kKfThreads) k_kf_count(KfArgs a) {
  pdl_begin();
  int x, y;
  float d;
  const bool sel = kf_selected(a, blockIdx.x * kKfThreads + threadIdx.x, x, y, d);
  const uint32_t c = __syncthreads_count(sel);
  if (threadIdx.x == 0) a.block_counts[blockIdx.x] = c;
}

__global__ void __launch_bounds__(1024) k_kf_scan(KfArgs a, int nblocks) {
  pdl_begin();
  __shared__ uint32_t s_warp[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t carry = 0;
  for (int base = 0; base < nblocks; base += 1024) {
    const int b = base + threadIdx.x;
    const uint32_t c = b < nblocks ? a.block_counts[b] : 0u;
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t wo = 0, tot = 0;
    for (int w = 0; w < 32; ++w) {
      wo += w < warp ? s_warp[w] : 0u;
      tot += s_warp[w];
    }
    __syncthreads();
    if (b < nblocks) a.block_counts[b] = carry + wo + incl - c;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    const int64_t room = a.capacity - a.first;
    *a.d_count = static_cast<uint32_t>(static_cast<int64_t>(carry) < room ? carry : (room > 0 ? room : 0));
  }
}

__global__ void __launch_bounds__(kKfThreads) k_kf_write(KfArgs a) {
  pdl_begin();
  __shared__ uint32_t s_warp[kKfThreads / 32];
  int x = 0, y = 0;
  float d = 0.0f;
  const bool sel = kf_selected(a, blockIdx.x * kKfThreads + threadIdx.x, x, y, d);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t ballot = __ballot_sync(0xffffffffu, sel);
  if (lane == 0) s_warp[warp] = __popc(ballot);
  __syncthreads();
  uint32_t rank = a.block_counts[blockIdx.x];
  for (int w = 0; w < warp; ++w) rank += s_warp[w];
  rank += __popc(ballot & ((1u << lane) - 1u));
  if (!sel || rank >= *a.d_count) return;
  const int64_t o = a.first + rank;
  const gs_camera_t c = *a.cam;
  // camera-space point of the pixel centre at depth d, then world = R^T (p_c - t)
  const float pc[3] = {(static_cast<float>(x) + 0.5f - c.cx) / c.fx * d, (static_cast<float>(y) + 0.5f - c.cy) / c.fy * d,
                       d};
  const float q[3] = {pc[0] - c.t[0], pc[1] - c.t[1], pc[2] - c.t[2]};
#pragma unroll
  for (int j = 0; j < 3; ++j) a.means[3 * o + j] = c.R[j] * q[0] + c.R[3 + j] * q[1] + c.R[6 + j] * q[2];
  const float ls = logf(a.scale_factor * static_cast<float>(a.stride) * d / (0.5f * (c.fx + c.fy)));
#pragma unroll
  for (int j = 0; j < 3; ++j) a.log_scales[3 * o + j] = ls;
  a.quats[4 * o + 0] = 1.0f;
  a.quats[4 * o + 1] = a.quats[4 * o + 2] = a.quats[4 * o + 3] = 0.0f;
  a.logits[o] = a.logit0;
  const int64_t HW = static_cast<int64_t>(a.W) * a.H, pix = static_cast<int64_t>(y) * a.W + x;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) a.colours[3 * o + ch] = a.rgb[ch * HW + pix];
}

int num_sms_dev() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status_t gs_map_adam_step(int64_t N, float* means, float* log_scales, float* quats,
                                        float* opacity_logits, float* rgb, const gs_grads_t* grads, float* state,
                                        const gs_adam_t* hp, const gs_gaussians_t* storage, void* stream) {
  if (N < 0 || !grads || !state || !hp) return GS_ERR_INVALID_ARG;
  if (N > 0 && (!means || !log_scales || !quats || !opacity_logits || !rgb || !grads->means || !grads->log_scales ||
                !grads->quats || !grads->opacity_logits || !grads->rgb))
    return GS_ERR_INVALID_ARG;
  if (!(hp->beta1 >= 0.0f && hp->beta1 < 1.0f) || !(hp->beta2 >= 0.0f && hp->beta2 < 1.0f) || !(hp->eps > 0.0f))
    return GS_ERR_INVALID_ARG;
  AdamArgs a{};
  float* p[kGroups] = {means, log_scales, quats, opacity_logits, rgb};
  const float* g[kGroups] = {grads->means, grads->log_scales, grads->quats, grads->opacity_logits, grads->rgb};
  const float lr[kGroups] = {hp->lr_means, hp->lr_log_scales, hp->lr_quats, hp->lr_opacity, hp->lr_rgb};
  if (hp->color_width < 0) return GS_ERR_INVALID_ARG;
  const int width[kGroups] = {3, 3, 4, 1, hp->color_width > 0 ? hp->color_width : 3};
  const void* st[kGroups] = {storage ? storage->means : nullptr, storage ? storage->log_scales : nullptr,
                             storage ? storage->quats : nullptr, storage ? storage->opacity_logits : nullptr,
                             storage ? storage->rgb : nullptr};
  int64_t off = 0;
  for (int k = 0; k < kGroups; ++k) {
    a.p[k] = p[k];
    a.g[k] = g[k];
    a.lr[k] = lr[k];
    a.n[k] = N * width[k];
    a.off[k] = off;
    off += a.n[k];
    a.store_dtype[k] = storage ? (k == 0 ? storage->means_dtype : storage->dtype) : GS_F32;
    // a storage array that is the master itself needs no copy
    a.store[k] = (st[k] && st[k] != static_cast<const void*>(p[k])) ? const_cast<void*>(st[k]) : nullptr;
  }
  if (storage && (storage->dtype < GS_F32 || storage->dtype > GS_F16 || storage->means_dtype < GS_F32 ||
                  storage->means_dtype > GS_F16))
    return GS_ERR_INVALID_ARG;
  a.total = off;
  a.m = state;
  a.v = state + off;
  a.step = state + 2 * off;
  a.beta1 = hp->beta1;
  a.beta2 = hp->beta2;
  a.eps = hp->eps;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t blocks = (off + kAdamThreads - 1) / kAdamThreads;
  const int64_t cap = static_cast<int64_t>(num_sms_dev()) * 8;
  if (off > 0) launch(k_map_adam, static_cast<unsigned>(blocks < cap ? blocks : cap), kAdamThreads, 0, s, a);
  launch(k_adam_tick, 1, 1, 0, s, state + 2 * off);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

extern "C" gs_status_t gs_map_adam_state_size(int64_t N, int32_t color_width, int64_t* floats) {
  if (N < 0 || color_width < 0 || !floats) return GS_ERR_INVALID_ARG;
  *floats = 2 * (11 + static_cast<int64_t>(color_width > 0 ? color_width : 3)) * N + 1;
  return GS_OK;
}

extern "C" gs_status_t gs_keyframe_tmp_size(int32_t width, int32_t height, int32_t stride, size_t* bytes) {
  if (width < 1 || height < 1 || stride < 1 || !bytes) return GS_ERR_INVALID_ARG;
  const int64_t gw = (width + stride - 1) / stride, gh = (height + stride - 1) / stride;
  *bytes = static_cast<size_t>((gw * gh + kKfThreads - 1) / kKfThreads) * 4 + 256;
  return GS_OK;
}

extern "C" gs_status_t gs_keyframe_insert(const gs_camera_t* d_cam, const float* rgb, const float* depth, const float* T,
                                          int32_t width, int32_t height, int32_t stride, float near_plane, float t_min,
                                          float scale_factor, float logit0, float* means, float* log_scales,
                                          float* quats, float* opacity_logits, float* colours, int64_t first,
                                          int64_t capacity, uint32_t* d_count, void* tmp, size_t tmp_bytes,
                                          void* stream) {
  if (!d_cam || !rgb || !depth || !means || !log_scales || !quats || !opacity_logits || !colours || !d_count || !tmp)
    return GS_ERR_INVALID_ARG;
  if (width < 1 || height < 1 || stride < 1 || first < 0 || capacity < first || !(scale_factor > 0.0f))
    return GS_ERR_INVALID_ARG;
  size_t need = 0;
  gs_keyframe_tmp_size(width, height, stride, &need);
  if (tmp_bytes < need) return GS_ERR_WORKSPACE_TOO_SMALL;
  KfArgs a{};
  a.cam = d_cam;
  a.rgb = rgb;
  a.depth = depth;
  a.T = T;
  a.W = width;
  a.H = height;
  a.stride = stride;
  a.gw = (width + stride - 1) / stride;
  a.gh = (height + stride - 1) / stride;
  a.near = near_plane;
  a.t_min = t_min;
  a.scale_factor = scale_factor;
  a.logit0 = logit0;
  a.block_counts = static_cast<uint32_t*>(tmp);
  a.d_count = d_count;
  a.means = means;
  a.log_scales = log_scales;
  a.quats = quats;
  a.logits = opacity_logits;
  a.colours = colours;
  a.first = first;
  a.capacity = capacity;
  const int nblocks = (a.gw * a.gh + kKfThreads - 1) / kKfThreads;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  launch(k_kf_count, nblocks, kKfThreads, 0, s, a);
  launch(k_kf_scan, 1, 1024, 0, s, a, nblocks);
  launch(k_kf_write, nblocks, kKfThreads, 0, s, a);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
