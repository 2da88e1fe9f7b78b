// C ABI entry points (include/gs.h): argument checks, workspace layout, launches.
#include <nvtx3/nvToolsExt.h>
#include <string.h>

#include "gs_internal.cuh"

namespace gs {

namespace {
constexpr size_t kAlign = 256;
// An NVTX range around each entry point that enqueues work (visible to nsys / ncu timelines;
// a no-op when no tool is attached).
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
};
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
int ceil_log2(int64_t x) {  // smallest b with 2^b >= x (x >= 1)
  int b = 0;
  while ((int64_t{1} << b) < x) ++b;
  return b;
}
}  // namespace

bool make_layout(const gs_config_t* cfg, Layout* L) {
  if (!cfg || !L) return false;
  if (cfg->tile != kTile) return false;
  if (cfg->width < 1 || cfg->width > 16384 || cfg->height < 1 || cfg->height > 16384) return false;
  if (cfg->num_views < 1 || cfg->num_views > 1024) return false;
  if (cfg->num_gaussians < 0 || cfg->num_gaussians > 0x7fffffffLL) return false;
  if (cfg->pair_capacity < 1 || cfg->pair_capacity > (1LL << 30) - 1) return false;
  if (!(cfg->near_plane > 0.0f)) return false;
  memset(L, 0, sizeof(*L));
  L->N = cfg->num_gaussians;
  L->K = cfg->num_views;
  L->KN = L->N * L->K;
  if (L->KN > 0x7fffffffLL) return false;  // item indices k N + g are 31-bit
  L->W = cfg->width;
  L->H = cfg->height;
  L->Tx = (L->W + kTile - 1) / kTile;
  L->Ty = (L->H + kTile - 1) / kTile;
  L->n_tiles = static_cast<int64_t>(L->K) * L->Tx * L->Ty;
  L->tile_bits = ceil_log2(L->n_tiles);
  L->key_bits = 32 + L->tile_bits;
  L->passes = (L->tile_bits + 7) / 8;
  L->cap = cfg->pair_capacity;
  L->near_plane = cfg->near_plane;
  L->lambda_depth = cfg->lambda_depth;
  if (cfg->fwd_px_per_thread < 0 || cfg->fwd_px_per_thread > 4 || cfg->fwd_px_per_thread == 3) return false;
  if (cfg->bwd_px_per_thread < 0 || cfg->bwd_px_per_thread > 4 || cfg->bwd_px_per_thread == 3) return false;
  L->fwd_px = cfg->fwd_px_per_thread;
  L->bwd_px = cfg->bwd_px_per_thread;
  if (cfg->fwd_chunk != 0 && cfg->fwd_chunk != 64 && cfg->fwd_chunk != 128 && cfg->fwd_chunk != 256) return false;
  if (cfg->bwd_chunk != 0 && cfg->bwd_chunk != 32 && cfg->bwd_chunk != 64 && cfg->bwd_chunk != 128) return false;
  L->fwd_chunk = cfg->fwd_chunk;
  L->bwd_chunk = cfg->bwd_chunk;
  if (cfg->raster_blocks_per_sm < 0 || cfg->raster_blocks_per_sm > 32) return false;
  L->raster_bps = cfg->raster_blocks_per_sm;
  if (cfg->color_mode != GS_COLOR_RGB && cfg->color_mode != GS_COLOR_SH) return false;
  if (cfg->color_mode == GS_COLOR_SH && (cfg->sh_degree < 0 || cfg->sh_degree > 3)) return false;
  L->color_mode = cfg->color_mode;
  L->sh_degree = cfg->color_mode == GS_COLOR_SH ? cfg->sh_degree : 0;
  L->sh_coeffs = (L->sh_degree + 1) * (L->sh_degree + 1);
  // colours depend on the view only through spherical harmonics of degree >= 1
  L->color_stride = (cfg->color_mode == GS_COLOR_SH && cfg->sh_degree > 0) ? L->N : 0;
  L->n_proj_blocks = L->KN > 0 ? (L->KN + kProjBlock - 1) / kProjBlock : 1;
  L->proj_items = kProjThreads;
  while (L->proj_items < kProjItemsMax && L->KN >= static_cast<int64_t>(2 * L->proj_items) * kProjTargetBlocks)
    L->proj_items *= 2;
  L->n_proj_groups = L->KN > 0 ? (L->KN + L->proj_items - 1) / L->proj_items : 1;
  L->item_sort_items = pick_sort_items(L->KN);
  L->pair_sort_items = pick_sort_items(L->cap);
  L->max_sort_tiles = sort_tiles(L->cap, L->pair_sort_items);
  L->max_item_tiles = sort_tiles(L->KN, L->item_sort_items);
  L->n_pose_blocks = L->N > 0 ? (L->N + kPoseBlock - 1) / kPoseBlock : 1;
  L->n_item_chunks = L->KN > 0 ? (L->KN + kPoseBlock - 1) / kPoseBlock : 1;
  const int64_t pixels = static_cast<int64_t>(L->K) * L->W * L->H;
  L->n_loss_blocks = (pixels + 255) / 256 < 1024 ? (pixels + 255) / 256 : 1024;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at_ = o;
    o = align_up(o + bytes);
    return at_;
  };
  const size_t KN = static_cast<size_t>(L->KN), N = static_cast<size_t>(L->N), cap = static_cast<size_t>(L->cap);
  L->status = take(sizeof(Status));
  L->proj_uv = take(KN * 16);
  L->proj_conic = take(KN * 16);
  L->proj_tiles = take(KN * 16);
  L->proj_depth_key = take(KN * 4);
  L->proj_radius = take(KN * 4);
  L->proj_rows = take(KN * 8);
  L->row_table = take(cap * 8);
  L->pair_valid = take((cap + 31) / 32 * 4);
  L->tile_loss = take(static_cast<size_t>(L->n_tiles) * 4);
  L->color_opacity = take((L->color_stride ? KN : N) * 16);
  L->block_sums = take(static_cast<size_t>(L->n_proj_blocks) * 4);
  L->block_offsets = take(static_cast<size_t>(L->n_proj_blocks) * 8);
  L->keys[0] = take(cap * 8);
  L->keys[1] = take(cap * 8);
  L->vals[0] = take(cap * 4);
  L->vals[1] = take(cap * 4);
  L->ranges = take(static_cast<size_t>(L->n_tiles) * 8);
  L->hist = take(kMaxSortPasses * 256 * 4);
  L->sort_status = take(static_cast<size_t>(L->passes) * L->max_sort_tiles * 256 * 4);
  L->pair_grads = take(cap * kPairGradStride * 4);
  L->pose_partials = take((static_cast<size_t>(L->n_item_chunks) + L->K) * 6 * 4);
  L->loss_partials = take(static_cast<size_t>(L->n_loss_blocks) * 4);
  L->item_keys[0] = take(KN * 4);
  L->item_keys[1] = take(KN * 4);
  L->item_vals[0] = take(KN * 4);
  L->item_vals[1] = take(KN * 4);
  L->item_hist = take(4 * 256 * 4);
  L->item_status = take(static_cast<size_t>(4) * L->max_item_tiles * 256 * 4);
  L->sorted_counts = take(static_cast<size_t>(L->n_proj_blocks) * kProjBlock * 4);
  L->item_offsets = take((KN + 1) * 4);
  L->item_rect = take(KN * 16);
  L->item_kg = take(KN * 8);
  L->tile_diff = take(static_cast<size_t>(L->K) * (L->Tx + 1) * (L->Ty + 1) * 4);
  L->n_emit_blocks = (L->cap + kEmitPairs - 1) / kEmitPairs;
  L->emit_first = take(static_cast<size_t>(L->n_emit_blocks) * 4);
  L->emit_last = take(static_cast<size_t>(L->n_emit_blocks) * 4);
  L->live_mask = take((KN + 31) / 32 * 4);
  L->live_wpre = take((KN + 31) / 32 * 4);
  L->live_kg = take(KN * 4);
  L->live_count = take(KN * 4);
  L->live_rows = take(KN * 8);
  L->live_off = take(KN * 4);
  L->live_blocks = take(static_cast<size_t>(L->n_proj_groups) * 4);
  L->live_bases = take(static_cast<size_t>(L->n_proj_groups) * 4);
  L->view_lb = take(static_cast<size_t>(L->K) * 8);
  L->item_partials = take(KN * 16 * 4);
  L->total = o;
  return true;
}

namespace {

gs_status_t check(const gs_config_t* cfg, const void* ws, size_t ws_bytes, Layout* L) {
  if (!make_layout(cfg, L)) return GS_ERR_INVALID_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return GS_ERR_INVALID_ARG;
  if (ws_bytes < L->total) return GS_ERR_WORKSPACE_TOO_SMALL;
  return GS_OK;
}

bool gauss_ptrs(const gs_gaussians_t* g, int64_t N, GaussPtrs* out) {
  if (!g) return false;
  if (N > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->rgb)) return false;
  if (g->dtype < GS_F32 || g->dtype > GS_F16 || g->means_dtype < GS_F32 || g->means_dtype > GS_F16) return false;
  *out = GaussPtrs{g->means, g->log_scales, g->quats, g->opacity_logits, g->rgb, g->dtype, g->means_dtype};
  return true;
}

gs_status_t launched(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ERR_CUDA; }

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

gs_status_t gs_workspace_size(const gs_config_t* cfg, size_t* bytes) {
  Layout L;
  if (!bytes || !make_layout(cfg, &L)) return GS_ERR_INVALID_ARG;
  *bytes = L.total;
  return GS_OK;
}

gs_status_t gs_workspace_layout(const gs_config_t* cfg, gs_ws_layout_t* out) {
  Layout L;
  if (!out || !make_layout(cfg, &L)) return GS_ERR_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  out->total = L.total;
  out->status = L.status;
  out->proj_uv = L.proj_uv;
  out->proj_conic = L.proj_conic;
  out->proj_tiles = L.proj_tiles;
  out->proj_depth_key = L.proj_depth_key;
  out->proj_radius = L.proj_radius;
  out->color_opacity = L.color_opacity;
  out->keys_sorted = L.keys[L.passes & 1];
  out->vals_sorted = L.vals[L.passes & 1];
  out->ranges = L.ranges;
  out->pair_grads = L.pair_grads;
  out->pair_valid = L.pair_valid;
  out->sort_passes = L.passes;
  out->bin_sort_launches = bin_sort_launch_count(L);
  out->live_mask = L.live_mask;
  out->live_off = L.live_off;
  out->project_launches = 2;
  out->project_bwd_launches = 3;
  out->tiles_x = L.Tx;
  out->tiles_y = L.Ty;
  return GS_OK;
}

gs_status_t gs_read_status(const gs_config_t* cfg, const void* ws, size_t ws_bytes, uint32_t* err_word,
                           int64_t* num_pairs, int64_t* evals, void* stream) {
  Layout L;
  gs_status_t st = check(cfg, ws, ws_bytes, &L);
  if (st != GS_OK) return st;
  Status h;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&h, at<Status>(ws, L.status), sizeof(Status), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return GS_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GS_ERR_CUDA;
  if (err_word) *err_word = h.err;
  if (num_pairs) *num_pairs = static_cast<int64_t>(h.total_pairs);
  if (evals) *evals = static_cast<int64_t>(h.evals);
  if (h.err & GS_DEVERR_BOUNDS) return GS_ERR_INDEX_CHECK;
  if (h.err & GS_DEVERR_PAIR_OVERFLOW) return GS_ERR_CAPACITY_OVERFLOW;
  if (h.err & GS_DEVERR_TIMEOUT) return GS_ERR_DEVICE_TIMEOUT;
  if (h.err & GS_DEVERR_NONFINITE) return GS_ERR_NONFINITE;
  return GS_OK;
}

gs_status_t gs_project(const gs_config_t* cfg, const gs_gaussians_t* gaussians, const gs_camera_t* d_cams, void* ws,
                       size_t ws_bytes, void* stream) {
  const TraceRange trace_("gs_project");
  Layout L;
  gs_status_t st = check(cfg, ws, ws_bytes, &L);
  if (st != GS_OK) return st;
  GaussPtrs g;
  if (!d_cams || !gauss_ptrs(gaussians, L.N, &g)) return GS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(at<Status>(ws, L.status), 0, sizeof(Status), s) != cudaSuccess) return GS_ERR_CUDA;
  if (cudaMemsetAsync(at<uint32_t>(ws, L.item_hist), 0, 4 * 256 * 4, s) != cudaSuccess) return GS_ERR_CUDA;
  if (cudaMemsetAsync(at<int32_t>(ws, L.tile_diff), 0, static_cast<size_t>(L.K) * (L.Tx + 1) * (L.Ty + 1) * 4, s) !=
      cudaSuccess)
    return GS_ERR_CUDA;
  return launched(launch_project(L, g, d_cams, ws, s));
}

gs_status_t gs_bin_sort(const gs_config_t* cfg, void* ws, size_t ws_bytes, void* stream) {
  const TraceRange trace_("gs_bin_sort");
  Layout L;
  gs_status_t st = check(cfg, ws, ws_bytes, &L);
  if (st != GS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_item_sort(L, ws, s);
  if (e == cudaSuccess) e = launch_bin(L, ws, s);
  if (e == cudaSuccess) e = launch_sort_passes(L, ws, s);
  return launched(e);
}

gs_status_t gs_raster_fwd(const gs_config_t* cfg, void* ws, size_t ws_bytes, float* rgb, float* depth,
                          float* T_final, int32_t* last, void* stream) {
  const TraceRange trace_("gs_raster_fwd");
  Layout L;
  gs_status_t st = check(cfg, ws, ws_bytes, &L);
  if (st != GS_OK) return st;
  return launched(launch_raster_fwd(L, ws, rgb, depth, T_final, last, false, nullptr, static_cast<cudaStream_t>(stream)));
}

gs_status_t gs_raster_fwd_stats(const gs_config_t* cfg, void* ws, size_t ws_bytes, float* rgb, float* depth,
                                float* T_final, int32_t* last, void* stream) {
  const TraceRange trace_("gs_raster_fwd_stats");
  Layout L;
  gs_status_t st = check(cfg, ws, ws_bytes, &L);
  if (st != GS_OK) return st;
  return launched(launch_raster_fwd(L, ws, rgb, depth, T_final, last, true, nullptr, static_cast<cudaStream_t>(stream)));
}

gs_status_t gs_raster_fwd_occluded(const gs_config_t* cfg, void* ws, size_t ws_bytes, float* rgb, float* depth,
                                   float* T_final, int32_t* last, const float* ext_depth, const float* ext_rgb,
                                   void* stream) {
  const TraceRange trace_("gs_raster_fwd_occluded");
  Layout L;
  gs_status_t st = check(cfg, ws, ws_bytes, &L);
  if (st != GS_OK) return st;
  if (!ext_depth) return GS_ERR_INVALID_ARG;
  return launched(launch_raster_fwd(L, ws, rgb, depth, T_final, last, false, nullptr, static_cast<cudaStream_t>(stream),
                                    ext_depth, ext_rgb));
}

gs_status_t gs_raster_fwd_l1(const gs_config_t* cfg, void* ws, size_t ws_bytes, float* rgb, float* depth,
                             float* T_final, int32_t* last, const float* rgb_target, const float* depth_target,
                             float* dL_drgb, float* dL_ddepth, float* d_loss, void* stream) {
  const TraceRange trace_("gs_raster_fwd_l1");
  Layout L;
  gs_status_t st = check(cfg, ws, ws_bytes, &L);
  if (st != GS_OK) return st;
  if (!rgb || !depth || !rgb_target || !depth_target || !dL_drgb || !dL_ddepth || !d_loss) return GS_ERR_INVALID_ARG;
  const FusedLossArgs F{rgb_target, depth_target, dL_drgb, dL_ddepth, d_loss};
  return launched(launch_raster_fwd(L, ws, rgb, depth, T_final, last, false, &F, static_cast<cudaStream_t>(stream)));
}

gs_status_t gs_raster_fwd_l1_bwd(const gs_config_t* cfg, void* ws, size_t ws_bytes, float* rgb, float* depth,
                                 float* T_final, int32_t* last, const float* rgb_target, const float* depth_target,
                                 float* dL_drgb, float* dL_ddepth, float* d_loss, void* stream) {
  const TraceRange trace_("gs_raster_fwd_l1_bwd");
  Layout L;
  gs_status_t st = check(cfg, ws, ws_bytes, &L);
  if (st != GS_OK) return st;
  if (!rgb || !depth || !rgb_target || !depth_target || !dL_drgb || !dL_ddepth || !d_loss) return GS_ERR_INVALID_ARG;
  const FusedLossArgs F{rgb_target, depth_target, dL_drgb, dL_ddepth, d_loss};
  return launched(launch_raster_fwd_l1_bwd(L, ws, rgb, depth, T_final, last, F, static_cast<cudaStream_t>(stream)));
}

gs_status_t gs_loss_l1(const gs_config_t* cfg, const float* rgb, const float* depth, const float* rgb_target,
                       const float* depth_target, float* dL_drgb, float* dL_ddepth, float* d_loss, void* ws,
                       size_t ws_bytes, void* stream) {
  const TraceRange trace_("gs_loss_l1");
  Layout L;
  gs_status_t st = check(cfg, ws, ws_bytes, &L);
  if (st != GS_OK) return st;
  if (!rgb || !depth || !rgb_target || !depth_target || !dL_drgb || !dL_ddepth || !d_loss) return GS_ERR_INVALID_ARG;
  return launched(launch_loss(L, rgb, depth, rgb_target, depth_target, dL_drgb, dL_ddepth, d_loss, ws,
                              static_cast<cudaStream_t>(stream)));
}

gs_status_t gs_raster_bwd(const gs_config_t* cfg, void* ws, size_t ws_bytes, const float* rgb, const float* depth,
                          const float* T_final, const int32_t* last, const float* dL_drgb, const float* dL_ddepth,
                          const float* dL_dT, void* stream) {
  const TraceRange trace_("gs_raster_bwd");
  Layout L;
  gs_status_t st = check(cfg, ws, ws_bytes, &L);
  if (st != GS_OK) return st;
  if (!rgb || !depth || !last || !dL_drgb || !dL_ddepth || (dL_dT && !T_final)) return GS_ERR_INVALID_ARG;
  return launched(launch_raster_bwd(L, ws, rgb, depth, T_final, last, dL_drgb, dL_ddepth, dL_dT,
                                    static_cast<cudaStream_t>(stream)));
}

gs_status_t gs_project_bwd(const gs_config_t* cfg, const gs_gaussians_t* gaussians, const gs_camera_t* d_cams,
                           void* ws, size_t ws_bytes, const gs_grads_t* grads, void* stream) {
  const TraceRange trace_("gs_project_bwd");
  Layout L;
  gs_status_t st = check(cfg, ws, ws_bytes, &L);
  if (st != GS_OK) return st;
  GaussPtrs g;
  if (!d_cams || !grads || !gauss_ptrs(gaussians, L.N, &g)) return GS_ERR_INVALID_ARG;
  return launched(launch_project_bwd(L, g, d_cams, ws, *grads, static_cast<cudaStream_t>(stream)));
}

gs_status_t gs_screen_grads(const gs_config_t* cfg, const void* ws, size_t ws_bytes, float* d_mean2d, float* d_conic,
                            float* d_depth, float* d_opacity, float* d_rgb, void* stream) {
  const TraceRange trace_("gs_screen_grads");
  Layout L;
  gs_status_t st = check(cfg, ws, ws_bytes, &L);
  if (st != GS_OK) return st;
  return launched(launch_screen_grads(L, ws, d_mean2d, d_conic, d_depth, d_opacity, d_rgb,
                                      static_cast<cudaStream_t>(stream)));
}

// ---------------------------------------------------------------- sort primitive
namespace {
struct SortTmp {
  size_t keys, vals, hist, ctr, err, status, total;
  int64_t max_tiles;
  int items;
};
SortTmp sort_tmp_layout(int64_t n, int items) {
  SortTmp t{};
  t.items = items;
  t.max_tiles = sort_tiles(n, items);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at_ = o;
    o = align_up(o + bytes);
    return at_;
  };
  t.keys = take(static_cast<size_t>(n) * 8);
  t.vals = take(static_cast<size_t>(n) * 4);
  t.hist = take(kMaxSortPasses * 256 * 4);
  t.ctr = take(kMaxSortPasses * 4);
  t.err = take(4);
  t.status = take(static_cast<size_t>(kMaxSortPasses) * t.max_tiles * 256 * 4);
  t.total = o;
  return t;
}
}  // namespace

gs_status_t gs_sort_pairs_tmp_size(int64_t n, size_t* bytes) {
  if (!bytes || n < 0 || n > (1LL << 30) - 1) return GS_ERR_INVALID_ARG;
  *bytes = sort_tmp_layout(n, pick_sort_items(n)).total;
  return GS_OK;
}

gs_status_t gs_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int32_t key_bits, void* tmp, size_t tmp_bytes,
                          uint32_t* d_err_word, void* stream) {
  const TraceRange trace_("gs_sort_pairs");
  if (n < 0 || n > (1LL << 30) - 1 || key_bits < 1 || key_bits > 64) return GS_ERR_INVALID_ARG;
  if (n == 0) return GS_OK;
  if (!keys || !vals || !tmp || (reinterpret_cast<uintptr_t>(tmp) % kAlign) != 0) return GS_ERR_INVALID_ARG;
  const SortTmp t = sort_tmp_layout(n, pick_sort_items(n));
  if (tmp_bytes < t.total) return GS_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SortArgs a{};
  a.items = t.items;
  a.keys[0] = keys;
  a.vals[0] = vals;
  a.keys[1] = at<uint64_t>(tmp, t.keys);
  a.vals[1] = at<uint32_t>(tmp, t.vals);
  a.n_dev = nullptr;
  a.n_host = n;
  a.hist = at<uint32_t>(tmp, t.hist);
  a.tile_status = at<uint32_t>(tmp, t.status);
  a.tile_ctr = at<uint32_t>(tmp, t.ctr);
  a.err = d_err_word ? d_err_word : at<uint32_t>(tmp, t.err);
  a.max_tiles = t.max_tiles;
  a.passes = (key_bits + 7) / 8;
  a.key_bits = key_bits;
  cudaError_t e = launch_sort_prepare(a, s);
  if (e == cudaSuccess) e = launch_onesweep(a, s);
  if (e == cudaSuccess && (a.passes & 1)) {
    e = cudaMemcpyAsync(keys, a.keys[1], static_cast<size_t>(n) * 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vals, a.vals[1], static_cast<size_t>(n) * 4, cudaMemcpyDeviceToDevice, s);
  }
  return launched(e);
}

}  // extern "C"

// Diagnostic: one 8-bit pass of the pair sort with tile 0 withheld. Nothing ever publishes
// tile 0's look-back status, so tile 1's bounded wait must run out and set
// GS_DEVERR_TIMEOUT in d_err_word. The keys come out unsorted (but every write stays in
// bounds); the call exists to exercise the device-side error path.
extern "C" gs_status_t gs_sort_diag_withheld_tile(uint64_t* keys, uint32_t* vals, int64_t n, void* tmp, size_t tmp_bytes,
                                                  uint32_t* d_err_word, void* stream) {
  if (n < 2 * gs::kSortTileKeys || n > (1LL << 30) - 1 || !keys || !vals || !tmp || !d_err_word)
    return GS_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(tmp) % 256) != 0) return GS_ERR_INVALID_ARG;
  const SortTmp t = sort_tmp_layout(n, gs::kSortItems);
  if (tmp_bytes < t.total) return GS_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  gs::SortArgs a{};
  a.items = t.items;
  a.keys[0] = keys;
  a.vals[0] = vals;
  a.keys[1] = gs::at<uint64_t>(tmp, t.keys);
  a.vals[1] = gs::at<uint32_t>(tmp, t.vals);
  a.n_host = n;
  a.hist = gs::at<uint32_t>(tmp, t.hist);
  a.tile_status = gs::at<uint32_t>(tmp, t.status);
  a.tile_ctr = gs::at<uint32_t>(tmp, t.ctr);
  a.err = d_err_word;
  a.max_tiles = t.max_tiles;
  a.passes = 1;
  a.key_bits = 8;
  a.first_tile = 1;
  cudaError_t e = gs::launch_sort_prepare(a, s);
  if (e == cudaSuccess) e = gs::launch_onesweep(a, s);
  return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
