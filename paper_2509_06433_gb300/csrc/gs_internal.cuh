// Internal declarations of the sm_103a rasterizer library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/gs.h"

namespace gs {

constexpr int kTile = 16;             // tile side (pixels)
constexpr int kTilePixels = kTile * kTile;
constexpr int kProjBlock = 256;       // (view, Gaussian) items per scan chunk of the binning
constexpr int kProjItemsMax = 2048;   // (view, Gaussian) items per projection block: 256 to
                                      // this, a power of two, so that there are >= kProjTargetBlocks
constexpr int kProjTargetBlocks = 1216;
constexpr int kProjThreads = 256;     // threads of a projection block
constexpr int kEmitPairs = 1024;      // pairs emitted per emission block
constexpr int kProjGridCells = 6144;  // largest (Tx+1)(Ty+1) difference grid kept in shared memory
constexpr int kSortThreads = 256;     // onesweep block
constexpr int kSortItems = 15;        // keys per thread per onesweep tile (default; 8 also built)
constexpr int kSortTileKeys = kSortThreads * kSortItems;
constexpr int kMaxSortPasses = 8;
constexpr int kPairGradStride = 12;   // floats per pair gradient record (10 used)
constexpr int kPoseBlock = 256;       // Gaussians / live items per projection-backward block
constexpr uint32_t kSpinLimit = 1u << 21;  // bounded decoupled look-back (about a second of polling)
constexpr int kDefaultFwdPx = 2;      // pixels per thread of the compositing kernels when
constexpr int kDefaultBwdPx = 2;      // gs_config_t leaves the choice to the library

// Workspace status block (first 256 bytes of the workspace).
struct Status {
  uint32_t err;
  uint32_t num_pairs;       // min(total pairs, capacity)
  uint64_t total_pairs;     // unclamped
  uint64_t evals;           // Gaussian-pixel evaluations of the last forward raster
  uint32_t tile_ctr[kMaxSortPasses];  // onesweep dynamic tile counters: [0,4) item sort, [4,8) pair sort
  uint64_t composited;      // evaluations of the last forward raster that blended a splat
  uint32_t row_ctr;         // entries of the row-span table handed out by the projection
  uint32_t loss_ctr;        // blocks of the loss-fused forward done (reset by the last one)
  uint32_t n_live;          // live items: (view, Gaussian) items that emit at least one pair
  uint32_t view_ctr;        // tile-scan blocks started (one per view)
  uint32_t proj_done;       // projection blocks finished (the last one scans their live counts)
  uint32_t grad_chunk_ctr;  // chunks of live items taken by the backward projection's blocks
};
static_assert(sizeof(Status) <= 256, "status block");

// Everything a kernel needs to find its buffers; built on the host from gs_config_t.
struct Layout {
  int64_t N, KN, cap;
  int K, W, H, Tx, Ty;
  int64_t n_tiles;          // K * Tx * Ty
  int tile_bits, key_bits;
  int passes;               // pair-sort passes over the tile bits: ceil(tile_bits / 8)
  int item_sort_items, pair_sort_items;  // keys per thread of the onesweep tiles of the two sorts
  int64_t max_item_tiles;   // onesweep tiles of the per-item depth sort
  float near_plane, lambda_depth;
  int fwd_px, bwd_px;       // pixels per thread of the compositing kernels (0 = default)
  int fwd_chunk, bwd_chunk; // splats staged per chunk of the compositing kernels (0 = default)
  int raster_bps;           // cap on resident compositing blocks per SM (0 = none)
  int color_mode, sh_degree, sh_coeffs;  // gs_color_mode_t; SH degree and (degree + 1)^2
  int64_t color_stride;     // index of (view k, Gaussian g) in color_opacity = k * color_stride + g
  int64_t n_proj_blocks;    // ceil(KN / kProjBlock)
  int64_t n_proj_groups;    // ceil(KN / proj_items): projection blocks
  int proj_items;           // items per projection block
  int64_t max_sort_tiles;   // onesweep tiles of the pair sort at capacity
  int64_t n_pose_blocks;    // ceil(N / kPoseBlock)
  int64_t n_item_chunks;    // ceil(KN / kPoseBlock): chunks of live items of the projection backward
  int64_t n_loss_blocks;
  // byte offsets into the workspace
  size_t status, proj_uv, proj_conic, proj_tiles, proj_depth_key, proj_radius, color_opacity, block_sums,
      block_offsets, keys[2], vals[2], ranges, hist, sort_status, pair_grads, pose_partials, loss_partials;
  // per-item depth sort (u32 depth key, u32 item index), its histograms and look-back status,
  // and the tiles touched by each item in depth order
  size_t item_keys[2], item_vals[2], item_hist, item_status, sorted_counts;
  // in depth order: exclusive pair offset of each item (KN + 1 entries), its row-span
  // table entries (int4: first entry, number of entries, -, -), its (view, Gaussian id)
  size_t item_offsets, item_rect, item_kg;
  // row-span table: per live item, its rows from the first to the last non-empty one, each an
  // int2 (pairs of the item in earlier rows, first column | row << 16); proj_rows: per live item
  // (first entry, number of entries). Entries are handed out by an atomic counter; at most
  // pair_capacity of them (more is reported as a pair overflow).
  size_t row_table, proj_rows;
  // one bit per pair slot: set by gs_raster_bwd for every record it writes (pairs in front of
  // every pixel's last contributor of their tile); the other records are never written, their
  // gradient is zero. Cleared by the emission.
  size_t pair_valid;
  size_t tile_loss;         // float [n_tiles]: per-tile loss partials of the loss-fused forward
  // per view a (Ty+1) x (Tx+1) grid: +1 / -1 at the first / one-past-last tile of every
  // emitted row span; its row-wise prefix sum is the number of pairs of each tile
  size_t tile_diff;
  int64_t n_emit_blocks;    // ceil(cap / kEmitPairs)
  size_t emit_first, emit_last;  // u32 [n_emit_blocks]: items holding each emission block's first / last pair
  // Live items (those that emit at least one pair) and their compaction. Only live items get
  // projection records (proj_uv, proj_conic, proj_tiles, proj_depth_key, proj_radius, proj_rows);
  // the others are marked dead and nothing reads their records. A live item's position among
  // the live items (in increasing k N + g order) is its rank in live_mask: live_wpre[i / 32] +
  // the set bits of word i / 32 below bit i & 31 (live_rank).
  //   live_mask  u32 [ceil(KN / 32)]: bit (i & 31) of word i / 32 set when item i = k N + g is live
  //   live_wpre  u32 [ceil(KN / 32)]: live items before word i / 32
  //   live_kg    u32 [KN]: the live items in increasing k N + g order (valid prefix n_live)
  //   live_count u32 [KN]: tiles emitted by each of them
  //   live_rows  uint2 [KN]: their row-span table entries (first entry, number of entries)
  //   live_off   u32 [KN]: their first pair index (emission order), clamped to the capacity
  //   live_blocks, live_bases  u32 [n_proj_groups]: live items of each projection block, and
  //              the block's first position among all live items (scanned by the last block)
  //   view_lb    u64 [K]: look-back status of the per-view pair totals (tile scan)
  //   item_partials float [KN][16]: the projection backward's per-live-item partial gradients
  size_t live_mask, live_wpre, live_kg, live_count, live_rows, live_off, live_blocks, live_bases, view_lb,
      item_partials;
  size_t total;
};

// Decoupled look-back over a sequence of blocks numbered in their start order (Merrill &
// Garland, "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016), on 64-bit
// status words: the top two bits flag an aggregate (1) or an inclusive prefix (2), the low 62
// bits hold the value; 0 = not published yet. Called by all 32 lanes of one warp of block
// `id`, which first publishes the block's aggregate; the lanes then read kLbWindows * 32
// predecessors per round (independent loads), consume the aggregates in front of the nearest
// inclusive prefix (or in front of the nearest unpublished block, which is read again next
// round), and return to every lane the sum of the
// aggregates of blocks [0, id), after publishing the block's inclusive prefix. The wait for an
// unpublished predecessor is bounded: after kSpinLimit polls without progress it sets
// GS_DEVERR_TIMEOUT in *err and returns what it has.
constexpr uint64_t kLbAggregate = 1ull << 62;
constexpr uint64_t kLbPrefix = 2ull << 62;
constexpr uint64_t kLbValue = (1ull << 62) - 1;
__device__ __forceinline__ uint64_t lb_load(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void lb_store(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
constexpr int kLbWindows = 8;  // 32-block windows read per round (loads in flight together)
__device__ __forceinline__ uint64_t lb_exclusive_warp(uint64_t* status, uint32_t id, uint64_t aggregate,
                                                      uint32_t* err) {
  const int lane = threadIdx.x & 31;
  if (id == 0) {
    if (lane == 0) lb_store(&status[0], kLbPrefix | aggregate);
    return 0;
  }
  if (lane == 0) lb_store(&status[id], kLbAggregate | aggregate);
  uint64_t excl = 0;
  uint32_t spins = 0;
  int64_t j = static_cast<int64_t>(id) - 1;  // window q, lane l: block j - 32 q - l
  bool done = false;
  while (!done) {
    uint64_t v[kLbWindows];
#pragma unroll
    for (int q = 0; q < kLbWindows; ++q) {
      const int64_t jj = j - 32 * q - lane;
      v[q] = jj >= 0 ? lb_load(&status[jj]) : kLbPrefix;  // before block 0: a zero prefix
    }
    int64_t consumed = 0;
#pragma unroll
    for (int q = 0; q < kLbWindows; ++q) {
      if (done) break;
      const uint64_t f = v[q] & ~kLbValue;
      const uint32_t pref = __ballot_sync(0xffffffffu, f == kLbPrefix);
      const uint32_t blocked = __ballot_sync(0xffffffffu, f == 0);
      const int p = pref ? __ffs(pref) - 1 : 32, b = blocked ? __ffs(blocked) - 1 : 32;
      if (p < b) {  // every block in front of the nearest prefix has published: done
        excl += warp_sum_u64(lane <= p ? (v[q] & kLbValue) : 0);
        done = true;
        break;
      }
      excl += warp_sum_u64(lane < b ? (v[q] & kLbValue) : 0);  // the aggregates in front of the gap
      consumed += b;
      if (b < 32) break;  // an unpublished block: read again from it
    }
    if (done) break;
    j -= consumed;
    if (consumed == 0 && ++spins > kSpinLimit) {
      if (lane == 0) atomicOr(err, GS_DEVERR_TIMEOUT);
      break;
    }
  }
  if (lane == 0) lb_store(&status[id], kLbPrefix | (excl + aggregate));
  return excl;
}

// Whether item kg is live (emits pairs); its projection records exist only then.
__device__ __forceinline__ bool item_live(const uint32_t* live_mask, int64_t kg) {
  return (live_mask[kg >> 5] >> (kg & 31)) & 1u;
}
// Position of live item kg among the live items.
__device__ __forceinline__ uint32_t live_rank(const uint32_t* live_mask, const uint32_t* live_wpre, int64_t kg) {
  return live_wpre[kg >> 5] + __popc(live_mask[kg >> 5] & ((1u << (kg & 31)) - 1u));
}

bool make_layout(const gs_config_t* cfg, Layout* L);

template <class T>
__host__ __device__ inline T* at(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<uint8_t*>(ws) + off);
}
template <class T>
__host__ __device__ inline const T* at(const void* ws, size_t off) {
  return reinterpret_cast<const T*>(static_cast<const uint8_t*>(ws) + off);
}

struct GaussPtrs {
  const void* means;
  const void* log_scales;
  const void* quats;
  const void* logits;
  const void* rgb;
  int dtype, means_dtype;
};

// Debug builds (-DGS_DEBUG) check the data-dependent indices of gathers and scatters: a failed
// check sets GS_DEVERR_BOUNDS in the error word and the access is skipped (no trap). Release
// builds compile the checks away.
#ifdef GS_DEBUG
#define GS_INDEX_OK(cond, err) ((cond) ? true : (atomicOr((err), GS_DEVERR_BOUNDS), false))
#else
#define GS_INDEX_OK(cond, err) true
#endif

// ---------------------------------------------------------------------------- launches
// Programmatic dependent launch: every kernel of the library begins with pdl_begin(), which
// waits until the preceding grid of the stream has completed (its writes are then visible)
// and lets the following grid start launching. Kernels are launched with the programmatic
// stream-serialization attribute, so the launch latency of each kernel overlaps the tail of
// the previous one. Outside such launches the two instructions are no-ops.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// For the long compositing kernels: wait at entry, but let the following grid launch only
// once this block's main loop is done (pdl_trigger), so its blocks do not sit on the SMs for
// the whole kernel.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Dynamic shared memory that caps `kernel` at `bps` resident blocks per multiprocessor (0: no
// cap, none added): the multiprocessor's shared memory divided by bps, less the kernel's static
// shared memory and the per-block reserve, rounded down to 128 bytes (0 when the cap is above
// what fits anyway). Raises the kernel's dynamic shared memory limit when the padding needs it.
template <typename... KArgs>
inline size_t cap_smem(void (*kernel)(KArgs...), int bps) {
  if (bps <= 0) return 0;
  int dev = 0, per_sm = 0, reserve = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return 0;
  long pad = static_cast<long>(per_sm) / bps - static_cast<long>(fa.sharedSizeBytes) - reserve;
  const long room = static_cast<long>(optin) - static_cast<long>(fa.sharedSizeBytes);
  pad = (pad < room ? pad : room) / 128 * 128;
  if (pad <= 0) return 0;
  if (pad > fa.maxDynamicSharedSizeBytes &&
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(pad)) != cudaSuccess)
    return 0;
  return static_cast<size_t>(pad);
}

// ---------------------------------------------------------------------------- device helpers
__device__ __forceinline__ float load_attr(const void* p, int64_t i, int dtype) {
  if (dtype == GS_F32) return static_cast<const float*>(p)[i];
  if (dtype == GS_BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
  return __half2float(static_cast<const __half*>(p)[i]);
}

// ---------------------------------------------------------------------------- pair culling
// The widened ellipse of a projected Gaussian inside which its opacity can reach 1/255, as
// the discrete projection evaluates it in binary32: E = {d : d^T Sigma2^-1 d <= kap} with
// kap = 2 (ln(255 o) + 0.02 |ln(255 o)| + 1.5e-4), o = 1 / (1 + exp(-logit)). Stored: the
// mean (u, v), Sigma2's off-diagonal b, 1 / c (c: Sigma2's yy entry), sqrt(det Sigma2), the
// half-extents hx = sqrt(kap a), hy = sqrt(kap c), and kxy = b / a (the y offset, per unit
// x offset, of E's leftmost / rightmost points).
struct Ellipse {
  float u, v, b, inv_c, sdet, hx, hy, kxy;
};

// Tile columns [xa, xb] (returned as x, y; xa > xb: none) of tile row ty whose square of
// pixel centres, widened by 0.05 px + 0.2% of the half-extent, meets E; clamped to [x0, x1).
// E's part inside the row's strip is convex, so its x-extent ends at E's leftmost /
// rightmost point when that lies inside the strip, else where E's boundary crosses the
// strip edge on that point's side. Every step is one binary32 rounding in a fixed order,
// so the projection (counts) and the emission (tiles) reproduce each other bit for bit.
__device__ __forceinline__ float ellipse_cross(const Ellipse& E, float Ye, float sgn) {
  const float dye = __fsub_rn(Ye, E.v);
  const float ad = fabsf(dye);
  const float w = __fsqrt_rn(fmaxf(__fmul_rn(__fsub_rn(E.hy, ad), __fadd_rn(E.hy, ad)), 0.0f));
  return __fadd_rn(E.u, __fmul_rn(__fmaf_rn(__fmul_rn(sgn, E.sdet), w, __fmul_rn(E.b, dye)), E.inv_c));
}
__device__ __forceinline__ int2 row_span(const Ellipse& E, int ty, int x0, int x1) {
  const int2 none = make_int2(1, 0);
  const float tf = static_cast<float>(kTile);
  const float mgx = __fmaf_rn(0.002f, E.hx, 0.05f);
  const float mgy = __fmaf_rn(0.002f, E.hy, 0.05f);
  const float y_lo = __fmul_rn(static_cast<float>(ty), tf);
  const float Y0 = __fsub_rn(__fadd_rn(y_lo, 0.5f), mgy);
  const float Y1 = __fadd_rn(__fadd_rn(y_lo, __fsub_rn(tf, 0.5f)), mgy);
  if (__fadd_rn(E.v, E.hy) < Y0 || __fsub_rn(E.v, E.hy) > Y1) return none;
  const float yR = __fmaf_rn(E.kxy, E.hx, E.v);
  const float yL = __fmaf_rn(-E.kxy, E.hx, E.v);
  const float xr = (yR >= Y0 && yR <= Y1) ? __fadd_rn(E.u, E.hx)
                                          : (yR > Y1 ? ellipse_cross(E, Y1, 1.0f) : ellipse_cross(E, Y0, 1.0f));
  const float xl = (yL >= Y0 && yL <= Y1) ? __fsub_rn(E.u, E.hx)
                                          : (yL > Y1 ? ellipse_cross(E, Y1, -1.0f) : ellipse_cross(E, Y0, -1.0f));
  const float inv_t = 1.0f / tf;
  float fa = ceilf(__fmul_rn(__fsub_rn(__fsub_rn(xl, mgx), __fsub_rn(tf, 0.5f)), inv_t));
  float fb = floorf(__fmul_rn(__fsub_rn(__fadd_rn(xr, mgx), 0.5f), inv_t));
  fa = fmaxf(fa, static_cast<float>(x0));
  fb = fminf(fb, static_cast<float>(x1 - 1));
  if (!(fa <= fb)) return none;
  return make_int2(static_cast<int>(fa), static_cast<int>(fb));
}

// Launchers (each defined in its own translation unit). All return cudaGetLastError().
cudaError_t launch_project(const Layout& L, const GaussPtrs& g, const gs_camera_t* cams, void* ws, cudaStream_t s);
cudaError_t launch_bin(const Layout& L, void* ws, cudaStream_t s);
cudaError_t launch_item_sort(const Layout& L, void* ws, cudaStream_t s);
cudaError_t launch_sort_passes(const Layout& L, void* ws, cudaStream_t s);

struct FusedLossArgs {
  const float* rgb_t;
  const float* depth_t;
  float* g_rgb;
  float* g_depth;
  float* d_loss;
};
cudaError_t launch_raster_fwd(const Layout& L, void* ws, float* rgb, float* depth, float* T_final, int32_t* last,
                              bool stats, const FusedLossArgs* loss, cudaStream_t s, const float* ext_depth = nullptr,
                              const float* ext_rgb = nullptr);
// the loss-fused forward continuing, block by block, into the backward pass (dL_dT = 0)
cudaError_t launch_raster_fwd_l1_bwd(const Layout& L, void* ws, float* rgb, float* depth, float* T_final, int32_t* last,
                                     const FusedLossArgs& loss, cudaStream_t s);
cudaError_t launch_raster_bwd(const Layout& L, void* ws, const float* rgb, const float* depth, const float* T_final,
                              const int32_t* last, const float* dL_drgb, const float* dL_ddepth, const float* dL_dT,
                              cudaStream_t s);
cudaError_t launch_loss(const Layout& L, const float* rgb, const float* depth, const float* rgb_t,
                        const float* depth_t, float* g_rgb, float* g_depth, float* d_loss, void* ws, cudaStream_t s);
cudaError_t launch_project_bwd(const Layout& L, const GaussPtrs& g, const gs_camera_t* cams, void* ws,
                               const gs_grads_t& out, cudaStream_t s);
cudaError_t launch_screen_grads(const Layout& L, const void* ws, float* d_mean2d, float* d_conic, float* d_depth,
                                float* d_opacity, float* d_rgb, cudaStream_t s);

// Generic stable onesweep sort of (key, u32 value) pairs: u64 keys for the (tile, depth) pairs
// and gs_sort_pairs, u32 keys for the per-item depth sort of gs_bin_sort.
template <class KeyT>
struct SortArgsT {
  KeyT* keys[2];
  uint32_t* vals[2];
  const uint32_t* n_dev;  // device pair count (nullptr: use n_host)
  int64_t n_host;         // host pair count or capacity bound
  uint32_t* hist;         // [passes][256] global digit counts (filled before the passes)
  uint32_t* tile_status;  // [passes][max_tiles][256]
  uint32_t* tile_ctr;     // [passes]
  uint32_t* err;
  int64_t max_tiles;
  int passes;
  int key_bits;   // the last pass only looks at the bits below key_bits
  int first_bit;  // pass p sorts on bits [first_bit + 8p, first_bit + 8p + 8)
  const uint64_t* total_dev;  // if set and *total_dev > n_host (capacity overflow), do nothing
  uint32_t first_tile;        // diagnostic: 1 withholds tile 0, so its successors' waits run out
  int items;                  // keys per thread per tile: 8 or 15 (0: kSortItems)
};
__host__ __device__ inline int sort_items(int items) { return (items == 4 || items == 8) ? items : kSortItems; }
// onesweep tiles of n keys at `items` keys per thread
__host__ __device__ inline int64_t sort_tiles(int64_t n, int items) {
  const int64_t tk = static_cast<int64_t>(kSortThreads) * sort_items(items);
  return n > 0 ? (n + tk - 1) / tk : 1;
}
// Keys per thread for a sort of up to n keys: small sorts take short tiles, so that enough
// blocks share the work.
// keys per thread: small sorts take small tiles (more blocks, shorter per-tile latency)
inline int pick_sort_items(int64_t n) { return n <= 200000 ? 4 : (n <= 600000 ? 8 : kSortItems); }
using SortArgs = SortArgsT<uint64_t>;
using SortArgs32 = SortArgsT<uint32_t>;
cudaError_t launch_onesweep(const SortArgs& a, cudaStream_t s);
cudaError_t launch_onesweep(const SortArgs32& a, cudaStream_t s);
cudaError_t launch_sort_prepare(const SortArgs& a, cudaStream_t s);  // zero status, build histogram
int bin_sort_launch_count(const Layout& L);  // kernels one gs_bin_sort launches
int device_sms();  // multiprocessors of the current device (cached per device)

}  // namespace gs
