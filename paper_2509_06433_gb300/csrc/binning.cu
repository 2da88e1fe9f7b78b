// Tile binning of the projected Gaussians, after the (view, Gaussian) items have been
// stably sorted by camera depth: tiles touched per item in depth order, exclusive scan,
// emission of one (key, value) pair per (view, Gaussian, tile) in depth order, digit
// histograms of the pair sort, and per-tile [start, end) ranges of the sorted list.
//
// key   = ((k * Tx * Ty + ty * Tx + tx) << 32) | bits(camera depth)   (depth > 0, so the
//         float bit pattern orders like the depth)
// value = Gaussian id g.
// Emission runs over the items in (depth bits, k*N + g) order, tiles row-major inside each
// rectangle. The pair sort then only orders the tile bits (stable), which leaves every
// tile's pairs in (depth bits, k*N + g) order: the order of a stable sort of the full keys.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kScanThreads = 1024;

// Tiles touched by each item in depth order, and per-block totals for the scan.
__global__ void __launch_bounds__(kProjBlock) k_sorted_counts(Layout L, uint8_t* __restrict__ ws) {
  const int64_t s = static_cast<int64_t>(blockIdx.x) * kProjBlock + threadIdx.x;
  uint32_t cnt = 0;
  if (s < L.KN) {
    const uint32_t kg = at<uint32_t>(ws, L.item_vals[0])[s];
    cnt = static_cast<uint32_t>(at<int4>(ws, L.proj_tiles)[kg].w);
  }
  at<uint32_t>(ws, L.sorted_counts)[s] = cnt;
  __shared__ uint32_t warp_sums[kProjBlock / 32];
  uint32_t v = cnt;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int w = 0; w < kProjBlock / 32; ++w) tot += warp_sums[w];
    at<uint32_t>(ws, L.block_sums)[blockIdx.x] = tot;
  }
}

// Exclusive scan of the per-block pair totals; total pair count, capacity check; clears the
// pair-sort digit histograms and tile counters.
__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(Layout L, uint8_t* __restrict__ ws) {
  const uint32_t* sums = at<uint32_t>(ws, L.block_sums);
  uint64_t* offs = at<uint64_t>(ws, L.block_offsets);
  __shared__ uint64_t warp_tot[kScanThreads / 32];
  __shared__ uint64_t carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < L.n_proj_blocks; base += kScanThreads) {
    const int64_t i = base + threadIdx.x;
    const uint64_t x = (i < L.n_proj_blocks) ? sums[i] : 0;
    uint64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      uint64_t w = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const uint64_t warp_excl = warp ? warp_tot[warp - 1] : 0;
    if (i < L.n_proj_blocks) offs[i] = carry + warp_excl + incl - x;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_tot[kScanThreads / 32 - 1];
    __syncthreads();
  }
  Status* st = at<Status>(ws, L.status);
  if (threadIdx.x == 0) {
    st->total_pairs = carry;
    st->num_pairs = static_cast<uint32_t>(carry < static_cast<uint64_t>(L.cap) ? carry : L.cap);
    if (carry > static_cast<uint64_t>(L.cap)) atomicOr(&st->err, GS_DEVERR_PAIR_OVERFLOW);
  }
  uint32_t* hist = at<uint32_t>(ws, L.hist);
  for (int i = threadIdx.x; i < kMaxSortPasses * 256; i += kScanThreads) hist[i] = 0;
  if (threadIdx.x < 4) st->tile_ctr[4 + threadIdx.x] = 0;
}

// One block per kProjBlock depth-sorted items. The block's pairs are written as one
// contiguous, coalesced run: thread j of the block handles pair j of the run and finds its
// item by binary search over the block-local exclusive scan.
__global__ void __launch_bounds__(kProjBlock) k_emit(Layout L, uint8_t* __restrict__ ws) {
  __shared__ uint32_t s_excl[kProjBlock + 1];
  __shared__ uint32_t s_rect_x[kProjBlock], s_rect_y[kProjBlock], s_key[kProjBlock], s_gid[kProjBlock];
  __shared__ uint32_t s_warp[kProjBlock / 32];
  __shared__ int s_view[kProjBlock];
  __shared__ uint32_t s_hist[4 * 256];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t s = static_cast<int64_t>(blockIdx.x) * kProjBlock + t;
  int4* tiles = at<int4>(ws, L.proj_tiles);
  const uint32_t cnt = at<uint32_t>(ws, L.sorted_counts)[s];
  uint32_t kg = 0;
  int4 tl = make_int4(0, 0, 0, 0);
  if (cnt) {
    kg = at<uint32_t>(ws, L.item_vals[0])[s];
    tl = tiles[kg];
  }
  // block exclusive scan of cnt
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  for (int i = t; i < 4 * 256; i += kProjBlock) s_hist[i] = 0;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = (lane < kProjBlock / 32) ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kProjBlock / 32) s_warp[lane] = w;
  }
  __syncthreads();
  const uint32_t excl = (warp ? s_warp[warp - 1] : 0) + incl - cnt;
  const uint32_t block_total = s_warp[kProjBlock / 32 - 1];
  const uint64_t base = at<uint64_t>(ws, L.block_offsets)[blockIdx.x];
  const uint64_t cap = static_cast<uint64_t>(L.cap);
  s_excl[t] = excl;
  if (t == 0) s_excl[kProjBlock] = block_total;
  const int k = static_cast<int>(kg / static_cast<uint64_t>(L.N > 0 ? L.N : 1));
  s_rect_x[t] = static_cast<uint32_t>(tl.y);
  s_rect_y[t] = static_cast<uint32_t>(tl.z);
  s_key[t] = cnt ? at<uint32_t>(ws, L.proj_depth_key)[kg] : 0u;
  s_gid[t] = static_cast<uint32_t>(kg - static_cast<int64_t>(k) * L.N);
  s_view[t] = k;
  if (cnt) {
    const uint64_t off = base + excl;
    tiles[kg].x = static_cast<int>(off < cap ? off : cap);
  }
  __syncthreads();

  uint64_t* keys = at<uint64_t>(ws, L.keys[0]);
  uint32_t* vals = at<uint32_t>(ws, L.vals[0]);
  const uint64_t tiles_per_view = static_cast<uint64_t>(L.Tx) * L.Ty;
  // the loop trip count is uniform over the block so that whole warps reach the
  // warp-aggregated histogram update (neighbouring pairs mostly share their tile digits)
  for (uint32_t j0 = 0; j0 < block_total; j0 += kProjBlock) {
    const uint32_t j = j0 + t;
    const uint64_t pos = base + j;
    const bool active = j < block_total && pos < cap;
    uint32_t tid32 = 0;
    if (active) {
      // last item with s_excl <= j
      int lo = 0, hi = kProjBlock;  // invariant: s_excl[lo] <= j < s_excl[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_excl[mid] <= j) lo = mid; else hi = mid;
      }
      const uint32_t r = j - s_excl[lo];
      const uint32_t rx = s_rect_x[lo], ry = s_rect_y[lo];
      const uint32_t x0 = rx & 0xffffu, w = (rx >> 16) - x0;
      const uint32_t y0 = ry & 0xffffu;
      const uint32_t ty = y0 + r / w, tx = x0 + r % w;
      const uint64_t tid = static_cast<uint64_t>(s_view[lo]) * tiles_per_view + static_cast<uint64_t>(ty) * L.Tx + tx;
      keys[pos] = (tid << 32) | s_key[lo];
      vals[pos] = s_gid[lo];
      tid32 = static_cast<uint32_t>(tid);
    }
    for (int p = 0; p < L.passes; ++p) {
      const uint32_t d = active ? ((tid32 >> (8 * p)) & 0xffu) : 0x100u;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      if (active && lane == __ffs(peers) - 1) atomicAdd(&s_hist[p * 256 + d], static_cast<uint32_t>(__popc(peers)));
    }
  }
  __syncthreads();
  uint32_t* hist = at<uint32_t>(ws, L.hist);
  for (int i = t; i < L.passes * 256; i += kProjBlock)
    if (s_hist[i]) atomicAdd(&hist[i], s_hist[i]);

  // clear the tile ranges and the pair sort's look-back status
  const Status* st = at<Status>(ws, L.status);
  const uint64_t n = st->num_pairs;
  const uint64_t used_tiles = (n + kSortTileKeys - 1) / kSortTileKeys;
  const uint64_t gsize = static_cast<uint64_t>(gridDim.x) * kProjBlock;
  const uint64_t gtid = static_cast<uint64_t>(blockIdx.x) * kProjBlock + t;
  uint32_t* ranges = at<uint32_t>(ws, L.ranges);
  for (uint64_t i = gtid; i < 2 * static_cast<uint64_t>(L.n_tiles); i += gsize) ranges[i] = 0;
  uint32_t* sstat = at<uint32_t>(ws, L.sort_status);
  for (int p = 0; p < L.passes; ++p) {
    uint32_t* sp = sstat + static_cast<uint64_t>(p) * L.max_sort_tiles * 256;
    for (uint64_t i = gtid; i < used_tiles * 256; i += gsize) sp[i] = 0;
  }
}

// ranges[t] = [first, last + 1) of tile t in the sorted keys (tiles without pairs stay [0, 0)).
__global__ void k_ranges(Layout L, uint8_t* __restrict__ ws, const uint64_t* __restrict__ keys) {
  const uint32_t n = at<Status>(ws, L.status)->num_pairs;
  uint32_t* ranges = at<uint32_t>(ws, L.ranges);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t tcur = static_cast<uint32_t>(keys[i] >> 32);
    if (i == 0 || static_cast<uint32_t>(keys[i - 1] >> 32) != tcur) ranges[2 * tcur] = i;
    if (i == n - 1 || static_cast<uint32_t>(keys[i + 1] >> 32) != tcur) ranges[2 * tcur + 1] = i + 1;
  }
}

int num_sms_bin() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

}  // namespace

cudaError_t launch_bin(const Layout& L, void* ws, cudaStream_t s) {
  auto* w = static_cast<uint8_t*>(ws);
  k_sorted_counts<<<static_cast<unsigned>(L.n_proj_blocks), kProjBlock, 0, s>>>(L, w);
  k_scan_blocks<<<1, kScanThreads, 0, s>>>(L, w);
  k_emit<<<static_cast<unsigned>(L.n_proj_blocks), kProjBlock, 0, s>>>(L, w);
  return cudaGetLastError();
}

cudaError_t launch_ranges(const Layout& L, void* ws, cudaStream_t s) {
  auto* w = static_cast<uint8_t*>(ws);
  const uint64_t* keys = at<uint64_t>(ws, L.keys[L.passes & 1]);
  const int64_t want = (L.cap + 255) / 256;
  const int blocks = static_cast<int>(want < 8 * num_sms_bin() ? (want > 0 ? want : 1) : 8 * num_sms_bin());
  k_ranges<<<blocks, 256, 0, s>>>(L, w, keys);
  return cudaGetLastError();
}

}  // namespace gs
