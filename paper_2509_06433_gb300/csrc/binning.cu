// Tile binning of the projected Gaussians, after the (view, Gaussian) items have been
// stably sorted by camera depth:
//   k_sorted_counts   tiles emitted per item in depth order, per-block totals
//   k_scan_blocks     exclusive scan of the block totals, pair count, capacity check
//   k_item_offsets    per item (depth order): first pair index, rectangle, ids
//   k_tile_scan       row-wise prefix sum of each view's span grid = pairs per tile, then the
//                     tile ranges [start, end) and the digit histograms of the pair sort
//   k_emit_pairs      one (key, value) pair per emitted (view, Gaussian, tile), 1024 pairs per block
//
// An item emits, row by row through its tile rectangle, the tiles of each row's span that
// its widened alpha >= 1/255 ellipse meets (row_span).
// key   = ((k * Tx * Ty + ty * Tx + tx) << 32) | g
// value = the pair's emission index (its slot in the per-pair gradient buffer).
// Pairs are emitted item by item in (depth bits, k*N + g) order. The pair sort then orders
// the tile bits only (stable), which leaves every tile's pairs in (depth bits, k*N + g)
// order: the order of a stable sort of ((tile << 32) | depth bits) keys emitted in (k, g)
// order. Because the sort orders by tile, the ranges are the exclusive scan of the per-tile
// pair counts.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kEmitThreads = 256;

// Tiles touched by each live item in depth order, and per-chunk totals for the scan (chunks of
// kProjBlock items; the blocks stride over the chunks of the n_live live items). Block 0 also
// resets what the tile scan accumulates into: the pair sort's digit histograms, the per-view
// look-back status and the view counter.
__global__ void __launch_bounds__(kProjBlock) k_sorted_counts(Layout L, uint8_t* __restrict__ ws) {
  pdl_begin();
  Status* st = at<Status>(ws, L.status);
  if (blockIdx.x == 0) {
    uint32_t* hist = at<uint32_t>(ws, L.hist);
    for (int i = threadIdx.x; i < 4 * 256; i += kProjBlock) hist[i] = 0;
    uint64_t* vlb = at<uint64_t>(ws, L.view_lb);
    for (int i = threadIdx.x; i < L.K; i += kProjBlock) vlb[i] = 0;
    if (threadIdx.x == 0) st->view_ctr = 0;
  }
  const int64_t n_live = st->n_live;
  const int64_t chunks = (n_live + kProjBlock - 1) / kProjBlock;
  __shared__ uint32_t warp_sums[kProjBlock / 32];
  for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
    const int64_t s = c * kProjBlock + threadIdx.x;
    uint32_t cnt = 0;
    if (s < n_live) cnt = at<uint32_t>(ws, L.live_count)[at<uint32_t>(ws, L.item_vals[0])[s]];
    at<uint32_t>(ws, L.sorted_counts)[s] = cnt;
    uint32_t v = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t tot = 0;
      for (int w = 0; w < kProjBlock / 32; ++w) tot += warp_sums[w];
      at<uint32_t>(ws, L.block_sums)[c] = tot;
    }
    __syncthreads();
  }
}

// Inclusive scan of x over a 1024-thread block; tmp: 32 words. Returns the inclusive value;
// *total receives the block total.
__device__ __forceinline__ uint64_t block_inclusive_scan1024(uint64_t x, uint64_t* tmp, uint64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = tmp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    tmp[lane] = w;
  }
  __syncthreads();
  const uint64_t r = (warp ? tmp[warp - 1] : 0) + incl;
  *total = tmp[31];
  __syncthreads();
  return r;
}

// Exclusive scan of the per-block pair totals; total pair count, capacity check; clears the
// pair sort's tile counters.
__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(Layout L, uint8_t* __restrict__ ws) {
  pdl_begin();
  const uint32_t* sums = at<uint32_t>(ws, L.block_sums);
  uint64_t* offs = at<uint64_t>(ws, L.block_offsets);
  Status* st = at<Status>(ws, L.status);
  const int64_t chunks = (static_cast<int64_t>(st->n_live) + kProjBlock - 1) / kProjBlock;
  __shared__ uint64_t tmp[32];
  // each thread sums a run of consecutive totals, one block-wide scan of the runs' sums gives
  // every run its start, and the thread then writes its run's offsets (one barrier round, not
  // one per 1024 totals)
  const int64_t per = (chunks + kScanThreads - 1) / kScanThreads;
  const int64_t b0 = threadIdx.x * per, b1 = b0 + per < chunks ? b0 + per : chunks;
  uint64_t run = 0;
  for (int64_t i = b0; i < b1; ++i) run += sums[i];
  uint64_t carry;
  uint64_t start = block_inclusive_scan1024(run, tmp, &carry) - run;
  for (int64_t i = b0; i < b1; ++i) {
    offs[i] = start;
    start += sums[i];
  }
  if (threadIdx.x == 0) {
    st->total_pairs = carry;
    st->num_pairs = static_cast<uint32_t>(carry < static_cast<uint64_t>(L.cap) ? carry : L.cap);
    if (carry > static_cast<uint64_t>(L.cap)) atomicOr(&st->err, GS_DEVERR_PAIR_OVERFLOW);
  }
  if (threadIdx.x < 4) st->tile_ctr[4 + threadIdx.x] = 0;
}

// Per live item in depth order: its first pair index (clamped to the capacity), and the compact
// record the pair-parallel emission reads. Also stores the offset with the projection record
// (the backward pass finds a pair's gradient slot from it). The blocks stride over the chunks.
__global__ void __launch_bounds__(kProjBlock) k_item_offsets(Layout L, uint8_t* __restrict__ ws) {
  pdl_begin();
  __shared__ uint32_t s_warp[kProjBlock / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const Status* st = at<Status>(ws, L.status);
  const int64_t n_live = st->n_live;
  const int64_t chunks = (n_live + kProjBlock - 1) / kProjBlock;
  const uint64_t cap = static_cast<uint64_t>(L.cap);
  const uint64_t n = st->num_pairs;
  uint32_t* offsets = at<uint32_t>(ws, L.item_offsets);
  if (blockIdx.x == 0 && t == 0 && n_live == 0) offsets[0] = 0;
  for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
    const int64_t s = c * kProjBlock + t;
    const uint32_t cnt = at<uint32_t>(ws, L.sorted_counts)[s];
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t wo = 0;
#pragma unroll
    for (int w = 0; w < kProjBlock / 32; ++w) wo += (w < warp) ? s_warp[w] : 0u;
    __syncthreads();
    const uint64_t off = at<uint64_t>(ws, L.block_offsets)[c] + wo + incl - cnt;
    if (s < n_live && cnt) {
      // the emission blocks (kEmitPairs pairs each) whose first or last pair is one of this item's
      // pairs learn here which item that is (the block's window of items)
      const uint64_t lo = off, hi = off + cnt < n ? off + cnt : n;
      uint32_t* first_item = at<uint32_t>(ws, L.emit_first);
      uint32_t* last_item = at<uint32_t>(ws, L.emit_last);
      for (uint64_t b = lo / kEmitPairs; b * kEmitPairs < hi; ++b) {
        const uint64_t b0 = b * kEmitPairs;
        const uint64_t b1 = (b0 + kEmitPairs < n ? b0 + kEmitPairs : n) - 1;
        if (b0 >= lo) first_item[b] = static_cast<uint32_t>(s);
        if (b1 < hi) last_item[b] = static_cast<uint32_t>(s);
      }
    }
    if (s < n_live) {
      offsets[s] = static_cast<uint32_t>(off < cap ? off : cap);
      if (s == n_live - 1) offsets[n_live] = static_cast<uint32_t>(off + cnt < cap ? off + cnt : cap);
      const uint32_t pos = at<uint32_t>(ws, L.item_vals[0])[s];
      const uint32_t kg = at<uint32_t>(ws, L.live_kg)[pos];
      at<uint32_t>(ws, L.live_off)[pos] = static_cast<uint32_t>(off < cap ? off : cap);
      const uint32_t k = static_cast<uint32_t>(kg / static_cast<uint64_t>(L.N));
      const uint2 rows = at<uint2>(ws, L.live_rows)[pos];
      at<int4>(ws, L.item_rect)[s] = make_int4(static_cast<int>(rows.x), static_cast<int>(rows.y), 0, 0);
      at<uint2>(ws, L.item_kg)[s] = make_uint2(k, kg - k * static_cast<uint32_t>(L.N));
    }
  }
}

// One block per view (views numbered in block start order): the row-wise prefix sum of the
// view's (Ty+1) x (Tx+1) span grid (cell (ty, tx) then holds the number of pairs of tile (ty, tx);
// staged in shared memory when it fits, else summed in place in global memory), the view's pair
// total, the pair offset of the view (decoupled look-back over the lower-numbered views), then
// the exclusive scan of the per-tile pair counts over the view's tiles: ranges (clamped to the
// pairs actually emitted; [0, 0) for an empty tile) and the digit histograms of the pair sort.
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(Layout L, uint8_t* __restrict__ ws) {
  pdl_begin();
  __shared__ uint64_t tmp[32];
  __shared__ uint32_t s_hist[4 * 256];
  __shared__ int32_t sg[kProjGridCells];
  __shared__ uint32_t s_view;
  __shared__ uint64_t s_base;
  Status* st = at<Status>(ws, L.status);
  if (threadIdx.x == 0) s_view = atomicAdd(&st->view_ctr, 1u);
  for (int i = threadIdx.x; i < 4 * 256; i += kScanThreads) s_hist[i] = 0;
  __syncthreads();
  const int k = static_cast<int>(s_view);
  if (k >= L.K) return;
  // after a capacity overflow the pair sort does not run: leave every tile empty
  const uint64_t n = st->total_pairs > static_cast<uint64_t>(L.cap) ? 0 : st->num_pairs;
  uint32_t* ranges = at<uint32_t>(ws, L.ranges);
  const int stride = L.Tx + 1;
  const int cells = stride * (L.Ty + 1);
  const bool in_smem = cells <= kProjGridCells;
  const int64_t per_view = static_cast<int64_t>(L.Tx) * L.Ty;
  int32_t* gg = at<int32_t>(ws, L.tile_diff) + static_cast<int64_t>(k) * cells;
  int32_t* g = in_smem ? sg : gg;
  if (in_smem)
    for (int i = threadIdx.x; i < cells; i += kScanThreads) sg[i] = gg[i];
  __syncthreads();
  // row-wise prefix sums, and the view's total (each thread sums the rows it owns)
  uint64_t mine = 0;
  for (int y = threadIdx.x; y < L.Ty; y += kScanThreads) {
    int32_t acc = 0;
    for (int x = 0; x <= L.Tx; ++x) {
      acc += g[y * stride + x];
      g[y * stride + x] = acc;
      if (x < L.Tx) mine += static_cast<uint32_t>(acc);
    }
  }
  uint64_t total;
  block_inclusive_scan1024(mine, tmp, &total);
  if (threadIdx.x < 32) {
    const uint64_t base = lb_exclusive_warp(at<uint64_t>(ws, L.view_lb), static_cast<uint32_t>(k), total, &st->err);
    if (threadIdx.x == 0) s_base = base;
  }
  __syncthreads();
  uint64_t carry = s_base;
  for (int64_t base = 0; base < per_view; base += kScanThreads) {
    const int64_t r = base + threadIdx.x;
    uint32_t c = 0;
    if (r < per_view) {
      const int64_t ty = r / L.Tx, tx = r - ty * L.Tx;
      c = static_cast<uint32_t>(g[ty * stride + tx]);
    }
    uint64_t tot;
    const uint64_t incl = block_inclusive_scan1024(c, tmp, &tot);
    if (r < per_view) {
      const int64_t tg = k * per_view + r;
      const uint64_t start = c ? carry + incl - c : 0, end = c ? carry + incl : 0;
      ranges[2 * tg] = static_cast<uint32_t>(start < n ? start : n);
      ranges[2 * tg + 1] = static_cast<uint32_t>(end < n ? end : n);
      if (c)
        for (int p = 0; p < L.passes; ++p)
          atomicAdd(&s_hist[p * 256 + ((static_cast<uint32_t>(tg) >> (8 * p)) & 0xffu)], c);
    }
    carry += tot;
  }
  __syncthreads();
  uint32_t* hist = at<uint32_t>(ws, L.hist);
  for (int i = threadIdx.x; i < L.passes * 256; i += kScanThreads)
    if (s_hist[i]) atomicAdd(&hist[i], s_hist[i]);
}

// Pairs [b * kEmitPairs, (b + 1) * kEmitPairs) of the emission order (window b; the blocks
// stride over the windows). The block stages its window of items (pair offsets, row-table ranges, view and Gaussian ids) and, when they fit,
// the window items' row-span entries in shared memory; each pair then finds its item and its
// row by binary searches in shared memory.
constexpr int kEmitRows = 1024;  // row-span entries staged per block (else read from the table)

__global__ void __launch_bounds__(kEmitThreads) k_emit_pairs(Layout L, uint8_t* __restrict__ ws) {
  pdl_wait();
  constexpr int kPerThread = (kEmitPairs + 1 + kEmitThreads - 1) / kEmitThreads;  // items per thread in the scan
  __shared__ uint32_t s_off[kEmitPairs + 2];
  __shared__ uint32_t s_rt[kEmitPairs + 1];    // first row-table entry of each window item
  __shared__ uint32_t s_nk[kEmitPairs + 1];    // entries | view << 16
  __shared__ uint32_t s_g[kEmitPairs + 1];     // Gaussian id
  __shared__ uint32_t s_rbase[kEmitPairs + 1];  // first staged entry of each window item
  __shared__ int2 s_rows[kEmitRows];
  __shared__ uint32_t s_warp[kEmitThreads / 32];
  __shared__ int64_t s_lo, s_hi;
  const uint64_t n = at<Status>(ws, L.status)->num_pairs;
  // clear the pair sort's look-back status (grid-stride over the tiles in use)
  {
    const uint64_t used = static_cast<uint64_t>(sort_tiles(static_cast<int64_t>(n), L.pair_sort_items)) * 256;
    const uint64_t gsize = static_cast<uint64_t>(gridDim.x) * kEmitThreads;
    uint32_t* sstat = at<uint32_t>(ws, L.sort_status);
    for (int p = 0; p < L.passes; ++p)
      for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * kEmitThreads + threadIdx.x; i < used; i += gsize)
        sstat[static_cast<uint64_t>(p) * L.max_sort_tiles * 256 + i] = 0;
    // and the per-pair record bits of the backward pass
    uint32_t* valid = at<uint32_t>(ws, L.pair_valid);
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * kEmitThreads + threadIdx.x; i < (n + 31) / 32; i += gsize)
      valid[i] = 0;
  }
  // the blocks stride over the windows of kEmitPairs pairs that hold emitted pairs
  const uint64_t n_windows = (n + kEmitPairs - 1) / kEmitPairs;
  for (uint64_t win_id = blockIdx.x; win_id < n_windows; win_id += gridDim.x) {
  __syncthreads();  // the previous window's shared staging is no longer read
  const uint64_t start = win_id * kEmitPairs;
  const uint64_t end = start + kEmitPairs < n ? start + kEmitPairs : n;
  const uint32_t* offsets = at<uint32_t>(ws, L.item_offsets);
  if (threadIdx.x == 0) {  // the items holding the window's first and last pairs (k_item_offsets)
    s_lo = at<uint32_t>(ws, L.emit_first)[win_id];
    s_hi = at<uint32_t>(ws, L.emit_last)[win_id];
  }
  __syncthreads();
  const int64_t lo = s_lo;
  // every item of the window emits (items that emit nothing sort last), so win <= kEmitPairs
  const int win = static_cast<int>(s_hi - lo + 1);
  const int4* rects = at<int4>(ws, L.item_rect);
  const uint2* kgs = at<uint2>(ws, L.item_kg);
  const int2* rowtab = at<int2>(ws, L.row_table);
  for (int i = threadIdx.x; i <= win; i += kEmitThreads) s_off[i] = offsets[lo + i];
  for (int i = threadIdx.x; i < win; i += kEmitThreads) {
    const int4 rc = rects[lo + i];  // (first row-table entry, entries)
    const uint2 kg = kgs[lo + i];
    s_rt[i] = static_cast<uint32_t>(rc.x);
    s_nk[i] = static_cast<uint32_t>(rc.y) | (kg.x << 16);
    s_g[i] = kg.y;
  }
  __syncthreads();
  // exclusive scan of the window items' entry counts (kPerThread consecutive items per thread)
  uint32_t loc[kPerThread], sum = 0;
#pragma unroll
  for (int q = 0; q < kPerThread; ++q) {
    const int i = threadIdx.x * kPerThread + q;
    loc[q] = i < win ? (s_nk[i] & 0xffffu) : 0u;
    sum += loc[q];
  }
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t base = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kEmitThreads / 32; ++w) {
      base += w < warp ? s_warp[w] : 0u;
      total += s_warp[w];
    }
    base += incl - sum;
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
      const int i = threadIdx.x * kPerThread + q;
      if (i < win) s_rbase[i] = base;
      base += loc[q];
    }
    __syncthreads();
    if (total <= static_cast<uint32_t>(kEmitRows)) {
      for (int i = threadIdx.x; i < win; i += kEmitThreads) {
        const uint32_t nr = s_nk[i] & 0xffffu, b = s_rbase[i], rt = s_rt[i];
        for (uint32_t r = 0; r < nr; ++r) s_rows[b + r] = rowtab[rt + r];
      }
    } else if (threadIdx.x == 0) {
      s_warp[0] = 0xffffffffu;  // marker: entries stay in global memory
    }
    __syncthreads();
  }
  const bool staged = s_warp[0] != 0xffffffffu;
  uint64_t* keys = at<uint64_t>(ws, L.keys[0]);
  uint32_t* vals = at<uint32_t>(ws, L.vals[0]);
  const uint64_t tiles_per_view = static_cast<uint64_t>(L.Tx) * L.Ty;
  for (uint64_t j = start + threadIdx.x; j < end; j += kEmitThreads) {
    const uint32_t jj = static_cast<uint32_t>(j);
    int a = 0, b = win;  // s_off[a] <= j < s_off[b]
    while (b - a > 1) {
      const int mid = (a + b) >> 1;
      if (s_off[mid] <= jj) a = mid; else b = mid;
    }
    const uint32_t nk = s_nk[a];
    const int nrows = static_cast<int>(nk & 0xffffu);
    // the pair's tile: its row is the last entry whose earlier-row pair count is <= r
    const int r = static_cast<int>(jj - s_off[a]);
    int tx = 0, ty = 0;
    if (nrows > 0) {
      const int2* tab = staged ? s_rows + s_rbase[a] : rowtab + s_rt[a];
      int p = 0, q = nrows;  // tab[p].x <= r, and r < tab[q].x or q = entries
      while (q - p > 1) {
        const int mid = (p + q) >> 1;
        if (tab[mid].x <= r) p = mid; else q = mid;
      }
      const int2 e = tab[p];
      tx = (e.y & 0xffff) + (r - e.x);
      ty = static_cast<int>(static_cast<uint32_t>(e.y) >> 16);
    }
    const uint64_t tid = static_cast<uint64_t>(nk >> 16) * tiles_per_view + static_cast<uint64_t>(ty) * L.Tx + tx;
    if (!GS_INDEX_OK(tid < static_cast<uint64_t>(L.n_tiles) && tx < L.Tx && ty < L.Ty && j < static_cast<uint64_t>(L.cap),
                     &at<Status>(ws, L.status)->err))
      continue;
    keys[j] = (tid << 32) | s_g[a];
    vals[j] = jj;
  }
  }  // windows
  pdl_trigger();
}

}  // namespace

cudaError_t launch_bin(const Layout& L, void* ws, cudaStream_t s) {
  auto* w = static_cast<uint8_t*>(ws);
  // the live items are counted on the device: the per-item kernels stride over their chunks
  const int64_t resident = static_cast<int64_t>(device_sms()) * (2048 / kProjBlock);
  const unsigned item_grid = static_cast<unsigned>(L.n_proj_blocks < resident ? L.n_proj_blocks : resident);
  launch(k_sorted_counts, item_grid, kProjBlock, 0, s, L, w);
  launch(k_scan_blocks, 1, kScanThreads, 0, s, L, w);
  launch(k_item_offsets, item_grid, kProjBlock, 0, s, L, w);
  launch(k_tile_scan, static_cast<unsigned>(L.K), kScanThreads, 0, s, L, w);
  // the emission's blocks stride over the windows of emitted pairs (their number is on the device);
  // enough blocks that a typical count takes one window per block (a block looping over several
  // windows serialises their latency-bound searches), few enough that surplus blocks cost little
  const int64_t emit_resident = static_cast<int64_t>(device_sms()) * 128;
  launch(k_emit_pairs, static_cast<unsigned>(L.n_emit_blocks < emit_resident ? L.n_emit_blocks : emit_resident),
         kEmitThreads, 0, s, L, w);
  return cudaGetLastError();
}

}  // namespace gs
