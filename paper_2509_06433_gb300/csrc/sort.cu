// Stable LSD radix sort of (key, u32 value) pairs, one "onesweep" kernel per 8-bit digit
// (Adinets & Merrill, "Onesweep: A Faster Least Significant Digit Radix Sort for GPUs",
// 2022): the global digit histograms of all passes are counted up front; each pass then
// ranks a tile of keys in shared memory, obtains the tile's global offset per digit by a
// decoupled look-back over the preceding tiles, and scatters through shared memory so that
// runs of equal digits are written contiguously. Keys are u64 ((tile, depth) pairs and the
// gs_sort_pairs primitive) or u32 (the per-item depth sort of gs_bin_sort).
//
// Stability: inside a tile, keys are ranked in (warp, item, lane) order, which is their
// input order; tiles are numbered by a dynamic counter and the look-back sums the counts
// of all lower-numbered tiles. The look-back spin is bounded: past kSpinLimit polls it
// sets GS_DEVERR_TIMEOUT and stops waiting (all writes stay inside [0, n)).
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr uint32_t kFlagAggregate = 1u << 30;
constexpr uint32_t kFlagPrefix = 2u << 30;
constexpr uint32_t kValueMask = (1u << 30) - 1;
constexpr int kWarps = kSortThreads / 32;

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Exclusive scan of one value per thread over a kSortThreads block. tmp: kWarps words.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* tmp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  uint32_t off = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) off += (w < warp) ? tmp[w] : 0u;
  __syncthreads();
  return off + incl - x;
}

template <class KeyT, int IT>
struct SortSmem {
  KeyT keys[kSortThreads * IT];
  uint32_t vals[kSortThreads * IT];
  uint32_t warp_hist[kWarps][256];
  uint32_t bucket[256];       // exclusive scan of this pass's global digit histogram
  uint32_t global_base[256];  // destination of the tile's first key of each digit
  uint32_t local_start[256];  // first slot of each digit in the tile's shared-memory copy
  uint32_t scan_tmp[kWarps];
  uint32_t tile;
};

template <class KeyT>
__device__ __forceinline__ uint32_t digit_mask(const SortArgsT<KeyT>& a, int pass) {
  const int rem = a.key_bits - (a.first_bit + 8 * pass);
  return rem >= 8 ? 0xffu : ((1u << rem) - 1u);
}

// Decoupled look-back for digit t of tile `tile` (> 0): the sum of the counts of all
// lower-numbered tiles. The statuses of kLookahead predecessors are loaded together (one
// round trip) and consumed in order until one is not published yet (polled again) or
// carries an inclusive prefix (done). Gives up after kSpinLimit polls without progress.
constexpr int kLookahead = 16;  // wider polling loads the L2 more than it saves round trips
__device__ __forceinline__ uint32_t look_back(const uint32_t* status, uint32_t tile, int t, uint32_t* err) {
  uint32_t excl = 0, spins = 0;
  int64_t j = static_cast<int64_t>(tile) - 1;
  for (;;) {
    uint32_t v[kLookahead];
#pragma unroll
    for (int q = 0; q < kLookahead; ++q)
      v[q] = (j - q >= 0) ? ld_relaxed(&status[static_cast<size_t>(j - q) * 256 + t]) : kFlagPrefix;
    int consumed = 0;
    bool found = false, blocked = false;
#pragma unroll
    for (int q = 0; q < kLookahead; ++q) {
      const uint32_t f = v[q] & ~kValueMask;
      if (found || blocked) continue;
      if (f == 0) {
        blocked = true;
        continue;
      }
      excl += v[q] & kValueMask;
      ++consumed;
      found = (f == kFlagPrefix);
    }
    if (found) return excl;
    j -= consumed;
    if (consumed == 0 && ++spins > kSpinLimit) {
      atomicOr(err, GS_DEVERR_TIMEOUT);
      return excl;
    }
  }
}

// One pass over 8 digit bits. Tiles of kSortThreads * IT keys; a block takes tiles from a
// dynamic counter until none are left. Per tile: rank the keys (warp histograms, ordered by
// (warp, item, lane)), publish the tile's digit counts, place the keys in digit order in
// shared memory, look back for the tile's global digit offsets, write the keys out.
// 64-bit keys (the pair sort): compiled for 3 resident blocks per SM (80 registers; 2 at the
// unconstrained 128), which runs its passes 4-6% faster; the 32-bit depth sort is faster at 2.
template <class KeyT, int IT>
__global__ void __launch_bounds__(kSortThreads, sizeof(KeyT) == 8 ? 3 : 1) k_onesweep(SortArgsT<KeyT> a, int pass) {
  pdl_wait();
  constexpr int kTileKeys = kSortThreads * IT;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  SortSmem<KeyT, IT>& S = *reinterpret_cast<SortSmem<KeyT, IT>*>(smem_raw);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // (selects, not a dynamic index into the parameter arrays, which would copy them to local memory)
  const bool odd = pass & 1;
  const KeyT* __restrict__ kin = odd ? a.keys[1] : a.keys[0];
  const uint32_t* __restrict__ vin = odd ? a.vals[1] : a.vals[0];
  KeyT* __restrict__ kout = odd ? a.keys[0] : a.keys[1];
  uint32_t* __restrict__ vout = odd ? a.vals[0] : a.vals[1];
  if (a.total_dev && *a.total_dev > static_cast<uint64_t>(a.n_host)) return;  // overflowed: reported, not sorted
  uint32_t n = static_cast<uint32_t>(a.n_host);
  if (a.n_dev) n = min(*a.n_dev, n);
  const uint32_t n_tiles = (n + kTileKeys - 1) / kTileKeys;
  const int shift = a.first_bit + 8 * pass;
  const uint32_t dmask = digit_mask(a, pass);
  uint32_t* status = a.tile_status + static_cast<size_t>(pass) * a.max_tiles * 256;

  S.bucket[t] = block_exclusive_scan(a.hist[pass * 256 + t], S.scan_tmp);

  for (;;) {
    if (t == 0) S.tile = atomicAdd(&a.tile_ctr[pass], 1u) + a.first_tile;
    __syncthreads();
    const uint32_t tile = S.tile;
    if (tile >= n_tiles) break;
    for (int d = lane; d < 256; d += 32) S.warp_hist[warp][d] = 0;
    __syncwarp();
    const uint32_t wbase = tile * kTileKeys + warp * (32 * IT);
    uint32_t rr[IT], dd[IT], cnt = 0;
    {
      KeyT kr[IT];
      uint32_t vr[IT];
#pragma unroll
      for (int it = 0; it < IT; ++it) {
        const uint32_t i = wbase + it * 32 + lane;
        const bool valid = i < n;
        kr[it] = valid ? kin[i] : static_cast<KeyT>(~static_cast<KeyT>(0));
        vr[it] = valid ? vin[i] : 0u;
      }
#pragma unroll
      for (int it = 0; it < IT; ++it) {
        const uint32_t i = wbase + it * 32 + lane;
        const bool valid = i < n;
        const uint32_t d = valid ? static_cast<uint32_t>(kr[it] >> shift) & dmask : 256u;
        dd[it] = d;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t prior = valid ? S.warp_hist[warp][d] : 0u;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) S.warp_hist[warp][d] = prior + __popc(peers);
        __syncwarp();
        rr[it] = prior + __popc(peers & lanemask_lt());
      }
      __syncthreads();
      // thread t owns digit t: prefix over warps and the tile's count
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = S.warp_hist[w][t];
        S.warp_hist[w][t] = cnt;
        cnt += c;
      }
      // publish early: successors can look back past this tile while it places its keys
      if (tile == 0)
        st_relaxed(&status[t], kFlagPrefix | cnt);
      else
        st_relaxed(&status[static_cast<size_t>(tile) * 256 + t], kFlagAggregate | cnt);
      S.local_start[t] = block_exclusive_scan(cnt, S.scan_tmp);
      __syncthreads();
#pragma unroll
      for (int it = 0; it < IT; ++it) {
        if (dd[it] < 256u) {
          const uint32_t pos = S.local_start[dd[it]] + S.warp_hist[warp][dd[it]] + rr[it];
          S.keys[pos] = kr[it];
          S.vals[pos] = vr[it];
        }
      }
    }
    {
      uint32_t excl = 0;
      if (tile != 0) {
        excl = look_back(status, tile, t, a.err);
        st_relaxed(&status[static_cast<size_t>(tile) * 256 + t], kFlagPrefix | (excl + cnt));
      }
      S.global_base[t] = S.bucket[t] + excl;
    }
    __syncthreads();
    const uint32_t rem = n - tile * kTileKeys;
    const uint32_t tile_n = rem < static_cast<uint32_t>(kTileKeys) ? rem : kTileKeys;
    for (uint32_t j = t; j < tile_n; j += kSortThreads) {
      const KeyT key = S.keys[j];
      const uint32_t d = static_cast<uint32_t>(key >> shift) & dmask;
      const uint32_t dst = S.global_base[d] + (j - S.local_start[d]);
      if (!GS_INDEX_OK(dst < n, a.err)) continue;
      kout[dst] = key;
      vout[dst] = S.vals[j];
    }
    __syncthreads();
  }
  pdl_trigger();
}

// Digit histograms of every pass, and clearing of the look-back status of the used tiles.
__global__ void k_sort_hist(SortArgs a) {
  pdl_begin();
  __shared__ uint32_t s_hist[kMaxSortPasses * 256];
  for (int i = threadIdx.x; i < a.passes * 256; i += blockDim.x) s_hist[i] = 0;
  __syncthreads();
  const uint64_t n = static_cast<uint64_t>(a.n_host);
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  const uint64_t gtid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  for (uint64_t i = gtid; i < n; i += stride) {
    const uint64_t key = a.keys[0][i];
    for (int p = 0; p < a.passes; ++p)
      atomicAdd(&s_hist[p * 256 + ((key >> (a.first_bit + 8 * p)) & digit_mask(a, p))], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < a.passes * 256; i += blockDim.x)
    if (s_hist[i]) atomicAdd(&a.hist[i], s_hist[i]);
  const uint64_t used = static_cast<uint64_t>(sort_tiles(static_cast<int64_t>(n), a.items));
  for (int p = 0; p < a.passes; ++p) {
    uint32_t* sp = a.tile_status + static_cast<uint64_t>(p) * a.max_tiles * 256;
    for (uint64_t i = gtid; i < used * 256; i += stride) sp[i] = 0;
  }
}

// Per-device launch facts, looked up once per device (a process may drive several GPUs).
constexpr int kMaxDevices = 64;

int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
  return dev;
}

int num_sms() { return device_sms(); }

template <class KeyT, int IT>
int sort_grid(int64_t max_tiles) {
  static int blocks_per_sm[kMaxDevices] = {};
  const int dev = current_device();
  if (!blocks_per_sm[dev]) {
    int b = 0;
    cudaFuncSetAttribute(k_onesweep<KeyT, IT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(sizeof(SortSmem<KeyT, IT>)));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_onesweep<KeyT, IT>, kSortThreads, sizeof(SortSmem<KeyT, IT>));
    blocks_per_sm[dev] = b > 0 ? b : 1;
  }
  const int64_t resident = static_cast<int64_t>(blocks_per_sm[dev]) * num_sms();
  const int64_t g = max_tiles < resident ? max_tiles : resident;
  return static_cast<int>(g > 0 ? g : 1);
}

template <class KeyT, int IT>
cudaError_t onesweep_passes_it(const SortArgsT<KeyT>& a, cudaStream_t s) {
  const int grid = sort_grid<KeyT, IT>(a.max_tiles);
  for (int p = 0; p < a.passes; ++p)
    launch(k_onesweep<KeyT, IT>, grid, kSortThreads, sizeof(SortSmem<KeyT, IT>), s, a, p);
  return cudaGetLastError();
}

template <class KeyT>
cudaError_t onesweep_passes(const SortArgsT<KeyT>& a, cudaStream_t s) {
  switch (sort_items(a.items)) {
    case 4: return onesweep_passes_it<KeyT, 4>(a, s);
    case 8: return onesweep_passes_it<KeyT, 8>(a, s);
    default: return onesweep_passes_it<KeyT, kSortItems>(a, s);
  }
}

}  // namespace

int device_sms() {
  static int sms[kMaxDevices] = {};
  const int dev = current_device();
  if (!sms[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = n > 0 ? n : 1;
  }
  return sms[dev];
}

cudaError_t launch_onesweep(const SortArgs& a, cudaStream_t s) { return onesweep_passes(a, s); }

int bin_sort_launch_count(const Layout& L) {
  // counts, scan, item offsets, tile scan, emission; 4 item passes; pair passes
  return 5 + (L.KN > 0 ? 4 : 0) + L.passes;
}
cudaError_t launch_onesweep(const SortArgs32& a, cudaStream_t s) { return onesweep_passes(a, s); }

cudaError_t launch_sort_prepare(const SortArgs& a, cudaStream_t s) {
  cudaMemsetAsync(a.hist, 0, sizeof(uint32_t) * 256 * a.passes, s);
  cudaMemsetAsync(a.tile_ctr, 0, sizeof(uint32_t) * kMaxSortPasses, s);
  int64_t blocks = (a.n_host + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  launch(k_sort_hist, static_cast<unsigned>(blocks), 256, 0, s, a);
  return cudaGetLastError();
}

// gs_bin_sort: (1) stable depth sort of the K*N (view, Gaussian) items, (2) per-item pair
// counts in depth order, scan, emission of the pairs in depth order, (3) stable sort of the
// pairs on the tile bits only, (4) ranges. Pairs sharing a tile leave step (3) ordered by
// (depth bits, k*N + g), exactly the order of a stable sort of the full 64-bit keys emitted
// in (k, g) order.
cudaError_t launch_item_sort(const Layout& L, void* ws, cudaStream_t s) {
  SortArgs32 a{};
  a.keys[0] = at<uint32_t>(ws, L.item_keys[0]);
  a.keys[1] = at<uint32_t>(ws, L.item_keys[1]);
  a.vals[0] = at<uint32_t>(ws, L.item_vals[0]);
  a.vals[1] = at<uint32_t>(ws, L.item_vals[1]);
  Status* st = at<Status>(ws, L.status);
  a.n_dev = &st->n_live;  // the live items, compacted by the projection
  a.n_host = L.KN;
  a.hist = at<uint32_t>(ws, L.item_hist);
  a.tile_status = at<uint32_t>(ws, L.item_status);
  a.tile_ctr = st->tile_ctr;
  a.err = &st->err;
  a.max_tiles = L.max_item_tiles;
  a.items = L.item_sort_items;
  a.passes = 4;
  a.key_bits = 32;
  a.first_bit = 0;
  if (L.KN == 0) return cudaSuccess;
  return launch_onesweep(a, s);
}

cudaError_t launch_sort_passes(const Layout& L, void* ws, cudaStream_t s) {
  if (L.passes == 0) return cudaSuccess;  // a single tile: the emission order is final
  SortArgs a{};
  a.keys[0] = at<uint64_t>(ws, L.keys[0]);
  a.keys[1] = at<uint64_t>(ws, L.keys[1]);
  a.vals[0] = at<uint32_t>(ws, L.vals[0]);
  a.vals[1] = at<uint32_t>(ws, L.vals[1]);
  Status* st = at<Status>(ws, L.status);
  a.n_dev = &st->num_pairs;
  a.n_host = L.cap;
  a.hist = at<uint32_t>(ws, L.hist);
  a.tile_status = at<uint32_t>(ws, L.sort_status);
  a.tile_ctr = st->tile_ctr + 4;
  a.err = &st->err;
  a.max_tiles = L.max_sort_tiles;
  a.items = L.pair_sort_items;
  a.passes = L.passes;
  a.key_bits = L.key_bits;
  a.first_bit = 32;
  a.total_dev = &st->total_pairs;
  return launch_onesweep(a, s);
}

}  // namespace gs
