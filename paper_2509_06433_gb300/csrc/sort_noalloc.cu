// gs_sort_pairs_noalloc: the stable pair sort of gs_sort_pairs with its temporary storage
// in a file-scope device array, so that the call needs no memory from the caller and
// allocates none.
//
// Who needs this: callers that cannot allocate device memory at the point of the call. A
// renderer plugin inside a host application (for instance a viewer process that receives
// the shared Gaussian map and its output buffers from the host engine) does not own the
// device allocator; a real-time tracking loop cannot afford cudaMalloc's implicit device
// synchronisation and unbounded latency. They can still pass their keys and values.
//
// The scratch array holds GS_SORT_NOALLOC_MAX_PAIRS pairs (about 14 MB) and is resident
// on every GPU that loads this library until the process exits. All calls share it, so
// calls whose work overlaps on the GPU (different streams, or different host threads on
// the same device) race on it; serialise them. Each call clears the parts that must start
// at zero (digit histograms, tile counters, look-back status of the tiles it uses, the
// internal error word).
//
// Host code cannot use the array's name as a device address: it is a host-side stand-in.
// The device address is looked up with cudaGetSymbolAddress, with the device current, on
// every call made outside a stream capture (the lookup is cheap, and a context that was torn
// down and re-created, e.g. after cudaDeviceReset, may place the array elsewhere), and kept
// per device for calls made while a stream is being captured. So the first call on a device
// must come before any stream capture that contains a call.
#include <mutex>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int64_t kMaxPairs = GS_SORT_NOALLOC_MAX_PAIRS;
constexpr int64_t kMaxTiles = (kMaxPairs + kSortTileKeys - 1) / kSortTileKeys;
constexpr size_t kAlignment = 256;
constexpr size_t round_up(size_t x) { return (x + kAlignment - 1) / kAlignment * kAlignment; }
constexpr size_t kOffKeys = 0;
constexpr size_t kOffVals = round_up(kOffKeys + static_cast<size_t>(kMaxPairs) * 8);
constexpr size_t kOffHist = round_up(kOffVals + static_cast<size_t>(kMaxPairs) * 4);
constexpr size_t kOffCtr = round_up(kOffHist + kMaxSortPasses * 256 * 4);
constexpr size_t kOffErr = round_up(kOffCtr + kMaxSortPasses * 4);
constexpr size_t kOffStatus = round_up(kOffErr + 4);
constexpr size_t kScratchBytes = round_up(kOffStatus + static_cast<size_t>(kMaxSortPasses) * kMaxTiles * 256 * 4);

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device: looked up again unless `stream` is
// being captured, then the address of the last lookup on this device.
cudaError_t scratch_address(cudaStream_t stream, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cs);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  } else if (!g_scratch_addr[dev]) {
    return cudaErrorStreamCaptureUnsupported;  // no lookup on this device before the capture
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace gs

extern "C" gs_status_t gs_sort_pairs_noalloc(uint64_t* keys, uint32_t* vals, int64_t n, int32_t key_bits,
                                             uint32_t* d_err_word, void* stream) {
  using namespace gs;
  if (n < 0 || key_bits < 1 || key_bits > 64) return GS_ERR_INVALID_ARG;
  if (n > kMaxPairs) return GS_ERR_SIZE_LIMIT;
  if (n == 0) return GS_OK;
  if (!keys || !vals) return GS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* base = nullptr;
  if (scratch_address(s, &base) != cudaSuccess) return GS_ERR_CUDA;
  SortArgs a{};
  a.keys[0] = keys;
  a.vals[0] = vals;
  a.keys[1] = at<uint64_t>(base, kOffKeys);
  a.vals[1] = at<uint32_t>(base, kOffVals);
  a.n_dev = nullptr;
  a.n_host = n;
  a.hist = at<uint32_t>(base, kOffHist);
  a.tile_status = at<uint32_t>(base, kOffStatus);
  a.tile_ctr = at<uint32_t>(base, kOffCtr);
  a.err = d_err_word;
  if (!a.err) {
    a.err = at<uint32_t>(base, kOffErr);
    if (cudaMemsetAsync(a.err, 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
  }
  a.max_tiles = kMaxTiles;
  a.passes = (key_bits + 7) / 8;
  a.key_bits = key_bits;
  cudaError_t e = launch_sort_prepare(a, s);
  if (e == cudaSuccess) e = launch_onesweep(a, s);
  if (e == cudaSuccess && (a.passes & 1)) {
    e = cudaMemcpyAsync(keys, a.keys[1], static_cast<size_t>(n) * 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vals, a.vals[1], static_cast<size_t>(n) * 4, cudaMemcpyDeviceToDevice, s);
  }
  return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
