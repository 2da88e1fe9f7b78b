// Sharing a Gaussian map between processes on one GPU (Sec. III, Fig. 5: the map optimiser and
// the interactive viewer run as separate processes, each with its own renderer, and both read
// the map where it lives in GPU memory through CUDA IPC).
//
// Memory: the exporter names any device pointer inside a cudaMalloc allocation; the handle
// carries the allocation's IPC handle plus the pointer's offset and the byte count, so a
// sub-range of a larger allocation (a caching allocator's block) can be shared. The importer
// maps the allocation and gets the same bytes back at its own address.
// Ordering: an interprocess event (no timing). The exporter records it on its stream after an
// update of the map; the importer makes its stream wait on it before reading, so a render
// starts after the last update recorded before the wait was enqueued. The exporter is not held
// back by the importer: an update enqueued after that record may run while the importer reads
// (a render can see a mix of two consecutive updates).
#include <cuda.h>
#include <string.h>

#include <mutex>
#include <unordered_map>

#include "gs_internal.cuh"

namespace gs {
namespace {

struct MemHandle {
  cudaIpcMemHandle_t h;
  uint64_t offset, bytes;
};
static_assert(sizeof(MemHandle) <= sizeof(gs_ipc_mem_handle_t), "IPC memory handle does not fit");
static_assert(sizeof(cudaIpcEventHandle_t) <= sizeof(gs_ipc_event_handle_t), "IPC event handle does not fit");

std::mutex g_mu;
std::unordered_map<uintptr_t, void*>& imported() {  // imported pointer -> mapped allocation base
  static std::unordered_map<uintptr_t, void*> m;
  return m;
}

using GetRangeFn = CUresult (*)(CUdeviceptr*, size_t*, CUdeviceptr);

bool allocation_range(const void* p, uintptr_t* base, size_t* size) {
  static GetRangeFn fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f)
      return false;
    fn = reinterpret_cast<GetRangeFn>(f);
  }
  CUdeviceptr b = 0;
  size_t s = 0;
  if (fn(&b, &s, reinterpret_cast<CUdeviceptr>(p)) != CUDA_SUCCESS) return false;
  *base = static_cast<uintptr_t>(b);
  *size = s;
  return true;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status_t gs_ipc_export(const void* d_ptr, size_t bytes, gs_ipc_mem_handle_t* out) {
  if (!d_ptr || !out || bytes == 0) return GS_ERR_INVALID_ARG;
  uintptr_t base = 0;
  size_t size = 0;
  if (!allocation_range(d_ptr, &base, &size)) return GS_ERR_CUDA;
  const uintptr_t p = reinterpret_cast<uintptr_t>(d_ptr);
  if (p < base || p + bytes > base + size) return GS_ERR_INVALID_ARG;
  MemHandle h{};
  if (cudaIpcGetMemHandle(&h.h, reinterpret_cast<void*>(base)) != cudaSuccess) return GS_ERR_CUDA;
  h.offset = p - base;
  h.bytes = bytes;
  memset(out, 0, sizeof(*out));
  memcpy(out->bytes, &h, sizeof(h));
  return GS_OK;
}

extern "C" gs_status_t gs_ipc_import(const gs_ipc_mem_handle_t* handle, void** d_ptr, size_t* bytes) {
  if (!handle || !d_ptr) return GS_ERR_INVALID_ARG;
  MemHandle h;
  memcpy(&h, handle->bytes, sizeof(h));
  if (h.bytes == 0) return GS_ERR_INVALID_ARG;
  void* base = nullptr;
  if (cudaIpcOpenMemHandle(&base, h.h, cudaIpcMemLazyEnablePeerAccess) != cudaSuccess) return GS_ERR_CUDA;
  void* p = static_cast<uint8_t*>(base) + h.offset;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    imported()[reinterpret_cast<uintptr_t>(p)] = base;
  }
  *d_ptr = p;
  if (bytes) *bytes = h.bytes;
  return GS_OK;
}

extern "C" gs_status_t gs_ipc_release(void* d_ptr) {
  if (!d_ptr) return GS_ERR_INVALID_ARG;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = imported().find(reinterpret_cast<uintptr_t>(d_ptr));
    if (it == imported().end()) return GS_ERR_INVALID_ARG;
    base = it->second;
    imported().erase(it);
  }
  return cudaIpcCloseMemHandle(base) == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

extern "C" gs_status_t gs_ipc_event_create(void** event, gs_ipc_event_handle_t* out) {
  if (!event || !out) return GS_ERR_INVALID_ARG;
  cudaEvent_t e = nullptr;
  if (cudaEventCreateWithFlags(&e, cudaEventInterprocess | cudaEventDisableTiming) != cudaSuccess) return GS_ERR_CUDA;
  cudaIpcEventHandle_t h;
  if (cudaIpcGetEventHandle(&h, e) != cudaSuccess) {
    cudaEventDestroy(e);
    return GS_ERR_CUDA;
  }
  memset(out, 0, sizeof(*out));
  memcpy(out->bytes, &h, sizeof(h));
  *event = e;
  return GS_OK;
}

extern "C" gs_status_t gs_ipc_event_open(const gs_ipc_event_handle_t* handle, void** event) {
  if (!handle || !event) return GS_ERR_INVALID_ARG;
  cudaIpcEventHandle_t h;
  memcpy(&h, handle->bytes, sizeof(h));
  cudaEvent_t e = nullptr;
  if (cudaIpcOpenEventHandle(&e, h) != cudaSuccess) return GS_ERR_CUDA;
  *event = e;
  return GS_OK;
}

extern "C" gs_status_t gs_ipc_event_record(void* event, void* stream) {
  if (!event) return GS_ERR_INVALID_ARG;
  return cudaEventRecord(static_cast<cudaEvent_t>(event), static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? GS_OK
             : GS_ERR_CUDA;
}

extern "C" gs_status_t gs_ipc_stream_wait(void* stream, void* event) {
  if (!event) return GS_ERR_INVALID_ARG;
  return cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), static_cast<cudaEvent_t>(event), 0) == cudaSuccess
             ? GS_OK
             : GS_ERR_CUDA;
}

extern "C" gs_status_t gs_ipc_event_destroy(void* event) {
  if (!event) return GS_ERR_INVALID_ARG;
  return cudaEventDestroy(static_cast<cudaEvent_t>(event)) == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
