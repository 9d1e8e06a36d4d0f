// dls_compress_noalloc: compression for callers that cannot allocate device
// memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the
// moment they want to compress: an in-situ compression hook running inside a
// simulation that has already handed all device memory to its own pools, a
// host callback where CUDA API allocation is not allowed, or a real-time loop
// with a fixed memory budget.  This entry point gives them the same
// compression as dls_compress with the workspace taken from a statically sized
// device array that lives in this library, so the caller passes only the input
// field and the output buffer.
//
// The array is 64 MiB and every GPU on which this library is loaded keeps it
// until the process exits.  Under CUDA's lazy module loading (the default) the
// array is placed in device memory when the first call on a device looks up
// its address, so that first call needs 64 MiB of free device memory: make it
// before the caller's pools take the device (or load modules eagerly with
// CUDA_MODULE_LOADING=EAGER).  All calls share it: overlapping calls (two
// streams, two host threads) race on it and must be serialised by the caller.
// The previous call's contents are left in it; dls_compress clears the status
// words it reads and writes every other workspace entry before reading it.
#include <mutex>

#include "dls_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;

// Device-side scratch.  In host code `g_noalloc_scratch` is only a host-side
// stand-in for the symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};

// Resolves the scratch address on the current device, once per device.
int scratch_on_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DLS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DLS_ERR_CUDA;
    g_dev_ptr[dev] = p;
  }
  *out = g_dev_ptr[dev];
  return DLS_OK;
}

}  // namespace

extern "C" int dls_compress_noalloc(const dls_params* p, const void* d_in, void* d_out, size_t out_cap,
                                    size_t* out_bytes, dls_stream_t stream) {
  // invalid parameters report what dls_compress would report for them
  dls::Plan P;
  const int pst = dls::make_plan(p, &P);
  if (pst != DLS_OK) return pst;
  const size_t need = dls_workspace_size(p);
  if (need == 0) return DLS_ERR_INVALID_ARG;
  if (need > kNoAllocScratchBytes) return DLS_ERR_WORKSPACE;
  void* ws = nullptr;
  const int st = scratch_on_current_device(&ws);
  if (st != DLS_OK) return st;
  return dls_compress(p, d_in, d_out, out_cap, out_bytes, ws, kNoAllocScratchBytes, stream);
}
