// static_ws.cu -- hull_compute_static: the whole method on at most
// HULL_STATIC_MAX_POINTS points with its workspace in a file-scope device
// array, so that the call allocates nothing.
//
// Callers that cannot allocate: a latency-bound loop (cudaMalloc and cudaFree
// may synchronise the whole device and stall every other stream), and a host
// program that reserved all of the device's memory up front or has no
// allocator of its own to size a workspace with.  Such a caller gets a fixed,
// modest scratch (about 26 MiB, in the module's static data) instead of a
// caller-owned workspace.
//
// The kernels are those of hull_compute; only the workspace differs.  The
// parts of the scratch that must start at zero (the header: status flags,
// survivor and escalation counters, the refinement bins) are cleared by every
// call on its stream before its first kernel; everything else is written
// before it is read.  One scratch per device: calls on one device that may
// overlap on the GPU race on it.
#include <mutex>

#include "internal.cuh"

namespace {

// The workspace of hull_compute for HULL_STATIC_MAX_POINTS points is
// 27,027,456 bytes; the margin keeps the size a whole number of MiB.
constexpr size_t STATIC_SCRATCH_BYTES = size_t(26) << 20;

static __device__ __align__(256) unsigned char g_scratch[STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_ptr[MAX_DEVICES] = {};

// Set-up, once per device, with that device current: the device address of
// g_scratch.  Returns nullptr when the query fails.  The address is cached
// for the process; cudaDeviceReset unloads the module and makes it stale,
// so the header tells callers not to use this entry point on a device after
// resetting it.
void* scratch_of_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return nullptr;
    g_ptr[dev] = ptr;
  }
  return g_ptr[dev];
}

}  // namespace

extern "C" hull_status hull_compute_static(const float* d_xy, int64_t n, uint32_t* d_hull_idx, int64_t* d_n_hull,
                                           const hull_options* opt, void* stream) {
  if (n < 0) return HULL_ERR_INVALID_ARG;
  if (n > HULL_STATIC_MAX_POINTS) return HULL_ERR_BUDGET;
  if (hull_workspace_bytes(n, opt) > STATIC_SCRATCH_BYTES) return HULL_ERR_BUDGET;
  void* ws = scratch_of_current_device();
  if (!ws) return HULL_ERR_CUDA;
  return hull_compute(d_xy, n, ws, STATIC_SCRATCH_BYTES, d_hull_idx, d_n_hull, opt, stream);
}
