// Coarse solve for callers that may not allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they need a coarse solve: code that runs
// under a memory manager that forbids allocations outside its own pool, code on a latency path
// where cudaMalloc's implicit device synchronisation is not acceptable, or code that has
// already handed the rest of the device to another allocator.  amg_coarse_solve allocates its
// Krylov workspace on first use; this variant instead uses a fixed scratch array compiled into
// the library, so it allocates nothing.
//
// The scratch is a file-scope __device__ array of AMG_NOALLOC_SCRATCH_BYTES.  Every GPU that
// loads the library holds it until the process exits, and every call shares it: two calls whose
// kernels overlap on the GPU (different streams, or different host threads on one device)
// overwrite each other's workspace.  Each call clears the parts of the array that must start at
// zero (the convergence flags and counters) before use.
//
// Host code may not hand the array's name to a kernel: on the host that name is only a
// stand-in for the device symbol.  The device address is looked up with cudaGetSymbolAddress
// once per device, with that device current, on the first call made on that device; that first
// call should therefore come before any stream capture begins.  The looked-up address is kept
// until the process exits: after a cudaDeviceReset it is stale (as is every handle), so a
// process that resets a device must not call the library on it again.
//
// The call never stops early on the host: it queues every application of the max_applies
// budget, and kernels queued after convergence return at once.
#include "amg_internal.cuh"

#include <mutex>

#define AMG_NOALLOC_SCRATCH_BYTES (16u << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[AMG_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_scratch_ptr[kMaxDevices] = {};

amg_status scratch_address(void** out) {
  int dev = 0;
  AMG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return AMG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    AMG_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return AMG_OK;
}

}  // namespace

extern "C" {

amg_status amg_coarse_solve_noalloc(amg_handle h, const void* d_b, void* d_x, int nrhs, double tol,
                                    int restart, int max_applies, void* stream, double* info) {
  if (!h || !d_b || !d_x || d_b == d_x || !aligned16(d_b) || !aligned16(d_x)) return AMG_ERR_INVALID_ARG;
  if (nrhs < 1 || nrhs > h->p.max_nrhs || nrhs > 16 || !(tol >= 0)) return AMG_ERR_INVALID_ARG;
  if (restart < 1 || restart > AMG_MAX_NTV || max_applies < 1) return AMG_ERR_INVALID_ARG;
  const size_t need = amg_internal_solve_bytes(h, nrhs, restart);
  if (need > AMG_NOALLOC_SCRATCH_BYTES) {
    amg_note_error("amg_coarse_solve_noalloc: workspace of %zu bytes exceeds the %u-byte scratch array",
                   need, AMG_NOALLOC_SCRATCH_BYTES);
    return AMG_ERR_INVALID_ARG;
  }
  void* ws = nullptr;
  amg_status s = scratch_address(&ws);
  if (s != AMG_OK) return s;
  h->last_stream = (cudaStream_t)stream;
  return amg_internal_solve_ws(h, d_b, d_x, nrhs, tol, restart, max_applies, (cudaStream_t)stream, info, ws,
                               false);
}

size_t amg_noalloc_scratch_bytes(void) { return AMG_NOALLOC_SCRATCH_BYTES; }

}  // extern "C"
