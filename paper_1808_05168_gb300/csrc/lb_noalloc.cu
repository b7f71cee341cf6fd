// lb_noalloc.cu -- lb_power_spectrum_noalloc: the one-snapshot power spectrum for callers that
// must not allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point where they need
// a spectrum: code running while a CUDA graph is being captured on a stream it does not own,
// code in a process whose device memory pool is owned by another framework, or a real-time loop
// that must never block on the allocator.  This entry point uses a fixed scratch area compiled
// into the library instead: a file-scope __device__ array of kNoAllocMaxPoints complex doubles
// (4 MiB), which every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "lb_internal.cuh"

namespace {

constexpr int kNoAllocMaxPoints = 1 << 18;  // Lx * Lz limit (LB_NOALLOC_MAX_POINTS in lb.h)
static_assert(kNoAllocMaxPoints == LB_NOALLOC_MAX_POINTS, "limit out of sync with lb.h");

// Intermediate row transforms (Lx * Lz complex values).  Each call overwrites the part it uses
// before reading it, so nothing needs clearing between calls; calls that overlap on the GPU
// (two streams, or two host threads) race on it.
static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocMaxPoints];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// Once per device, with that device current: the array's device address (the host-side name of
// g_noalloc_scratch is only a stand-in and must never reach a kernel) and the kernels'
// shared-memory attributes.
int setup_current_device(void** scratch) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LB_ERR_CUDA;
  {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return LB_ERR_CUDA;
      }
      g_scratch_addr[dev] = p;
    }
    *scratch = g_scratch_addr[dev];
  }
  return lbk::prepare_power_spectrum_current_device();
}

}  // namespace

extern "C" int lb_power_spectrum_noalloc(const double* field, int Lx, int Lz, double* out, void* stream) {
  // the checks of lb_power_spectrum (sizes 2..8192, powers of two, device memory of the current
  // device: LB_ERR_BAD_PARAM), then the array's own limit (LB_ERR_SIZE)
  int rc = lbk::power_spectrum_args_ok(field, Lx, Lz, out);
  if (rc) return rc;
  if ((long long)Lx * Lz > kNoAllocMaxPoints) return LB_ERR_SIZE;
  void* scratch = nullptr;
  rc = setup_current_device(&scratch);
  if (rc) return rc;
  if (lbk::launch_power_spectrum(field, Lx, Lz, out, scratch, (cudaStream_t)stream) != cudaSuccess)
    return LB_ERR_CUDA;
  return LB_OK;
}
