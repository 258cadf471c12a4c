// noalloc.cu -- mpcg_solve_static: mpcg_solve with its scratch carved from a
// fixed device array of this library instead of a caller's workspace.  It
// allocates nothing (no cudaMalloc, no cudaFree); the array is mapped when
// the library's device code is loaded on the device.
#include <mutex>

#include "internal.h"

namespace {

// One array per device (a __device__ variable is instantiated per device).
// 256-byte alignment is what the workspace carving requires.
static __device__ __align__(256) unsigned char g_static_ws[MPCG_STATIC_WS_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices];  // device address of g_static_ws, looked up once per device

// Address of g_static_ws on the current device; nullptr on failure.
void* static_ws_address() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    // the current device is `dev`: the lookup resolves the symbol there
    if (cudaGetSymbolAddress(&p, g_static_ws) != cudaSuccess) return nullptr;
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

}  // namespace

extern "C" int32_t mpcg_solve_static(const mpcg_csr_t* A, const double* b, double* x,
                                     const mpcg_sample_t* sample, const mpcg_options_t* opts,
                                     mpcg_result_t* res, mpcg_stream_t stream) {
  if (!A || !b || !x || !res || !opts) return MPCG_ERR_INVALID_ARG;
  const size_t need = mpcg_workspace_bytes(A->n, A->nnz, opts);
  if (need == 0) return MPCG_ERR_INVALID_ARG;
  if (need > (size_t)MPCG_STATIC_WS_BYTES) return MPCG_ERR_WORKSPACE;  // too large for the array
  void* ws = static_ws_address();
  if (!ws) return MPCG_ERR_CUDA;
  // mpcg_solve clears the control block (the only part of the scratch that
  // must start at zero) on `stream` before its first kernel; every other
  // region is written before it is read.
  return mpcg_solve(A, b, x, sample, opts, ws, (size_t)MPCG_STATIC_WS_BYTES, res, stream);
}
