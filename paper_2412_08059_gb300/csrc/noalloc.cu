// noalloc.cu -- mpcg_solve_static: mpcg_solve with its scratch carved from a
// fixed device array of this library instead of a caller's workspace.  It
// allocates nothing (no cudaMalloc, no cudaFree); the array is mapped when
// the library's device code is loaded on the device.
#include "internal.h"

namespace {

// One array per device (a __device__ variable is instantiated per device).
// 256-byte alignment is what the workspace carving requires.
static __device__ __align__(256) unsigned char g_static_ws[MPCG_STATIC_WS_BYTES];

}  // namespace

extern "C" int32_t mpcg_solve_static(const mpcg_csr_t* A, const double* b, double* x,
                                     const mpcg_sample_t* sample, const mpcg_options_t* opts,
                                     mpcg_result_t* res, mpcg_stream_t stream) {
  // The checks mpcg_solve makes on its own arguments come first, so that a
  // bad option is reported as such and not as a size problem.
  if (!A || !b || !x || !res || !mpcg::options_ok(opts)) return MPCG_ERR_INVALID_ARG;
  const size_t need = mpcg_workspace_bytes(A->n, A->nnz, opts);
  if (need == 0) return MPCG_ERR_INVALID_ARG;
  if (need > (size_t)MPCG_STATIC_WS_BYTES) return MPCG_ERR_WORKSPACE;  // too large for the array
  // The host-side name g_static_ws is not a device address.  The address is
  // looked up on every call, in the caller's current context: a cached one
  // could name the array of another context (a non-primary one, or one
  // created after cudaDeviceReset) and the kernels would then write to
  // memory that is not theirs.  The lookup costs far less than a solve.
  void* ws = nullptr;
  if (cudaGetSymbolAddress(&ws, g_static_ws) != cudaSuccess || !ws) {
    (void)cudaGetLastError();  // leave no pending error for the caller's next launch
    return MPCG_ERR_CUDA;
  }
  // mpcg_solve clears the control block (the only part of the scratch that
  // must start at zero) on `stream` before its first kernel; every other
  // region is written before it is read.
  return mpcg_solve(A, b, x, sample, opts, ws, (size_t)MPCG_STATIC_WS_BYTES, res, stream);
}
