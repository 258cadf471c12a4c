// api.cu -- the C ABI of libmpcg (declared in include/mpcg.h): argument
// checks on the host, workspace carving, and the stream-ordered sequence of
// kernels for each entry point.  No call synchronises the host; numerical
// outcomes reach the caller through the device-side result record.
#include <stdint.h>
#include <string.h>

#include "internal.h"

using namespace mpcg;

namespace {

// Barrier-counter slots of the persistent launches within one call.
enum Slot { kSlotCg64 = 0, kSlotPd = 1, kSlotCgK0 = 2, kSlotCg32 = 3, kSlotBfs = 4 };

}  // namespace

namespace mpcg {

bool options_ok(const mpcg_options_t* o) {
  if (!o) return false;
  if (!(o->eps2 >= 0.0)) return false;
  if (o->k0 < 0 || o->knn_k < 1 || o->knn_k > MPCG_KNN_MAX_K) return false;
  if (o->grid_blocks < 0 || o->timeout_ms < 0) return false;
  if (o->bfs_starts < 0) return false;
  if (o->precond != 0 && o->precond != 1) return false;
  if (o->stop_true_residual != 0 && o->stop_true_residual != 1) return false;
  if (o->acc32 != 0 && o->acc32 != 1) return false;
  if (o->spmv_variant != 0 && o->spmv_variant != 1) return false;
  return true;
}

bool sample_ok(const mpcg_sample_t* s) {
  return s && s->feat && s->cls && s->count >= 1 && s->count <= MPCG_KNN_MAX_SAMPLE;
}

}  // namespace mpcg

namespace {

int grid_size(int requested) {
  const void* kernels[1] = {bfs_kernel()};
  int g = kMaxGrid;
  for (const void* k : kernels) {
    int gk = persistent_grid(k, kCgThreads, requested);
    if (gk < g) g = gk;
  }
  return g;
}

int32_t prepare(const mpcg_csr_t* A, void* ws, size_t ws_bytes, mpcg_stream_t stream,
                int grid_req, Launch* L, int precond = 0) {
  if (!A || A->n <= 0 || A->nnz < 0 || !A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))
    return MPCG_ERR_INVALID_ARG;
  Dims d;
  if (!dims_for(A->n, A->nnz, &d)) return MPCG_ERR_INVALID_ARG;
  const size_t need = carve(d, nullptr, nullptr);
  if (!ws || ((uintptr_t)ws & 255u) || ws_bytes < need + precond_bytes(d.n, precond))
    return MPCG_ERR_WORKSPACE;
  carve(d, (char*)ws, &L->ws);
  L->precond = precond ? 1 : 0;
  L->true_res = 0;
  L->dinv64 = nullptr;
  L->dinv32 = nullptr;
  L->z32 = nullptr;
  if (precond) {  // the preconditioner arrays, past the workspace map (256-byte aligned)
    char* p = (char*)ws + need;
    const size_t n = (size_t)d.n;
    L->dinv64 = (double*)p;
    p += (sizeof(double) * n + 255) & ~(size_t)255;
    L->dinv32 = (float*)p;
    p += (sizeof(float) * n + 255) & ~(size_t)255;
    L->z32 = (float*)p;
  }
  L->d = d;
  L->A = A;
  L->st = (cudaStream_t)stream;
  L->grid_req = grid_req;
  L->grid = grid_size(grid_req);
  if (L->grid <= 0 || cg_grid(grid_req) <= 0) return MPCG_ERR_CUDA;
  return MPCG_OK;
}

int32_t cuda_status(cudaError_t e) { return e == cudaSuccess ? MPCG_OK : MPCG_ERR_CUDA; }

}  // namespace

extern "C" {

mpcg_options_t mpcg_options_default(void) {
  mpcg_options_t o;
  memset(&o, 0, sizeof(o));
  o.eps1 = -1.0;
  o.eps2 = 1e-10;
  o.k0 = 10;
  o.knn_k = 5;
  o.weighted = 1;
  o.tol_relative = 1;
  o.max_it_fp32 = 0;
  o.max_it_fp64 = 0;
  o.max_true_restarts = 2;
  o.feat_mask = 0xFu;
  o.fp64_only = 0;
  o.grid_blocks = 0;
  o.timeout_ms = 20000;
  o.bfs_starts = 1;
  o.precond = 0;
  o.stop_true_residual = 0;
  o.acc32 = 0;
  o.spmv_variant = 0;
  return o;
}

const char* mpcg_status_string(int32_t s) {
  switch (s) {
    case MPCG_OK: return "ok";
    case MPCG_WARN_EPS1_NOT_REACHED: return "warning: eps1 not reached in single precision";
    case MPCG_WARN_TRUE_RESID_RESTARTED: return "warning: FP64 stage restarted on the true residual";
    case MPCG_ERR_INVALID_ARG: return "invalid argument";
    case MPCG_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case MPCG_ERR_BREAKDOWN: return "breakdown: d^T A d <= 0 (matrix not SPD)";
    case MPCG_ERR_NAN: return "non-finite value";
    case MPCG_ERR_NOT_CONVERGED:
      return "FP64 stage did not reach eps2 (iteration cap, or true residual after the last restart)";
    case MPCG_ERR_TIMEOUT: return "device-side wait timed out";
    case MPCG_ERR_CUDA: return "CUDA error";
    case MPCG_ERR_CANCELLED: return "cancelled";
    case MPCG_ERR_UNIMPLEMENTED: return "unimplemented";
    default: return "unknown status";
  }
}

size_t mpcg_workspace_bytes(int32_t n, int32_t nnz, const mpcg_options_t* opts) {
  Dims d;
  if (!dims_for(n, nnz, &d)) return 0;
  return carve(d, nullptr, nullptr) + precond_bytes(d.n, opts ? opts->precond : 0);
}

int32_t mpcg_features(const mpcg_csr_t* A, const double* b, const mpcg_options_t* opts,
                      void* ws, size_t ws_bytes, mpcg_features_t* out, mpcg_stream_t stream) {
  if (!b || !out || !options_ok(opts)) return MPCG_ERR_INVALID_ARG;
  Launch L;
  int32_t st = prepare(A, ws, ws_bytes, stream, opts->grid_blocks, &L, opts->precond);
  if (st != MPCG_OK) return st;
  L.true_res = opts->stop_true_residual;
  cudaError_t e;
  if ((e = launch_init(L, *opts, 0)) != cudaSuccess) return cuda_status(e);
  if ((e = launch_prep(L, b)) != cudaSuccess) return cuda_status(e);
  if (L.precond && (e = launch_jacobi(L)) != cudaSuccess) return cuda_status(e);
  if ((e = launch_pseudo_diameter(L, kSlotPd)) != cudaSuccess) return cuda_status(e);
  if ((e = launch_cg32(L, kCgK0, kSlotCgK0)) != cudaSuccess) return cuda_status(e);
  return cuda_status(launch_finalize(L, nullptr, out));
}

int32_t mpcg_choose_eps1(const mpcg_features_t* f, const mpcg_sample_t* sample,
                         const mpcg_options_t* opts, double* eps1_out, int32_t* cls_out,
                         mpcg_stream_t stream) {
  if (!f || !options_ok(opts) || !sample_ok(sample) || (!eps1_out && !cls_out))
    return MPCG_ERR_INVALID_ARG;
  return cuda_status(launch_knn((cudaStream_t)stream, (const double*)f, *sample, *opts, nullptr,
                                eps1_out, cls_out));
}

int32_t mpcg_knn_batch(const mpcg_sample_t* sample, const double* chi, int32_t count,
                       const mpcg_options_t* opts, int32_t* cls_out, int32_t* nbr_out,
                       mpcg_stream_t stream) {
  if (count < 0 || (count > 0 && (!chi || !cls_out)) || !options_ok(opts) || !sample_ok(sample))
    return MPCG_ERR_INVALID_ARG;
  return cuda_status(launch_knn_batch((cudaStream_t)stream, *sample, *opts, chi, count, cls_out,
                                      nbr_out));
}

int32_t mpcg_solve(const mpcg_csr_t* A, const double* b, double* x, const mpcg_sample_t* sample,
                   const mpcg_options_t* opts, void* ws, size_t ws_bytes, mpcg_result_t* res,
                   mpcg_stream_t stream) {
  if (!b || !x || !res || !options_ok(opts)) return MPCG_ERR_INVALID_ARG;
  const int fp64_only = opts->fp64_only != 0;
  const int auto_eps1 = !fp64_only && !(opts->eps1 > 0.0);
  if (auto_eps1 && !sample_ok(sample)) return MPCG_ERR_INVALID_ARG;
  Launch L;
  int32_t st = prepare(A, ws, ws_bytes, stream, opts->grid_blocks, &L, opts->precond);
  if (st != MPCG_OK) return st;
  L.true_res = opts->stop_true_residual;
  cudaError_t e;
  if ((e = launch_init(L, *opts, fp64_only)) != cudaSuccess) return cuda_status(e);
  if ((e = launch_prep(L, b)) != cudaSuccess) return cuda_status(e);
  if (L.precond && (e = launch_jacobi(L)) != cudaSuccess) return cuda_status(e);
  if (!fp64_only && auto_eps1 && (L.precond || L.true_res)) {
    // Algorithm II with Jacobi PCG or with the stop test on b - A x, its
    // steps as separate launches in the paper's order: 2BFS, k0 iterations
    // (v), kNN, stage 1 from iterate k0
    if ((e = launch_pseudo_diameter(L, kSlotPd)) != cudaSuccess) return cuda_status(e);
    if ((e = launch_cg32(L, kCgK0, kSlotCgK0)) != cudaSuccess) return cuda_status(e);
    if ((e = launch_knn(L.st, nullptr, *sample, *opts, L.ws.ctl, nullptr, nullptr)) != cudaSuccess)
      return cuda_status(e);
    if ((e = launch_cg32(L, kCgContinue, kSlotCg32)) != cudaSuccess) return cuda_status(e);
  } else if (!fp64_only) {
    if (auto_eps1) {  // Algorithm II: features, kNN and stage 1 in one fused launch
      if ((e = launch_stage1(L, *sample, *opts, kSlotCg32, kSlotPd)) != cudaSuccess)
        return cuda_status(e);
    } else {  // Algorithm I
      if ((e = launch_cg32(L, kCgToEps1, kSlotCg32)) != cudaSuccess) return cuda_status(e);
    }
  }
  if (opts->stage1_only && !fp64_only) {
    if ((e = launch_promote(L, x)) != cudaSuccess) return cuda_status(e);
  } else {
    if ((e = launch_cg64(L, b, x, fp64_only, kSlotCg64)) != cudaSuccess) return cuda_status(e);
  }
  return cuda_status(launch_finalize(L, res, nullptr));
}

int32_t mpcg_spmv(const mpcg_csr_t* A, int32_t fp32, const void* x, void* y, void* ws,
                  size_t ws_bytes, mpcg_stream_t stream) {
  if (!x || !y) return MPCG_ERR_INVALID_ARG;
  Launch L;
  mpcg_options_t o = mpcg_options_default();
  int32_t st = prepare(A, ws, ws_bytes, stream, 0, &L);
  if (st != MPCG_OK) return st;
  cudaError_t e;
  if ((e = launch_init(L, o, 0)) != cudaSuccess) return cuda_status(e);
  if ((e = launch_prep(L, nullptr)) != cudaSuccess) return cuda_status(e);
  return cuda_status(launch_spmv(L, fp32, x, y));
}

int32_t mpcg_bfs(const mpcg_csr_t* A, int32_t src, int32_t* dist, void* ws, size_t ws_bytes,
                 mpcg_stream_t stream) {
  if (!dist || !A || src < 0 || src >= A->n) return MPCG_ERR_INVALID_ARG;
  Launch L;
  mpcg_options_t o = mpcg_options_default();
  int32_t st = prepare(A, ws, ws_bytes, stream, 0, &L);
  if (st != MPCG_OK) return st;
  cudaError_t e;
  if ((e = launch_init(L, o, 0)) != cudaSuccess) return cuda_status(e);
  if ((e = launch_prep(L, nullptr)) != cudaSuccess) return cuda_status(e);
  return cuda_status(launch_bfs_only(L, src, dist, kSlotBfs));
}

int32_t mpcg_pseudo_diameter(const mpcg_csr_t* A, int32_t* out, void* ws, size_t ws_bytes,
                             mpcg_stream_t stream) {
  if (!out) return MPCG_ERR_INVALID_ARG;
  Launch L;
  mpcg_options_t o = mpcg_options_default();
  int32_t st = prepare(A, ws, ws_bytes, stream, 0, &L);
  if (st != MPCG_OK) return st;
  cudaError_t e;
  if ((e = launch_init(L, o, 0)) != cudaSuccess) return cuda_status(e);
  if ((e = launch_prep(L, nullptr)) != cudaSuccess) return cuda_status(e);
  if ((e = launch_pseudo_diameter(L, kSlotPd)) != cudaSuccess) return cuda_status(e);
  return cuda_status(launch_copy_pdiam(L, out));
}

}  // extern "C"
