// internal.h -- host-side interfaces between the translation units of libmpcg.
#pragma once
#include <cuda_runtime.h>

#include "bfs_core.cuh"
#include "common.cuh"
#include "knn_core.cuh"

namespace mpcg {

// Layout parameters that depend only on (n, nnz): rows per slice is fixed at
// 32; a slice stores at most `wcap` entries per row in the sliced arrays,
// and the rest of a longer row is read from the caller's CSR.
struct Dims {
  int n, nnz, nslices, wcap;
  long long pcap;  // capacity of the sliced arrays (elements)
};

bool dims_for(int n, int nnz, Dims* d);
size_t carve(const Dims& d, char* base, Ws* ws);  // base == nullptr: size only

struct Launch {
  Dims d;
  Ws ws;
  const mpcg_csr_t* A;
  cudaStream_t st;
  int grid;      // persistent grid of the BFS / component kernels
  int grid_req;  // requested grid (0 = one full wave)
  // Jacobi preconditioning (option precond), carved past the workspace map
  int precond;
  double* dinv64;  // 1 / a_ii
  float* dinv32;   // 1 / float32(a_ii)
  float* z32;      // z = dinv32 r of the single-precision stage
  int true_res;    // stop tests on b - A x (option stop_true_residual)
};

// Bytes of the preconditioner arrays past the workspace map (0 without).
size_t precond_bytes(int n, int precond);

int persistent_grid(const void* kernel, int threads, int requested, size_t dyn_smem = 0);

// api.cu: host checks shared by the entry points
bool options_ok(const mpcg_options_t* o);
bool sample_ok(const mpcg_sample_t* s);

// prep.cu
cudaError_t launch_init(const Launch& L, const mpcg_options_t& o, int fp64_only);
cudaError_t launch_jacobi(const Launch& L);
cudaError_t launch_prep(const Launch& L, const double* b);
cudaError_t launch_finalize(const Launch& L, mpcg_result_t* res, mpcg_features_t* feat);

// cg.cu
enum Cg32Mode { kCgK0 = 0, kCgToEps1 = 1, kCgContinue = 2 };
cudaError_t launch_cg32(const Launch& L, int mode, int slot);
cudaError_t launch_cg64(const Launch& L, const double* b, double* x, int from_zero, int slot);
cudaError_t launch_spmv(const Launch& L, int fp32, const void* x, void* y);
cudaError_t launch_promote(const Launch& L, double* x);
// Fused stage 1 of Algorithm II: 2BFS + k0 iterations + kNN + CG to eps1.
cudaError_t launch_stage1(const Launch& L, const mpcg_sample_t& S, const mpcg_options_t& o,
                          int slot, int bfs_slot);
const void* stage1_kernel();
const void* cg32_kernel();
const void* cg64_kernel();
int cg_grid(int requested);

// bfs.cu
BfsGraph bfs_graph(const Launch& L);
cudaError_t launch_pseudo_diameter(const Launch& L, int slot);
cudaError_t launch_bfs_only(const Launch& L, int src, int32_t* dist, int slot);
cudaError_t launch_copy_pdiam(const Launch& L, int32_t* out);
const void* bfs_kernel();

// knn.cu
KnnSpec knn_spec(const mpcg_sample_t& S, const mpcg_options_t& o);
cudaError_t launch_knn(cudaStream_t st, const double* feat4, const mpcg_sample_t& S,
                       const mpcg_options_t& o, Ctl* ctl, double* eps1_out, int32_t* cls_out);
cudaError_t launch_knn_batch(cudaStream_t st, const mpcg_sample_t& S, const mpcg_options_t& o,
                             const double* chi4, int count, int32_t* cls, int32_t* nbr);

}  // namespace mpcg
