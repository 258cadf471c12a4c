// knn.cu -- standalone kernel for the choice of eps1 by kNN (Sec. 11); the
// vote itself is knn_warp in knn_core.cuh.
#include "internal.h"
#include "knn_core.cuh"

namespace mpcg {

// q4: device query (n, m, l~, v); nullptr: take it from the control block.
// ctl nullable: then errors are reported as cls_out = -1, eps1_out = NaN.
__global__ void k_knn(KnnSpec s, Ctl* ctl, const double* q4, double* eps1_out,
                      int32_t* cls_out) {
  if (ctl && volatile_status(ctl) != 0) return;
  double chi[4];
  if (q4) {
    for (int c = 0; c < 4; ++c) chi[c] = q4[c];
  } else {
    chi[0] = (double)ctl->n;
    chi[1] = (double)ctl->nnz;
    chi[2] = (double)ctl->pdiam;
    chi[3] = ctl->v;
  }
  const int t = knn_warp(s, chi);
  if (threadIdx.x != 0) return;
  if (t < 0) {
    if (ctl) set_status(ctl, MPCG_ERR_INVALID_ARG);
    if (cls_out) *cls_out = -1;
    if (eps1_out) *eps1_out = NAN;
  } else {
    if (ctl) {
      ctl->cls = t;
      ctl->eps1 = pow10_neg(t);
    }
    if (cls_out) *cls_out = t;
    if (eps1_out) *eps1_out = pow10_neg(t);
  }
  if (ctl) ctl->t_features = globaltimer();
}

KnnSpec knn_spec(const mpcg_sample_t& S, const mpcg_options_t& o) {
  KnnSpec s{};
  s.feat = S.feat;
  s.cls = S.cls;
  s.count = S.count;
  s.k = o.knn_k;
  s.weighted = o.weighted;
  s.mask = o.feat_mask;
  for (int c = 0; c < 4; ++c) {
    s.fmin[c] = S.fmin[c];
    s.fmax[c] = S.fmax[c];
  }
  return s;
}

// Many queries (the classification of a test set, Sec. 12): one warp per
// query, grid-stride.  chi: [count][4]; cls: [count]; nbr: [count][k] or null.
__global__ void k_knn_batch(KnnSpec s, const double* chi4, int count, int32_t* cls,
                            int32_t* nbr) {
  const int warps = (int)(gridDim.x * blockDim.x) >> 5;
  const int w0 = (int)(blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int qi = w0; qi < count; qi += warps) {  // warp-uniform
    double chi[4];
    for (int c = 0; c < 4; ++c) chi[c] = chi4[4 * (size_t)qi + c];
    const int t = knn_warp(s, chi);
    if ((threadIdx.x & 31) == 0) cls[qi] = t;
    if (nbr && !knn_neighbours_warp(s, chi, nbr + (size_t)qi * s.k) && (threadIdx.x & 31) == 0)
      for (int j = 0; j < s.k; ++j) nbr[(size_t)qi * s.k + j] = -1;
  }
}

cudaError_t launch_knn_batch(cudaStream_t st, const mpcg_sample_t& S, const mpcg_options_t& o,
                             const double* chi4, int count, int32_t* cls, int32_t* nbr) {
  if (count <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaErrorUnknown;
  const int threads = 256;                                   // 8 queries per block at a time
  const int need = (count + threads / 32 - 1) / (threads / 32);
  const int grid = need < 8 * sms ? need : 8 * sms;
  k_knn_batch<<<grid, threads, 0, st>>>(knn_spec(S, o), chi4, count, cls, nbr);
  return cudaGetLastError();
}

cudaError_t launch_knn(cudaStream_t st, const double* feat4, const mpcg_sample_t& S,
                       const mpcg_options_t& o, Ctl* ctl, double* eps1_out, int32_t* cls_out) {
  k_knn<<<1, 32, 0, st>>>(knn_spec(S, o), ctl, feat4, eps1_out, cls_out);
  return cudaGetLastError();
}

}  // namespace mpcg
