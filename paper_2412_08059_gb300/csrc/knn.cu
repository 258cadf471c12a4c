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

cudaError_t launch_knn(cudaStream_t st, const double* feat4, const mpcg_sample_t& S,
                       const mpcg_options_t& o, Ctl* ctl, double* eps1_out, int32_t* cls_out) {
  k_knn<<<1, 32, 0, st>>>(knn_spec(S, o), ctl, feat4, eps1_out, cls_out);
  return cudaGetLastError();
}

}  // namespace mpcg
