// knn.cu -- choice of eps1 by the k-nearest-neighbours vote of Sec. 11.
//
// One block, no scratch memory: distances are recomputed in each selection
// round (the same arithmetic, so the same values).  Each feature component is min-max scaled with the sample's
// min and max (Sec. 11.1; the query is not clamped; a constant component
// maps to 0).  The squared Euclidean distance (Sec. 11.5) is summed over the
// selected components in index order.  The k nearest are the k smallest
// pairs (d2, index), found by k block-wide selections of the smallest pair
// above the previous one.  Vote: weight 1/sqrt(d2) (Eq. 23) or 1 (Eq. 22),
// summed in selection order; when a selected neighbour is at distance 0
// only the zero-distance neighbours vote, by count; ties go to the smallest
// class t.  Every operation is an explicit IEEE-rounded intrinsic, so the
// result does not depend on compiler contraction.
#include <math.h>

#include "internal.h"

namespace mpcg {

constexpr int kKnnThreads = 1024;

__device__ __constant__ double kPow10Neg[16] = {1e0,  1e-1,  1e-2,  1e-3,  1e-4,  1e-5,
                                                 1e-6, 1e-7,  1e-8,  1e-9,  1e-10, 1e-11,
                                                 1e-12, 1e-13, 1e-14, 1e-15};

struct KnnArgs {
  Ctl* ctl;          // nullable: then errors are reported as cls_out = -1
  const double* q4;  // device query (n, m, l~, v); nullptr: take it from ctl
  const double* feat;
  const int8_t* cls;
  int count, k, weighted;
  unsigned mask;
  double fmin[4], fmax[4];
  double* eps1_out;
  int32_t* cls_out;
};

__device__ __forceinline__ double scale_comp(double v, double lo, double hi) {
  return hi > lo ? __ddiv_rn(__dsub_rn(v, lo), __dsub_rn(hi, lo)) : 0.0;
}

// (d, i) < (e, j) lexicographically
__device__ __forceinline__ bool pair_less(double d, int i, double e, int j) {
  return d < e || (d == e && i < j);
}

__device__ __forceinline__ double sample_d2(const KnnArgs& a, const double* q, int i) {
  double d2 = 0.0;
  for (int c = 0; c < 4; ++c) {
    if (!((a.mask >> c) & 1u)) continue;
    const double p = scale_comp(a.feat[4 * (size_t)i + c], a.fmin[c], a.fmax[c]);
    const double diff = __dsub_rn(q[c], p);
    d2 = __dadd_rn(d2, __dmul_rn(diff, diff));
  }
  return d2;
}

__device__ void knn_fail(const KnnArgs& a) {
  if (a.ctl) set_status(a.ctl, MPCG_ERR_INVALID_ARG);
  if (a.cls_out) *a.cls_out = -1;
  if (a.eps1_out) *a.eps1_out = NAN;
}

__global__ void __launch_bounds__(kKnnThreads) k_knn(KnnArgs a) {
  __shared__ double sd[32];
  __shared__ int si[32];
  __shared__ double q[4];
  __shared__ double sel_d[MPCG_KNN_MAX_K];
  __shared__ int sel_i[MPCG_KNN_MAX_K];
  __shared__ int bad;
  Ctl* ctl = a.ctl;
  if (ctl && volatile_status(ctl) != 0) return;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) {
    double chi[4];
    if (a.q4) {
      for (int c = 0; c < 4; ++c) chi[c] = a.q4[c];
    } else {
      chi[0] = (double)ctl->n;
      chi[1] = (double)ctl->nnz;
      chi[2] = (double)ctl->pdiam;
      chi[3] = ctl->v;
    }
    bad = 0;
    for (int c = 0; c < 4; ++c) {
      if (((a.mask >> c) & 1u) && !isfinite(chi[c])) bad = 1;
      q[c] = scale_comp(chi[c], a.fmin[c], a.fmax[c]);
    }
  }
  __syncthreads();
  if (bad) {
    if (t == 0) knn_fail(a);
    return;
  }
  for (int i = t; i < a.count; i += blockDim.x) {
    const double d2 = sample_d2(a, q, i);
    if (!(d2 == d2)) atomicExch(&bad, 1);
  }
  __syncthreads();
  if (bad) {
    if (t == 0) knn_fail(a);
    return;
  }
  const int k = a.k < a.count ? a.k : a.count;
  double last_d = -INFINITY;
  int last_i = -1;
  for (int j = 0; j < k; ++j) {
    double bd = INFINITY;
    int bi = 0x7fffffff;
    for (int i = t; i < a.count; i += blockDim.x) {
      const double d = sample_d2(a, q, i);
      if (pair_less(last_d, last_i, d, i) && pair_less(d, i, bd, bi)) {
        bd = d;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double od = __shfl_xor_sync(0xffffffffu, bd, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (pair_less(od, oi, bd, bi)) {
        bd = od;
        bi = oi;
      }
    }
    if (lane == 0) {
      sd[warp] = bd;
      si[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
      bd = lane < (int)(blockDim.x >> 5) ? sd[lane] : INFINITY;
      bi = lane < (int)(blockDim.x >> 5) ? si[lane] : 0x7fffffff;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double od = __shfl_xor_sync(0xffffffffu, bd, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (pair_less(od, oi, bd, bi)) {
          bd = od;
          bi = oi;
        }
      }
      if (lane == 0) {
        sel_d[j] = bd;
        sel_i[j] = bi;
      }
    }
    __syncthreads();
    last_d = sel_d[j];
    last_i = sel_i[j];
  }
  if (t == 0) {
    double sc[16];
    int present[16];
    for (int c = 0; c < 16; ++c) {
      sc[c] = 0.0;
      present[c] = 0;
    }
    const bool zero = k > 0 && sel_d[0] == 0.0;
    int result = -1;
    for (int j = 0; j < k; ++j) {
      const int c = a.cls[sel_i[j]];
      if (c < 0 || c > 15) {
        result = -2;
        break;
      }
      const double d2 = sel_d[j];
      if (zero) {
        if (d2 == 0.0) {
          sc[c] = __dadd_rn(sc[c], 1.0);
          present[c] = 1;
        }
      } else {
        sc[c] = __dadd_rn(sc[c], a.weighted ? __ddiv_rn(1.0, __dsqrt_rn(d2)) : 1.0);
        present[c] = 1;
      }
    }
    if (result != -2) {
      double best = -1.0;
      for (int c = 0; c < 16; ++c)
        if (present[c] && sc[c] > best) {
          best = sc[c];
          result = c;
        }
    }
    if (result < 0) {
      knn_fail(a);
    } else {
      if (ctl) {
        ctl->cls = result;
        ctl->eps1 = kPow10Neg[result];
      }
      if (a.eps1_out) *a.eps1_out = kPow10Neg[result];
      if (a.cls_out) *a.cls_out = result;
    }
    if (ctl) ctl->t_features = globaltimer();
  }
}

cudaError_t launch_knn(cudaStream_t st, const double* feat4, const mpcg_sample_t& S,
                       const mpcg_options_t& o, Ctl* ctl, double* eps1_out, int32_t* cls_out) {
  KnnArgs a{};
  a.ctl = ctl;
  a.q4 = feat4;
  a.feat = S.feat;
  a.cls = S.cls;
  a.count = S.count;
  a.k = o.knn_k;
  a.weighted = o.weighted;
  a.mask = o.feat_mask;
  for (int c = 0; c < 4; ++c) {
    a.fmin[c] = S.fmin[c];
    a.fmax[c] = S.fmax[c];
  }
  a.eps1_out = eps1_out;
  a.cls_out = cls_out;
  k_knn<<<1, kKnnThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace mpcg
