// knn_core.cuh -- choice of eps1 by the k-nearest-neighbours vote of
// Sec. 11, run by one warp, with no scratch memory.
//
// Each feature component is min-max scaled with the sample's min and max
// (Sec. 11.1; the query is not clamped; a constant component maps to 0).
// The squared Euclidean distance (Sec. 11.5) is summed over the selected
// components in index order.  The k nearest are the k smallest pairs
// (d2, index), found by k warp-wide selections of the smallest pair above the
// previous one (distances are recomputed in each round: same arithmetic,
// same values).  Vote: weight 1/sqrt(d2) (Eq. 23) or 1 (Eq. 22), summed in
// selection order; when a selected neighbour is at distance 0 only the
// zero-distance neighbours vote, by count; ties go to the smallest class t.
// Every operation is an explicit IEEE-rounded intrinsic, so the result does
// not depend on compiler contraction.
#pragma once
#include <math.h>

#include "common.cuh"

namespace mpcg {

struct KnnSpec {
  const double* feat;  // [count][4], device
  const int8_t* cls;   // [count], device
  int count, k, weighted;
  unsigned mask;
  double fmin[4], fmax[4];
};

__device__ __forceinline__ double knn_scale(double v, double lo, double hi) {
  return hi > lo ? __ddiv_rn(__dsub_rn(v, lo), __dsub_rn(hi, lo)) : 0.0;
}

__device__ __forceinline__ bool knn_pair_less(double d, int i, double e, int j) {
  return d < e || (d == e && i < j);
}

__device__ __forceinline__ double knn_d2(const KnnSpec& s, const double q[4], int i) {
  double d2 = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (!((s.mask >> c) & 1u)) continue;
    const double p = knn_scale(s.feat[4 * (size_t)i + c], s.fmin[c], s.fmax[c]);
    const double diff = __dsub_rn(q[c], p);
    d2 = __dadd_rn(d2, __dmul_rn(diff, diff));
  }
  return d2;
}

// Class t in [0, 15] chosen for the raw query chi; -1 if the query, the
// sample or a label is invalid.  All 32 lanes of the warp must call it; the
// result is returned in every lane.
__device__ inline int knn_warp(const KnnSpec& s, const double chi[4]) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  double q[4];
  int bad = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (((s.mask >> c) & 1u) && !isfinite(chi[c])) bad = 1;
    q[c] = knn_scale(chi[c], s.fmin[c], s.fmax[c]);
  }
  if (s.count <= 0 || s.k <= 0 || s.k > MPCG_KNN_MAX_K) bad = 1;
  if (!bad) {
    for (int i = lane; i < s.count; i += 32) {
      const double d2 = knn_d2(s, q, i);
      if (!(d2 == d2)) bad = 1;
    }
  }
  if (__any_sync(full, bad)) return -1;
  const int k = s.k < s.count ? s.k : s.count;
  // lane j keeps the j-th and (j+32)-th selected neighbours
  double sel_d_lo = 0.0, sel_d_hi = 0.0;
  int sel_i_lo = 0, sel_i_hi = 0;
  double last_d = -INFINITY;
  int last_i = -1;
  for (int j = 0; j < k; ++j) {
    double bd = INFINITY;
    int bi = 0x7fffffff;
    for (int i = lane; i < s.count; i += 32) {
      const double d = knn_d2(s, q, i);
      if (knn_pair_less(last_d, last_i, d, i) && knn_pair_less(d, i, bd, bi)) {
        bd = d;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double od = __shfl_xor_sync(full, bd, o);
      const int oi = __shfl_xor_sync(full, bi, o);
      if (knn_pair_less(od, oi, bd, bi)) {
        bd = od;
        bi = oi;
      }
    }
    if (lane == (j & 31)) {
      if (j < 32) {
        sel_d_lo = bd;
        sel_i_lo = bi;
      } else {
        sel_d_hi = bd;
        sel_i_hi = bi;
      }
    }
    last_d = bd;
    last_i = bi;
  }
  // vote in selection order (lane 0 gathers the selection through shuffles)
  double sc[16];
  int present[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    sc[c] = 0.0;
    present[c] = 0;
  }
  const double d_first = __shfl_sync(full, sel_d_lo, 0);
  const bool zero = k > 0 && d_first == 0.0;
  int result = -1;
  for (int j = 0; j < k; ++j) {
    const double d2 = j < 32 ? __shfl_sync(full, sel_d_lo, j & 31) : __shfl_sync(full, sel_d_hi, j & 31);
    const int idx = j < 32 ? __shfl_sync(full, sel_i_lo, j & 31) : __shfl_sync(full, sel_i_hi, j & 31);
    const int c = s.cls[idx];
    if (c < 0 || c > 15) {
      result = -2;
      break;
    }
    if (zero) {
      if (d2 == 0.0) {
        sc[c] = __dadd_rn(sc[c], 1.0);
        present[c] = 1;
      }
    } else {
      sc[c] = __dadd_rn(sc[c], s.weighted ? __ddiv_rn(1.0, __dsqrt_rn(d2)) : 1.0);
      present[c] = 1;
    }
  }
  if (result == -2) return -1;
  double best = -1.0;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    if (present[c] && sc[c] > best) {
      best = sc[c];
      result = c;
    }
  }
  return result;
}

// The k nearest sample points of a query (the same selection as knn_warp:
// the k smallest pairs (d2, index), in order), written to nbr[0..k) by lane
// 0, with -1 past min(k, count).  Used to report the neighbours of a query
// (the localization measure of Sec. 11.4); kept apart from knn_warp so that
// the solve kernels that vote carry no code for it.  Returns false in every
// lane if the query or the sample is invalid (nothing written).
__device__ inline bool knn_neighbours_warp(const KnnSpec& s, const double chi[4], int* nbr) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  double q[4];
  int bad = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (((s.mask >> c) & 1u) && !isfinite(chi[c])) bad = 1;
    q[c] = knn_scale(chi[c], s.fmin[c], s.fmax[c]);
  }
  if (s.count <= 0 || s.k <= 0 || s.k > MPCG_KNN_MAX_K) bad = 1;
  if (__any_sync(full, bad)) return false;
  const int k = s.k < s.count ? s.k : s.count;
  double last_d = -INFINITY;
  int last_i = -1;
  for (int j = 0; j < k; ++j) {
    double bd = INFINITY;
    int bi = 0x7fffffff;
    for (int i = lane; i < s.count; i += 32) {
      const double d = knn_d2(s, q, i);
      if (knn_pair_less(last_d, last_i, d, i) && knn_pair_less(d, i, bd, bi)) {
        bd = d;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double od = __shfl_xor_sync(full, bd, o);
      const int oi = __shfl_xor_sync(full, bi, o);
      if (knn_pair_less(od, oi, bd, bi)) {
        bd = od;
        bi = oi;
      }
    }
    if (lane == 0) nbr[j] = bi;
    last_d = bd;
    last_i = bi;
  }
  if (lane == 0)
    for (int j = k; j < s.k; ++j) nbr[j] = -1;
  return true;
}

// eps1 = 10^-t as the correctly rounded decimal literal.
__device__ __forceinline__ double pow10_neg(int t) {
  switch (t) {
    case 0: return 1e0;
    case 1: return 1e-1;
    case 2: return 1e-2;
    case 3: return 1e-3;
    case 4: return 1e-4;
    case 5: return 1e-5;
    case 6: return 1e-6;
    case 7: return 1e-7;
    case 8: return 1e-8;
    case 9: return 1e-9;
    case 10: return 1e-10;
    case 11: return 1e-11;
    case 12: return 1e-12;
    case 13: return 1e-13;
    case 14: return 1e-14;
    default: return 1e-15;
  }
}

}  // namespace mpcg
