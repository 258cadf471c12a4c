// cg.cu -- persistent conjugate-gradient kernels (CG procedure of Sec. 3) for
// the two stages of Algorithm I / II.
//
// One cooperative launch runs a whole stage.  Every warp owns a fixed,
// contiguous range of 32-row slices; in the SpMV each lane owns one row of a
// slice, so a row is summed in its stored order by one thread (bit-identical
// to a sequential fused-multiply-add chain).  The convergence test is taken
// on the device after each grid-wide reduction, identically in every block.
//
// Memory-level parallelism: a warp first loads the widths and offsets of up
// to 32 of its slices (one per lane), then streams two slices at a time with
// fully unrolled loads of up to 8 entries per row held in registers: the
// next slice's columns and values are in flight while the current slice's
// gathers and FMAs run.  The per-row update phases use 16-byte vector loads.
//
// Single-precision stage (float32(A), float32(b)), per iteration:
//   P1  d_k = r_k + beta_k d_{k-1} formed on the fly for every gathered
//       column and stored for the warp's own rows (double-buffered d);
//       q = A d_k; partial d_k^T q                        -> grid reduction
//   P2  x += alpha d_k; r -= alpha q; partial r^T r          -> grid reduction
// Dot products are accumulated as float-float sums (error-free products and
// sums in single precision) and combined in double: double-accurate norms
// (Remark 3 of Sec. 9) without loading the FP64 units.  alpha and beta are
// the double quotients rounded once to float.
//
// Double-precision stage: d is stored explicitly (forming it on the fly would
// cost one FP64 FMA per stored entry), so the iteration has a third phase
//   P3  d = r + beta d  followed by a grid barrier.
#include <math.h>

#include "internal.h"

namespace mpcg {

constexpr int kFastW = 8;  // rows up to this width take the unrolled path
constexpr unsigned kFull = 0xffffffffu;

struct CgArgs {
  Ctl* ctl;
  double* partials;
  const uint32_t* slice_w;
  const int32_t* slice_ptr;
  const int32_t* scol;
  const float* sv32;
  const double* sv64;
  const int32_t* rp;
  const int32_t* col;
  const double* val;
  int n, nslices, slot, mode;
  const float* b32;
  float *x32, *r32, *da, *db, *q32;
  const double* b64;
  double *x64, *r64, *d64, *q64;
};

// Slice range [lo, hi) of the calling warp: contiguous per warp, warps of a
// block adjacent.
__device__ __forceinline__ void warp_slices(int nslices, int& lo, int& hi) {
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  lo = (int)(nslices * gw / nw);
  hi = (int)(nslices * (gw + 1) / nw);
}

// Grid-wide double sum of the block partials (the block partial is in every
// thread).  Alternating halves of `partials`.
__device__ __forceinline__ double grid_total(double block_part, double* partials, int& red,
                                             Ctl* ctl, int slot, unsigned long long& round,
                                             double* sm, bool& ok) {
  double* buf = partials + (red & 1) * kMaxGrid;
  ++red;
  if (threadIdx.x == 0) buf[blockIdx.x] = block_part;
  ok = grid_barrier(ctl, slot, round);
  return block_sum_global(buf, gridDim.x, sm);
}

__device__ __forceinline__ double ff_block(FF v, double* sm) {
  v = ff_warp_sum(v);
  return block_sum_warp_values((double)v.hi + (double)v.lo, sm);
}

__device__ __forceinline__ double stop_measure(double rr, double bnorm, int rel) {
  return rel ? sqrt(rr) / bnorm : sqrt(rr);
}

__device__ __forceinline__ bool fast_slice(uint32_t wf) {
  return !(wf & kOverflowBit) && (int)wf <= kFastW;
}

// ---------------------------------------------------------------------------------------
// Sliced SpMV rows, generic over the value type.  G(c) is the gathered vector
// entry for column c (d, or r + beta d formed on the fly).
// ---------------------------------------------------------------------------------------
template <typename T>
struct SliceBuf {
  int c[kFastW];
  T v[kFastW];
};

template <typename T>
__device__ __forceinline__ const T* svals(const CgArgs& a);
template <>
__device__ __forceinline__ const float* svals<float>(const CgArgs& a) { return a.sv32; }
template <>
__device__ __forceinline__ const double* svals<double>(const CgArgs& a) { return a.sv64; }

template <typename T>
__device__ __forceinline__ void slice_load(const CgArgs& a, uint32_t wf, int p, SliceBuf<T>& b) {
  if (!fast_slice(wf)) return;
  const int w = (int)wf;
  const T* sv = svals<T>(a);
#pragma unroll
  for (int k = 0; k < kFastW; ++k) {
    if (k < w) {
      b.c[k] = ld_stream(a.scol + p + kSlice * k);
      b.v[k] = ld_stream(sv + p + kSlice * k);
    }
  }
}

// Row i = 32 s + lane: returns sum_k v_k G(c_k) in stored order.
template <typename T, class Gather>
__device__ __forceinline__ T slice_row(const CgArgs& a, int i, uint32_t wf, int p,
                                       const SliceBuf<T>& b, Gather G) {
  T acc = (T)0;
  if (fast_slice(wf)) {
    const int w = (int)wf;
#pragma unroll
    for (int k = 0; k < kFastW; ++k)
      if (k < w) acc = fma(b.v[k], G(b.c[k]), acc);
  } else {
    const int w = (int)(wf & ~kOverflowBit);
    const T* sv = svals<T>(a);
    for (int k = 0; k < w; ++k)
      acc = fma(ld_stream(sv + p + kSlice * k), G(ld_stream(a.scol + p + kSlice * k)), acc);
    if ((wf & kOverflowBit) && i < a.n) {
      const int e1 = a.rp[i + 1];
      for (int e = a.rp[i] + w; e < e1; ++e) acc = fma((T)a.val[e], G(a.col[e]), acc);
    }
  }
  return acc;
}

// Walk the warp's slices two at a time; Row(i, acc) consumes each row.  With
// DB (double buffering) the next slice's loads are issued before the current
// slice's gathers; without it only the slice metadata is preloaded.
template <typename T, bool DB, class Gather, class Row>
__device__ __forceinline__ void spmv_slices(const CgArgs& a, int s_lo, int s_hi, int lane,
                                            Gather G, Row R) {
  if (!DB) {
    for (int cb = s_lo; cb < s_hi; cb += 32) {
      const int cnt = min(32, s_hi - cb);
      const uint32_t mw = lane < cnt ? a.slice_w[cb + lane] : 0u;
      const int mp = lane < cnt ? a.slice_ptr[cb + lane] : 0;
      for (int j = 0; j < cnt; ++j) {
        const uint32_t wf = __shfl_sync(kFull, mw, j);
        const int p = __shfl_sync(kFull, mp, j) + lane;
        SliceBuf<T> A;
        slice_load<T>(a, wf, p, A);
        const int i = (cb + j) * kSlice + lane;
        R(i, slice_row<T>(a, i, wf, p, A, G));
      }
    }
    return;
  }
  for (int cb = s_lo; cb < s_hi; cb += 32) {
    const int cnt = min(32, s_hi - cb);
    const uint32_t mw = lane < cnt ? a.slice_w[cb + lane] : 0u;
    const int mp = lane < cnt ? a.slice_ptr[cb + lane] : 0;
    SliceBuf<T> A, B;
    uint32_t wa = __shfl_sync(kFull, mw, 0);
    int pa = __shfl_sync(kFull, mp, 0) + lane;
    slice_load<T>(a, wa, pa, A);
    for (int j = 0; j < cnt; j += 2) {
      const bool hb = j + 1 < cnt;
      const uint32_t wb = __shfl_sync(kFull, mw, (j + 1) & 31);
      const int pb = __shfl_sync(kFull, mp, (j + 1) & 31) + lane;
      if (hb) slice_load<T>(a, wb, pb, B);
      {
        const int i = (cb + j) * kSlice + lane;
        R(i, slice_row<T>(a, i, wa, pa, A, G));
      }
      if (j + 2 < cnt) {
        wa = __shfl_sync(kFull, mw, j + 2);
        pa = __shfl_sync(kFull, mp, j + 2) + lane;
        slice_load<T>(a, wa, pa, A);
      }
      if (hb) {
        const int i = (cb + j + 1) * kSlice + lane;
        R(i, slice_row<T>(a, i, wb, pb, B, G));
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Single-precision stage.
//   mode kCgK0:      start from x = 0; at most k0 iterations; stop early when
//                    the residual reaches eps2 or 0; accumulate Eq. (13).
//   mode kCgToEps1:  start from x = 0; iterate to eps1 (Algorithm I).
//   mode kCgContinue continue the state left by kCgK0 to eps1 (Algorithm II).
// ---------------------------------------------------------------------------------------
template <bool FIRST>
__device__ __forceinline__ void p1_32(const CgArgs& a, int s_lo, int s_hi, int lane,
                                      const float* r, const float* dold, float* dnew, float beta,
                                      FF& pdq) {
  const int n = a.n;
  float* q = a.q32;
  auto G = [&](int c) -> float {
    if (FIRST) return r[c];
    return __fmaf_rn(beta, dold[c], r[c]);
  };
  auto R = [&](int i, float acc) {
    if (i < n) {
      const float di = G(i);
      dnew[i] = di;
      q[i] = acc;
      ff_add_prod(pdq, di, acc);
    }
  };
  spmv_slices<float, false>(a, s_lo, s_hi, lane, G, R);
}

// x += alpha d, r -= alpha q, r^T r over the warp's rows, four rows per lane.
__device__ __forceinline__ void p2_32(const CgArgs& a, int s_lo, int s_hi, int lane,
                                      const float* d, float alpha, FF& prr) {
  const int R0 = s_lo * kSlice, R1 = min(s_hi * kSlice, a.n);
  for (int base = R0 + 4 * lane; base < R1; base += 4 * kSlice) {
    if (base + 4 <= R1) {
      const float4 d4 = *reinterpret_cast<const float4*>(d + base);
      const float4 q4 = *reinterpret_cast<const float4*>(a.q32 + base);
      float4 x4 = *reinterpret_cast<const float4*>(a.x32 + base);
      float4 r4 = *reinterpret_cast<const float4*>(a.r32 + base);
      x4.x = __fmaf_rn(alpha, d4.x, x4.x);
      x4.y = __fmaf_rn(alpha, d4.y, x4.y);
      x4.z = __fmaf_rn(alpha, d4.z, x4.z);
      x4.w = __fmaf_rn(alpha, d4.w, x4.w);
      r4.x = __fmaf_rn(-alpha, q4.x, r4.x);
      r4.y = __fmaf_rn(-alpha, q4.y, r4.y);
      r4.z = __fmaf_rn(-alpha, q4.z, r4.z);
      r4.w = __fmaf_rn(-alpha, q4.w, r4.w);
      *reinterpret_cast<float4*>(a.x32 + base) = x4;
      *reinterpret_cast<float4*>(a.r32 + base) = r4;
      ff_add_prod(prr, r4.x, r4.x);
      ff_add_prod(prr, r4.y, r4.y);
      ff_add_prod(prr, r4.z, r4.z);
      ff_add_prod(prr, r4.w, r4.w);
    } else {
      for (int i = base; i < R1; ++i) {
        a.x32[i] = __fmaf_rn(alpha, d[i], a.x32[i]);
        const float ri = __fmaf_rn(-alpha, a.q32[i], a.r32[i]);
        a.r32[i] = ri;
        ff_add_prod(prr, ri, ri);
      }
    }
  }
}

__global__ void __launch_bounds__(kCgThreads, 2) k_cg32(CgArgs a) {
  __shared__ double sm[33];
  Ctl* ctl = a.ctl;
  if (volatile_status(ctl) != 0 || ctl->trivial) return;
  if (a.mode == kCgContinue && ctl->broke32) {  // stage 1 already ended in the k0 phase
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (ctl->res32 > ctl->eps1) ctl->warn_eps1 = 1;
      ctl->t_fp32 = globaltimer();
    }
    return;
  }
  const int lane = threadIdx.x & 31;
  int s_lo, s_hi;
  warp_slices(a.nslices, s_lo, s_hi);
  const int n = a.n;
  const int rel = ctl->tol_relative;
  unsigned long long round = 0;
  int red = 0;
  bool ok = true;

  double rr, bnorm;
  float beta;
  int first, parity, it;
  if (a.mode != kCgContinue) {
    // CG line 1: x0 = 0, r0 = b - A x0 = b~, d0 = r0.
    FF acc{0.f, 0.f};
    const int R0 = s_lo * kSlice, R1 = min(s_hi * kSlice, n);
    for (int i = R0 + lane; i < R1; i += kSlice) {
      const float bi = a.b32[i];
      a.x32[i] = 0.0f;
      a.r32[i] = bi;
      ff_add_prod(acc, bi, bi);
    }
    rr = grid_total(ff_block(acc, sm), a.partials, red, ctl, a.slot, round, sm, ok);
    bnorm = sqrt(rr);  // ||b~|| = ||r0||
    first = 1;
    parity = 0;
    beta = 0.0f;
    it = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl->bnorm32 = bnorm;
      if (!isfinite(bnorm)) set_status(ctl, MPCG_ERR_NAN);
    }
    if (!isfinite(bnorm)) ok = false;
  } else {
    rr = ctl->rr;
    bnorm = ctl->bnorm32;
    beta = ctl->beta32;
    first = ctl->first;
    parity = ctl->parity;
    it = ctl->n1;
  }
  const double eps = a.mode == kCgK0 ? ctl->eps2 : ctl->eps1;
  const int limit = a.mode == kCgK0 ? min(ctl->k0, ctl->max1) : ctl->max1;
  double vsum = 0.0;
  int k0done = 0, broke = 0;
  double m = stop_measure(rr, bnorm, rel);

  while (ok) {
    m = stop_measure(rr, bnorm, rel);
    if (isnan(m)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_status(ctl, MPCG_ERR_NAN);
      break;
    }
    if (m <= eps || it >= limit) break;
    if (a.mode == kCgK0 && rr == 0.0) break;

    // ---- P1: q = A d_k with d_k = r_k + beta_k d_{k-1} formed on the fly ----
    // Plain (coherent) pointers: these vectors change between iterations of
    // this launch, so they must not go through the read-only data path.
    const float* dold = parity ? a.db : a.da;
    float* dnew = parity ? a.da : a.db;
    FF pdq{0.f, 0.f};
    if (first)
      p1_32<true>(a, s_lo, s_hi, lane, a.r32, dold, dnew, beta, pdq);
    else
      p1_32<false>(a, s_lo, s_hi, lane, a.r32, dold, dnew, beta, pdq);
    const double dq = grid_total(ff_block(pdq, sm), a.partials, red, ctl, a.slot, round, sm, ok);
    if (!ok) break;
    if (!isfinite(dq)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_status(ctl, MPCG_ERR_NAN);
      break;
    }
    if (!(dq > 0.0)) {  // stage 1 ends here; x and r are unchanged
      broke = 1;
      break;
    }
    const float alpha = (float)(rr / dq);

    // ---- P2: x += alpha d_k, r -= alpha q, r^T r ----
    FF prr{0.f, 0.f};
    p2_32(a, s_lo, s_hi, lane, dnew, alpha, prr);
    const double rrn = grid_total(ff_block(prr, sm), a.partials, red, ctl, a.slot, round, sm, ok);
    if (!ok) break;
    if (!isfinite(rrn)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_status(ctl, MPCG_ERR_NAN);
      break;
    }
    if (a.mode == kCgK0) {
      vsum += sqrt(rrn) / sqrt(rr);  // Eq. (13) ratio ||r_i|| / ||r_{i-1}||
      ++k0done;
    }
    beta = (float)(rrn / rr);
    rr = rrn;
    parity ^= 1;
    first = 0;
    ++it;
  }

  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->rr = rr;
    ctl->beta32 = beta;
    ctl->first = first;
    ctl->parity = parity;
    ctl->n1 = it;
    ctl->res32 = stop_measure(rr, bnorm, rel);
    if (broke) ctl->broke32 = 1;
    if (a.mode == kCgK0) {
      ctl->k0_done = k0done;
      ctl->vsum = vsum;
      ctl->v = k0done > 0 ? vsum / (double)k0done : 0.0;
    } else {
      if (ctl->res32 > ctl->eps1) ctl->warn_eps1 = 1;
      ctl->t_fp32 = globaltimer();
    }
  }
}

// ---------------------------------------------------------------------------------------
// Double-precision stage (restart of Algorithm I/II, or pure FP64 CG).
// ---------------------------------------------------------------------------------------

// r = b - A v (and d = r) over the warp's rows; returns the partial r^T r.
// out_r / out_d may be null.
__device__ __forceinline__ double residual64(const CgArgs& a, int s_lo, int s_hi, int lane,
                                             const double* v, double* out_r, double* out_d) {
  double p = 0.0;
  auto G = [&](int c) -> double { return v[c]; };
  auto R = [&](int i, double acc) {
    if (i < a.n) {
      const double ri = a.b64[i] - acc;
      if (out_r) out_r[i] = ri;
      if (out_d) out_d[i] = ri;
      p = __fma_rn(ri, ri, p);
    }
  };
  spmv_slices<double, false>(a, s_lo, s_hi, lane, G, R);
  return p;
}

// q = A d over the warp's rows; returns the partial d^T q.
__device__ __forceinline__ double p1_64(const CgArgs& a, int s_lo, int s_hi, int lane) {
  double pdq = 0.0;
  const double* d = a.d64;
  double* q = a.q64;
  const int n = a.n;
  auto G = [&](int c) -> double { return d[c]; };
  auto R = [&](int i, double acc) {
    if (i < n) {
      q[i] = acc;
      pdq = __fma_rn(d[i], acc, pdq);
    }
  };
  spmv_slices<double, false>(a, s_lo, s_hi, lane, G, R);
  return pdq;
}

__global__ void __launch_bounds__(kCgThreads, 2) k_cg64(CgArgs a) {
  __shared__ double sm[33];
  Ctl* ctl = a.ctl;
  const int lane = threadIdx.x & 31;
  int s_lo, s_hi;
  warp_slices(a.nslices, s_lo, s_hi);
  const int n = a.n;
  const int R0 = s_lo * kSlice, R1 = min(s_hi * kSlice, n);
  if (volatile_status(ctl) != 0) return;
  if (ctl->trivial) {  // b = 0: x = 0 solves A x = b exactly
    for (int i = R0 + lane; i < R1; i += kSlice) a.x64[i] = 0.0;
    return;
  }
  const int rel = ctl->tol_relative;
  const double bnorm = ctl->bnorm64;
  const double eps2 = ctl->eps2;
  const int max2 = ctl->max2;
  const int max_restarts = ctl->max_restarts;
  unsigned long long round = 0;
  int red = 0;
  bool ok = true;
  int it = 0, restarts = 0, failed = 0;

  // Promote: x0 = float64(x~) (or 0); restart: r0 = b - A x0, d0 = r0.
  for (int i = R0 + lane; i < R1; i += kSlice) a.x64[i] = a.mode ? 0.0 : (double)a.x32[i];
  ok = grid_barrier(ctl, a.slot, round);
  double rr = grid_total(block_sum_warp_values(warp_sum(residual64(a, s_lo, s_hi, lane, a.x64,
                                                                   a.r64, a.d64)), sm),
                         a.partials, red, ctl, a.slot, round, sm, ok);
  double m = stop_measure(rr, bnorm, rel);
  double true_rel = NAN;

  while (ok) {
    m = stop_measure(rr, bnorm, rel);
    if (isnan(m)) {
      failed = MPCG_ERR_NAN;
      break;
    }
    if (m <= eps2) {
      // True residual ||b - A x|| (FP64); restart from x if it misses eps2.
      const double tt = grid_total(
          block_sum_warp_values(warp_sum(residual64(a, s_lo, s_hi, lane, a.x64, a.q64, nullptr)),
                                sm),
          a.partials, red, ctl, a.slot, round, sm, ok);
      if (!ok) break;
      true_rel = bnorm > 0.0 ? sqrt(tt) / bnorm : sqrt(tt);
      const double tm = rel ? true_rel : sqrt(tt);
      if (!(tm > eps2) || restarts >= max_restarts) break;
      ++restarts;
      for (int i = R0 + lane; i < R1; i += kSlice) {
        const double ri = a.q64[i];
        a.r64[i] = ri;
        a.d64[i] = ri;
      }
      rr = tt;
      ok = grid_barrier(ctl, a.slot, round);
      continue;
    }
    if (it >= max2) {
      failed = MPCG_ERR_NOT_CONVERGED;
      break;
    }
    // ---- P1: q = A d, d^T q ----
    const double pdq = p1_64(a, s_lo, s_hi, lane);
    const double dq = grid_total(block_sum_warp_values(warp_sum(pdq), sm), a.partials, red, ctl,
                                 a.slot, round, sm, ok);
    if (!ok) break;
    if (!isfinite(dq)) {
      failed = MPCG_ERR_NAN;
      break;
    }
    if (!(dq > 0.0)) {
      failed = MPCG_ERR_BREAKDOWN;
      break;
    }
    const double alpha = rr / dq;
    // ---- P2: x += alpha d, r -= alpha q, r^T r (two rows per lane) ----
    double prr = 0.0;
    for (int base = R0 + 2 * lane; base < R1; base += 2 * kSlice) {
      if (base + 2 <= R1) {
        const double2 d2 = *reinterpret_cast<const double2*>(a.d64 + base);
        const double2 q2 = *reinterpret_cast<const double2*>(a.q64 + base);
        double2 x2 = *reinterpret_cast<const double2*>(a.x64 + base);
        double2 r2 = *reinterpret_cast<const double2*>(a.r64 + base);
        x2.x = __fma_rn(alpha, d2.x, x2.x);
        x2.y = __fma_rn(alpha, d2.y, x2.y);
        r2.x = __fma_rn(-alpha, q2.x, r2.x);
        r2.y = __fma_rn(-alpha, q2.y, r2.y);
        *reinterpret_cast<double2*>(a.x64 + base) = x2;
        *reinterpret_cast<double2*>(a.r64 + base) = r2;
        prr = __fma_rn(r2.x, r2.x, prr);
        prr = __fma_rn(r2.y, r2.y, prr);
      } else {
        a.x64[base] = __fma_rn(alpha, a.d64[base], a.x64[base]);
        const double ri = __fma_rn(-alpha, a.q64[base], a.r64[base]);
        a.r64[base] = ri;
        prr = __fma_rn(ri, ri, prr);
      }
    }
    const double rrn = grid_total(block_sum_warp_values(warp_sum(prr), sm), a.partials, red, ctl,
                                  a.slot, round, sm, ok);
    if (!ok) break;
    if (!isfinite(rrn)) {
      failed = MPCG_ERR_NAN;
      break;
    }
    const double beta = rrn / rr;
    rr = rrn;
    // ---- P3: d = r + beta d ----
    for (int base = R0 + 2 * lane; base < R1; base += 2 * kSlice) {
      if (base + 2 <= R1) {
        double2 d2 = *reinterpret_cast<const double2*>(a.d64 + base);
        const double2 r2 = *reinterpret_cast<const double2*>(a.r64 + base);
        d2.x = __fma_rn(beta, d2.x, r2.x);
        d2.y = __fma_rn(beta, d2.y, r2.y);
        *reinterpret_cast<double2*>(a.d64 + base) = d2;
      } else {
        a.d64[base] = __fma_rn(beta, a.d64[base], a.r64[base]);
      }
    }
    ok = grid_barrier(ctl, a.slot, round);
    ++it;
  }

  if (failed == MPCG_ERR_NOT_CONVERGED && ok) {
    const double tt = grid_total(
        block_sum_warp_values(warp_sum(residual64(a, s_lo, s_hi, lane, a.x64, nullptr, nullptr)),
                              sm),
        a.partials, red, ctl, a.slot, round, sm, ok);
    true_rel = bnorm > 0.0 ? sqrt(tt) / bnorm : sqrt(tt);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (failed) set_status(ctl, failed);
    ctl->n2 = it;
    ctl->restarts = restarts;
    if (restarts) ctl->warn_restart = 1;
    ctl->res64 = m;
    ctl->true_rel = true_rel;
    ctl->rr = rr;
    ctl->t_fp64 = globaltimer();
  }
}

// Promotion only (stage-1-only solves): x = float64(x~).
__global__ void k_promote(const Ctl* c, const float* __restrict__ x32, double* __restrict__ x64,
                          int n) {
  const bool zero = c->trivial != 0;
  if (c->status != 0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x64[i] = zero ? 0.0 : (double)x32[i];
}

// ---------------------------------------------------------------------------------------
// Stand-alone SpMV through the sliced layout (verification entry point).
// ---------------------------------------------------------------------------------------
__global__ void k_spmv(CgArgs a, int fp32, const void* xv, void* yv) {
  if (volatile_status(a.ctl) != 0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = i >> 5, lane = i & 31;
  if (s >= a.nslices || i >= a.n) return;
  const uint32_t wf = a.slice_w[s];
  const int p = a.slice_ptr[s] + lane;
  if (fp32) {
    const float* x = (const float*)xv;
    SliceBuf<float> b;
    slice_load<float>(a, wf, p, b);
    ((float*)yv)[i] = slice_row<float>(a, i, wf, p, b, [&](int c) { return x[c]; });
  } else {
    const double* x = (const double*)xv;
    SliceBuf<double> b;
    slice_load<double>(a, wf, p, b);
    ((double*)yv)[i] = slice_row<double>(a, i, wf, p, b, [&](int c) { return x[c]; });
  }
}

static CgArgs make_args(const Launch& L, int slot, int mode) {
  CgArgs a{};
  a.ctl = L.ws.ctl;
  a.partials = L.ws.partials;
  a.slice_w = L.ws.slice_w;
  a.slice_ptr = L.ws.slice_ptr;
  a.scol = L.ws.scol;
  a.sv32 = L.ws.sv32;
  a.sv64 = L.ws.sv64;
  a.rp = L.A->row_ptr;
  a.col = L.A->col;
  a.val = L.A->val;
  a.n = L.d.n;
  a.nslices = L.d.nslices;
  a.slot = slot;
  a.mode = mode;
  a.b32 = L.ws.b32;
  a.x32 = L.ws.x32;
  a.r32 = L.ws.r32;
  a.da = L.ws.d32a;
  a.db = L.ws.d32b;
  a.q32 = L.ws.q32;
  a.r64 = L.ws.r64;
  a.d64 = L.ws.d64;
  a.q64 = L.ws.q64;
  return a;
}

const void* cg32_kernel() { return (const void*)k_cg32; }
const void* cg64_kernel() { return (const void*)k_cg64; }

cudaError_t launch_cg32(const Launch& L, int mode, int slot) {
  CgArgs a = make_args(L, slot, mode);
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)k_cg32, dim3(L.grid), dim3(kCgThreads), args, 0,
                                    L.st);
}

cudaError_t launch_cg64(const Launch& L, const double* b, double* x, int from_zero, int slot) {
  CgArgs a = make_args(L, slot, from_zero);
  a.b64 = b;
  a.x64 = x;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)k_cg64, dim3(L.grid), dim3(kCgThreads), args, 0,
                                    L.st);
}

cudaError_t launch_promote(const Launch& L, double* x) {
  int blocks = (L.d.n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_promote<<<blocks, 256, 0, L.st>>>(L.ws.ctl, L.ws.x32, x, L.d.n);
  return cudaGetLastError();
}

cudaError_t launch_spmv(const Launch& L, int fp32, const void* x, void* y) {
  CgArgs a = make_args(L, 0, 0);
  const int threads = 256;
  const int blocks = (int)(((long long)L.d.nslices * kSlice + threads - 1) / threads);
  k_spmv<<<blocks, threads, 0, L.st>>>(a, fp32, x, y);
  return cudaGetLastError();
}

}  // namespace mpcg
