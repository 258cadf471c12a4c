// cg.cu -- persistent conjugate-gradient kernels (CG procedure of Sec. 3) for
// the two stages of Algorithm I / II.
//
// One cooperative launch runs a whole stage: every block owns a fixed,
// contiguous range of 32-row slices; each lane owns one row of a slice, so a
// row is summed in its stored order by one thread (bit-identical to a
// sequential fused-multiply-add chain).  The convergence test is taken on the
// device after each grid-wide reduction, identically in every block.
//
// Single-precision stage (float32(A), float32(b)), per iteration:
//   P1  d_k = r_k + beta_k d_{k-1} formed on the fly for every gathered
//       column and stored for the block's own rows (double-buffered d);
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

// Grid-wide double sum of one value per thread-group partial (the block
// partial is in every thread).  Alternating halves of `partials`.
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

// ---------------------------------------------------------------------------------------
// Single-precision stage.
//   mode kCgK0:      start from x = 0; at most k0 iterations; stop early when
//                    the residual reaches eps2 or 0; accumulate Eq. (13).
//   mode kCgToEps1:  start from x = 0; iterate to eps1 (Algorithm I).
//   mode kCgContinue continue the state left by kCgK0 to eps1 (Algorithm II).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kCgThreads) k_cg32(CgArgs a) {
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
    for (int s = s_lo; s < s_hi; ++s) {
      const int i = s * kSlice + lane;
      if (i < n) {
        const float bi = a.b32[i];
        a.x32[i] = 0.0f;
        a.r32[i] = bi;
        ff_add_prod(acc, bi, bi);
      }
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
    const float* r = a.r32;
    FF pdq{0.f, 0.f};
    for (int s = s_lo; s < s_hi; ++s) {
      const int i = s * kSlice + lane;
      if (i >= n) continue;
      const uint32_t wf = a.slice_w[s];
      const int w = (int)(wf & ~kOverflowBit);
      const int base = a.slice_ptr[s] + lane;
      float acc = 0.0f;
      if (first) {
#pragma unroll 4
        for (int k = 0; k < w; ++k) {
          const int c = ld_stream(a.scol + base + kSlice * k);
          const float av = ld_stream(a.sv32 + base + kSlice * k);
          acc = __fmaf_rn(av, r[c], acc);
        }
      } else {
#pragma unroll 4
        for (int k = 0; k < w; ++k) {
          const int c = ld_stream(a.scol + base + kSlice * k);
          const float av = ld_stream(a.sv32 + base + kSlice * k);
          acc = __fmaf_rn(av, __fmaf_rn(beta, dold[c], r[c]), acc);
        }
      }
      if (wf & kOverflowBit) {
        const int e1 = a.rp[i + 1];
        for (int e = a.rp[i] + w; e < e1; ++e) {
          const int c = a.col[e];
          const float av = (float)a.val[e];
          const float dj = first ? r[c] : __fmaf_rn(beta, dold[c], r[c]);
          acc = __fmaf_rn(av, dj, acc);
        }
      }
      const float di = first ? r[i] : __fmaf_rn(beta, dold[i], r[i]);
      dnew[i] = di;
      a.q32[i] = acc;
      ff_add_prod(pdq, di, acc);
    }
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
    for (int s = s_lo; s < s_hi; ++s) {
      const int i = s * kSlice + lane;
      if (i >= n) continue;
      const float di = dnew[i];
      const float qi = a.q32[i];
      const float xi = __fmaf_rn(alpha, di, a.x32[i]);
      const float ri = __fmaf_rn(-alpha, qi, a.r32[i]);
      a.x32[i] = xi;
      a.r32[i] = ri;
      ff_add_prod(prr, ri, ri);
    }
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
__device__ __forceinline__ double spmv64_row(const CgArgs& a, int s, int i, int lane,
                                             const double* v) {
  const uint32_t wf = a.slice_w[s];
  const int w = (int)(wf & ~kOverflowBit);
  const int base = a.slice_ptr[s] + lane;
  double acc = 0.0;
#pragma unroll 4
  for (int k = 0; k < w; ++k) {
    const int c = ld_stream(a.scol + base + kSlice * k);
    const double av = ld_stream(a.sv64 + base + kSlice * k);
    acc = __fma_rn(av, v[c], acc);
  }
  if (wf & kOverflowBit) {
    const int e1 = a.rp[i + 1];
    for (int e = a.rp[i] + w; e < e1; ++e) acc = __fma_rn(a.val[e], v[a.col[e]], acc);
  }
  return acc;
}

__global__ void __launch_bounds__(kCgThreads) k_cg64(CgArgs a) {
  __shared__ double sm[33];
  Ctl* ctl = a.ctl;
  const int lane = threadIdx.x & 31;
  int s_lo, s_hi;
  warp_slices(a.nslices, s_lo, s_hi);
  const int n = a.n;
  if (volatile_status(ctl) != 0) return;
  if (ctl->trivial) {  // b = 0: x = 0 solves A x = b exactly
    for (int s = s_lo; s < s_hi; ++s) {
      const int i = s * kSlice + lane;
      if (i < n) a.x64[i] = 0.0;
    }
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
  for (int s = s_lo; s < s_hi; ++s) {
    const int i = s * kSlice + lane;
    if (i < n) a.x64[i] = a.mode ? 0.0 : (double)a.x32[i];
  }
  ok = grid_barrier(ctl, a.slot, round);
  double rr = 0.0;
  {
    double p = 0.0;
    for (int s = s_lo; s < s_hi; ++s) {
      const int i = s * kSlice + lane;
      if (i >= n) continue;
      const double ri = a.b64[i] - spmv64_row(a, s, i, lane, a.x64);
      a.r64[i] = ri;
      a.d64[i] = ri;
      p = __fma_rn(ri, ri, p);
    }
    rr = grid_total(block_sum_warp_values(warp_sum(p), sm), a.partials, red, ctl, a.slot, round,
                    sm, ok);
  }
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
      double p = 0.0;
      for (int s = s_lo; s < s_hi; ++s) {
        const int i = s * kSlice + lane;
        if (i >= n) continue;
        const double ri = a.b64[i] - spmv64_row(a, s, i, lane, a.x64);
        a.q64[i] = ri;
        p = __fma_rn(ri, ri, p);
      }
      const double tt = grid_total(block_sum_warp_values(warp_sum(p), sm), a.partials, red, ctl,
                                   a.slot, round, sm, ok);
      if (!ok) break;
      true_rel = bnorm > 0.0 ? sqrt(tt) / bnorm : sqrt(tt);
      const double tm = rel ? true_rel : sqrt(tt);
      if (!(tm > eps2) || restarts >= max_restarts) break;
      ++restarts;
      for (int s = s_lo; s < s_hi; ++s) {
        const int i = s * kSlice + lane;
        if (i >= n) continue;
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
    double pdq = 0.0;
    for (int s = s_lo; s < s_hi; ++s) {
      const int i = s * kSlice + lane;
      if (i >= n) continue;
      const double qi = spmv64_row(a, s, i, lane, a.d64);
      a.q64[i] = qi;
      pdq = __fma_rn(a.d64[i], qi, pdq);
    }
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
    // ---- P2: x += alpha d, r -= alpha q, r^T r ----
    double prr = 0.0;
    for (int s = s_lo; s < s_hi; ++s) {
      const int i = s * kSlice + lane;
      if (i >= n) continue;
      a.x64[i] = __fma_rn(alpha, a.d64[i], a.x64[i]);
      const double ri = __fma_rn(-alpha, a.q64[i], a.r64[i]);
      a.r64[i] = ri;
      prr = __fma_rn(ri, ri, prr);
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
    for (int s = s_lo; s < s_hi; ++s) {
      const int i = s * kSlice + lane;
      if (i < n) a.d64[i] = __fma_rn(beta, a.d64[i], a.r64[i]);
    }
    ok = grid_barrier(ctl, a.slot, round);
    ++it;
  }

  if (failed == MPCG_ERR_NOT_CONVERGED && ok) {
    double p = 0.0;
    for (int s = s_lo; s < s_hi; ++s) {
      const int i = s * kSlice + lane;
      if (i >= n) continue;
      const double ri = a.b64[i] - spmv64_row(a, s, i, lane, a.x64);
      p = __fma_rn(ri, ri, p);
    }
    const double tt = grid_total(block_sum_warp_values(warp_sum(p), sm), a.partials, red, ctl,
                                 a.slot, round, sm, ok);
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

// ---------------------------------------------------------------------------------------
// Stand-alone SpMV through the sliced layout (verification entry point).
// ---------------------------------------------------------------------------------------
__global__ void k_spmv(CgArgs a, int fp32, const void* xv, void* yv) {
  if (volatile_status(a.ctl) != 0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = i >> 5, lane = i & 31;
  if (s >= a.nslices || i >= a.n) return;
  if (fp32) {
    const float* x = (const float*)xv;
    const uint32_t wf = a.slice_w[s];
    const int w = (int)(wf & ~kOverflowBit);
    const int base = a.slice_ptr[s] + lane;
    float acc = 0.0f;
    for (int k = 0; k < w; ++k)
      acc = __fmaf_rn(a.sv32[base + kSlice * k], x[a.scol[base + kSlice * k]], acc);
    if (wf & kOverflowBit)
      for (int e = a.rp[i] + w; e < a.rp[i + 1]; ++e) acc = __fmaf_rn((float)a.val[e], x[a.col[e]], acc);
    ((float*)yv)[i] = acc;
  } else {
    ((double*)yv)[i] = spmv64_row(a, s, i, lane, (const double*)xv);
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

cudaError_t launch_spmv(const Launch& L, int fp32, const void* x, void* y) {
  CgArgs a = make_args(L, 0, 0);
  const int threads = 256;
  const int blocks = (int)(((long long)L.d.nslices * kSlice + threads - 1) / threads);
  k_spmv<<<blocks, threads, 0, L.st>>>(a, fp32, x, y);
  return cudaGetLastError();
}

}  // namespace mpcg
