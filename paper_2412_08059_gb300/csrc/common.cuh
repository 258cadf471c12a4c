// common.cuh -- device-side building blocks shared by the libmpcg kernels:
// the per-solve control block, the workspace map, bounded grid barriers,
// deterministic reductions and float-float accumulation.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mpcg.h"

namespace mpcg {

constexpr int kSlice = 32;          // rows per slice of the sliced layout (one warp)
constexpr int kCgThreads = 512;     // threads per block of the persistent kernels
constexpr int kMaxGrid = 2048;      // upper bound on persistent grid blocks
constexpr int kBarSlots = 8;        // barrier counters per control block
constexpr uint32_t kOverflowBit = 0x80000000u;

// ---------------------------------------------------------------------------------------
// Control block: all state of one solve that lives on the device.  Zeroed by
// the host (cudaMemsetAsync) at the start of every call, then initialised.
// ---------------------------------------------------------------------------------------
// A grid-barrier arrival counter alone in a 128-byte line: the blocks that
// arrive at and poll one barrier do not contend with those of another (the
// fused stage 1 runs two barriers at once, the CG's and the 2BFS's).
struct alignas(128) BarSlot {
  unsigned long long v;
};

struct Ctl {
  BarSlot bar[kBarSlots];             // monotone grid-barrier arrival counters
  int status;                         // first error wins (atomicCAS from 0)
  int trivial;                        // b == 0: x = 0 and nothing else runs
  int warn_eps1;
  int warn_restart;
  // problem and options
  int n, nnz, nslices, wcap;
  int k0, max1, max2, max_restarts, tol_relative;
  int acc32;  // single-precision inner products summed in float (option acc32)
  double eps1, eps2;
  long long timeout_ns;
  // norms
  double bnorm32, bnorm64;
  // CG state carried between launches
  double rr;          // r^T r of the current residual
  float beta32;       // pending beta of the single-precision stage
  int first;          // next iteration starts with d = r
  int parity;         // current d buffer of the single-precision stage
  int broke32;        // stage 1 ended by d^T A d <= 0
  int n1, n2, k0_done, restarts;
  double vsum, v;
  double res32, res64, true_rel;
  // features and kNN
  int pdiam, far_t, reached, ncomp, connected;
  // the 2BFS's atomically updated counters, in a line of their own
  alignas(128) unsigned long long key;
  int qsize[3];
  int qsizeB[3];   // frontier counters of the second, speculative search
  int ccflag[2];
  alignas(128) int cls;
  int eps1_ready;  // fused stage 1: 0 pending, t + 1 when the kNN chose t, -1 on failure
  int x32_src;     // stage-1 result: -1 = x32, s >= 0 = snapshot slot s
  // device clock marks (ns)
  unsigned long long t_start, t_prep, t_features, t_fp32, t_fp64, t_end;
  unsigned long long t_s2;  // team kernels: start of the double-precision stage (0: not marked)
  int bfs_starts;  // 2BFS runs for l~ (the repeated 2BFS of Sec. 6; 1 = the single run)
  double rz;       // r^T z of the preconditioned single-precision stage (carried to Continue)
  const volatile int* cancel;  // the caller's cancel word (option `cancel`), or null
  // One-warp mode of the dual 2BFS (bfs_core.cuh): mode word and the state
  // that a hand-back or the end publishes to the rest of the group
  alignas(128) int nmode;
  int nla, nlb;
  long long nreached;
  // Column format of the sliced layout: 1 = int16 offsets (column - row), set
  // by the fill when every stored entry's offset fits; 0 = int32 columns.
  // (Team workspaces keep the int32 columns and add the int16 copy.)
  int col16;
  int colwide;  // some stored entry's offset does not fit in int16, or 32-bit columns asked for
  int colbits;  // 16 or 32 once the fill has written the layout, else 0 (result record)
};

// ---------------------------------------------------------------------------------------
// Workspace map (device pointers carved from the caller's buffer).
// ---------------------------------------------------------------------------------------
struct Ws {
  Ctl* ctl;
  double* partials;      // [4][kMaxGrid]
  uint32_t* slice_w;     // width | overflow flag
  int32_t* slice_ptr;    // [nslices + 1] element offsets
  int32_t* scol;         // sliced column indices (int32), or int16 offsets (Ctl::col16)
  int16_t* scol16;       // team workspaces: 16-bit offsets beside scol (Ctl::col16)
  float* sv32;           // sliced values, single
  double* sv64;          // sliced values, double
  float *b32, *x32, *r32, *d32a, *d32b, *q32;
  double *r64, *d64, *q64;
  int32_t *dist, *dist2, *fq0, *fq1, *label;
  int32_t *fq2, *fq3;        // frontier queues of the speculative second search
  unsigned long long* ckey;  // per-component farthest-vertex keys
  float* snap;               // stage-1 snapshots of x~ at candidate crossings [6][n]
  size_t bytes;
};

// ---------------------------------------------------------------------------------------
// Small device helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void set_status(Ctl* c, int s) { atomicCAS(&c->status, 0, s); }

// Stop measure of the CG procedure: ||r|| / ||b|| (relative) or ||r||.
__device__ __forceinline__ double stop_measure(double rr, double bnorm, int rel) {
  return rel ? sqrt(rr) / bnorm : sqrt(rr);
}

// The stop test stop_measure(rr) <= eps without a square root and a division
// per iteration.  stop_measure is non-decreasing in rr, so the test passes
// exactly for rr up to some threshold near t = (eps ||b||)^2 (or eps^2).
// rr <= lo passes and rr > hi fails for certain (the band of 1e-12 relative
// covers the rounding of t and of the exact test); in the band the exact
// test decides.  Where t is not a normal number the exact test always
// decides.  The outcome is that of the exact test for every rr.
struct StopThr {
  double lo, hi, eps, bnorm;
  int rel;
};
__device__ __forceinline__ StopThr stop_thr(double eps, double bnorm, int rel) {
  const double s = rel ? eps * bnorm : eps;
  const double t = s * s;
  StopThr T{-1.0, INFINITY, eps, bnorm, rel};
  if (t >= 1e-290 && t <= 1e290) {
    T.lo = t * (1.0 - 1e-12);
    T.hi = t * (1.0 + 1e-12);
  }
  return T;
}
__device__ __forceinline__ bool stop_pass(const StopThr& T, double rr) {
  if (rr <= T.lo) return true;
  if (rr > T.hi) return false;
  return stop_measure(rr, T.bnorm, T.rel) <= T.eps;
}

__device__ __forceinline__ int volatile_status(const Ctl* c) {
  return *reinterpret_cast<const volatile int*>(&c->status);
}

// Cancellation: the caller's cancel word, when set, ends the call's work with
// MPCG_ERR_CANCELLED (first error wins).  Read in the periodic checks of the
// bounded waits and, through cancel_word, at the head of every CG iteration.
__device__ __forceinline__ int cancel_word(const Ctl* c) {
  const volatile int* w = c->cancel;
  return w ? *w : 0;
}
__device__ __forceinline__ bool poll_cancel(Ctl* c) {
  if (cancel_word(c) == 0) return false;
  set_status(c, MPCG_ERR_CANCELLED);
  return true;
}

// Streaming (read-once-per-sweep) loads for the matrix: evict-first in L1/L2.
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }

// Grid barrier for a cooperative (co-resident) launch.  `slot` selects a
// counter that the host zeroed before the launch; `round` counts the
// barriers this launch has passed on that slot.  Every wait is bounded by
// ctl->timeout_ns of device time; on timeout the status becomes
// MPCG_ERR_TIMEOUT and the function returns false in every thread.
//
// Ordering: the block's writes are ordered before thread 0's release-add by
// the CTA barrier; thread 0's acquire load, followed by the second CTA
// barrier, orders every thread's later loads after all blocks' writes.
__device__ __forceinline__ bool grid_barrier(Ctl* ctl, int slot, unsigned long long& round) {
  __shared__ int s_ok;
  __syncthreads();
  round += 1;
  if (threadIdx.x == 0) {
    const unsigned long long target = round * (unsigned long long)gridDim.x;
    red_release_add(&ctl->bar[slot].v, 1ull);
    int ok = 1;
    if (ld_acquire(&ctl->bar[slot].v) < target) {
      const unsigned long long t0 = globaltimer();
      unsigned spins = 0;
      while (ld_acquire(&ctl->bar[slot].v) < target) {
        if ((++spins & 1023u) == 0) {
          if (volatile_status(ctl) != 0 || poll_cancel(ctl)) {  // another block failed
            ok = 0;
            break;
          }
          if (globaltimer() - t0 > (unsigned long long)ctl->timeout_ns) {
            set_status(ctl, MPCG_ERR_TIMEOUT);
            ok = 0;
            break;
          }
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------------------
// Shared-memory mbarriers and 1-D bulk asynchronous copies (TMA engine).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait for the completion of the phase with the given parity.
// Returns false on timeout (status set) or when *stop becomes non-zero.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity, Ctl* ctl,
                                          const volatile int* stop) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  unsigned spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++spins & 63u) == 0) {
      if (stop && *stop) return false;
      if (globaltimer() - t0 > (unsigned long long)ctl->timeout_ns) {
        set_status(ctl, MPCG_ERR_TIMEOUT);
        return false;
      }
    }
  }
  return true;
}
__device__ __forceinline__ unsigned long long l2_policy_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// global -> shared bulk copy; bytes and both addresses multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         unsigned long long* bar, unsigned long long policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

// ---------------------------------------------------------------------------------------
// Float-float accumulation (error-free transformations in single precision).
// A product of two floats is split exactly into p + e; sums are carried as
// (hi, lo).  The result is converted to double once per warp.
// ---------------------------------------------------------------------------------------
struct FF {
  float hi, lo;
};

// With `f32` (option acc32) the compensation is left out: the product and
// every add round to float, in the same order and the same tree.
__device__ __forceinline__ void ff_add_prod(FF& s, float a, float b, bool f32) {
  if (f32) {
    s.hi = __fadd_rn(s.hi, __fmul_rn(a, b));
    return;
  }
  float p = a * b;
  float e = __fmaf_rn(a, b, -p);             // a*b = p + e exactly
  float t = s.hi + p;                         // two-sum(s.hi, p)
  float bp = t - s.hi;
  float err = (s.hi - (t - bp)) + (p - bp);
  s.hi = t;
  s.lo += err + e;
}

__device__ __forceinline__ FF ff_add(FF a, FF b, bool f32) {
  if (f32) return FF{__fadd_rn(a.hi, b.hi), 0.f};
  float t = a.hi + b.hi;
  float bp = t - a.hi;
  float err = (a.hi - (t - bp)) + (b.hi - bp);
  float lo = a.lo + b.lo + err;
  float hi = t + lo;                          // fast two-sum renormalisation
  lo = lo - (hi - t);
  return {hi, lo};
}

__device__ __forceinline__ FF ff_warp_sum(FF v, bool f32) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    FF w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = ff_add(v, w, f32);
  }
  return v;
}

// Butterfly sum of one float per lane, every add rounded to float (all lanes
// end with the same value: a + b and b + a round alike).
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum of one double per warp (`w` valid in lane 0 of
// each warp).  Returns the total in every thread.  Uses `sm` (>= 32 doubles).
__device__ __forceinline__ double block_sum_warp_values(double w, double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sm[warp] = w;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < nw ? sm[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) sm[32] = t;
  }
  __syncthreads();
  return sm[32];
}

// Sum of `count` doubles in global memory, identical in every block that
// calls it (fixed assignment and tree order).  Plain loads: the caller has
// passed a grid barrier after the values were written.
__device__ __forceinline__ double block_sum_global(const double* v, int count, double* sm) {
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) s += v[i];
  s = warp_sum(s);
  return block_sum_warp_values(s, sm);
}

// Key for the farthest-vertex choice of 2BFS: larger distance first, then
// smaller vertex index.
__device__ __forceinline__ unsigned long long far_key(int dist, int v) {
  return ((unsigned long long)(unsigned)dist << 32) | (unsigned long long)(0xffffffffu - (unsigned)v);
}
__device__ __forceinline__ int far_key_vertex(unsigned long long k) {
  return (int)(0xffffffffu - (unsigned)(k & 0xffffffffull));
}

}  // namespace mpcg
