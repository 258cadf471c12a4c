// cg.cu -- persistent conjugate-gradient kernels (CG procedure of Sec. 3) for
// the two stages of Algorithm I / II.
//
// One cooperative launch runs a whole stage, one block per SM.  A block
// owns a contiguous range of 32-row slices and is warp-specialised:
//   * a producer warp (one elected thread) streams the block's part of the
//     sliced matrix -- columns and values, a contiguous element range --
//     through a ring of shared-memory stages with 1-D bulk asynchronous
//     copies (TMA engine, cp.async.bulk) completing on mbarriers.  The matrix
//     does not change, so the producer streams it cyclically, pass after
//     pass, and keeps prefetching the next pass while the consumers are in a
//     grid barrier or in the per-row update phases;
//   * consumer warps take the block's slices round-robin; in the SpMV each
//     lane owns one row of a slice and sums it in stored order (the same
//     chain of fused multiply-adds as a sequential loop, so the SpMV result is
//     bit-identical), reading columns and values from shared memory and
//     gathering the vector from L1/L2.  Consumers synchronise among
//     themselves with a named barrier, never with the producer.
// The convergence test is taken after each grid-wide reduction, identically
// in every block.  Every wait is bounded in device time.
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
//
// Kernels: k_cg32 (single-precision stage of Algorithm I, and the k0 phase
// for mpcg_features), k_stage1 (the single-precision stage of Algorithm II
// with the 2BFS and the kNN running alongside; described at the kernel),
// k_cg64 (double-precision stage), k_promote and k_spmv.
#include <math.h>

#include <type_traits>

#include "internal.h"

namespace mpcg {

constexpr int kNC = 15;                       // consumer warps per block
constexpr int kTmaThreads = (kNC + 1) * 32;   // + one producer warp
constexpr int kLogCH = 12;
constexpr int kCH = 1 << kLogCH;              // elements per streamed chunk
constexpr int kFastW = 8;                     // rows up to this width take the unrolled path

template <typename T>
struct StageCfg;
template <>
struct StageCfg<float> {
  static constexpr int kStages = 5;
};
template <>
struct StageCfg<double> {
  static constexpr int kStages = 4;
};
template <typename T>
__host__ __device__ constexpr size_t stage_bytes() {
  return (size_t)kCH * (sizeof(int32_t) + sizeof(T));
}
template <typename T>
__host__ __device__ constexpr size_t ring_smem_bytes() {
  return StageCfg<T>::kStages * stage_bytes<T>() + 2 * StageCfg<T>::kStages * 8 + 16;
}

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
  float* snap;  // stage-1 snapshots of x~ ([slot][n]); ctl->x32_src picks one
  // Jacobi preconditioning (the k_cg32 / k_cg64 instances with kPc)
  const double* dinv64;
  const float* dinv32;
  float* z32;
};

template <typename T>
__device__ __forceinline__ const T* svals(const CgArgs& a);
template <>
__device__ __forceinline__ const float* svals<float>(const CgArgs& a) { return a.sv32; }
template <>
__device__ __forceinline__ const double* svals<double>(const CgArgs& a) { return a.sv64; }


// ---------------------------------------------------------------------------------------
// Consumer-group synchronisation (named barrier 1, consumer warps only).
// ---------------------------------------------------------------------------------------
template <int NC>
__device__ __forceinline__ void cbar() {
  asm volatile("bar.sync 1, %0;" ::"r"(NC * 32) : "memory");
}

// Shared scratch of the consumer group: per-thread partials and the values
// that thread 0 broadcasts after each reduction.  Scalars of the iteration
// (alpha, beta, the stop test) are computed once per block by thread 0 (they
// are the same in every block: same totals, same operations), which keeps
// the slow FP64 units free of redundant work.
template <int NC>
struct CShared {
  double part[NC * 32];
  float ffp[2 * NC];
  double rr, val;
  float alpha, beta;
  int dec;
  int ok;
  int aux;
};

// Block partial of float-float sums, valid in thread 0 (float ops only until
// the final conversion).
template <int NC>
__device__ __forceinline__ double block_ff(FF v, CShared<NC>& S, bool f32) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = ff_warp_sum(v, f32);
  if (lane == 0) {
    S.ffp[2 * warp] = v.hi;
    S.ffp[2 * warp + 1] = v.lo;
  }
  cbar<NC>();
  double r = 0.0;
  if (warp == 0) {
    FF t = lane < NC ? FF{S.ffp[2 * lane], S.ffp[2 * lane + 1]} : FF{0.f, 0.f};
    t = ff_warp_sum(t, f32);
    r = (double)t.hi + (double)t.lo;
  }
  return r;
}

// Block partial of per-thread doubles, valid in thread 0 (one warp adds them
// in a fixed order).
template <int NC>
__device__ __forceinline__ double block_d(double p, CShared<NC>& S) {
  const int lane = threadIdx.x & 31;
  S.part[threadIdx.x] = p;
  cbar<NC>();
  double r = 0.0;
  if (threadIdx.x < 32) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < NC; ++j) s += S.part[lane + 32 * j];
    r = warp_sum(s);
  }
  return r;
}

// The waiting part of a grid barrier (thread 0): poll the arrival counter
// until it reaches target; bounded in device time; gives up when another
// block has recorded an error or the caller's cancel word is set.  Kept out
// of line so that its registers do not weigh on the CG loops.
__device__ __noinline__ int cgrid_wait(Ctl* ctl, int slot, unsigned long long target) {
  const unsigned long long t0 = globaltimer();
  unsigned spins = 0;
  while (ld_acquire(&ctl->bar[slot].v) < target) {
    if ((++spins & 1023u) == 0) {
      if (volatile_status(ctl) != 0 || poll_cancel(ctl)) return 0;
      if (globaltimer() - t0 > (unsigned long long)ctl->timeout_ns) {
        set_status(ctl, MPCG_ERR_TIMEOUT);
        return 0;
      }
    }
  }
  return 1;
}

// Grid barrier among the consumer groups of all blocks; bounded; also stops
// when another block has recorded an error.
template <int NC>
__device__ __forceinline__ bool cgrid_barrier(Ctl* ctl, int slot, unsigned long long& round,
                                              int* s_ok) {
  cbar<NC>();
  round += 1;
  if (threadIdx.x == 0) {
    const unsigned long long target = round * (unsigned long long)gridDim.x;
    red_release_add(&ctl->bar[slot].v, 1ull);
    int ok = 1;
    if (ld_acquire(&ctl->bar[slot].v) < target) ok = cgrid_wait(ctl, slot, target);
    *s_ok = ok;
  }
  cbar<NC>();
  return *s_ok != 0;
}

// Grid-wide sum of the block partials (block partial valid in thread 0;
// alternating halves of `partials`).  The total is valid in thread 0; the
// caller derives its scalars there and broadcasts them with cbar().
template <int NC>
__device__ __forceinline__ double cgrid_total(double block_part, double* partials, int& red,
                                              Ctl* ctl, int slot, unsigned long long& round,
                                              CShared<NC>& S, bool& ok, bool f32 = false,
                                              double* extra = nullptr) {
  double* buf = partials + (red & 1) * kMaxGrid;
  ++red;
  if (threadIdx.x == 0) buf[blockIdx.x] = block_part;
  ok = cgrid_barrier<NC>(ctl, slot, round, &S.ok);
  // extra (thread 0): the slot after the partials, which block 0 wrote before
  // the barrier; loaded beside them rather than after the sum
  if (extra && threadIdx.x == 0) *extra = buf[gridDim.x];
  double s = 0.0;
  if (threadIdx.x < 32) {
    if (f32) {  // option acc32: the blocks' float partials summed in float
      float sf = 0.0f;
      for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) sf = __fadd_rn(sf, (float)buf[i]);
      s = (double)warp_sum_f(sf);
    } else {
      for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) s += buf[i];
      s = warp_sum(s);
    }
  }
  return s;
}

// ---------------------------------------------------------------------------------------
// The streamed matrix ring.
// ---------------------------------------------------------------------------------------
template <typename T>
struct Ring {
  static constexpr int S = StageCfg<T>::kStages;
  char* base;                   // stage s: columns at base + s*stage_bytes, values after them
  unsigned long long* full;     // [S]
  unsigned long long* empty;    // [S]
  volatile int* stop;
  int E0, E1;                   // element range of the block
  unsigned nch;                 // chunks per pass
  int c16;                      // columns are int16 offsets from the row (Ctl::col16)
  __device__ __forceinline__ const int32_t* cols(int s) const {
    return reinterpret_cast<const int32_t*>(base + (size_t)s * stage_bytes<T>());
  }
  __device__ __forceinline__ const int16_t* cols16(int s) const {
    return reinterpret_cast<const int16_t*>(base + (size_t)s * stage_bytes<T>());
  }
  __device__ __forceinline__ const T* vals(int s) const {
    return reinterpret_cast<const T*>(base + (size_t)s * stage_bytes<T>() + kCH * sizeof(int32_t));
  }
};

// Producer: one thread.  Streams chunks g = 0, 1, 2, ... (chunk g % nch of the
// block's elements) until the consumers raise `stop`; then waits for every
// copy it issued before the block's shared memory can be released.
template <typename T>
__device__ void ring_producer(const CgArgs& a, Ring<T>& R) {
  constexpr int S = Ring<T>::S;
  if (R.nch == 0) return;
  const unsigned long long pol = l2_policy_evict_first();
  const T* sv = svals<T>(a);
  long long issued[S];
  for (int s = 0; s < S; ++s) issued[s] = -1;
  for (unsigned g = 0;; ++g) {
    if (*R.stop) break;
    const int st = (int)(g % S);
    const unsigned use = g / S;
    if (use >= 1 && !mbar_wait(&R.empty[st], (use - 1) & 1u, a.ctl, R.stop)) break;
    const unsigned c = g % R.nch;
    const int e = R.E0 + (int)(c << kLogCH);
    const int cnt = min(kCH, R.E1 - e);
    // int16 offsets: 2 bytes a column (element offsets and counts are
    // multiples of 32, so the copies stay 16-byte aligned)
    const uint32_t cb = R.c16 ? 2u : 4u;
    const void* csrc = R.c16 ? (const void*)(reinterpret_cast<const int16_t*>(a.scol) + e)
                             : (const void*)(a.scol + e);
    mbar_arrive_expect_tx(&R.full[st], (uint32_t)cnt * (cb + (uint32_t)sizeof(T)));
    bulk_g2s(const_cast<int32_t*>(R.cols(st)), csrc, (uint32_t)cnt * cb, &R.full[st], pol);
    bulk_g2s(const_cast<T*>(R.vals(st)), sv + e, (uint32_t)cnt * sizeof(T), &R.full[st], pol);
    issued[st] = g;
  }
  for (int s = 0; s < S; ++s)
    if (issued[s] >= 0) mbar_wait(&R.full[s], (unsigned)(issued[s] / S) & 1u, a.ctl, nullptr);
}

// Consumer-side cursor: chunks below `waited_plus1` are known full; chunks
// below `rel` have been released by this warp.
struct Cursor {
  unsigned pass_base, waited_plus1, rel;
};

// Release every chunk below g.  A chunk is released only after it has been
// filled: the producer fills chunk h only once every warp released chunk
// h - S, so an arrival for h always lands in the empty-barrier phase of h
// (a warp that skips chunks would otherwise count its arrival for h towards
// the phase of h - S while another warp still reads h - S).
template <typename T>
__device__ __forceinline__ bool ring_release_below(Ring<T>& R, Cursor& C, unsigned g, int lane,
                                                   Ctl* ctl) {
  while (C.rel < g) {
    if (C.rel >= C.waited_plus1) {
      if (!mbar_wait(&R.full[C.rel % Ring<T>::S], (C.rel / Ring<T>::S) & 1u, ctl, nullptr))
        return false;
      C.waited_plus1 = C.rel + 1;
    }
    if (lane == 0) mbar_arrive(&R.empty[C.rel % Ring<T>::S]);
    ++C.rel;
  }
  return true;
}

template <typename T>
__device__ __forceinline__ bool ring_acquire(Ring<T>& R, Cursor& C, unsigned g_lo, unsigned g_hi,
                                             Ctl* ctl) {
  unsigned g = C.waited_plus1 > g_lo ? C.waited_plus1 : g_lo;
  for (; g <= g_hi; ++g)
    if (!mbar_wait(&R.full[g % Ring<T>::S], (g / Ring<T>::S) & 1u, ctl, nullptr)) return false;
  if (g_hi + 1 > C.waited_plus1) C.waited_plus1 = g_hi + 1;
  return true;
}

// Chunk range [lo, hi] of a slice's k-rows (w > 0) relative to the pass.
__device__ __forceinline__ void slice_chunks(int r0, int w, unsigned& lo, unsigned& hi) {
  lo = (unsigned)r0 >> kLogCH;
  hi = (unsigned)(r0 + kSlice * (w - 1)) >> kLogCH;
}

// Load the (column, value) pairs of one slice row from the ring.  A slice
// spans at most two chunks: the stage of its first chunk and the next one.
// C16: the ring holds int16 offsets from the row index i.
template <typename T, bool C16>
__device__ __forceinline__ void ring_load_t(const Ring<T>& R, const Cursor& C, int r0, int w,
                                            int lane, int i, int (&c)[kFastW], T (&v)[kFastW]) {
  using CT = typename std::conditional<C16, int16_t, int32_t>::type;
  const unsigned g0 = C.pass_base + ((unsigned)r0 >> kLogCH);
  const int st0 = (int)(g0 % Ring<T>::S);
  const int st1 = st0 + 1 == Ring<T>::S ? 0 : st0 + 1;
  const int off0 = (r0 & (kCH - 1)) + lane;
  const int base = C16 ? i : 0;
  const CT* c0p = reinterpret_cast<const CT*>(R.cols(st0));
  const T* v0p = R.vals(st0);
  if ((r0 & (kCH - 1)) + kSlice * kFastW <= kCH) {  // the slice lies in one chunk
    const CT* cp = c0p + off0;
    const T* vp = v0p + off0;
#pragma unroll
    for (int k = 0; k < kFastW; ++k) {
      if (k < w) {
        c[k] = base + (int)cp[kSlice * k];
        v[k] = vp[kSlice * k];
      }
    }
    return;
  }
  const CT* c1p = reinterpret_cast<const CT*>(R.cols(st1));
  const T* v1p = R.vals(st1);
#pragma unroll
  for (int k = 0; k < kFastW; ++k) {
    if (k < w) {
      const int off = off0 + kSlice * k;
      const bool second = off >= kCH;
      const int o = second ? off - kCH : off;
      c[k] = base + (int)(second ? c1p[o] : c0p[o]);
      v[k] = second ? v1p[o] : v0p[o];
    }
  }
}
template <typename T>
__device__ __forceinline__ void ring_load(const Ring<T>& R, const Cursor& C, int r0, int w,
                                          int lane, int i, int (&c)[kFastW], T (&v)[kFastW]) {
  if (R.c16) ring_load_t<T, true>(R, C, r0, w, lane, i, c, v);
  else ring_load_t<T, false>(R, C, r0, w, lane, i, c, v);
}

// Row sum of one slice row, generic width, from the ring (plus the tail of an
// overflowing row from the caller's CSR).
template <typename T, class Gather>
__device__ __forceinline__ T ring_row_generic(const CgArgs& a, const Ring<T>& R, const Cursor& C,
                                              int r0, uint32_t wf, int i, int lane, Gather G) {
  const int w = (int)(wf & ~kOverflowBit);
  T acc = (T)0;
  for (int k = 0; k < w; ++k) {
    const int rr = r0 + kSlice * k + lane;
    const int st = (int)((C.pass_base + ((unsigned)rr >> kLogCH)) % Ring<T>::S);
    const int off = rr & (kCH - 1);
    const int cc = R.c16 ? i + (int)R.cols16(st)[off] : R.cols(st)[off];
    acc = fma(R.vals(st)[off], G(cc), acc);
  }
  if ((wf & kOverflowBit) && i < a.n) {
    const int e1 = a.rp[i + 1];
    for (int e = a.rp[i] + w; e < e1; ++e) acc = fma((T)a.val[e], G(a.col[e]), acc);
  }
  return acc;
}

__device__ __forceinline__ bool fast_w(uint32_t wf) {
  return !(wf & kOverflowBit) && (int)wf <= kFastW;
}

// One SpMV pass over the block's slices by the consumer warps.  For every
// row i of the block's slices (padding rows included), Rw(i, acc) receives
// sum_k v_k G(c_k) in stored order.  A warp takes two slices (s, s + kNC) per
// step when both fit in two chunks, so that the gathers of both rows are in
// flight together; a step never needs more than two chunks at once (the ring
// has at least four), which keeps the producer/consumer ring free of
// deadlock.  Returns false if a wait failed.
template <int NC, typename T, class Gather, class Row>
__device__ __forceinline__ bool ring_spmv(const CgArgs& a, Ring<T>& R, Cursor& C, int S0, int S1,
                                          Gather G, Row Rw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool ok = true;
  for (int s0 = S0 + warp; s0 < S1; s0 += 2 * NC) {
    const int s1 = s0 + NC;
    const bool h1 = s1 < S1;
    const uint32_t wf0 = a.slice_w[s0];
    const uint32_t wf1 = h1 ? a.slice_w[s1] : 0u;
    const int w0 = (int)(wf0 & ~kOverflowBit), w1 = (int)(wf1 & ~kOverflowBit);
    const int r00 = a.slice_ptr[s0] - R.E0;
    const int r01 = h1 ? a.slice_ptr[s1] - R.E0 : 0;
    const int i0 = s0 * kSlice + lane, i1 = s1 * kSlice + lane;
    unsigned lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
    if (w0 > 0) slice_chunks(r00, w0, lo0, hi0);
    if (w1 > 0) slice_chunks(r01, w1, lo1, hi1);
    const bool pair = h1 && w0 > 0 && w1 > 0 && fast_w(wf0) && fast_w(wf1) && hi1 <= lo0 + 1;
    if (pair) {
      if (ok) ok = ring_release_below(R, C, C.pass_base + lo0, lane, a.ctl);
      if (ok) ok = ring_acquire(R, C, C.pass_base + lo0, C.pass_base + hi1, a.ctl);
      T acc0 = (T)0, acc1 = (T)0;
      if (ok) {
        int c0[kFastW], c1[kFastW];
        T v0[kFastW], v1[kFastW];
        ring_load(R, C, r00, w0, lane, i0, c0, v0);
        ring_load(R, C, r01, w1, lane, i1, c1, v1);
#pragma unroll
        for (int k = 0; k < kFastW; ++k) {
          if (k < w0) acc0 = fma(v0[k], G(c0[k]), acc0);
          if (k < w1) acc1 = fma(v1[k], G(c1[k]), acc1);
        }
      }
      Rw(i0, acc0);
      Rw(i1, acc1);
      continue;
    }
    for (int j = 0; j < 2; ++j) {  // one slice at a time
      const bool hj = j == 0 || h1;
      if (!hj) break;
      const uint32_t wf = j ? wf1 : wf0;
      const int w = j ? w1 : w0;
      const int r0 = j ? r01 : r00;
      const int i = j ? i1 : i0;
      T acc = (T)0;
      if (w > 0) {
        const unsigned lo = j ? lo1 : lo0, hi = j ? hi1 : hi0;
        if (ok) ok = ring_release_below(R, C, C.pass_base + lo, lane, a.ctl);
        if (ok) ok = ring_acquire(R, C, C.pass_base + lo, C.pass_base + hi, a.ctl);
      }
      if (ok) {
        if (fast_w(wf)) {
          int c[kFastW];
          T v[kFastW];
          ring_load(R, C, r0, w, lane, i, c, v);
#pragma unroll
          for (int k = 0; k < kFastW; ++k)
            if (k < w) acc = fma(v[k], G(c[k]), acc);
        } else {
          acc = ring_row_generic(a, R, C, r0, wf, i, lane, G);
        }
      }
      Rw(i, acc);
    }
  }
  C.pass_base += R.nch;
  if (ok) ok = ring_release_below(R, C, C.pass_base, lane, a.ctl);
  return ok;
}

// Set-up common to both stages: the ring in dynamic shared memory, the
// block's slice range and element range, barrier initialisation.
template <int NC, typename T>
__device__ __forceinline__ void ring_setup(const CgArgs& a, char* smem, Ring<T>& R, int& S0,
                                           int& S1) {
  constexpr int S = Ring<T>::S;
  R.base = smem;
  R.full = reinterpret_cast<unsigned long long*>(smem + S * stage_bytes<T>());
  R.empty = R.full + S;
  R.stop = reinterpret_cast<volatile int*>(R.empty + S);
  S0 = (int)((long long)a.nslices * blockIdx.x / gridDim.x);
  S1 = (int)((long long)a.nslices * (blockIdx.x + 1) / gridDim.x);
  R.E0 = a.slice_ptr[S0];
  R.E1 = a.slice_ptr[S1];
  R.nch = (unsigned)((R.E1 - R.E0 + kCH - 1) >> kLogCH);
  R.c16 = a.ctl->col16;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&R.full[s], 1);
      mbar_init(&R.empty[s], NC);
    }
    *R.stop = 0;
    mbar_fence_init();
  }
  __syncthreads();
}

// Rows [R0, R1) of consumer warp `warp` inside the block's row range.
template <int NC>
__device__ __forceinline__ void warp_rows(int S0, int S1, int n, int& R0, int& R1) {
  const int warp = threadIdx.x >> 5;
  const int B0 = S0 * kSlice, B1 = min(S1 * kSlice, n);
  const int rows = max(0, B1 - B0);
  // split in multiples of 4 rows so that 16-byte vectors stay aligned
  const int q4 = (rows + 3) >> 2;
  R0 = B0 + 4 * (int)((long long)q4 * warp / NC);
  R1 = min(B1, B0 + 4 * (int)((long long)q4 * (warp + 1) / NC));
}

// ---------------------------------------------------------------------------------------
// Single-precision stage.
//   mode kCgK0:      start from x = 0; at most k0 iterations; stop early when
//                    the residual reaches eps2 or 0; accumulate Eq. (13).
//   mode kCgToEps1:  start from x = 0; iterate to eps1 (Algorithm I).
//   mode kCgContinue continue the state left by kCgK0 to eps1 (Algorithm II).
// ---------------------------------------------------------------------------------------

// x += alpha d, r -= alpha q, r^T r over rows [R0, R1): four rows per lane,
// two groups of four in flight.
// x += alpha d, r -= alpha q, r^T r for four rows whose operands are loaded.
__device__ __forceinline__ void upd32(const CgArgs& a, int i, float4 d4, float4 q4, float4 x4,
                                      float4 r4, float alpha, FF& prr, bool f32) {
  x4.x = __fmaf_rn(alpha, d4.x, x4.x);
  x4.y = __fmaf_rn(alpha, d4.y, x4.y);
  x4.z = __fmaf_rn(alpha, d4.z, x4.z);
  x4.w = __fmaf_rn(alpha, d4.w, x4.w);
  r4.x = __fmaf_rn(-alpha, q4.x, r4.x);
  r4.y = __fmaf_rn(-alpha, q4.y, r4.y);
  r4.z = __fmaf_rn(-alpha, q4.z, r4.z);
  r4.w = __fmaf_rn(-alpha, q4.w, r4.w);
  *reinterpret_cast<float4*>(a.x32 + i) = x4;
  *reinterpret_cast<float4*>(a.r32 + i) = r4;
  ff_add_prod(prr, r4.x, r4.x, f32);
  ff_add_prod(prr, r4.y, r4.y, f32);
  ff_add_prod(prr, r4.z, r4.z, f32);
  ff_add_prod(prr, r4.w, r4.w, f32);
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// Rows [R0, R1): four rows per lane, two groups of four; every operand of
// both groups is loaded before the first store (stores to x and r could
// alias later loads, so the compiler would not reorder them).
__device__ __forceinline__ void p2_32(const CgArgs& a, int R0, int R1, int lane, const float* d,
                                      float alpha, FF& prr, bool f32) {
  for (int base = R0 + 4 * lane; base < R1; base += 8 * kSlice) {
    const int b2 = base + 4 * kSlice;
    if (b2 + 4 <= R1) {
      const float4 d4 = ld4(d + base), q4 = ld4(a.q32 + base);
      const float4 x4 = ld4(a.x32 + base), r4 = ld4(a.r32 + base);
      const float4 e4 = ld4(d + b2), s4 = ld4(a.q32 + b2);
      const float4 y4 = ld4(a.x32 + b2), t4 = ld4(a.r32 + b2);
      upd32(a, base, d4, q4, x4, r4, alpha, prr, f32);
      upd32(a, b2, e4, s4, y4, t4, alpha, prr, f32);
    } else {
      for (int g = base; g < R1 && g <= b2; g += 4 * kSlice) {
        if (g + 4 <= R1) {
          upd32(a, g, ld4(d + g), ld4(a.q32 + g), ld4(a.x32 + g), ld4(a.r32 + g), alpha, prr, f32);
        } else {
          for (int i = g; i < R1; ++i) {
            a.x32[i] = __fmaf_rn(alpha, d[i], a.x32[i]);
            const float ri = __fmaf_rn(-alpha, a.q32[i], a.r32[i]);
            a.r32[i] = ri;
            ff_add_prod(prr, ri, ri, f32);
          }
        }
      }
    }
  }
}

// Preconditioned form: also z = dinv r (stored; the next P1 forms d from it)
// and r^T z.  Four rows per lane, every operand loaded before the stores.
__device__ __forceinline__ void p2_32_pc(const CgArgs& a, int R0, int R1, int lane, const float* d,
                                         float alpha, FF& prr, FF& prz, bool f32) {
  for (int base = R0 + 4 * lane; base < R1; base += 4 * kSlice) {
    if (base + 4 <= R1) {
      const float4 d4 = ld4(d + base), q4 = ld4(a.q32 + base), m4 = ld4(a.dinv32 + base);
      float4 x4 = ld4(a.x32 + base), r4 = ld4(a.r32 + base), z4;
      x4.x = __fmaf_rn(alpha, d4.x, x4.x);
      x4.y = __fmaf_rn(alpha, d4.y, x4.y);
      x4.z = __fmaf_rn(alpha, d4.z, x4.z);
      x4.w = __fmaf_rn(alpha, d4.w, x4.w);
      r4.x = __fmaf_rn(-alpha, q4.x, r4.x);
      r4.y = __fmaf_rn(-alpha, q4.y, r4.y);
      r4.z = __fmaf_rn(-alpha, q4.z, r4.z);
      r4.w = __fmaf_rn(-alpha, q4.w, r4.w);
      z4.x = __fmul_rn(m4.x, r4.x);
      z4.y = __fmul_rn(m4.y, r4.y);
      z4.z = __fmul_rn(m4.z, r4.z);
      z4.w = __fmul_rn(m4.w, r4.w);
      *reinterpret_cast<float4*>(a.x32 + base) = x4;
      *reinterpret_cast<float4*>(a.r32 + base) = r4;
      *reinterpret_cast<float4*>(a.z32 + base) = z4;
      ff_add_prod(prr, r4.x, r4.x, f32);
      ff_add_prod(prr, r4.y, r4.y, f32);
      ff_add_prod(prr, r4.z, r4.z, f32);
      ff_add_prod(prr, r4.w, r4.w, f32);
      ff_add_prod(prz, r4.x, z4.x, f32);
      ff_add_prod(prz, r4.y, z4.y, f32);
      ff_add_prod(prz, r4.z, z4.z, f32);
      ff_add_prod(prz, r4.w, z4.w, f32);
    } else {
      for (int i = base; i < R1; ++i) {
        a.x32[i] = __fmaf_rn(alpha, d[i], a.x32[i]);
        const float ri = __fmaf_rn(-alpha, a.q32[i], a.r32[i]);
        const float zi = __fmul_rn(a.dinv32[i], ri);
        a.r32[i] = ri;
        a.z32[i] = zi;
        ff_add_prod(prr, ri, ri, f32);
        ff_add_prod(prz, ri, zi, f32);
      }
    }
  }
}

enum Dec { kGo = 0, kStop = 1, kNan = 2, kBroke = 3, kBreakdown = 4, kCancel = 5 };

// kPc: Jacobi-preconditioned CG (the PCG form of Sec. 5): z = dinv r is
// kept beside r, d is formed from z, alpha = r^T z / d^T q and
// beta = r'^T z' / r^T z; the stop test and v stay on r.
// kTrue: the stop test as the CG procedure of Sec. 3 prints it, on
// ||b~ - A~ x~|| of the current iterate: one more pass over the matrix at the
// head of every iteration, t = b~ - A~ x~ rounded in single precision and
// t^T t summed like the other norms.  v (Eq. 13) stays on the recursive r.
// A stage whose recursive r has fallen 1e3 times below ||b - A x|| is taken
// as stagnated (the true residual of Sec. 7, Fig. 2, no longer falls) and
// ends as at its iteration cap.  The paper gives no such rule; the factor
// 1e3 is this implementation's choice.
constexpr double kStagnationRR = 1e-6;  // on squares: r^T r <= 1e-6 ||b - A x||^2

template <bool kPc, bool kTrue>
__global__ void __launch_bounds__(kTmaThreads, 1) k_cg32(CgArgs a) {
  constexpr int NC = kNC;
  extern __shared__ __align__(128) char smem[];
  __shared__ CShared<NC> S;
  Ctl* ctl = a.ctl;
  if (volatile_status(ctl) != 0 || ctl->trivial) return;
  if (a.mode == kCgContinue && ctl->broke32) {  // stage 1 already ended in the k0 phase
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (ctl->res32 > ctl->eps1) ctl->warn_eps1 = 1;
      ctl->t_fp32 = globaltimer();
    }
    return;
  }
  Ring<float> R;
  int S0, S1;
  ring_setup<NC>(a, smem, R, S0, S1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == NC) {
    if (lane == 0) ring_producer(a, R);
    return;
  }
  const bool lead = threadIdx.x == 0;           // computes the block's scalars
  const bool lead0 = lead && blockIdx.x == 0;   // writes the control block
  Cursor C{0u, 0u, 0u};
  int R0, R1;
  warp_rows<NC>(S0, S1, a.n, R0, R1);
  const int n = a.n;
  const int rel = ctl->tol_relative;
  const bool f32 = ctl->acc32 != 0;  // inner products summed in float (option acc32)
  unsigned long long round = 0;
  int red = 0;
  bool ok = true;

  double rr, bnorm;  // identical in every thread after each broadcast
  double rz = 0.0;   // r^T z (kPc; thread 0)
  float beta;
  int first, parity, it;
  if (a.mode != kCgContinue) {
    // CG line 1: x0 = 0, r0 = b - A x0 = b~, d0 = r0 (kPc: z0 = dinv r0, d0 = z0).
    FF acc{0.f, 0.f}, accz{0.f, 0.f};
    for (int i = R0 + lane; i < R1; i += kSlice) {
      const float bi = a.b32[i];
      a.x32[i] = 0.0f;
      a.r32[i] = bi;
      a.da[i] = 0.0f;  // d_{-1}
      ff_add_prod(acc, bi, bi, f32);
      if constexpr (kPc) {
        const float zi = __fmul_rn(a.dinv32[i], bi);
        a.z32[i] = zi;
        ff_add_prod(accz, bi, zi, f32);
      }
    }
    const double tot = cgrid_total(block_ff(acc, S, f32), a.partials, red, ctl, a.slot, round, S, ok, f32);
    if constexpr (kPc) rz = cgrid_total(block_ff(accz, S, f32), a.partials, red, ctl, a.slot, round, S, ok, f32);
    if (lead) {
      S.rr = tot;
      S.val = sqrt(tot);  // ||b~|| = ||r0||
      if (lead0) {
        ctl->bnorm32 = S.val;
        if (!isfinite(S.val)) set_status(ctl, MPCG_ERR_NAN);
      }
    }
    cbar<NC>();
    rr = S.rr;
    bnorm = S.val;
    first = 1;
    parity = 0;
    beta = 0.0f;
    it = 0;
    if (!isfinite(bnorm)) ok = false;
  } else {
    rr = ctl->rr;
    bnorm = ctl->bnorm32;
    beta = ctl->beta32;
    first = ctl->first;
    parity = ctl->parity;
    it = ctl->n1;
    if constexpr (kPc) rz = ctl->rz;
  }
  const double eps = a.mode == kCgK0 ? ctl->eps2 : ctl->eps1;
  const int limit = a.mode == kCgK0 ? min(ctl->k0, ctl->max1) : ctl->max1;
  const StopThr thr = stop_thr(eps, bnorm, rel);  // used by thread 0
  double vsum = 0.0;  // thread 0
  int k0done = 0, broke = 0;
  double trr = 0.0;   // kTrue: ||b~ - A~ x~||^2 of the current iterate (thread 0)
  int cw = 0;         // the cancel word as block 0's thread 0 read it during the last pass

  while (ok) {
    if constexpr (kTrue) {
      FF pt{0.f, 0.f};
      const float* xv = a.x32;
      const float* bv = a.b32;
      auto Gx = [&](int c) -> float { return xv[c]; };
      auto Rt = [&](int i, float acc) {
        if (i < n) {
          const float t = __fsub_rn(bv[i], acc);
          ff_add_prod(pt, t, t, f32);
        }
      };
      if (!ring_spmv<NC, float>(a, R, C, S0, S1, Gx, Rt)) set_status(ctl, MPCG_ERR_TIMEOUT);
      trr = cgrid_total(block_ff(pt, S, f32), a.partials, red, ctl, a.slot, round, S, ok, f32);
      if (!ok) break;
    }
    if (lead) {
      const double rs = kTrue ? trr : rr;  // the stop test's r^T r
      int dec = kGo;
      if (isnan(rr) || isnan(rs)) dec = kNan;
      else if (stop_pass(thr, rs) || it >= limit || (a.mode == kCgK0 && rr == 0.0) ||
               (kTrue && rr <= kStagnationRR * rs))
        dec = kStop;
      if (lead0 && cw != 0) {  // the caller cancelled; the other blocks stop at their next wait
        set_status(ctl, MPCG_ERR_CANCELLED);
        dec = kCancel;
      }
      S.dec = dec;
      if (dec == kNan && lead0) set_status(ctl, MPCG_ERR_NAN);
    }
    cbar<NC>();
    if (S.dec != kGo) break;
    if (lead0) cw = cancel_word(ctl);  // consumed at the next loop head: latency hidden

    // ---- P1: q = A d_k with d_k = r_k + beta_k d_{k-1} formed on the fly ----
    // Plain (coherent) pointers: these vectors change between iterations of
    // this launch, so they must not go through the read-only data path.
    const float* dold = parity ? a.db : a.da;
    float* dnew = parity ? a.da : a.db;
    const float* r = kPc ? a.z32 : a.r32;  // d is formed from z under kPc
    float* q = a.q32;
    FF pdq{0.f, 0.f};
    // d_0 = r_0 is the same formula with beta = 0 and d_{-1} = 0 (zeroed at
    // the start): fma(0, 0, r) = r.
    const float bt = first ? 0.0f : beta;
    auto G = [&](int c) -> float { return __fmaf_rn(bt, dold[c], r[c]); };
    auto Rw = [&](int i, float acc) {
      if (i < n) {
        const float di = __fmaf_rn(bt, dold[i], r[i]);
        dnew[i] = di;
        q[i] = acc;
        ff_add_prod(pdq, di, acc, f32);
      }
    };
    const bool pass_ok = ring_spmv<NC, float>(a, R, C, S0, S1, G, Rw);
    if (!pass_ok) set_status(ctl, MPCG_ERR_TIMEOUT);
    {
      const double dq = cgrid_total(block_ff(pdq, S, f32), a.partials, red, ctl, a.slot, round, S, ok, f32);
      if (lead) {
        int dec = kGo;
        if (!isfinite(dq)) dec = kNan;
        else if (!(dq > 0.0)) dec = kBroke;  // stage 1 ends here; x and r are unchanged
        else S.alpha = (float)((kPc ? rz : rr) / dq);
        S.dec = dec;
        if (dec == kNan && lead0) set_status(ctl, MPCG_ERR_NAN);
      }
      cbar<NC>();
    }
    if (!ok) break;
    if (S.dec == kBroke) {
      broke = 1;
      break;
    }
    if (S.dec != kGo) break;
    const float alpha = S.alpha;

    // ---- P2: x += alpha d_k, r -= alpha q, r^T r (kPc: also z = dinv r, r^T z) ----
    FF prr{0.f, 0.f}, prz{0.f, 0.f};
    if constexpr (kPc) p2_32_pc(a, R0, R1, lane, dnew, alpha, prr, prz, f32);
    else p2_32(a, R0, R1, lane, dnew, alpha, prr, f32);
    {
      const double rrn = cgrid_total(block_ff(prr, S, f32), a.partials, red, ctl, a.slot, round, S, ok, f32);
      double rzn = 0.0;
      if constexpr (kPc)
        rzn = cgrid_total(block_ff(prz, S, f32), a.partials, red, ctl, a.slot, round, S, ok, f32);
      if (lead) {
        int dec = kGo;
        if (!isfinite(rrn) || (kPc && !isfinite(rzn))) {
          dec = kNan;
          if (lead0) set_status(ctl, MPCG_ERR_NAN);
        } else {
          if (a.mode == kCgK0) vsum += sqrt(rrn) / sqrt(rr);  // Eq. (13) ratio
          if constexpr (kPc) {
            S.beta = (float)(rzn / rz);
            rz = rzn;
          } else {
            S.beta = (float)(rrn / rr);
          }
          S.rr = rrn;
        }
        S.dec = dec;
      }
      cbar<NC>();
    }
    if (!ok || S.dec != kGo) break;
    if (a.mode == kCgK0) ++k0done;
    beta = S.beta;
    rr = S.rr;
    parity ^= 1;
    first = 0;
    ++it;
  }
  if (lead) *R.stop = 1;

  if (lead0) {
    ctl->rr = rr;
    if constexpr (kPc) ctl->rz = rz;
    ctl->beta32 = beta;
    ctl->first = first;
    ctl->parity = parity;
    ctl->n1 = it;
    ctl->res32 = stop_measure(kTrue ? trr : rr, bnorm, rel);
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

__device__ __forceinline__ double2 ld2(const double* p) {
  return *reinterpret_cast<const double2*>(p);
}

// P2: r -= alpha q and r^T r over rows [R0, R1), both pairs of a step loaded
// first.  (x += alpha d waits for P3, which reads d anyway.)
__device__ __forceinline__ double p2_64(const CgArgs& a, int R0, int R1, int lane, double alpha) {
  double prr = 0.0;
  for (int base = R0 + 2 * lane; base < R1; base += 4 * kSlice) {
    const int g1 = base + 2 * kSlice;
    if (g1 + 2 <= R1) {
      const double2 q0 = ld2(a.q64 + base), q1 = ld2(a.q64 + g1);
      double2 r0 = ld2(a.r64 + base), r1 = ld2(a.r64 + g1);
      r0.x = __fma_rn(-alpha, q0.x, r0.x);
      r0.y = __fma_rn(-alpha, q0.y, r0.y);
      r1.x = __fma_rn(-alpha, q1.x, r1.x);
      r1.y = __fma_rn(-alpha, q1.y, r1.y);
      *reinterpret_cast<double2*>(a.r64 + base) = r0;
      *reinterpret_cast<double2*>(a.r64 + g1) = r1;
      prr = __fma_rn(r0.x, r0.x, prr);
      prr = __fma_rn(r0.y, r0.y, prr);
      prr = __fma_rn(r1.x, r1.x, prr);
      prr = __fma_rn(r1.y, r1.y, prr);
      continue;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = base + h * 2 * kSlice;
      if (g + 2 <= R1) {
        const double2 q2 = ld2(a.q64 + g);
        double2 r2 = ld2(a.r64 + g);
        r2.x = __fma_rn(-alpha, q2.x, r2.x);
        r2.y = __fma_rn(-alpha, q2.y, r2.y);
        *reinterpret_cast<double2*>(a.r64 + g) = r2;
        prr = __fma_rn(r2.x, r2.x, prr);
        prr = __fma_rn(r2.y, r2.y, prr);
      } else if (g < R1) {
        const double ri = __fma_rn(-alpha, a.q64[g], a.r64[g]);
        a.r64[g] = ri;
        prr = __fma_rn(ri, ri, prr);
      }
    }
  }
  return prr;
}

// P3: x += alpha d (the step of P2, with the d it used), then d = r + beta d,
// over rows [R0, R1), both pairs of a step loaded first.
__device__ __forceinline__ void p3_64(const CgArgs& a, int R0, int R1, int lane, double alpha,
                                      double beta) {
  for (int base = R0 + 2 * lane; base < R1; base += 4 * kSlice) {
    const int g1 = base + 2 * kSlice;
    if (g1 + 2 <= R1) {
      double2 d0 = ld2(a.d64 + base), d1 = ld2(a.d64 + g1);
      double2 x0 = ld2(a.x64 + base), x1 = ld2(a.x64 + g1);
      const double2 r0 = ld2(a.r64 + base), r1 = ld2(a.r64 + g1);
      x0.x = __fma_rn(alpha, d0.x, x0.x);
      x0.y = __fma_rn(alpha, d0.y, x0.y);
      x1.x = __fma_rn(alpha, d1.x, x1.x);
      x1.y = __fma_rn(alpha, d1.y, x1.y);
      d0.x = __fma_rn(beta, d0.x, r0.x);
      d0.y = __fma_rn(beta, d0.y, r0.y);
      d1.x = __fma_rn(beta, d1.x, r1.x);
      d1.y = __fma_rn(beta, d1.y, r1.y);
      *reinterpret_cast<double2*>(a.x64 + base) = x0;
      *reinterpret_cast<double2*>(a.x64 + g1) = x1;
      *reinterpret_cast<double2*>(a.d64 + base) = d0;
      *reinterpret_cast<double2*>(a.d64 + g1) = d1;
      continue;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = base + h * 2 * kSlice;
      if (g + 2 <= R1) {
        double2 d2 = ld2(a.d64 + g), x2 = ld2(a.x64 + g);
        const double2 r2 = ld2(a.r64 + g);
        x2.x = __fma_rn(alpha, d2.x, x2.x);
        x2.y = __fma_rn(alpha, d2.y, x2.y);
        d2.x = __fma_rn(beta, d2.x, r2.x);
        d2.y = __fma_rn(beta, d2.y, r2.y);
        *reinterpret_cast<double2*>(a.x64 + g) = x2;
        *reinterpret_cast<double2*>(a.d64 + g) = d2;
      } else if (g < R1) {
        const double dg = a.d64[g];
        a.x64[g] = __fma_rn(alpha, dg, a.x64[g]);
        a.d64[g] = __fma_rn(beta, dg, a.r64[g]);
      }
    }
  }
}

// Preconditioned P2: r -= alpha q; returns r^T r and, in *prz, r^T z with
// z = dinv r (z is not stored: P3 forms it again; x waits for P3 too).
__device__ __forceinline__ double p2_64_pc(const CgArgs& a, int R0, int R1, int lane, double alpha,
                                           double* prz) {
  double prr = 0.0, pz = 0.0;
  for (int g = R0 + 2 * lane; g < R1; g += 2 * kSlice) {
    if (g + 2 <= R1) {
      const double2 q2 = ld2(a.q64 + g), m2 = ld2(a.dinv64 + g);
      double2 r2 = ld2(a.r64 + g);
      r2.x = __fma_rn(-alpha, q2.x, r2.x);
      r2.y = __fma_rn(-alpha, q2.y, r2.y);
      *reinterpret_cast<double2*>(a.r64 + g) = r2;
      prr = __fma_rn(r2.x, r2.x, prr);
      prr = __fma_rn(r2.y, r2.y, prr);
      pz = __fma_rn(r2.x, __dmul_rn(m2.x, r2.x), pz);
      pz = __fma_rn(r2.y, __dmul_rn(m2.y, r2.y), pz);
    } else if (g < R1) {
      const double ri = __fma_rn(-alpha, a.q64[g], a.r64[g]);
      a.r64[g] = ri;
      prr = __fma_rn(ri, ri, prr);
      pz = __fma_rn(ri, __dmul_rn(a.dinv64[g], ri), pz);
    }
  }
  *prz = pz;
  return prr;
}

// Preconditioned P3: x += alpha d, then d = dinv r + beta d.
__device__ __forceinline__ void p3_64_pc(const CgArgs& a, int R0, int R1, int lane, double alpha,
                                         double beta) {
  for (int g = R0 + 2 * lane; g < R1; g += 2 * kSlice) {
    if (g + 2 <= R1) {
      double2 d2 = ld2(a.d64 + g), x2 = ld2(a.x64 + g);
      const double2 r2 = ld2(a.r64 + g), m2 = ld2(a.dinv64 + g);
      x2.x = __fma_rn(alpha, d2.x, x2.x);
      x2.y = __fma_rn(alpha, d2.y, x2.y);
      d2.x = __fma_rn(beta, d2.x, __dmul_rn(m2.x, r2.x));
      d2.y = __fma_rn(beta, d2.y, __dmul_rn(m2.y, r2.y));
      *reinterpret_cast<double2*>(a.x64 + g) = x2;
      *reinterpret_cast<double2*>(a.d64 + g) = d2;
    } else if (g < R1) {
      const double dg = a.d64[g];
      a.x64[g] = __fma_rn(alpha, dg, a.x64[g]);
      a.d64[g] = __fma_rn(beta, dg, __dmul_rn(a.dinv64[g], a.r64[g]));
    }
  }
}

// Kinds of SpMV pass in the double-precision stage.
enum Pass64 { kRestart = 0, kTrueRes = 1, kIterate = 2, kFinalRes = 3, kDone = 4, kCheck = 5 };

// kPc: Jacobi-preconditioned CG (the PCG form of Sec. 5): restarts set
// d = z = dinv r, alpha = r^T z / d^T q, beta = r'^T z' / r^T z and
// d = z + beta d; the stop test and the true residual stay on r.
// kTrue: the stop test as the CG procedure of Sec. 3 prints it: a kCheck
// pass computes ||b - A x||^2 at the head of every iteration and decides on
// it, so the stage ends on its true residual (no true-residual restart), or
// as not converged at the cap or once stagnated (as k_cg32).
template <bool kPc, bool kTrue>
__global__ void __launch_bounds__(kTmaThreads, 1) k_cg64(CgArgs a) {
  constexpr int NC = kNC;
  extern __shared__ __align__(128) char smem[];
  __shared__ CShared<NC> S;
  Ctl* ctl = a.ctl;
  if (volatile_status(ctl) != 0) return;
  Ring<double> R;
  int S0, S1;
  ring_setup<NC>(a, smem, R, S0, S1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = a.n;
  if (ctl->trivial) {  // b = 0: x = 0 solves A x = b exactly
    if (warp < NC) {
      int R0, R1;
      warp_rows<NC>(S0, S1, n, R0, R1);
      for (int i = R0 + lane; i < R1; i += kSlice) a.x64[i] = 0.0;
    }
    return;
  }
  if (warp == NC) {
    if (lane == 0) ring_producer(a, R);
    return;
  }
  const bool lead = threadIdx.x == 0;
  const bool lead0 = lead && blockIdx.x == 0;
  Cursor C{0u, 0u, 0u};
  int R0, R1;
  warp_rows<NC>(S0, S1, n, R0, R1);
  const int rel = ctl->tol_relative;
  const double bnorm = ctl->bnorm64;
  const double eps2 = ctl->eps2;
  const int max2 = ctl->max2;
  const int max_restarts = ctl->max_restarts;
  unsigned long long round = 0;
  int red = 0;
  bool ok = true;
  int it = 0, restarts = 0;
  int failed = 0;                  // thread 0
  double true_rel = NAN;  // thread 0
  double trr = NAN;       // kTrue: ||b - A x||^2 of the last check (thread 0)
  const StopThr thr2 = stop_thr(eps2, bnorm, rel);  // used by thread 0
  double rr = 0.0;                 // thread 0
  double rz = 0.0;                 // r^T z (kPc; thread 0)

  // Promote: x0 = float64(x~) (or 0).
  {
    const int src = ctl->x32_src;
    const float* xs = src >= 0 ? a.snap + (size_t)src * n : a.x32;
    for (int i = R0 + lane; i < R1; i += kSlice) a.x64[i] = a.mode ? 0.0 : (double)xs[i];
  }
  ok = cgrid_barrier<NC>(ctl, a.slot, round, &S.ok);

  // One SpMV pass per step; its kind is decided by thread 0 and broadcast.
  //   kRestart:  r = b - A x, d = r, r^T r      (CG line 1 from x)
  //   kTrueRes:  q = b - A x, ||q||^2           (true residual at eps2)
  //   kIterate:  q = A d, d^T q; then the x, r update and d = r + beta d
  //   kFinalRes: ||b - A x||^2 after the cap
  //   kCheck:    ||b - A x||^2, the stop test of kTrue
  int kind = kRestart;
  const double* x = a.x64;
  int cw = 0;  // the cancel word as block 0's thread 0 read it during the last pass
  while (ok && kind != kDone) {
    if (lead0) cw = cancel_word(ctl);  // consumed at the next loop head: latency hidden
    const double* gv = kind == kIterate ? a.d64 : x;
    double p = 0.0, pz = 0.0;
    {
      const int knd = kind;
      double* r = a.r64;
      double* d = a.d64;
      double* q = a.q64;
      const double* b = a.b64;
      auto G = [&](int c) -> double { return gv[c]; };
      auto Rw = [&](int i, double acc) {
        if (i < n) {
          if (knd == kIterate) {
            q[i] = acc;
            p = __fma_rn(d[i], acc, p);
          } else {
            const double ri = b[i] - acc;
            if (knd == kRestart) {
              r[i] = ri;
              if constexpr (kPc) {
                const double zi = __dmul_rn(a.dinv64[i], ri);
                d[i] = zi;
                pz = __fma_rn(ri, zi, pz);
              } else {
                d[i] = ri;
              }
            } else if (knd == kTrueRes) {
              q[i] = ri;
            }
            p = __fma_rn(ri, ri, p);
          }
        }
      };
      if (!ring_spmv<NC, double>(a, R, C, S0, S1, G, Rw)) set_status(ctl, MPCG_ERR_TIMEOUT);
    }
    const double tot = cgrid_total(block_d(p, S), a.partials, red, ctl, a.slot, round, S, ok);
    if constexpr (kPc) {
      if (kind == kRestart) {  // uniform: r^T z of the restart
        const double tz = cgrid_total(block_d(pz, S), a.partials, red, ctl, a.slot, round, S, ok);
        if (lead) rz = tz;
      }
    }
    if (!ok) break;

    // ---- thread 0: the scalars and the next pass ----
    if (lead) {
      int next = kDone;
      if (kTrue && kind == kCheck) {
        true_rel = bnorm > 0.0 ? sqrt(tot) / bnorm : sqrt(tot);
        trr = tot;
        if (isnan(tot)) failed = MPCG_ERR_NAN;
        else if (stop_pass(thr2, tot)) next = kDone;
        else if (it >= max2 || rr <= kStagnationRR * tot) failed = MPCG_ERR_NOT_CONVERGED;
        else next = kIterate;
      } else if (kind == kFinalRes) {
        true_rel = bnorm > 0.0 ? sqrt(tot) / bnorm : sqrt(tot);
      } else if (kind == kTrueRes) {
        true_rel = bnorm > 0.0 ? sqrt(tot) / bnorm : sqrt(tot);
        const double tm = rel ? true_rel : sqrt(tot);
        if (tm > eps2) {
          if (restarts < max_restarts) {
            next = kTrueRes + 100;  // restart from x: r = d = q, then the loop head
            rr = tot;
          } else {
            failed = MPCG_ERR_NOT_CONVERGED;  // the last restart still missed eps2
          }
        }
      } else if (kind == kIterate) {
        if (!isfinite(tot)) {
          failed = MPCG_ERR_NAN;
        } else if (!(tot > 0.0)) {
          failed = MPCG_ERR_BREAKDOWN;
        } else {
          S.val = (kPc ? rz : rr) / tot;  // alpha
          next = kIterate;
        }
      } else {  // kRestart
        rr = tot;
        next = -1;  // loop head
      }
      S.dec = next;
    }
    cbar<NC>();
    int next = S.dec;

    if (kind == kIterate && next == kIterate) {
      // ---- P2: r -= alpha q, r^T r ----
      const double alpha = S.val;
      double przl = 0.0;
      double prr;
      if constexpr (kPc) prr = p2_64_pc(a, R0, R1, lane, alpha, &przl);
      else prr = p2_64(a, R0, R1, lane, alpha);
      const double rrn = cgrid_total(block_d(prr, S), a.partials, red, ctl, a.slot, round, S, ok);
      double rzn = 0.0;
      if constexpr (kPc)
        rzn = cgrid_total(block_d(przl, S), a.partials, red, ctl, a.slot, round, S, ok);
      if (lead) {
        if (!isfinite(rrn) || (kPc && !isfinite(rzn))) {
          failed = MPCG_ERR_NAN;
          S.dec = kDone;
        } else {
          if constexpr (kPc) {
            S.val = rzn / rz;  // beta
            rz = rzn;
          } else {
            S.val = rrn / rr;  // beta
          }
          rr = rrn;
          S.dec = -1;
        }
      }
      cbar<NC>();
      if (!ok || S.dec == kDone) break;
      // ---- P3: x += alpha d, d = r + beta d (kPc: d = dinv r + beta d) ----
      if constexpr (kPc) p3_64_pc(a, R0, R1, lane, alpha, S.val);
      else p3_64(a, R0, R1, lane, alpha, S.val);
      ok = cgrid_barrier<NC>(ctl, a.slot, round, &S.ok);
      ++it;
      next = -1;
    } else if (next == kTrueRes + 100) {
      ++restarts;
      double pzr = 0.0;
      for (int i = R0 + lane; i < R1; i += kSlice) {
        const double ri = a.q64[i];
        a.r64[i] = ri;
        if constexpr (kPc) {
          const double zi = __dmul_rn(a.dinv64[i], ri);
          a.d64[i] = zi;
          pzr = __fma_rn(ri, zi, pzr);
        } else {
          a.d64[i] = ri;
        }
      }
      if constexpr (kPc) {
        const double tz = cgrid_total(block_d(pzr, S), a.partials, red, ctl, a.slot, round, S, ok);
        if (lead) rz = tz;
      } else {
        ok = cgrid_barrier<NC>(ctl, a.slot, round, &S.ok);
      }
      next = -1;
    }
    if (next == -1) {  // loop head: stop test on the recursive residual
      if (lead) {
        int nk = kIterate;
        if (lead0 && cw != 0) {  // the caller cancelled; the other blocks stop at their next wait
          failed = MPCG_ERR_CANCELLED;
          set_status(ctl, MPCG_ERR_CANCELLED);
          nk = kDone;
        } else if (isnan(rr)) {
          failed = MPCG_ERR_NAN;
          nk = kDone;
        } else if (kTrue) {
          nk = kCheck;  // the decision follows the check pass
        } else if (stop_pass(thr2, rr)) {
          nk = kTrueRes;
        } else if (it >= max2) {
          failed = MPCG_ERR_NOT_CONVERGED;
          nk = kFinalRes;
        }
        S.dec = nk;
      }
      cbar<NC>();
      next = S.dec;
    }
    kind = next;
  }

  if (lead) *R.stop = 1;
  if (lead0) {
    if (failed) set_status(ctl, failed);
    ctl->n2 = it;
    ctl->restarts = restarts;
    if (restarts) ctl->warn_restart = 1;
    ctl->res64 = stop_measure(kTrue ? trr : rr, bnorm, rel);
    ctl->true_rel = true_rel;
    ctl->rr = rr;
    ctl->t_fp64 = globaltimer();
  }
}


// ---------------------------------------------------------------------------------------
// Fused single-precision stage of Algorithm II.
//
// The 2BFS of Sec. 6 is a chain of grid-wide levels (latency-bound); CG is
// bandwidth-bound.  This kernel runs them side by side: in every block one
// feature warp runs the 2BFS (with the component rule) on its own bounded
// barrier, and in block 0 it then runs the kNN vote once v (Eq. 13) is
// known; fourteen consumer warps run CG from x~0 = 0 meanwhile.
//
// Past the k0 iterations the consumers keep iterating before the label is
// known.  For every class t present in the sample they record the first
// iteration j >= k0 whose stop measure is <= 10^-t and keep a snapshot of x~
// there.  Once the label t is known, stage 1 ends at its recorded iteration
// with its snapshot, or iterates on until 10^-t is met.  The iterates of CG
// do not depend on when eps1 becomes known, so this gives the same N1 and the
// same x~ as running k0 iterations, the kNN, and CG from iterate k0 to eps1.
// When every present class has been met, or the snapshot slots run out, or
// the iteration cap is reached, the consumers wait for the label (bounded).
// The label reaches every block at the same reduction through the reduction
// buffer (one extra slot written by block 0), so all blocks take the same
// decisions.
// ---------------------------------------------------------------------------------------
constexpr int kNC1 = 14;      // consumer warps; warp 14 = feature warp, warp 15 = producer
constexpr int kSnapSlots = 6; // snapshots of x~ kept in the workspace

struct Stage1Args {
  CgArgs a;
  BfsGraph g;
  int32_t *d1, *d2;
  KnnSpec knn;
  int bfs_slot;
};

// Thread 0: wait (bounded) until the feature warp has published the label.
// Returns t >= 0, or -1 on failure (status set).
__device__ __forceinline__ int wait_label(Ctl* ctl) {
  const volatile int* p = &ctl->eps1_ready;
  const unsigned long long t0 = globaltimer();
  unsigned spins = 0;
  while (true) {
    const int label = *p;
    if (label > 0) return label - 1;
    if (label < 0) return -1;
    if ((++spins & 255u) == 0) {
      if (volatile_status(ctl) != 0 || poll_cancel(ctl)) return -1;
      if (globaltimer() - t0 > (unsigned long long)ctl->timeout_ns) {
        set_status(ctl, MPCG_ERR_TIMEOUT);
        return -1;
      }
    }
  }
}

// The feature warp's 2BFS (out of line: its registers are its own).  The
// block's consumers join its levels once stage 1 waits for nothing but the
// label (help_begin); the release ends their part on every path.
__device__ __noinline__ bool stage1_pdiam(const BfsGraph g, int32_t* d1, int32_t* d2, Ctl* ctl,
                                          int slot, int* hstate, HelpLevel* hl, int nhelp) {
  WarpGroupHelped sync{{ctl, slot, 0ull}, hstate, hl, nhelp};
  const bool ok = pseudo_diameter_run(g, d1, d2, blockIdx.x * 32 + (threadIdx.x & 31),
                                      gridDim.x * 32, sync);
  help_release(sync);
  return ok;
}

__global__ void __launch_bounds__(kTmaThreads, 1) k_stage1(Stage1Args sa) {
  constexpr int NC = kNC1;
  extern __shared__ __align__(128) char smem[];
  __shared__ CShared<NC> S;
  __shared__ volatile int s_k0_ready;
  __shared__ double s_v;
  __shared__ unsigned s_cmask;
  __shared__ int s_help;       // the consumers' part in the 2BFS (kHelpNone / Joined / Closed)
  __shared__ HelpLevel s_hl;   // the level the feature warp publishes to them
  const CgArgs& a = sa.a;
  Ctl* ctl = a.ctl;
  if (volatile_status(ctl) != 0 || ctl->trivial) return;
  if (threadIdx.x == 0) {
    s_k0_ready = 0;
    s_cmask = 0u;
    s_help = kHelpNone;
    s_hl.cmd = 0;
  }
  Ring<float> R;
  int S0, S1;
  ring_setup<NC>(a, smem, R, S0, S1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == NC + 1) {
    if (lane == 0) ring_producer(a, R);
    return;
  }
  if (warp == NC) {
    // ---- feature warp: 2BFS over the grid's feature warps ----
    const bool ok = stage1_pdiam(sa.g, sa.d1, sa.d2, ctl, sa.bfs_slot, &s_help, &s_hl, NC);
    if (blockIdx.x != 0) return;
    // ---- block 0: wait for v from this block's consumers, then the kNN ----
    int have_v = 0;
    if (ok && lane == 0) {
      const unsigned long long t0 = globaltimer();
      unsigned spins = 0;
      while (true) {
        if (s_k0_ready) {
          have_v = 1;
          break;
        }
        if ((++spins & 255u) == 0) {
          if (volatile_status(ctl) != 0 || poll_cancel(ctl)) break;
          if (globaltimer() - t0 > (unsigned long long)ctl->timeout_ns) {
            set_status(ctl, MPCG_ERR_TIMEOUT);
            break;
          }
        }
      }
    }
    // lane 0 wrote l~ (the last 2BFS level) and observed v; it broadcasts both
    double pd = 0.0, v = 0.0;
    if (have_v) {
      __threadfence_block();
      pd = (double)*reinterpret_cast<volatile int*>(&ctl->pdiam);
      v = *reinterpret_cast<volatile double*>(&s_v);
    }
    have_v = __shfl_sync(0xffffffffu, have_v, 0);
    pd = __shfl_sync(0xffffffffu, pd, 0);
    v = __shfl_sync(0xffffffffu, v, 0);
    int t = -1;
    if (have_v) {
      const double chi[4] = {(double)a.n, (double)ctl->nnz, pd, v};
      t = knn_warp(sa.knn, chi);
    }
    if (lane == 0) {
      if (t >= 0) {
        ctl->cls = t;
        ctl->eps1 = pow10_neg(t);
      } else if (have_v) {
        set_status(ctl, MPCG_ERR_INVALID_ARG);  // invalid query, sample or label
      }
      ctl->t_features = globaltimer();
      __threadfence();
      atomicExch(&ctl->eps1_ready, t >= 0 ? t + 1 : -1);
    }
    return;
  }

  // ---- consumers ----
  const bool lead = threadIdx.x == 0;
  const bool lead0 = lead && blockIdx.x == 0;
  Cursor C{0u, 0u, 0u};
  int R0, R1;
  warp_rows<NC>(S0, S1, a.n, R0, R1);
  const int n = a.n;
  const int rel = ctl->tol_relative;
  const bool f32 = ctl->acc32 != 0;  // inner products summed in float (option acc32)
  const int k0 = ctl->k0, max1 = ctl->max1;
  const double eps2 = ctl->eps2;
  unsigned long long round = 0;
  int red = 0;
  bool ok = true;

  // Classes present in the sample (block 0 reads the labels; the mask rides
  // along the first reduction).
  if (blockIdx.x == 0) {
    unsigned cm = 0u;
    for (int i = threadIdx.x; i < sa.knn.count; i += NC * 32) {
      const int c = sa.knn.cls[i];
      if (c >= 0 && c < 16) cm |= 1u << c;
    }
    cm = __reduce_or_sync(0xffffffffu, cm);
    if (lane == 0 && cm) atomicOr(&s_cmask, cm);
  }

  // CG line 1: x0 = 0, r0 = b~, d_{-1} = 0 (so that d_0 = fma(0, 0, r0) = r0).
  FF acc{0.f, 0.f};
  for (int i = R0 + lane; i < R1; i += kSlice) {
    const float bi = a.b32[i];
    a.x32[i] = 0.0f;
    a.r32[i] = bi;
    a.da[i] = 0.0f;
    ff_add_prod(acc, bi, bi, f32);
  }
  double rr, bnorm;
  // thread 0: the classes present in the sample, and those met so far (in
  // shared memory: registers are scarce here)
  __shared__ unsigned cmask, met;
  {
    double* buf = a.partials + (red & 1) * kMaxGrid;
    const double bp = block_ff(acc, S, f32);  // all consumer warps past the mask
    if (lead0) buf[gridDim.x] = (double)s_cmask;
    const double tot = cgrid_total(bp, a.partials, red, ctl, a.slot, round, S, ok, f32);
    if (lead) {
      cmask = (unsigned)buf[gridDim.x];
      met = 0u;
      S.rr = tot;
      S.val = sqrt(tot);
      if (lead0) {
        ctl->bnorm32 = S.val;
        if (!isfinite(S.val)) set_status(ctl, MPCG_ERR_NAN);
      }
    }
    cbar<NC>();
    rr = S.rr;
    bnorm = S.val;
    if (!isfinite(bnorm)) ok = false;
  }
  float beta = 0.0f;
  int parity = 0, first = 1, it = 0;
  // thread 0 only:
  double vsum = 0.0;
  int k0done = 0, in_k0 = 1, cls = -1, nslots = 0;
  // Thread 0's record of the candidate crossings, in shared memory: as a
  // thread-local array it lived in local memory, whose lines the gathers
  // evict from L1, so the decision at every loop head waited on L2 round
  // trips (measured at 128^3: the loop head took 3.65 us per iteration,
  // 1.9 us with the record here, against 0.55 us in k_cg32).
  __shared__ int nt[16], snap_it[kSnapSlots];
  __shared__ double res_at[16];
  if (lead)
    for (int t = 0; t < 16; ++t) {
      nt[t] = -1;
      res_at[t] = 0.0;
    }
  enum { kGoOn = 0, kEnd = 1, kFailed = 2, kBrokeDown = 3, kEndForLabel = 4 };
  int broke = 0;
  // thread 0: stop thresholds of eps2 (slot 16) and of every candidate
  // eps1 = 10^-t (slots 0..15), kept in shared memory
  __shared__ double s_lo[17], s_hi[17];
  if (lead) {
    for (int t = 0; t <= 16; ++t) {
      const StopThr c = stop_thr(t < 16 ? pow10_neg(t) : eps2, bnorm, rel);
      s_lo[t] = c.lo;
      s_hi[t] = c.hi;
    }
  }

  int cw = 0;  // the cancel word as block 0's thread 0 read it during the last pass
  bool help = false;  // stage 1 is over and waits for the label only
  while (ok) {
    if (lead) {
      int dec = kGoOn, snap_slot = -1;
      if (lead0 && cw != 0) {  // the caller cancelled; the other blocks stop at their next wait
        dec = kFailed;
        set_status(ctl, MPCG_ERR_CANCELLED);
      } else if (isnan(rr)) {
        dec = kFailed;
        if (lead0) set_status(ctl, MPCG_ERR_NAN);
      } else {
        if (in_k0 && (it >= min(k0, max1) || rr == 0.0 || rr <= s_lo[16] ||
                      (rr <= s_hi[16] && stop_measure(rr, bnorm, rel) <= eps2))) {
          in_k0 = 0;  // end of the k0 phase: v of Eq. (13) for the kNN
          if (lead0) {
            ctl->k0_done = k0done;
            ctl->vsum = vsum;
            ctl->v = k0done > 0 ? vsum / (double)k0done : 0.0;
            s_v = ctl->v;
            __threadfence_block();
            s_k0_ready = 1;
          }
        }
        if (!in_k0) {
          // Candidates are met in the order of t (a smaller eps1 has the
          // smaller threshold): while r^T r stays above the upper bracket of
          // the lowest present class not met yet, none is met this iteration.
          bool fresh = false;
          const unsigned open = cmask & ~met;
          if (open && rr <= s_hi[__ffs(open) - 1]) {
            for (int t = 0; t < 16; ++t) {
              if (!((open >> t) & 1u)) continue;
              if (rr <= s_lo[t] ||
                  (rr <= s_hi[t] && stop_measure(rr, bnorm, rel) <= pow10_neg(t))) {
                nt[t] = it;
                res_at[t] = stop_measure(rr, bnorm, rel);
                met |= 1u << t;
                fresh = true;
              }
            }
          }
          const bool all = (cmask & ~met) == 0u;  // every present class is met
          if (cls < 0 && (all || it >= max1)) {
            // Stage 1 ends here whatever the label (every present class is
            // met, or the cap): the loop ends, and the consumers help the
            // 2BFS before thread 0 waits for the label.
            dec = kEndForLabel;
          } else if (cls < 0 && fresh && nslots >= kSnapSlots) {
            cls = wait_label(ctl);
            if (cls < 0) dec = kFailed;
          }
          if (dec == kGoOn) {
            if (cls < 0) {
              if (fresh) {
                snap_slot = nslots;
                snap_it[nslots++] = it;
              }
            } else if (nt[cls] >= 0 || it >= max1) {
              dec = kEnd;
            }
          }
        }
      }
      S.dec = dec;
      S.aux = snap_slot;
    }
    cbar<NC>();
    const int dec = S.dec;
    const int snap_slot = S.aux;
    if (snap_slot >= 0) {
      float* dst = a.snap + (size_t)snap_slot * n;
      for (int i = R0 + lane; i < R1; i += kSlice) dst[i] = a.x32[i];
    }
    if (dec != kGoOn) {
      if (dec == kFailed) ok = false;
      if (dec == kEndForLabel) help = true;
      break;
    }

    if (lead0) cw = cancel_word(ctl);  // consumed at the next loop head: latency hidden

    // ---- P1: q = A d_k with d_k = r_k + beta_k d_{k-1} formed on the fly ----
    const float* dold = parity ? a.db : a.da;
    float* dnew = parity ? a.da : a.db;
    const float* r = a.r32;
    float* q = a.q32;
    FF pdq{0.f, 0.f};
    const float bt = first ? 0.0f : beta;
    auto G = [&](int c) -> float { return __fmaf_rn(bt, dold[c], r[c]); };
    auto Rw = [&](int i, float accv) {
      if (i < n) {
        const float di = __fmaf_rn(bt, dold[i], r[i]);
        dnew[i] = di;
        q[i] = accv;
        ff_add_prod(pdq, di, accv, f32);
      }
    };
    if (!ring_spmv<NC, float>(a, R, C, S0, S1, G, Rw)) set_status(ctl, MPCG_ERR_TIMEOUT);
    {
      const double dq = cgrid_total(block_ff(pdq, S, f32), a.partials, red, ctl, a.slot, round, S, ok, f32);
      if (lead) {
        int d2 = kGoOn;
        if (!isfinite(dq)) {
          d2 = kFailed;
          if (lead0) set_status(ctl, MPCG_ERR_NAN);
        } else if (!(dq > 0.0)) {
          d2 = kBrokeDown;  // stage 1 ends here; x~ and r are unchanged
        } else {
          S.alpha = (float)(rr / dq);
        }
        S.dec = d2;
      }
      cbar<NC>();
    }
    if (!ok || S.dec == kFailed) {
      ok = false;
      break;
    }
    if (S.dec == kBrokeDown) {
      broke = 1;
      break;
    }
    const float alpha = S.alpha;

    // ---- P2: x += alpha d_k, r -= alpha q, r^T r; the label rides along ----
    // Block 0 reads the label flag before its updates, so that the read's
    // latency overlaps them; once the label is known it is no longer read.
    int label_now = 0;
    if (lead0) label_now = cls >= 0 ? cls + 1 : *reinterpret_cast<volatile int*>(&ctl->eps1_ready);
    FF prr{0.f, 0.f};
    p2_32(a, R0, R1, lane, dnew, alpha, prr, f32);
    {
      double* buf = a.partials + (red & 1) * kMaxGrid;
      const double bp = block_ff(prr, S, f32);
      if (lead0) buf[gridDim.x] = (double)label_now;
      double label_slot = 0.0;
      const double rrn = cgrid_total(bp, a.partials, red, ctl, a.slot, round, S, ok, f32, &label_slot);
      if (lead) {
        const int label = (int)label_slot;
        int d3 = kGoOn;
        if (label < 0) {
          d3 = kFailed;
        } else if (!isfinite(rrn)) {
          d3 = kFailed;
          if (lead0) set_status(ctl, MPCG_ERR_NAN);
        } else {
          if (label > 0) cls = label - 1;
          if (in_k0) {
            vsum += sqrt(rrn) / sqrt(rr);  // Eq. (13) ratio ||r_i|| / ||r_{i-1}||
            ++k0done;
          }
          S.beta = (float)(rrn / rr);
          S.rr = rrn;
        }
        S.dec = d3;
      }
      cbar<NC>();
    }
    if (!ok || S.dec != kGoOn) {
      ok = false;
      break;
    }
    beta = S.beta;
    rr = S.rr;
    parity ^= 1;
    first = 0;
    ++it;
  }

  if (ok && help) {  // the consumers join the 2BFS levels unless the search has ended
    if (lead) S.aux = atomicCAS(&s_help, kHelpNone, kHelpJoined);
    cbar<NC>();
    if (S.aux == kHelpNone) bfs_help(sa.g, &s_hl, NC, warp + 1);
  }
  if (lead) {
    if (ok && broke && in_k0 && lead0) {  // breakdown in the k0 phase: v over completed ratios
      ctl->k0_done = k0done;
      ctl->vsum = vsum;
      ctl->v = k0done > 0 ? vsum / (double)k0done : 0.0;
      s_v = ctl->v;
      __threadfence_block();
      s_k0_ready = 1;
    }
    if (ok && cls < 0) {
      cls = wait_label(ctl);
      if (cls < 0) ok = false;
    }
    if (lead0 && ok) {
      // Stage 1 ends at the first iteration >= k0 that met eps1 = 10^-t, with
      // its iterate; otherwise (iteration cap, breakdown) at the current one.
      const double eps1 = pow10_neg(cls);
      int n1 = it, src = -1;
      double res = stop_measure(rr, bnorm, rel);
      if (!in_k0 && nt[cls] >= 0 && nt[cls] < it) {
        n1 = nt[cls];
        res = res_at[cls];
        for (int k = 0; k < nslots; ++k)
          if (snap_it[k] == n1) src = k;
        if (src < 0) set_status(ctl, MPCG_ERR_INVALID_ARG);  // cannot happen: crossings are snapshotted
      }
      ctl->n1 = n1;
      ctl->x32_src = src;
      ctl->res32 = res;
      ctl->rr = rr;
      if (res > eps1) ctl->warn_eps1 = 1;
      ctl->t_fp32 = globaltimer();
    }
    *R.stop = 1;
  }
}

// Promotion only (stage-1-only solves): x = float64(x~).
__global__ void k_promote(const Ctl* c, const float* __restrict__ x32,
                          const float* __restrict__ snap, double* __restrict__ x64, int n) {
  const bool zero = c->trivial != 0;
  if (c->status != 0) return;
  const float* xs = c->x32_src >= 0 ? snap + (size_t)c->x32_src * n : x32;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x64[i] = zero ? 0.0 : (double)xs[i];
}

// ---------------------------------------------------------------------------------------
// Stand-alone SpMV through the sliced layout (verification entry point).
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T spmv_row_direct(const CgArgs& a, int s, int i, const T* x) {
  const uint32_t wf = a.slice_w[s];
  const int w = (int)(wf & ~kOverflowBit);
  const int p = a.slice_ptr[s] + (i & 31);
  const T* sv = svals<T>(a);
  const int16_t* sc16 = reinterpret_cast<const int16_t*>(a.scol);
  const bool c16 = a.ctl->col16 != 0;
  T acc = (T)0;
  for (int k = 0; k < w; ++k) {
    const int e = p + kSlice * k;
    acc = fma(sv[e], x[c16 ? i + (int)sc16[e] : a.scol[e]], acc);
  }
  if (wf & kOverflowBit)
    for (int e = a.rp[i] + w; e < a.rp[i + 1]; ++e) acc = fma((T)a.val[e], x[a.col[e]], acc);
  return acc;
}

__global__ void k_spmv(CgArgs a, int fp32, const void* xv, void* yv) {
  if (volatile_status(a.ctl) != 0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = i >> 5;
  if (s >= a.nslices || i >= a.n) return;
  if (fp32)
    ((float*)yv)[i] = spmv_row_direct<float>(a, s, i, (const float*)xv);
  else
    ((double*)yv)[i] = spmv_row_direct<double>(a, s, i, (const double*)xv);
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
  a.snap = L.ws.snap;
  a.dinv64 = L.dinv64;
  a.dinv32 = L.dinv32;
  a.z32 = L.z32;
  return a;
}

// Blocks of the stage kernels: one per SM (fewer when asked).  0 on failure.
int cg_grid(int requested) {
  // Per device: the shared-memory attribute and the occupancy are properties
  // of the device the kernels run on.  A benign race between host threads
  // computes the same values twice.
  constexpr int kMaxDevices = 64;
  static int cached[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
  if (!cached[dev]) {
    struct K {
      const void* f;
      size_t smem;
    } ks[9] = {{(const void*)k_cg32<false, false>, ring_smem_bytes<float>()},
               {(const void*)k_cg64<false, false>, ring_smem_bytes<double>()},
               {(const void*)k_stage1, ring_smem_bytes<float>()},
               {(const void*)k_cg32<true, false>, ring_smem_bytes<float>()},
               {(const void*)k_cg64<true, false>, ring_smem_bytes<double>()},
               {(const void*)k_cg32<false, true>, ring_smem_bytes<float>()},
               {(const void*)k_cg64<false, true>, ring_smem_bytes<double>()},
               {(const void*)k_cg32<true, true>, ring_smem_bytes<float>()},
               {(const void*)k_cg64<true, true>, ring_smem_bytes<double>()}};
    int sms = 0, per = 1 << 30;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return 0;
    for (const K& k : ks) {
      int g = 0;
      if (cudaFuncSetAttribute(k.f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem) !=
              cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g, k.f, kTmaThreads, k.smem) !=
              cudaSuccess)
        return 0;
      if (g < per) per = g;
    }
    int c = per > 0 ? sms * per : -1;
    if (c > kMaxGrid - 1) c = kMaxGrid - 1;  // one reduction slot stays free
    cached[dev] = c;
  }
  const int c = cached[dev];
  if (c <= 0) return 0;
  return (requested > 0 && requested < c) ? requested : c;
}

const void* cg32_kernel() { return (const void*)k_cg32<false, false>; }
const void* cg64_kernel() { return (const void*)k_cg64<false, false>; }
const void* stage1_kernel() { return (const void*)k_stage1; }

cudaError_t launch_cg32(const Launch& L, int mode, int slot) {
  CgArgs a = make_args(L, slot, mode);
  void* args[] = {&a};
  const int g = cg_grid(L.grid_req);
  if (g <= 0) return cudaErrorInvalidConfiguration;
  const void* k = L.true_res
                      ? (L.precond ? (const void*)k_cg32<true, true> : (const void*)k_cg32<false, true>)
                      : (L.precond ? (const void*)k_cg32<true, false> : (const void*)k_cg32<false, false>);
  return cudaLaunchCooperativeKernel(k, dim3(g), dim3(kTmaThreads), args, ring_smem_bytes<float>(),
                                     L.st);
}

cudaError_t launch_cg64(const Launch& L, const double* b, double* x, int from_zero, int slot) {
  CgArgs a = make_args(L, slot, from_zero);
  a.b64 = b;
  a.x64 = x;
  void* args[] = {&a};
  const int g = cg_grid(L.grid_req);
  if (g <= 0) return cudaErrorInvalidConfiguration;
  const void* k = L.true_res
                      ? (L.precond ? (const void*)k_cg64<true, true> : (const void*)k_cg64<false, true>)
                      : (L.precond ? (const void*)k_cg64<true, false> : (const void*)k_cg64<false, false>);
  return cudaLaunchCooperativeKernel(k, dim3(g), dim3(kTmaThreads), args,
                                     ring_smem_bytes<double>(), L.st);
}

cudaError_t launch_stage1(const Launch& L, const mpcg_sample_t& S, const mpcg_options_t& o,
                          int slot, int bfs_slot) {
  Stage1Args sa{};
  sa.a = make_args(L, slot, kCgToEps1);
  sa.g = bfs_graph(L);
  sa.d1 = L.ws.dist;
  sa.d2 = L.ws.dist2;
  sa.knn = knn_spec(S, o);
  sa.bfs_slot = bfs_slot;
  void* args[] = {&sa};
  const int g = cg_grid(L.grid_req);
  if (g <= 0) return cudaErrorInvalidConfiguration;
  return cudaLaunchCooperativeKernel((const void*)k_stage1, dim3(g), dim3(kTmaThreads), args,
                                    ring_smem_bytes<float>(), L.st);
}

cudaError_t launch_promote(const Launch& L, double* x) {
  int blocks = (L.d.n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_promote<<<blocks, 256, 0, L.st>>>(L.ws.ctl, L.ws.x32, L.ws.snap, x, L.d.n);
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
