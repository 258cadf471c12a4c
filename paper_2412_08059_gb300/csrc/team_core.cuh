// team_core.cuh -- the whole method for one system, run by a team of blocks
// of a persistent launch (the batched solve and the serving steps).
//
// A team is 1, 2, 4, ..., 128 blocks of one cooperative launch.  Teams
// synchronise with a bounded barrier over their own blocks (a block barrier
// for one-block teams).  Scalars are computed from team-wide sums that every
// block of the team forms in the same order, so all blocks take the same
// decisions.  The arithmetic is that of the single-system kernels: SpMV rows
// summed in stored order with fused multiply-adds, float-float dot products
// in single precision, alpha and beta rounded once to float.  The CG stages
// can stop after an iteration budget and continue in a later launch from
// the state kept in the system's workspace and control block.
#pragma once
#include <math.h>

#include <type_traits>
#include <vector>

#include "bfs_block.cuh"
#include "internal.h"

namespace mpcg {

constexpr int kBatchThreads = 512;
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int kTeamClasses = 8;                // team sizes 1, 2, 4, ..., 128 blocks
constexpr int kRowsPerBlock = 16384;           // planner default: target rows per block of a team
constexpr int kNoBudget = 0x7fffffff;          // iteration budget of a run-to-completion call
constexpr int kTeamFastW = 8;                  // widest slice whose pairs the SpMV stages
constexpr int kSpmvStep = 2;                   // slices per SpMV step (their gathers overlap)
constexpr int kStageWarpBytes = 2 * kSpmvStep * kSlice * kTeamFastW * (4 + 4);  // two float stages
constexpr int kBScanPer = 8;                   // slice widths per thread in the block scan
constexpr int kBScanTile = kBatchThreads * kBScanPer;
constexpr int kScanSmem = kBScanTile * 4 + kBatchThreads * 8;  // the scan's tile and partials
// Dynamic shared memory of a team launch: the scan at set-up; with a
// single-precision stage also the SpMV stages and the block-local 2BFS.
// 128 KB plus the static part keeps the 132 KB shared-memory carve-out, so
// the L1 cache keeps 124 KB of the 256 KB.
constexpr int kTeamSmem = kBatchWarps * kStageWarpBytes;
static_assert(kTeamSmem >= kScanSmem, "scan buffer");
constexpr int kBlockBfsMaxN = 1 << 18;         // larger systems run the 2BFS over the whole team

// One system of the batch (device copy written by the host).
struct BatchSys {
  mpcg_csr_t A;
  const double* b;
  double* x;
  mpcg_result_t* res;
  Ws w;  // the system's own workspace, carved by the host
  int n, nnz, nslices, wcap;
  double eps2;  // per-system final tolerance
};

// Shared state of the launch (device, zeroed by the host copy).
struct BatchHdr {
  unsigned long long bar[kMaxGrid];  // per-team barrier counters
  int next[kMaxGrid];                // system index broadcast by each team leader
  int head[kTeamClasses];            // queue heads (atomic)
  int qbase[kTeamClasses], qlen[kTeamClasses];
  int abort;                         // a team barrier timed out: every block leaves
  int pad;
};

struct BatchArgs {
  BatchHdr* h;
  const BatchSys* sys;
  const int* order;            // systems by class queue
  const int* team_of_block;    // [grid]
  const int* rank_of_block;    // [grid]
  const int* team_size;        // [nteams]
  const int* team_class;       // [nteams]
  KnnSpec knn;
  mpcg_options_t o;
  int auto_eps1;
  int smem_bytes;  // dynamic shared memory of the launch (0: none)
  int part;        // batch launches: 1 = set-up to the single-precision stage, 2 = the rest
};

// ---------------------------------------------------------------------------------------
// Team context: barrier, block-level scratch, deterministic team sums.
// ---------------------------------------------------------------------------------------
struct TeamShared {
  double dpart[kBatchWarps];
  float ffp[2 * kBatchWarps];
  double val[4];
  float fval[2];
  int ival[4];
  int ok;
};

struct Team {
  BatchHdr* h;
  unsigned long long* bar;
  int rank, size, team;
  unsigned long long round;
  long long timeout_ns;
  TeamShared* S;
};

// The launch's dynamic shared memory (the block-local 2BFS); its size is
// BatchArgs::smem_bytes.  Not kept in Team, so that it takes no register
// for the length of the kernel.
extern __shared__ __align__(16) unsigned char team_dyn[];

// Bounded barrier over the team's blocks.  False (in every thread of the
// block) on timeout or when another team has aborted the launch.
static __device__ bool team_sync(Team& t) {
  __syncthreads();
  if (t.size == 1) {
    if (threadIdx.x == 0) t.S->ok = *reinterpret_cast<volatile int*>(&t.h->abort) == 0;
    __syncthreads();
    return t.S->ok != 0;
  }
  t.round += 1;
  if (threadIdx.x == 0) {
    const unsigned long long target = t.round * (unsigned long long)t.size;
    red_release_add(t.bar, 1ull);
    int ok = 1;
    if (ld_acquire(t.bar) < target) {
      const unsigned long long t0 = globaltimer();
      unsigned spins = 0;
      while (ld_acquire(t.bar) < target) {
        if ((++spins & 1023u) == 0) {
          if (*reinterpret_cast<volatile int*>(&t.h->abort)) {
            ok = 0;
            break;
          }
          if (globaltimer() - t0 > (unsigned long long)t.timeout_ns) {
            atomicExch(&t.h->abort, 1);
            ok = 0;
            break;
          }
        }
      }
    }
    t.S->ok = ok;
  }
  __syncthreads();
  return t.S->ok != 0;
}

struct TeamSyncFn {
  static constexpr bool kWholeBlock = true;
  static constexpr bool kNarrow = false;  // team searches keep every level on the team
  static constexpr bool kHelpers = false;
  Team* t;
  __device__ bool operator()() { return team_sync(*t); }
};

// Team-wide sum of one double per thread, identical in every block: block
// partials in warp order, then the team's partials in rank order.  `buf`
// alternates between two halves of the system's partials array.
static __device__ bool team_sum_d(Team& t, double v, double* partials, int& red, double& out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) t.S->dpart[warp] = v;
  __syncthreads();
  double* buf = partials + (red & 1) * kMaxGrid;
  ++red;
  if (threadIdx.x < 32) {
    double s = lane < kBatchWarps ? t.S->dpart[lane] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) {
      if (t.size == 1) t.S->val[0] = s;
      else buf[t.rank] = s;
    }
  }
  if (t.size > 1) {
    if (!team_sync(t)) return false;
    if (threadIdx.x < 32) {
      double s = 0.0;
      for (int i = lane; i < t.size; i += 32) s += buf[i];
      s = warp_sum(s);
      if (threadIdx.x == 0) t.S->val[0] = s;
    }
  }
  __syncthreads();
  out = t.S->val[0];
  __syncthreads();
  return true;
}

// Same for float-float partial sums (single-precision stage).
static __device__ bool team_sum_ff(Team& t, FF v, double* partials, int& red, double& out,
                                   bool f32) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = ff_warp_sum(v, f32);
  if (lane == 0) {
    t.S->ffp[2 * warp] = v.hi;
    t.S->ffp[2 * warp + 1] = v.lo;
  }
  __syncthreads();
  double* buf = partials + (red & 1) * kMaxGrid;
  ++red;
  if (threadIdx.x < 32) {
    FF s = lane < kBatchWarps ? FF{t.S->ffp[2 * lane], t.S->ffp[2 * lane + 1]} : FF{0.f, 0.f};
    s = ff_warp_sum(s, f32);
    const double bs = (double)s.hi + (double)s.lo;
    if (threadIdx.x == 0) {
      if (t.size == 1) t.S->val[0] = bs;
      else buf[t.rank] = bs;
    }
  }
  if (t.size > 1) {
    if (!team_sync(t)) return false;
    if (threadIdx.x < 32) {
      double s = 0.0;
      if (f32) {  // option acc32: the blocks' float partials summed in float
        float sf = 0.0f;
        for (int i = lane; i < t.size; i += 32) sf = __fadd_rn(sf, (float)buf[i]);
        s = (double)warp_sum_f(sf);
      } else {
        for (int i = lane; i < t.size; i += 32) s += buf[i];
        s = warp_sum(s);
      }
      if (threadIdx.x == 0) t.S->val[0] = s;
    }
  }
  __syncthreads();
  out = t.S->val[0];
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------------------
// Per-system set-up by the team (the same steps as the set-up kernels of the
// single-system path).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int team_tid(const Team& t) { return t.rank * kBatchThreads + threadIdx.x; }
__device__ __forceinline__ int team_threads(const Team& t) { return t.size * kBatchThreads; }

// Control block of the system: zeroed and initialised by the team leader block.
static __device__ void sys_init(const Team& t, const BatchSys& s, const BatchArgs& a) {
  Ctl* c = s.w.ctl;
  if (t.rank != 0) return;
  int* ci = reinterpret_cast<int*>(c);
  for (int k = threadIdx.x; k < (int)(sizeof(Ctl) / sizeof(int)); k += blockDim.x) ci[k] = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    const mpcg_options_t& o = a.o;
    c->t_start = globaltimer();
    c->n = s.n;
    c->nnz = s.nnz;
    c->nslices = s.nslices;
    c->wcap = s.wcap;
    c->k0 = o.k0 > 0 ? o.k0 : 0;
    c->max1 = o.max_it_fp32 > 0 ? o.max_it_fp32 : s.n;
    const long long m2 = o.max_it_fp64 > 0 ? (long long)o.max_it_fp64 : 10ll * s.n;
    c->max2 = m2 > 0x7fffffffll ? 0x7fffffff : (int)m2;
    c->max_restarts = o.max_true_restarts > 0 ? o.max_true_restarts : 0;
    c->tol_relative = o.tol_relative ? 1 : 0;
    c->acc32 = o.acc32 ? 1 : 0;
    c->colwide = o.spmv_variant == 1 ? 1 : 0;  // 32-bit columns asked for
    c->eps1 = o.fp64_only ? 0.0 : (a.auto_eps1 ? -1.0 : o.eps1);
    c->eps2 = s.eps2;
    c->timeout_ns = (long long)(o.timeout_ms > 0 ? o.timeout_ms : 20000) * 1000000ll;
    c->cls = -1;
    c->first = 1;
    c->x32_src = -1;
  }
}

// CSR check, b~ = float32(b), slice widths (one warp per slice).  Also
// notes whether some entry kept in the slices (the first wcap of its row)
// lies more than 32767 columns from its row: the fill then writes no 16-bit
// copy of the columns.
static __device__ void sys_rows(const Team& t, const BatchSys& s) {
  Ctl* c = s.w.ctl;
  const int lane = threadIdx.x & 31;
  const int T = team_threads(t);
  const int32_t* rp = s.A.row_ptr;
  const int32_t* col = s.A.col;
  for (int base = team_tid(t) - lane; base < s.nslices * kSlice; base += T) {
    const int i = base + lane;
    int len = 0, ok = 1, wide = 0;
    if (i < s.n) {
      const int a0 = rp[i], e = rp[i + 1];
      if (a0 < 0 || e < a0 || e > s.nnz) {
        ok = 0;
      } else {
        len = e - a0;
        int prev = -1;
        for (int k = a0; k < e; ++k) {
          const int cc = col[k];
          if (cc < 0 || cc >= s.n || cc <= prev) {
            ok = 0;
            break;
          }
          if (k - a0 < s.wcap && (cc - i > 32767 || i - cc > 32768)) wide = 1;
          prev = cc;
        }
      }
      if (i == 0 && a0 != 0) ok = 0;
      if (i == s.n - 1 && e != s.nnz) ok = 0;
      s.w.b32[i] = (float)s.b[i];
    }
    if (!ok) {
      set_status(c, MPCG_ERR_INVALID_ARG);
      len = 0;
    }
    const int w = len < s.wcap ? len : s.wcap;
    const int wmax = __reduce_max_sync(0xffffffffu, w);
    const int any_ovf = __any_sync(0xffffffffu, len > s.wcap);
    if (lane == 0) s.w.slice_w[i >> 5] = (uint32_t)wmax | (any_ovf ? kOverflowBit : 0u);
    if (__any_sync(0xffffffffu, wide) && lane == 0) atomicExch(&c->colwide, 1);
  }
}

// Exclusive scan of 32 * width over the slices, by one block (tile and
// partials in the launch's dynamic shared memory).
static __device__ void block_scan_slices(const uint32_t* slice_w, int32_t* slice_ptr, int nslices) {
  int32_t* tile = reinterpret_cast<int32_t*>(team_dyn);
  long long* part = reinterpret_cast<long long*>(team_dyn + kBScanTile * 4);
  __shared__ long long carry_s;
  const int t = threadIdx.x;
  if (t == 0) carry_s = 0;
  __syncthreads();
  for (int base = 0; base < nslices; base += kBScanTile) {
    for (int j = t; j < kBScanTile; j += kBatchThreads) {
      const int sidx = base + j;
      tile[j] = sidx < nslices ? (int32_t)(kSlice * (slice_w[sidx] & ~kOverflowBit)) : 0;
    }
    __syncthreads();
    long long loc = 0;
    for (int j = 0; j < kBScanPer; ++j) loc += tile[t * kBScanPer + j];
    part[t] = loc;
    __syncthreads();
    for (int o = 1; o < kBatchThreads; o <<= 1) {
      const long long v = t >= o ? part[t - o] : 0;
      __syncthreads();
      part[t] += v;
      __syncthreads();
    }
    long long run = carry_s + part[t] - loc;
    for (int j = 0; j < kBScanPer; ++j) {
      const int v = tile[t * kBScanPer + j];
      tile[t * kBScanPer + j] = (int32_t)run;
      run += v;
    }
    __syncthreads();
    for (int j = t; j < kBScanTile; j += kBatchThreads) {
      const int sidx = base + j;
      if (sidx < nslices) slice_ptr[sidx] = tile[j];
    }
    if (t == kBatchThreads - 1) carry_s += part[kBatchThreads - 1];
    __syncthreads();
  }
  if (t == 0) slice_ptr[nslices] = (int32_t)carry_s;
  __syncthreads();
}

// Sliced arrays: entry k of row i at slice_ptr[s] + 32 k + (i mod 32); short
// rows padded with value 0 and their own column, the rows past n that fill
// the last slice with value 0 and column 0 (n - 1 in the 16-bit copy).
// narrow: the launch's single-precision SpMV is the staged one, which also
// gets a copy of the columns as 16-bit offsets from the row (Ctl::col16)
// when sys_rows found that every one fits and 32-bit columns were not asked
// for.  Both copies hold the same entries in the same order.
static __device__ void sys_fill(const Team& t, const BatchSys& s, bool narrow) {
  const int T = team_threads(t);
  const int32_t* rp = s.A.row_ptr;
  const bool c16 = narrow && *reinterpret_cast<volatile int*>(&s.w.ctl->colwide) == 0;
  if (t.rank == 0 && threadIdx.x == 0) {
    s.w.ctl->col16 = c16 ? 1 : 0;
    s.w.ctl->colbits = c16 ? 16 : 32;
  }
  for (int i = team_tid(t); i < s.nslices * kSlice; i += T) {
    const int sl = i >> 5, lane = i & 31;
    const int w = (int)(s.w.slice_w[sl] & ~kOverflowBit);
    const int base = s.w.slice_ptr[sl] + lane;
    int a0 = 0, len = 0;
    if (i < s.n) {
      a0 = rp[i];
      len = rp[i + 1] - a0;
    }
    for (int k = 0; k < w; ++k) {
      const int e = base + kSlice * k;
      double v = 0.0;
      int cc = i < s.n ? i : 0;
      if (k < len) {
        v = s.A.val[a0 + k];
        cc = s.A.col[a0 + k];
      }
      s.w.scol[e] = cc;
      if (c16) s.w.scol16[e] = (int16_t)((i < s.n ? cc : s.n - 1) - i);
      s.w.sv64[e] = v;
      s.w.sv32[e] = (float)v;
    }
  }
}

// ---------------------------------------------------------------------------------------
// CG stages over the team.  Warp gw of the team owns slices gw, gw + W, ...;
// lane l owns row 32 s + l of slice s in every phase, so the vector updates
// of a row are done by the thread that produced its SpMV result.
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ const T* bvals(const BatchSys& s);
template <>
__device__ __forceinline__ const float* bvals<float>(const BatchSys& s) { return s.w.sv32; }
template <>
__device__ __forceinline__ const double* bvals<double>(const BatchSys& s) { return s.w.sv64; }

// Overflow tail of row i (entries past the slice width, from the CSR).
template <typename T, class Gather>
__device__ __forceinline__ T btail(const BatchSys& s, int i, int w, T acc, Gather G) {
  const int e1 = s.A.row_ptr[i + 1];
  for (int e = s.A.row_ptr[i] + w; e < e1; ++e) acc = fma((T)s.A.val[e], G(s.A.col[e]), acc);
  return acc;
}

__device__ __forceinline__ int team_warp(const Team& t);
__device__ __forceinline__ int team_warps(const Team& t);

// Asynchronous 16-byte global -> shared copies (cached in L2 only), in
// per-thread groups: a thread waits for its own groups, then a __syncwarp
// makes every lane's copies visible to the warp.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Copy one slice's (column, value) pairs -- 32 w contiguous elements from
// element p0 (a multiple of 32, so every 16-byte copy is aligned) -- into a
// warp's stage.  CT: 32-bit columns or 16-bit offsets.
template <typename T, typename CT>
__device__ __forceinline__ void stage_slice(CT* cdst, T* vdst, const CT* sc, const T* sv, int p0,
                                            int w, int lane) {
  const int E = kSlice * w;
  constexpr int cper = 16 / (int)sizeof(CT);
  for (int q = lane; q < E / cper; q += 32) cp_async16(cdst + cper * q, sc + p0 + cper * q);
  constexpr int per = 16 / (int)sizeof(T);
  for (int q = lane; q < E / per; q += 32) cp_async16(vdst + per * q, sv + p0 + per * q);
}

// Column of a stored entry of row i: a 32-bit column, or a 16-bit offset
// from the row.
template <bool C16>
__device__ __forceinline__ int col_at(typename std::conditional<C16, int16_t, int32_t>::type c, int i) {
  if constexpr (C16) return i + (int)c;
  else return c;
}

// SpMV over the team's slices, pairs staged in shared memory (the single-
// precision stage): warp gw owns slices gw, gw + W, ...; lane l owns row
// 32 s + l.  Rw(i, acc, own) receives row i's sum in stored order (fused
// multiply-adds from zero, padding rows included) and the row's own values
// that P(i) loaded before the gathers (P gets i >= n for absent rows).
//
// The slices are taken kS at a time (a step).  The (column, value) pairs of
// the next step's slices are copied into the warp's shared-memory stage
// (two stages per warp in the launch's dynamic shared memory) while the
// current step runs, so a step costs one round trip for its gathers: the
// pairs come from shared memory and every gather of a row is issued at once.
// Slices wider than kTeamFastW, or with an overflow tail, read their pairs
// from global memory instead.  The metadata of 32 of the warp's slices is
// loaded at once (one slice per lane).
template <typename T, bool C16, class Gather, class Pre, class Row>
__device__ __forceinline__ void team_spmv_staged(const Team& t, const BatchSys& s, Gather G, Pre P,
                                                 Row Rw) {
  static_assert(sizeof(T) == 4, "the stages hold 4-byte values");
  using CT = typename std::conditional<C16, int16_t, int32_t>::type;
  constexpr int kS = kSpmvStep;
  constexpr int kE = kSlice * kTeamFastW;      // elements of a staged slice
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gw = team_warp(t), W = team_warps(t);
  const T* sv = bvals<T>(s);
  const CT* sc;
  if constexpr (C16) sc = s.w.scol16;
  else sc = s.w.scol;
  int32_t* stage = reinterpret_cast<int32_t*>(team_dyn + warp * kStageWarpBytes);
  CT* cbuf = reinterpret_cast<CT*>(stage);            // [2][kS][kE]
  T* vbuf = reinterpret_cast<T*>(stage + 2 * kS * kE);  // [2][kS][kE]
  for (int base = gw; base < s.nslices; base += 32 * W) {
    const int mine = base + lane * W;
    uint32_t mwf = 0u;
    int mp = 0;
    if (mine < s.nslices) {
      mwf = s.w.slice_w[mine];
      mp = s.w.slice_ptr[mine];
    }
    const int cnt = min(32, (s.nslices - base + W - 1) / W);
    const int nsteps = (cnt + kS - 1) / kS;
    auto issue = [&](int step) {  // the copies of a step, into stage step & 1
#pragma unroll
      for (int u = 0; u < kS; ++u) {
        const int jj = step * kS + u;
        if (jj < cnt) {  // warp-uniform
          const uint32_t wf = __shfl_sync(full, mwf, jj);
          const int pp = __shfl_sync(full, mp, jj);
          const int w = (int)(wf & ~kOverflowBit);
          if (!(wf & kOverflowBit) && w <= kTeamFastW) {
            const int slot = ((step & 1) * kS + u) * kE;
            stage_slice<T, CT>(cbuf + slot, vbuf + slot, sc, sv, pp, w, lane);
          }
        }
      }
      cp_async_commit();
    };
    issue(0);
    for (int step = 0; step < nsteps; ++step) {
      if (step + 1 < nsteps) issue(step + 1);
      else cp_async_commit();  // an empty group keeps the count: wait<1> below covers `step`
      int w[kS], p[kS], i[kS];
      uint32_t wf[kS];
      T a[kS];
      decltype(P(0)) own[kS];
#pragma unroll
      for (int u = 0; u < kS; ++u) {
        const int jj = step * kS + u;
        const int ju = min(jj, 31);
        wf[u] = __shfl_sync(full, mwf, ju);
        p[u] = __shfl_sync(full, mp, ju) + lane;
        w[u] = jj < cnt ? (int)(wf[u] & ~kOverflowBit) : 0;
        i[u] = (base + jj * W) * kSlice + lane;
        a[u] = (T)0;
        // the rows' own values, loaded before the gathers (the row callbacks
        // store, and later loads could not be moved above those stores)
        own[u] = P(jj < cnt ? i[u] : s.n);
      }
      cp_async_wait<1>();
      __syncwarp();
#pragma unroll
      for (int u = 0; u < kS; ++u) {
        if (!(wf[u] & kOverflowBit) && w[u] <= kTeamFastW) {
          const int slot = ((step & 1) * kS + u) * kE + lane;
          const CT* cs = cbuf + slot;
          const T* vs = vbuf + slot;
#pragma unroll
          for (int k = 0; k < kTeamFastW; ++k)
            if (k < w[u]) a[u] = fma(vs[kSlice * k], G(col_at<C16>(cs[kSlice * k], i[u])), a[u]);
        } else if (step * kS + u < cnt) {
          for (int k = 0; k < w[u]; ++k)
            a[u] = fma(sv[p[u] + kSlice * k], G(col_at<C16>(sc[p[u] + kSlice * k], i[u])), a[u]);
          if (i[u] < s.n) a[u] = btail<T>(s, i[u], w[u], a[u], G);
        }
      }
#pragma unroll
      for (int u = 0; u < kS; ++u)
        if (step * kS + u < cnt) Rw(i[u], a[u], own[u]);
      __syncwarp();  // the stage is read before step + 2 copies into it
    }
    cp_async_wait<0>();
  }
}

// SpMV over the team's slices, operands from global memory (the double-
// precision stage): warp gw owns slices gw, gw + W, ...; lane l
// owns row 32 s + l.  Rw(i, acc, own) receives row i's sum in stored order
// (fused multiply-adds from zero, padding rows included) and the row's own
// values that P(i) loaded before the gathers (P gets i >= n for absent rows).  The metadata of 32 of
// the warp's slices is loaded at once (one slice per lane) and kU slices are
// summed together so that their loads and gathers overlap.
template <typename T, class Gather, class Pre, class Row>
__device__ __forceinline__ void team_spmv_regs(const Team& t, const BatchSys& s, Gather G, Pre P,
                                               Row Rw) {
  constexpr int kU = 4;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int gw = team_warp(t), W = team_warps(t);
  const T* sv = bvals<T>(s);
  const int32_t* sc = s.w.scol;
  for (int base = gw; base < s.nslices; base += 32 * W) {
    const int mine = base + lane * W;
    uint32_t mwf = 0u;
    int mp = 0;
    if (mine < s.nslices) {
      mwf = s.w.slice_w[mine];
      mp = s.w.slice_ptr[mine];
    }
    const int cnt = min(32, (s.nslices - base + W - 1) / W);
    for (int j = 0; j < cnt; j += kU) {
      int w[kU], p[kU], i[kU];
      uint32_t wf[kU];
      T a[kU];
      int wm = 0;
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int ju = min(j + u, 31);
        wf[u] = __shfl_sync(full, mwf, ju);
        p[u] = __shfl_sync(full, mp, ju) + lane;
        w[u] = j + u < cnt ? (int)(wf[u] & ~kOverflowBit) : 0;
        i[u] = (base + (j + u) * W) * kSlice + lane;
        a[u] = (T)0;
        wm = max(wm, w[u]);
      }
      // the rows' own values, loaded before the gathers (the row callbacks
      // store, and later loads could not be moved above those stores)
      decltype(P(0)) own[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) own[u] = P(j + u < cnt ? i[u] : s.n);
#pragma unroll 2
      for (int k = 0; k < wm; ++k) {
#pragma unroll
        for (int u = 0; u < kU; ++u)
          if (k < w[u]) a[u] = fma(sv[p[u] + kSlice * k], G(sc[p[u] + kSlice * k]), a[u]);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        if (j + u < cnt) {
          if ((wf[u] & kOverflowBit) && i[u] < s.n) a[u] = btail<T>(s, i[u], w[u], a[u], G);
          Rw(i[u], a[u], own[u]);
        }
      }
    }
  }
}

// The SpMV of the team kernels.  The single-precision stage stages its
// pairs in shared memory; the double-precision stage loads them from global
// memory: staged double pairs would need 12 bytes an element, and the shared
// memory they take comes out of the L1 cache that the stage's gathers use
// (measured on the 512-system batch: the FP64 stage lost more to the
// smaller L1 than it gained from the staging).
//
// The staged SpMV reads the 16-bit copy of the columns when the set-up built
// one (Ctl::col16; each format has its own copy of the loop); the SpMV from
// global memory reads the 32-bit columns, so the double-precision loops keep
// the one form whose schedule was measured.
template <typename T, bool kStage, class Gather, class Pre, class Row>
__device__ __forceinline__ void team_spmv(const Team& t, const BatchSys& s, Gather G, Pre P,
                                          Row Rw) {
  if constexpr (kStage && sizeof(T) == 4) {
    if (s.w.ctl->col16) team_spmv_staged<T, true>(t, s, G, P, Rw);
    else team_spmv_staged<T, false>(t, s, G, P, Rw);
  } else {
    team_spmv_regs<T>(t, s, G, P, Rw);
  }
}

__device__ __forceinline__ int team_warp(const Team& t) { return t.rank * kBatchWarps + (threadIdx.x >> 5); }
__device__ __forceinline__ int team_warps(const Team& t) { return t.size * kBatchWarps; }

// Row phases over the team's rows, kR slices per step: Ld(i) loads a row's
// operands, then Op(i, v) computes and stores.  All the step's loads are
// issued before any of its stores (the stores may alias the arrays the next
// loads read, so the compiler could not reorder them itself).
template <class Ld, class Op>
__device__ __forceinline__ void team_rows(const Team& t, const BatchSys& s, Ld L, Op O) {
  const int lane = threadIdx.x & 31;
  const int gw = team_warp(t), W = team_warps(t);
  constexpr int kR = 4;
  for (int sl = gw; sl < s.nslices; sl += kR * W) {
    int i[kR];
    decltype(L(0)) v[kR];
#pragma unroll
    for (int u = 0; u < kR; ++u) {
      i[u] = (sl + u * W) * kSlice + lane;
      v[u] = (sl + u * W < s.nslices && i[u] < s.n) ? L(i[u]) : decltype(L(0)){};
    }
#pragma unroll
    for (int u = 0; u < kR; ++u)
      if (sl + u * W < s.nslices && i[u] < s.n) O(i[u], v[u]);
  }
}

// Broadcast of thread 0's decision (and scalars) to the block.
__device__ __forceinline__ int bcast_dec(Team& t, int dec) {
  if (threadIdx.x == 0) t.S->ival[0] = dec;
  __syncthreads();
  const int d = t.S->ival[0];
  __syncthreads();
  return d;
}

enum BDec { kBGo = 0, kBStop = 1, kBNan = 2, kBBroke = 3, kBBreakdown = 4, kBCap = 5, kBSuspend = 6 };

// Single-precision stage; modes as in the single-system kernel (kCgK0,
// kCgToEps1, kCgContinue).  The state needed to continue is kept in the
// control block.  Outside the k0 phase at most `budget` iterations run;
// *done is false when the budget ended the call before the stage ended.
// Returns false if the launch aborted.
template <bool kStage>
static __device__ bool sys_cg32(Team& t, const BatchSys& s, int mode, int& red, int budget, bool* done) {
  *done = true;
  Ctl* ctl = s.w.ctl;
  const int lane = threadIdx.x & 31;
  const int gw = team_warp(t), W = team_warps(t);
  const int n = s.n, rel = ctl->tol_relative;
  const bool f32 = ctl->acc32 != 0;  // inner products summed in float (option acc32)
  const bool lead = threadIdx.x == 0, lead0 = lead && t.rank == 0;
  if (mode == kCgContinue && ctl->broke32) {  // stage 1 already ended in the k0 phase
    if (lead0) {
      if (ctl->res32 > ctl->eps1) ctl->warn_eps1 = 1;
      ctl->t_fp32 = globaltimer();
    }
    return true;
  }
  float* x = s.w.x32;
  float* r = s.w.r32;
  float* q = s.w.q32;
  double rr, bnorm;
  float beta;
  int first, parity, it;
  if (mode != kCgContinue) {
    FF acc{0.f, 0.f};
    for (int sl = gw; sl < s.nslices; sl += W) {
      const int i = sl * kSlice + lane;
      if (i < n) {
        const float bi = s.w.b32[i];
        x[i] = 0.0f;
        r[i] = bi;
        s.w.d32a[i] = 0.0f;  // d_{-1}
        ff_add_prod(acc, bi, bi, f32);
      }
    }
    double tot;
    if (!team_sum_ff(t, acc, s.w.partials, red, tot, f32)) return false;
    rr = tot;
    if (lead) t.S->val[1] = sqrt(tot);
    __syncthreads();
    bnorm = t.S->val[1];
    __syncthreads();
    if (lead0) {
      ctl->bnorm32 = bnorm;
      if (!isfinite(bnorm)) set_status(ctl, MPCG_ERR_NAN);
    }
    if (!isfinite(bnorm)) return true;
    first = 1;
    parity = 0;
    beta = 0.0f;
    it = 0;
  } else {
    rr = ctl->rr;
    bnorm = ctl->bnorm32;
    beta = ctl->beta32;
    first = ctl->first;
    parity = ctl->parity;
    it = ctl->n1;
  }
  const double eps = mode == kCgK0 ? ctl->eps2 : ctl->eps1;
  const int limit = mode == kCgK0 ? min(ctl->k0, ctl->max1) : ctl->max1;
  const int it_start = it;
  // Every thread holds the team sums (identical in every block), so every
  // thread takes the loop's decisions itself, with no broadcast barrier.
  const StopThr thr = stop_thr(eps, bnorm, rel);
  double vsum = 0.0;  // thread 0
  int k0done = 0, broke = 0, suspended = 0;
  while (true) {
    int dec = kBGo;
    if (isnan(rr)) dec = kBNan;
    else if (stop_pass(thr, rr) || it >= limit || (mode == kCgK0 && rr == 0.0)) dec = kBStop;
    else if (mode != kCgK0 && it - it_start >= budget) dec = kBSuspend;
    if (dec == kBSuspend) {
      suspended = 1;
      break;
    }
    if (dec != kBGo) {
      if (dec == kBNan && lead0) set_status(ctl, MPCG_ERR_NAN);
      break;
    }
    // P1: q = A d_k, d_k = r_k + beta_k d_{k-1} formed for every gathered column
    const float* dold = parity ? s.w.d32b : s.w.d32a;
    float* dnew = parity ? s.w.d32a : s.w.d32b;
    const float bt = first ? 0.0f : beta;
    FF pdq{0.f, 0.f};
    team_spmv<float, kStage>(
        t, s, [&](int c) -> float { return __fmaf_rn(bt, dold[c], r[c]); },
        [&](int i) -> float2 { return i < n ? make_float2(dold[i], r[i]) : make_float2(0.f, 0.f); },
        [&](int i, float acc, float2 own) {
          if (i < n) {
            const float di = __fmaf_rn(bt, own.x, own.y);
            dnew[i] = di;
            q[i] = acc;
            ff_add_prod(pdq, di, acc, f32);
          }
        });
    double dq;
    if (!team_sum_ff(t, pdq, s.w.partials, red, dq, f32)) return false;
    dec = kBGo;
    if (!isfinite(dq)) dec = kBNan;
    else if (!(dq > 0.0)) dec = kBBroke;
    if (dec == kBNan) {
      if (lead0) set_status(ctl, MPCG_ERR_NAN);
      break;
    }
    if (dec == kBBroke) {  // stage 1 ends here; x~ and r unchanged
      broke = 1;
      break;
    }
    const float alpha = (float)(rr / dq);
    // P2: x += alpha d_k, r -= alpha q, r^T r
    FF prr{0.f, 0.f};
    team_rows(
        t, s, [&](int i) -> float4 { return make_float4(dnew[i], x[i], q[i], r[i]); },
        [&](int i, float4 v) {
          x[i] = __fmaf_rn(alpha, v.x, v.y);
          const float ri = __fmaf_rn(-alpha, v.z, v.w);
          r[i] = ri;
          ff_add_prod(prr, ri, ri, f32);
        });
    double rrn;
    if (!team_sum_ff(t, prr, s.w.partials, red, rrn, f32)) return false;
    if (!isfinite(rrn)) {
      if (lead0) set_status(ctl, MPCG_ERR_NAN);
      break;
    }
    if (lead && mode == kCgK0) vsum += sqrt(rrn) / sqrt(rr);  // Eq. (13) ratio
    beta = (float)(rrn / rr);
    rr = rrn;
    if (mode == kCgK0) ++k0done;
    parity ^= 1;
    first = 0;
    ++it;
  }
  if (suspended) *done = false;
  if (lead0) {
    ctl->rr = rr;
    ctl->beta32 = beta;
    ctl->first = first;
    ctl->parity = parity;
    ctl->n1 = it;
  }
  if (lead0 && !suspended) {
    ctl->res32 = stop_measure(rr, bnorm, rel);
    if (broke) ctl->broke32 = 1;
    if (mode == kCgK0) {
      ctl->k0_done = k0done;
      ctl->vsum = vsum;
      ctl->v = k0done > 0 ? vsum / (double)k0done : 0.0;
    } else {
      if (ctl->res32 > ctl->eps1) ctl->warn_eps1 = 1;
      ctl->t_fp32 = globaltimer();
    }
  }
  return true;
}

// Double-precision stage: x0 = float64(x~) (or 0), restart r = b - A x0,
// d = r; CG to eps2 on the recursive residual; then the true residual, and a
// restart from x when it misses eps2 (at most max_restarts times).  At most
// `budget` iterations run per call; with `resume` the call continues the
// iteration state kept in the workspace (x, r, d) and the control block
// (r^T r, iterations, restarts).  *done is false when the budget ended it.
static __device__ bool sys_cg64(Team& t, const BatchSys& s, int from_zero, int& red, int budget,
                         bool resume, bool* done) {
  *done = true;
  Ctl* ctl = s.w.ctl;
  const int lane = threadIdx.x & 31;
  const int gw = team_warp(t), W = team_warps(t);
  const int n = s.n, rel = ctl->tol_relative;
  const bool lead = threadIdx.x == 0, lead0 = lead && t.rank == 0;
  const double bnorm = ctl->bnorm64, eps2 = ctl->eps2;
  const int max2 = ctl->max2, max_restarts = ctl->max_restarts;
  double* x = s.x;
  double* r = s.w.r64;
  double* d = s.w.d64;
  double* q = s.w.q64;
  const double* b = s.b;
  if (!resume) {
    if (lead0) ctl->t_s2 = globaltimer();
    for (int sl = gw; sl < s.nslices; sl += W) {
      const int i = sl * kSlice + lane;
      if (i < n) x[i] = from_zero ? 0.0 : (double)s.w.x32[i];
    }
    if (!team_sync(t)) return false;
  }
  int it = resume ? ctl->n2 : 0, restarts = resume ? ctl->restarts : 0, failed = 0;
  const int it_start = it;
  double rr = resume ? ctl->rr : 0.0, true_rel = NAN;
  const StopThr thr2 = stop_thr(eps2, bnorm, rel);  // used by thread 0
  bool skip_restart = resume;
  for (;;) {
    // restart (CG line 1 from x): r = b - A x, d = r, r^T r
    if (!skip_restart) {
    double p = 0.0;
    team_spmv<double, false>(
        t, s, [&](int c) -> double { return x[c]; },
        [&](int i) -> double { return i < n ? b[i] : 0.0; },
        [&](int i, double acc, double bi) {
          if (i < n) {
            const double ri = bi - acc;
            r[i] = ri;
            d[i] = ri;
            p = __fma_rn(ri, ri, p);
          }
        });
    if (!team_sum_d(t, p, s.w.partials, red, rr)) return false;
    }
    skip_restart = false;
    bool converged = false;
    for (;;) {
      int dec = kBGo;
      if (lead) {
        if (isnan(rr)) dec = kBNan;
        else if (stop_pass(thr2, rr)) dec = kBStop;
        else if (it >= max2) dec = kBCap;
        else if (it - it_start >= budget) dec = kBSuspend;
      }
      dec = bcast_dec(t, dec);
      if (dec == kBSuspend) {  // keep the iteration state for the next call
        if (lead0) {
          ctl->rr = rr;
          ctl->n2 = it;
          ctl->restarts = restarts;
        }
        *done = false;
        return true;
      }
      if (dec == kBNan) {
        failed = MPCG_ERR_NAN;
        break;
      }
      if (dec == kBStop) {
        converged = true;
        break;
      }
      if (dec == kBCap) {
        failed = MPCG_ERR_NOT_CONVERGED;
        break;
      }
      // P1: q = A d, d^T q
      double pq = 0.0;
      team_spmv<double, false>(
          t, s, [&](int c) -> double { return d[c]; },
          [&](int i) -> double { return i < n ? d[i] : 0.0; },
          [&](int i, double acc, double di) {
            if (i < n) {
              q[i] = acc;
              pq = __fma_rn(di, acc, pq);
            }
          });
      double dq;
      if (!team_sum_d(t, pq, s.w.partials, red, dq)) return false;
      dec = kBGo;
      if (lead) {
        if (!isfinite(dq)) dec = kBNan;
        else if (!(dq > 0.0)) dec = kBBreakdown;
        else t.S->val[2] = rr / dq;
      }
      dec = bcast_dec(t, dec);
      if (dec != kBGo) {
        failed = dec == kBNan ? MPCG_ERR_NAN : MPCG_ERR_BREAKDOWN;
        break;
      }
      const double alpha = t.S->val[2];
      // P2: x += alpha d, r -= alpha q, r^T r
      double pr = 0.0;
      team_rows(
          t, s, [&](int i) -> double4 { return make_double4(d[i], x[i], q[i], r[i]); },
          [&](int i, double4 v) {
            x[i] = __fma_rn(alpha, v.x, v.y);
            const double ri = __fma_rn(-alpha, v.z, v.w);
            r[i] = ri;
            pr = __fma_rn(ri, ri, pr);
          });
      double rrn;
      if (!team_sum_d(t, pr, s.w.partials, red, rrn)) return false;
      dec = kBGo;
      if (lead) {
        if (!isfinite(rrn)) dec = kBNan;
        else t.S->val[3] = rrn / rr;
      }
      dec = bcast_dec(t, dec);
      if (dec == kBNan) {
        failed = MPCG_ERR_NAN;
        break;
      }
      const double beta = t.S->val[3];
      rr = rrn;
      // P3: d = r + beta d
      team_rows(
          t, s, [&](int i) -> double2 { return make_double2(d[i], r[i]); },
          [&](int i, double2 v) { d[i] = __fma_rn(beta, v.x, v.y); });
      if (!team_sync(t)) return false;
      ++it;
    }
    if (failed && failed != MPCG_ERR_NOT_CONVERGED) break;
    // true residual ||b - A x|| (also after the iteration cap)
    double pt = 0.0;
    team_spmv<double, false>(
        t, s, [&](int c) -> double { return x[c]; },
        [&](int i) -> double { return i < n ? b[i] : 0.0; },
        [&](int i, double acc, double bi) {
          if (i < n) {
            const double ri = bi - acc;
            pt = __fma_rn(ri, ri, pt);
          }
        });
    double tot;
    if (!team_sum_d(t, pt, s.w.partials, red, tot)) return false;
    int again = 0;  // 1: restart from x; 2: the last restart still missed eps2
    if (lead) {
      true_rel = bnorm > 0.0 ? sqrt(tot) / bnorm : sqrt(tot);
      const double tm = rel ? true_rel : sqrt(tot);
      if (converged && tm > eps2) again = restarts < max_restarts ? 1 : 2;
    }
    again = bcast_dec(t, again);
    if (again == 2) failed = MPCG_ERR_NOT_CONVERGED;
    if (again != 1) break;
    ++restarts;
  }
  if (lead0) {
    if (failed) set_status(ctl, failed);
    ctl->n2 = it;
    ctl->restarts = restarts;
    if (restarts) ctl->warn_restart = 1;
    ctl->res64 = stop_measure(rr, bnorm, rel);
    ctl->true_rel = true_rel;
    ctl->rr = rr;
    ctl->t_fp64 = globaltimer();
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// One system, start to finish, by the team.
// ---------------------------------------------------------------------------------------
static __device__ void sys_finalize(const Team& t, const BatchSys& s) {
  if (t.rank != 0 || threadIdx.x != 0) return;
  const Ctl* c = s.w.ctl;
  mpcg_result_t* res = s.res;
  int st = c->status;
  if (st == 0) st = c->warn_restart ? MPCG_WARN_TRUE_RESID_RESTARTED
                                    : (c->warn_eps1 ? MPCG_WARN_EPS1_NOT_REACHED : MPCG_OK);
  res->status = st;
  res->n1 = c->n1;
  res->n2 = c->n2;
  res->cls = c->cls;
  res->k0_done = c->k0_done;
  res->restarts = c->restarts;
  res->eps1 = c->eps1;
  res->true_rel_resid = c->true_rel;
  res->pdiam = (double)c->pdiam;
  res->v = c->v;
  res->res_fp32 = c->res32;
  res->res_fp64 = c->res64;
  res->t_start_ns = c->t_start;
  const unsigned long long t0 = c->t_prep ? c->t_prep : c->t_start;
  res->t_features_ns = c->t_features ? c->t_features : t0;
  res->t_fp32_ns = c->t_fp32 ? c->t_fp32 : res->t_features_ns;
  res->t_fp64_ns = c->t_fp64 ? c->t_fp64 : res->t_fp32_ns;
  res->t_end_ns = globaltimer();
  res->t_prep_ns = t0;
  res->t_stage2_ns = c->t_s2 ? c->t_s2 : res->t_fp32_ns;
  res->spmv_cols = c->colbits;
  res->team_blocks = t.size;
}

// Status of the system as seen after a team barrier (identical in every block).
__device__ __forceinline__ int sys_status(const BatchSys& s) { return volatile_status(s.w.ctl); }

// Leader: next system for a team of class c -- its own queue first, then
// the queues of smaller classes.  -1 when all are empty.
static __device__ int batch_take(BatchHdr* h, const int* order, int c) {
  for (int cc = c; cc >= 0; --cc) {
    if (*reinterpret_cast<volatile int*>(&h->head[cc]) >= h->qlen[cc]) continue;
    const int i = atomicAdd(&h->head[cc], 1);
    if (i < h->qlen[cc]) return order[h->qbase[cc] + i];
  }
  return -1;
}

// Block-local 2BFS of one system (every thread of the calling block):
// ctl->pdiam, far_t, reached and connected = 1 if the graph is connected,
// else only connected = 0.  Not inlined: its code then leaves the register
// allocation of the CG loops in the same kernel alone (measured: inlined, the
// FP64 stage of a 512-system batch ran 12 % slower), and only the system's
// pointer crosses the call, so the search itself keeps its state in
// registers.
static __device__ __noinline__ void block_bfs_system(const BatchSys* sp, int smem_bytes) {
  const BatchSys& s = *sp;
  Ctl* ctl = s.w.ctl;
  int32_t* const gq[4] = {s.w.fq0, s.w.fq1, s.w.fq2, s.w.fq3};
  const BlockBfs b = block_bfs_layout(s.A.row_ptr, s.A.col, s.n, team_dyn, smem_bytes,
                                      reinterpret_cast<uint32_t*>(s.w.ckey), gq);
  int pd = 0, tv = 0;
  const bool ok = block_pseudo_diameter(b, &pd, &tv);
  if (threadIdx.x == 0) {
    if (ok) {
      ctl->pdiam = pd;
      ctl->far_t = tv;
      ctl->reached = s.n;
    }
    ctl->connected = ok ? 1 : 0;
  }
}

// 2BFS pseudo-diameter of the system (Sec. 6): ctl->pdiam and ctl->far_t.
// Connected systems of up to kBlockBfsMaxN rows: the team's first block runs
// both searches alone in shared memory (bfs_block.cuh) while the others wait
// at the barrier.  Larger or disconnected systems (and launches without the
// shared buffer): the team version over all of the team's blocks.
static __device__ bool team_pseudo_diameter(Team& t, const BatchSys& s, int smem_bytes) {
  Ctl* ctl = s.w.ctl;
  if (s.n >= 1 && s.n <= kBlockBfsMaxN && smem_bytes > 0) {
    if (t.rank == 0) block_bfs_system(&s, smem_bytes);
    if (!team_sync(t)) return false;
    if (*reinterpret_cast<volatile int*>(&ctl->connected)) return true;
  }
  BfsGraph g{ctl, s.A.row_ptr, s.A.col, s.n, s.w.fq0, s.w.fq1, s.w.label, s.w.ckey,
             s.w.fq2, s.w.fq3};
  TeamSyncFn sync{&t};
  return pseudo_diameter_run<TeamSyncFn, false>(g, s.w.dist, s.w.dist2, team_tid(t),
                                                team_threads(t), sync);
}

// ---------------------------------------------------------------------------------------
// Host: plan of a team launch (batch.cu).
// ---------------------------------------------------------------------------------------
struct Plan {
  std::vector<int> team_of_block, rank_of_block, team_size, team_class, order;
  int qbase[kTeamClasses], qlen[kTeamClasses];
};
// Teams for a grid of `grid` blocks and the class queues of nsys systems of
// n rows with estimated work `work` (largest first within a class); a system
// goes to the smallest team with at most rows_per_block rows per block, or
// rows_sys[i] when that array is given and its entry is positive.
Plan make_plan(int nsys, const int* n, const double* work, int grid, int rows_per_block,
               const int32_t* rows_sys = nullptr);
// Dynamic shared memory of a team launch of `kernel`: kTeamSmem when it runs
// a single-precision stage (stage1 != 0), else only the scan's kScanSmem.
// Raises the kernel's limit on the current device; -1 on a CUDA error.
int team_smem(const void* kernel, int stage1);

}  // namespace mpcg
