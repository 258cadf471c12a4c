// bfs_core.cuh -- sparsity-graph features of Sec. 6 as device routines that
// any group of whole warps can run: breadth-first search, connected
// components and the 2BFS pseudo-diameter.  The group is given by a thread
// index tid in [0, T) (warp-aligned) and a bounded barrier `sync` over the
// group; the standalone kernels use a grid barrier over whole blocks, the
// fused stage-1 kernel one warp per block.
//
// BFS is level-synchronous: the frontier of level L is a queue; each thread
// expands one frontier vertex with a warp-uniform trip count, claims
// neighbours in groups of 8 with atomicCAS on dist, and reserves queue space
// for a whole warp with one atomicAdd.  Distances are exact and do not
// depend on scheduling.
//
// 2BFS readings: s = vertex 0 (the smallest vertex of its component); the
// farthest vertex t is the smallest index at maximal distance (atomicMax over
// the key (dist, ~index)).  The second search is started speculatively from
// vertex n - 1 together with the first (see pseudo_diameter_run).  If the first BFS misses vertices, components are
// labelled by their smallest vertex (label propagation with pointer
// jumping) and 2BFS runs in every component at once from multi-source
// frontiers; l~ is the largest second-BFS level.
#pragma once
#include "common.cuh"

namespace mpcg {

enum BfsSources { kSrcSingle = 0, kSrcRoots = 2, kSrcRootFar = 3 };
enum BfsRole { kRoleFirst = 0, kRoleSecond = 1, kRoleComponentFirst = 2, kRolePlain = 3 };

struct BfsGraph {
  Ctl* ctl;
  const int32_t* rp;
  const int32_t* col;
  int n;
  int32_t *fq0, *fq1, *label;
  unsigned long long* ckey;
  int32_t *fq2, *fq3;  // queues of the second search of bfs_dual
};

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Whole blocks, every thread of the grid: the library's grid barrier.
struct GridSync {
  static constexpr bool kWholeBlock = true;  // every thread of every block is in the group
  static constexpr bool kNarrow = true;      // narrow levels run by one warp
  static constexpr bool kHelpers = false;    // no other warps join the levels
  Ctl* ctl;
  int slot;
  unsigned long long round;
  __device__ bool operator()() { return grid_barrier(ctl, slot, round); }
};

// One warp per block: lane 0 arrives on the counter and polls (bounded).
struct WarpGroupSync {
  static constexpr bool kWholeBlock = false;  // one warp of every block is in the group
  static constexpr bool kNarrow = true;       // narrow levels run by one warp
  static constexpr bool kHelpers = false;     // no other warps join the levels
  Ctl* ctl;
  int slot;
  unsigned long long round;
  __device__ bool operator()() {
    __syncwarp();
    round += 1;
    int ok = 1;
    if ((threadIdx.x & 31) == 0) {
      const unsigned long long target = round * (unsigned long long)gridDim.x;
      red_release_add(&ctl->bar[slot].v, 1ull);
      if (ld_acquire(&ctl->bar[slot].v) < target) {
        const unsigned long long t0 = globaltimer();
        unsigned spins = 0;
        while (ld_acquire(&ctl->bar[slot].v) < target) {
          if ((++spins & 1023u) == 0) {
            if (volatile_status(ctl) != 0 || poll_cancel(ctl)) {
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
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
  }
};

// ---- helper warps ----
// Warps of a block that have nothing else to do (the consumers of the fused
// single-precision stage once their iterations wait for the label) can join
// the levels of the one-warp-per-block group.  The group's warp stays the only
// member of the grid barrier.  Per wide level it publishes the level in
// shared memory, meets the helpers at a block barrier, every warp of the
// block takes its share of the block's items, and a second block barrier
// closes the level before the grid barrier.  Which items a block owns does not
// change, so blocks with and without helpers mix freely.  The helpers' only
// unbounded waits are these block barriers, and the group's warp reaches them
// through bounded waits only: its release (help_release) ends every search.
struct HelpLevel {
  const int32_t* inA;
  const int32_t* inB;
  int32_t* outA;
  int32_t* outB;
  int32_t* dA;
  int32_t* dB;
  int* cntA;
  int* cntB;
  int sa, sb, level, cmd;  // cmd: 0 = run the level, 1 = leave
};

enum { kHelpNone = 0, kHelpJoined = 1, kHelpClosed = 2 };
constexpr int kHelpBarStart = 2;  // block barrier ids (1 is the consumers' own)
constexpr int kHelpBarEnd = 3;

__device__ __forceinline__ void named_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

struct WarpGroupHelped : WarpGroupSync {
  static constexpr bool kHelpers = true;
  volatile int* hstate;  // kHelpNone / kHelpJoined (set by the helpers) / kHelpClosed
  HelpLevel* hl;
  int nhelp;             // helper warps of the block
};

// One level of the dual search over the items [0, sa + sb) of the two
// frontiers (A's first): the warp whose chunk base is `wbase` takes the item
// pairs first_pair, first_pair + pair_step, ... of its chunk sequence (two
// items per lane, T apart, so that their loads and claims are in flight
// together).  A single search is the case sb = 0.
__device__ __forceinline__ void dual_level_items(const BfsGraph& g, const int32_t* inA,
                                                 const int32_t* inB, int32_t* outA, int32_t* outB,
                                                 int32_t* dA, int32_t* dB, int* cntA, int* cntB,
                                                 int sa, int sb, int level, int wbase, int T,
                                                 int first_pair, int pair_step) {
  const int lane = threadIdx.x & 31;
  const int total = sa + sb;
  for (int base = wbase + first_pair * 2 * T; base < total; base += pair_step * 2 * T) {
    int u[2], e0[2], deg[2];
    bool isB[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int idx = base + h * T + lane;
      isB[h] = idx >= sa;
      u[h] = -1;
      if (idx < total) u[h] = isB[h] ? inB[idx - sa] : inA[idx];
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      e0[h] = 0;
      deg[h] = 0;
      if (u[h] >= 0) {
        e0[h] = g.rp[u[h]];
        deg[h] = g.rp[u[h] + 1] - e0[h];
      }
    }
    const int maxdeg = __reduce_max_sync(0xffffffffu, max(deg[0], deg[1]));
    for (int k0 = 0; k0 < maxdeg; k0 += 8) {
      int w[2][8];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 8; ++j) w[h][j] = (k0 + j < deg[h]) ? g.col[e0[h] + k0 + j] : -1;
      bool push[2][8];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int32_t* dist = isB[h] ? dB : dA;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          push[h][j] =
              w[h][j] >= 0 && w[h][j] != u[h] && atomicCAS(&dist[w[h][j]], -1, level + 1) == -1;
      }
      int mA = 0, mB = 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int mine = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) mine += push[h][j] ? 1 : 0;
        if (isB[h]) mB += mine;
        else mA += mine;
      }
      // separate warp scans for the pushes into A's and into B's queue
      int incA = mA, incB = mB;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int ta = __shfl_up_sync(0xffffffffu, incA, o);
        const int tb = __shfl_up_sync(0xffffffffu, incB, o);
        if (lane >= o) {
          incA += ta;
          incB += tb;
        }
      }
      const int totA = __shfl_sync(0xffffffffu, incA, 31);
      const int totB = __shfl_sync(0xffffffffu, incB, 31);
      int bA = 0, bB = 0;
      if (lane == 0) {
        if (totA > 0) bA = atomicAdd(cntA, totA);
        if (totB > 0) bB = atomicAdd(cntB, totB);
      }
      bA = __shfl_sync(0xffffffffu, bA, 0);
      bB = __shfl_sync(0xffffffffu, bB, 0);
      int posA = bA + incA - mA, posB = bB + incB - mB;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (push[h][j]) {
            if (isB[h]) outB[posB++] = w[h][j];
            else outA[posA++] = w[h][j];
          }
        }
      }
    }
  }
}

// The group's warp at the start of a wide level: when helpers have joined
// and the level needs more than one round of the group's warps alone (two
// items a lane), publish the level and meet them.  Returns the warps of the
// block on it.
template <class Sync>
__device__ __forceinline__ int help_begin(Sync& s, const HelpLevel& L) {
  if constexpr (Sync::kHelpers) {
    if (L.sa + L.sb <= 64 * (int)gridDim.x) return 1;  // one round: more warps cannot shorten it
    int st = 0;
    if ((threadIdx.x & 31) == 0) st = *s.hstate;
    st = __shfl_sync(0xffffffffu, st, 0);
    if (st != kHelpJoined) return 1;
    // The other blocks' queue entries, acquired by lane 0 at the grid
    // barrier, reach the helpers through the block barrier (the same order
    // as the consumers' own grid barrier: acquire by one thread, then bar.sync).
    if ((threadIdx.x & 31) == 0) *s.hl = L;
    __syncwarp();
    named_bar(kHelpBarStart, (s.nhelp + 1) * 32);
    return s.nhelp + 1;
  } else {
    return 1;
  }
}

// The group's warp at the end of a level run with helpers: wait for their
// claims and pushes before the grid barrier publishes them.
template <class Sync>
__device__ __forceinline__ void help_end(Sync& s, int warps) {
  if constexpr (Sync::kHelpers) {
    if (warps > 1) {
      // the helpers' claims and pushes precede the barrier, and lane 0's
      // release at the grid barrier that follows covers them
      named_bar(kHelpBarEnd, (s.nhelp + 1) * 32);
      __syncwarp();
    }
  }
}

// The group's warp once its searches are over (on every path): no helper
// joins any more, and helpers that have joined are sent away.
template <class Sync>
__device__ void help_release(Sync& s) {
  if constexpr (Sync::kHelpers) {
    int old = 0;
    if ((threadIdx.x & 31) == 0) old = atomicCAS(const_cast<int*>(s.hstate), kHelpNone, kHelpClosed);
    old = __shfl_sync(0xffffffffu, old, 0);
    if (old == kHelpJoined) {
      if ((threadIdx.x & 31) == 0) {
        s.hl->cmd = 1;
        *s.hstate = kHelpClosed;
      }
      __syncwarp();
      named_bar(kHelpBarStart, (s.nhelp + 1) * 32);
    }
  }
}

// A helper warp (warp index gw >= 1 among the block's nhelp + 1) in the
// levels of the block's group until the release.
static __device__ __noinline__ void bfs_help(const BfsGraph g, const HelpLevel* hl, int nhelp, int gw) {
  const int wbase = blockIdx.x * 32, T = gridDim.x * 32;
  for (;;) {
    named_bar(kHelpBarStart, (nhelp + 1) * 32);
    const volatile HelpLevel* v = hl;
    if (v->cmd) break;
    dual_level_items(g, v->inA, v->inB, v->outA, v->outB, v->dA, v->dB, v->cntA, v->cntB, v->sa,
                     v->sb, v->level, wbase, T, gw, nhelp + 1);
    named_bar(kHelpBarEnd, (nhelp + 1) * 32);
  }
}

// One BFS over the group.  Writes dist (all n entries), and by role: the
// farthest-vertex key and the reached count (first), per-component keys
// (component-first) or the largest level (second) in the control block.
template <class Sync>
__device__ bool bfs_run(const BfsGraph& g, int32_t* dist, int sources, int src, int role, int tid,
                        int T, Sync& sync) {
  Ctl* ctl = g.ctl;
  const int n = g.n;
  const int lane = threadIdx.x & 31;
  const int wbase = tid - lane;
  for (int v = tid; v < n; v += T) dist[v] = -1;
  if (tid == 0) {
    ctl->qsize[0] = 0;
    ctl->qsize[1] = 0;
    ctl->qsize[2] = 0;
  }
  if (!sync()) return false;
  if (sources == kSrcSingle) {
    if (tid == 0) {
      dist[src] = 0;
      g.fq0[0] = src;
      ctl->qsize[0] = 1;
    }
  } else {
    for (int base = wbase; base < n; base += T) {  // warp-uniform bound
      const int v = base + lane;
      const bool root = v < n && g.label[v] == v;
      int s = v;
      if (root && sources == kSrcRootFar) s = far_key_vertex(g.ckey[v]);
      if (root) dist[s] = 0;
      const unsigned mask = __ballot_sync(0xffffffffu, root);
      if (mask) {
        int b0 = 0;
        if (lane == 0) b0 = atomicAdd(&ctl->qsize[0], __popc(mask));
        b0 = __shfl_sync(0xffffffffu, b0, 0);
        if (root) g.fq0[b0 + __popc(mask & ((1u << lane) - 1u))] = s;
      }
    }
  }
  if (!sync()) return false;

  int level = 0;
  long long reached = 0;
  for (;;) {
    const int32_t* in = (level & 1) ? g.fq1 : g.fq0;
    int32_t* out = (level & 1) ? g.fq0 : g.fq1;
    const int size = *reinterpret_cast<volatile int*>(&ctl->qsize[level % 3]);
    if (size == 0) break;
    reached += size;
    if (tid == 0) ctl->qsize[(level + 2) % 3] = 0;
    int* cnt = &ctl->qsize[(level + 1) % 3];
    if constexpr (Sync::kHelpers) {  // the dual level body with an empty second search
      const HelpLevel L{in, in, out, out, dist, dist, cnt, cnt, size, 0, level, 0};
      const int warps = help_begin(sync, L);
      dual_level_items(g, in, in, out, out, dist, dist, cnt, cnt, size, 0, level, wbase, T, 0,
                       warps);
      help_end(sync, warps);
    } else {
    for (int base = wbase; base < size; base += T) {
      const int idx = base + lane;
      int u = -1, e0 = 0, deg = 0;
      if (idx < size) {
        u = in[idx];
        e0 = g.rp[u];
        deg = g.rp[u + 1] - e0;
      }
      const int maxdeg = __reduce_max_sync(0xffffffffu, deg);
      for (int k0 = 0; k0 < maxdeg; k0 += 8) {
        int w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) w[j] = (k0 + j < deg) ? g.col[e0 + k0 + j] : -1;
        bool push[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
          push[j] = w[j] >= 0 && w[j] != u && atomicCAS(&dist[w[j]], -1, level + 1) == -1;
        int mine = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) mine += push[j] ? 1 : 0;
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (total > 0) {
          int b0 = 0;
          if (lane == 0) b0 = atomicAdd(cnt, total);
          int pos = __shfl_sync(0xffffffffu, b0, 0) + incl - mine;
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (push[j]) out[pos++] = w[j];
        }
      }
    }
    }
    ++level;
    if (!sync()) return false;
  }
  const int maxlevel = level - 1;  // levels 0 .. level-1 were non-empty

  if (role == kRoleFirst) {
    unsigned long long best = 0;
    for (int v = tid; v < n; v += T) {
      const int d = dist[v];
      if (d >= 0) {
        const unsigned long long k = far_key(d, v);
        best = k > best ? k : best;
      }
    }
    best = warp_max_u64(best);
    if (lane == 0 && best) atomicMax(&ctl->key, best);
    if (tid == 0) ctl->reached = (int)reached;
  } else if (role == kRoleComponentFirst) {
    for (int v = tid; v < n; v += T) {
      const int d = dist[v];
      if (d >= 0) atomicMax(&g.ckey[g.label[v]], far_key(d, v));
    }
  } else if (role == kRoleSecond) {
    if (tid == 0) ctl->pdiam = maxlevel > 0 ? maxlevel : 0;
  }
  return true;
}

// ---- one-warp mode of the dual search (narrow frontiers) ----
// A level whose two frontiers together hold at most kNarrowItems vertices is
// run by one warp of the group (tid < 32) alone: no group barrier, the
// frontier in shared memory, row pointers and columns through the read-only
// cache (a narrow frontier on a banded ordering reuses them level after
// level).  As nothing else writes the distance arrays meanwhile, a claim is
// a read of the candidate's distance, a shared-memory set that settles
// candidates reached twice in the level, and a plain store (levels with a
// row wider than kNarrowHashDeg claim by compare-and-swap instead).  The warp also writes every claimed vertex to the group's queue of
// the next level, so that when a frontier grows past kNarrowItems it hands the
// search back at that level with nothing to copy.  The rest of the group waits
// on the control block's mode word: one lane of one warp a block polls it with
// pauses (the one-warp levels are latency-bound and must not share the memory
// system with a crowd of pollers), and in a whole-block group passes it on
// through shared memory.
constexpr int kNarrowItems = 64;
constexpr int kNarrowHash = 2048;  // shared-memory set of the level's claims (load <= 1/2)
constexpr int kNarrowHashDeg = 16; // levels with a wider row claim by compare-and-swap
enum { kNmResume = 1, kNmDone = 2 };

// Whether the mode word ends the wait of the group left at level L: the
// search finished, or was handed back at a level after L (an earlier
// hand-back, at L or before, may still be in the word); -1 = a failed wait.
__device__ __forceinline__ bool nm_ends(int m, int L) {
  return m == -1 || (m & 3) == kNmDone || ((m & 3) == kNmResume && (m >> 2) > L);
}

template <bool kBlk>
__device__ int nm_wait(Ctl* ctl, int L, volatile int* s_mode) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool poller = !kBlk || warp == (blockIdx.x == 0 ? 1 : 0);
  int m = 0;
  if (lane == 0) {
    const unsigned long long t0 = globaltimer();
    unsigned spins = 0;
    for (;;) {
      if (poller) {
        m = *reinterpret_cast<volatile int*>(&ctl->nmode);
        if (nm_ends(m, L)) break;
        __nanosleep(1000);
        if ((++spins & 15u) == 0) {
          if (volatile_status(ctl) != 0 || poll_cancel(ctl)) {
            m = -1;
            break;
          }
          if (globaltimer() - t0 > (unsigned long long)ctl->timeout_ns) {
            set_status(ctl, MPCG_ERR_TIMEOUT);
            m = -1;
            break;
          }
        }
      } else {  // the block's poller relays the word (and a failure) in shared memory
        m = *s_mode;
        if (nm_ends(m, L)) break;
        __nanosleep(500);
        if (globaltimer() - t0 > (unsigned long long)ctl->timeout_ns + 100000000ull) {
          m = -1;  // the poller's own limit passed long ago (it records the status)
          break;
        }
      }
    }
    __threadfence();
    if (kBlk && poller) *s_mode = m;
  }
  m = __shfl_sync(0xffffffffu, m, 0);
  __syncwarp();
  return m;
}

// The one warp's levels, from level L whose frontiers (sizes sa, sb) are in
// the group's queues.  Updates la, lb, reached (search A's vertices) for the
// levels after L that it completes.  Returns the level at which the group
// resumes (its frontiers in the queues and counters), or -1 when both
// searches have ended.
static __device__ int narrow_levels(const BfsGraph& g, int32_t* dA, int32_t* dB, int L, int sa, int sb,
                             int& la, int& lb, long long& reached, int (*s_cur)[kNarrowItems],
                             int (*s_nxt)[kNarrowItems], int* s_hash) {
  Ctl* ctl = g.ctl;
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < kNarrowHash; i += 32) s_hash[i] = -1;
  {
    const int32_t* inA = (L & 1) ? g.fq1 : g.fq0;
    const int32_t* inB = (L & 1) ? g.fq3 : g.fq2;
    for (int i = lane; i < sa; i += 32) s_cur[0][i] = __ldcg(inA + i);
    for (int i = lane; i < sb; i += 32) s_cur[1][i] = __ldcg(inB + i);
  }
  __syncwarp();
  int nA = sa, nB = sb, cur = L;
  for (;;) {
    int32_t* outA = (cur & 1) ? g.fq0 : g.fq1;
    int32_t* outB = (cur & 1) ? g.fq2 : g.fq3;
    // two frontier items per lane: i = lane, lane + 32 over A's items then B's
    int u[2], e0[2], deg[2];
    bool isB[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = lane + 32 * h;
      isB[h] = i >= nA;
      u[h] = -1;
      e0[h] = 0;
      deg[h] = 0;
      if (i < nA + nB) u[h] = isB[h] ? s_cur[1][i - nA] : s_cur[0][i];
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (u[h] >= 0) {
        e0[h] = __ldg(g.rp + u[h]);
        deg[h] = __ldg(g.rp + u[h] + 1) - e0[h];
      }
    }
    const int maxdeg = __reduce_max_sync(0xffffffffu, max(deg[0], deg[1]));
    const bool hashed = maxdeg <= kNarrowHashDeg;
    int totA = 0, totB = 0;
    for (int k0 = 0; k0 < maxdeg; k0 += 8) {
      int w[2][8];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 8; ++j) w[h][j] = (k0 + j < deg[h]) ? __ldg(g.col + e0[h] + k0 + j) : -1;
      bool push[2][8];
      if (hashed) {
        // Only this warp writes the distances now: read them, and settle
        // duplicates among the level's unvisited candidates in the set.
        int dv[2][8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int32_t* dist = isB[h] ? dB : dA;
#pragma unroll
          for (int j = 0; j < 8; ++j)
            dv[h][j] = (w[h][j] >= 0 && w[h][j] != u[h]) ? __ldcg(dist + w[h][j]) : 0;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int32_t* dist = isB[h] ? dB : dA;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            push[h][j] = false;
            if (dv[h][j] == -1) {
              const int key = 2 * w[h][j] + (isB[h] ? 1 : 0);
              unsigned slot = ((unsigned)key * 2654435761u) & (kNarrowHash - 1);
              bool settled = false;
              // at most 64 items x 16 columns enter a set of 2048 slots, so a
              // free slot is near; the bound only guards the loop
              for (int probe = 0; probe < kNarrowHash && !settled; ++probe) {
                const int old = atomicCAS(&s_hash[slot], -1, key);
                if (old == -1) {
                  push[h][j] = true;
                  dist[w[h][j]] = cur + 1;
                  settled = true;
                } else if (old == key) {
                  settled = true;
                }
                slot = (slot + 1) & (kNarrowHash - 1);
              }
              if (!settled) push[h][j] = atomicCAS(&dist[w[h][j]], -1, cur + 1) == -1;
            }
          }
        }
      } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int32_t* dist = isB[h] ? dB : dA;
#pragma unroll
          for (int j = 0; j < 8; ++j)
            push[h][j] = w[h][j] >= 0 && w[h][j] != u[h] && atomicCAS(&dist[w[h][j]], -1, cur + 1) == -1;
        }
      }
      int mA = 0, mB = 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int mine = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) mine += push[h][j] ? 1 : 0;
        if (isB[h]) mB += mine;
        else mA += mine;
      }
      int incA = mA, incB = mB;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int ta = __shfl_up_sync(0xffffffffu, incA, o);
        const int tb = __shfl_up_sync(0xffffffffu, incB, o);
        if (lane >= o) {
          incA += ta;
          incB += tb;
        }
      }
      int posA = totA + incA - mA, posB = totB + incB - mB;
      totA += __shfl_sync(0xffffffffu, incA, 31);
      totB += __shfl_sync(0xffffffffu, incB, 31);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (push[h][j]) {
            if (isB[h]) {
              outB[posB] = w[h][j];
              if (posB < kNarrowItems) s_nxt[1][posB] = w[h][j];
              ++posB;
            } else {
              outA[posA] = w[h][j];
              if (posA < kNarrowItems) s_nxt[0][posA] = w[h][j];
              ++posA;
            }
          }
        }
      }
    }
    __syncwarp();
    if (hashed) {  // empty the set for the next level
      for (int i = lane; i < kNarrowHash; i += 32) s_hash[i] = -1;
      __syncwarp();
    }
    ++cur;
    if (totA == 0 && totB == 0) return -1;
    if (totA + totB > kNarrowItems) {  // hand back: the group runs level cur from the queues
      if (lane == 0) {
        ctl->qsize[cur % 3] = totA;
        ctl->qsizeB[cur % 3] = totB;
        ctl->qsize[(cur + 1) % 3] = 0;
        ctl->qsizeB[(cur + 1) % 3] = 0;
      }
      return cur;
    }
    reached += totA;
    if (totA) la = cur;
    if (totB) lb = cur;
    nA = totA;
    nB = totB;
    int (*t)[kNarrowItems] = s_cur;
    s_cur = s_nxt;
    s_nxt = t;
  }
}

// Two breadth-first searches advanced together, one barrier per level: A
// from srcA into dA (queues fq0/fq1, counters qsize), B from srcB into dB
// (queues fq2/fq3, counters qsizeB).  Each search is exactly the BFS that
// bfs_run gives; the levels run until both frontiers are empty.  Out (in
// every thread): the last non-empty level of each search and the vertices
// reached by A.
template <class Sync>
__device__ bool bfs_dual(const BfsGraph& g, int32_t* dA, int32_t* dB, int srcA, int srcB, int tid,
                         int T, Sync& sync, int* lastA, int* lastB, long long* reachedA) {
  Ctl* ctl = g.ctl;
  const int n = g.n;
  const int lane = threadIdx.x & 31;
  const int wbase = tid - lane;
  for (int v = tid; v < n; v += T) {
    dA[v] = -1;
    dB[v] = -1;
  }
  if (tid == 0) {
    for (int k = 0; k < 3; ++k) {
      ctl->qsize[k] = 0;
      ctl->qsizeB[k] = 0;
    }
    ctl->nmode = 0;
  }
  if (!sync()) return false;
  if (tid == 0) {
    dA[srcA] = 0;
    dB[srcB] = 0;
    g.fq0[0] = srcA;
    g.fq2[0] = srcB;
    ctl->qsize[0] = 1;
    ctl->qsizeB[0] = 1;
  }
  if (!sync()) return false;
  int level = 0, la = 0, lb = 0;
  long long reached = 0;
  for (;;) {
    const int sa = *reinterpret_cast<volatile int*>(&ctl->qsize[level % 3]);
    const int sb = *reinterpret_cast<volatile int*>(&ctl->qsizeB[level % 3]);
    if (sa == 0 && sb == 0) break;
    reached += sa;
    if (sa) la = level;
    if (sb) lb = level;
    if constexpr (Sync::kNarrow) {
    if (sa + sb <= kNarrowItems) {
      // ---- narrow frontiers: one warp runs the next levels alone ----
      __shared__ int s_nbuf[4][kNarrowItems];  // the warp's current and next frontiers
      __shared__ int s_hash[kNarrowHash];      // the warp's set of a level's claims
      __shared__ volatile int s_nmode;         // whole-block groups: the block's copy of the mode word
      if constexpr (Sync::kWholeBlock) {
        if (threadIdx.x == 0) s_nmode = 0;
        __syncthreads();  // every thread of the block is here (same level, same decision)
      }
      int resume;
      if (tid < 32) {
        resume = narrow_levels(g, dA, dB, level, sa, sb, la, lb, reached,
                               reinterpret_cast<int (*)[kNarrowItems]>(&s_nbuf[0][0]),
                               reinterpret_cast<int (*)[kNarrowItems]>(&s_nbuf[2][0]), s_hash);
        if (lane == 0) {
          ctl->nla = la;
          ctl->nlb = lb;
          ctl->nreached = reached;
          __threadfence();
          atomicExch(&ctl->nmode, resume < 0 ? kNmDone : ((resume << 2) | kNmResume));
        }
        __syncwarp();
      } else {
        const int m = nm_wait<Sync::kWholeBlock>(ctl, level, &s_nmode);
        if (m == -1) return false;
        la = *reinterpret_cast<volatile int*>(&ctl->nla);
        lb = *reinterpret_cast<volatile int*>(&ctl->nlb);
        reached = *reinterpret_cast<volatile long long*>(&ctl->nreached);
        resume = (m & 3) == kNmDone ? -1 : (m >> 2);
      }
      if (resume < 0) break;
      // resume: the loop's head reads the level's sizes from the counters
      // and adds them to the state (the published state stops before it);
      // the frontiers are larger than kNarrowItems, so the group runs it
      level = resume;
      continue;
    }
    }
    if (tid == 0) {
      ctl->qsize[(level + 2) % 3] = 0;
      ctl->qsizeB[(level + 2) % 3] = 0;
    }
    const int32_t* inA = (level & 1) ? g.fq1 : g.fq0;
    int32_t* outA = (level & 1) ? g.fq0 : g.fq1;
    const int32_t* inB = (level & 1) ? g.fq3 : g.fq2;
    int32_t* outB = (level & 1) ? g.fq2 : g.fq3;
    int* cntA = &ctl->qsize[(level + 1) % 3];
    int* cntB = &ctl->qsizeB[(level + 1) % 3];
    if constexpr (Sync::kHelpers) {
      const HelpLevel L{inA, inB, outA, outB, dA, dB, cntA, cntB, sa, sb, level, 0};
      const int warps = help_begin(sync, L);
      dual_level_items(g, inA, inB, outA, outB, dA, dB, cntA, cntB, sa, sb, level, wbase, T, 0,
                       warps);
      help_end(sync, warps);
    } else {
      dual_level_items(g, inA, inB, outA, outB, dA, dB, cntA, cntB, sa, sb, level, wbase, T, 0, 1);
    }
    ++level;
    if (!sync()) return false;
  }
  *lastA = la;
  *lastB = lb;
  *reachedA = reached;
  return true;
}

// Connected components: label[v] = smallest vertex of v's component.
// Rounds of (hook: for every edge with differing labels, lower the larger
// label's entry to the smaller label) and (pointer jumping to the root),
// until a hook round changes nothing.  Labels only decrease and always name
// a vertex of the same component, so a component's root is its smallest
// vertex.
template <class Sync>
__device__ bool cc_run(const BfsGraph& g, int tid, int T, Sync& sync) {
  Ctl* ctl = g.ctl;
  const int n = g.n;
  const int lane = threadIdx.x & 31;
  int32_t* label = g.label;
  for (int v = tid; v < n; v += T) {
    label[v] = v;
    g.ckey[v] = 0ull;
  }
  if (tid == 0) {
    ctl->ccflag[0] = 0;
    ctl->ccflag[1] = 0;
  }
  if (!sync()) return false;
  for (int r = 0;; ++r) {
    int changed = 0;
    for (int u = tid; u < n; u += T) {
      const int e1 = g.rp[u + 1];
      for (int e = g.rp[u]; e < e1; ++e) {
        const int v = g.col[e];
        if (v == u) continue;
        const int lu = label[u], lv = label[v];
        if (lu < lv) {
          atomicMin(&label[lv], lu);
          changed = 1;
        } else if (lv < lu) {
          atomicMin(&label[lu], lv);
          changed = 1;
        }
      }
    }
    if (__any_sync(0xffffffffu, changed) && lane == 0) atomicExch(&ctl->ccflag[r & 1], 1);
    if (!sync()) return false;
    if (tid == 0) ctl->ccflag[(r + 1) & 1] = 0;
    for (int v = tid; v < n; v += T) {
      int l = label[v];
      for (int ll = label[l]; ll != l; ll = label[l]) l = ll;
      label[v] = l;
    }
    if (!sync()) return false;
    if (*reinterpret_cast<volatile int*>(&ctl->ccflag[r & 1]) == 0) break;
  }
  return true;
}

// Runs r = 1 .. R-1 of the repeated 2BFS (the remark of Sec. 6; R =
// ctl->bfs_starts): one 2BFS from s_r = floor(r n / R) inside its component
// each (BFS from s_r, t_r = the smallest vertex at the largest distance, BFS
// from t_r); ctl->pdiam becomes the largest of all runs.  Not inlined: the
// kernels that compute features carry it as a call.
template <class Sync>
__device__ __noinline__ bool pseudo_diameter_repeats(const BfsGraph& g, int32_t* d1, int32_t* d2,
                                                     int tid, int T, Sync& sync) {
  Ctl* ctl = g.ctl;
  const int R = ctl->bfs_starts;
  for (int r = 1; r < R; ++r) {
    const int s = (int)(((long long)r * g.n) / R);
    // Every thread has read the previous run's farthest-vertex key before it
    // is reset: a thread that read the reset key would take another branch
    // (and another number of barriers) than the rest of the group.
    if (!sync()) return false;
    if (tid == 0) ctl->key = 0ull;
    if (!sync()) return false;
    const int prev = *reinterpret_cast<volatile int*>(&ctl->pdiam);
    if (!bfs_run(g, d1, kSrcSingle, s, kRoleFirst, tid, T, sync)) return false;
    if (!sync()) return false;
    const int t = far_key_vertex(*reinterpret_cast<volatile unsigned long long*>(&ctl->key));
    if (!bfs_run(g, d2, kSrcSingle, t, kRoleSecond, tid, T, sync)) return false;
    if (!sync()) return false;
    if (tid == 0) {
      const int cur = *reinterpret_cast<volatile int*>(&ctl->pdiam);
      ctl->pdiam = cur > prev ? cur : prev;
    }
    if (!sync()) return false;
  }
  return true;
}

// 2BFS pseudo-diameter with the per-component rule.  On return (true),
// ctl->pdiam holds l~ and ctl->far_t the farthest vertex found from vertex 0.
//
// The second BFS starts from t, which the first BFS determines.  It is run
// speculatively alongside the first, from t' = n - 1: in a grid graph
// numbered row by row the farthest vertex from vertex 0 is the opposite
// corner n - 1.  When the first BFS confirms t = t', the second search is
// exactly the BFS from t and l~ is its depth; otherwise the BFS from t runs
// afterwards.  Either way the result is that of the two searches in order.
// kRepeats: run the repeated 2BFS when ctl->bfs_starts > 1 (the team kernels
// instantiate it without, so that their code does not change).
template <class Sync, bool kRepeats = true>
__device__ bool pseudo_diameter_run(const BfsGraph& g, int32_t* d1, int32_t* d2, int tid, int T,
                                    Sync& sync) {
  Ctl* ctl = g.ctl;
  const int lane = threadIdx.x & 31;
  if (tid == 0) {
    ctl->key = 0ull;
    ctl->reached = 0;
  }
  if (!sync()) return false;
  const int guess = g.n - 1;
  int lastA = 0, lastB = 0;
  long long reached = 0;
  if (!bfs_dual(g, d1, d2, 0, guess, tid, T, sync, &lastA, &lastB, &reached)) return false;
  // farthest vertex of the first search: largest distance, then smallest index
  {
    unsigned long long best = 0;
    for (int v = tid; v < g.n; v += T) {
      const int d = d1[v];
      if (d >= 0) {
        const unsigned long long k = far_key(d, v);
        best = k > best ? k : best;
      }
    }
    best = warp_max_u64(best);
    if (lane == 0 && best) atomicMax(&ctl->key, best);
    if (tid == 0) ctl->reached = (int)reached;
  }
  if (!sync()) return false;
  const bool connected = reached == g.n;
  if (connected) {
    const int t = far_key_vertex(*reinterpret_cast<volatile unsigned long long*>(&ctl->key));
    if (tid == 0) ctl->far_t = t;
    if (t == guess) {
      if (tid == 0) ctl->pdiam = lastB > 0 ? lastB : 0;
    } else {
      if (!bfs_run(g, d2, kSrcSingle, t, kRoleSecond, tid, T, sync)) return false;
    }
  } else {
    if (!cc_run(g, tid, T, sync)) return false;
    if (!bfs_run(g, d1, kSrcRoots, 0, kRoleComponentFirst, tid, T, sync)) return false;
    if (!sync()) return false;
    if (!bfs_run(g, d2, kSrcRootFar, 0, kRoleSecond, tid, T, sync)) return false;
    if (tid == 0) ctl->far_t = far_key_vertex(g.ckey[0]);
  }
  if (tid == 0) ctl->connected = connected ? 1 : 0;
  if constexpr (kRepeats) {
    if (ctl->bfs_starts > 1) return pseudo_diameter_repeats(g, d1, d2, tid, T, sync);
  }
  return true;
}

}  // namespace mpcg
