// bfs_block.cuh -- the 2BFS pseudo-diameter of Sec. 6 run by ONE block, for
// the teams of the batched and serving kernels.
//
// The team version (bfs_core.cuh) pays, per BFS level, a team barrier and a
// chain of global-memory round trips (queue size, queue entry, row pointers,
// columns, the claim on dist, the queue counter).  Here a single block runs
// both searches with block barriers, visited BITMAPS (a claim is one atomicOr
// on a bit) and frontier queues and counters in shared memory, which leaves
// two dependent global loads per level (row pointers, then columns).  The
// other blocks of the team wait at the next team barrier.
//
// Storage (given by the caller): the bitmaps of the two searches in shared
// memory when they fit in half of the block's buffer, else in global scratch
// of n words; the four queues (A and B, even and odd levels) take the rest of
// the buffer, and entries past that capacity go to global queues of n
// entries.  So any n works; shared memory only makes it faster.
//
// Readings are those of bfs_core.cuh: search A from vertex 0; t = smallest
// vertex at the largest distance from 0 = smallest vertex of A's last
// non-empty level; l~ = last non-empty level of the BFS from t; the search
// from t is started speculatively from n - 1 with A.  Unlike the team
// version, B is dropped as soon as A ends with t != n - 1.  Only connected
// graphs are handled; otherwise the caller runs the team version.
#pragma once
#include <limits.h>

#include "common.cuh"

namespace mpcg {

struct BlockBfs {
  const int32_t* rp;
  const int32_t* col;
  int n;
  uint32_t* vis[2];  // visited bitmaps of searches A and B, (n + 31) / 32 words each
  int32_t* qs[4];    // shared queue heads: A even, A odd, B even, B odd (cap entries)
  int32_t* qg[4];    // global queues of n entries (entries at index >= cap)
  int cap;
  int* cnt;          // shared: A sizes [0..2] and B sizes [3..5] by level mod 3, [6] scratch
};

// Partition of a block's shared buffer (bytes, 16-aligned base) for n
// vertices.  vis_global: scratch of >= 2 * words words for the bitmaps when
// they do not fit.
static __device__ BlockBfs block_bfs_layout(const int32_t* rp, const int32_t* col, int n,
                                            unsigned char* smem, int smem_bytes,
                                            uint32_t* vis_global, int32_t* const gq[4]) {
  BlockBfs b;
  b.rp = rp;
  b.col = col;
  b.n = n;
  const int words = (n + 31) >> 5;
  b.cnt = reinterpret_cast<int*>(smem);
  unsigned char* p = smem + 64;
  int left = smem_bytes - 64;
  const long long vis_bytes = 2ll * words * 4;
  if (vis_bytes <= left / 2) {
    b.vis[0] = reinterpret_cast<uint32_t*>(p);
    b.vis[1] = b.vis[0] + words;
    const int used = (int)((vis_bytes + 15) & ~15ll);
    p += used;
    left -= used;
  } else {
    b.vis[0] = vis_global;
    b.vis[1] = vis_global + words;
  }
  b.cap = left / 16;
  if (b.cap > n) b.cap = n;
  for (int k = 0; k < 4; ++k) {
    b.qs[k] = reinterpret_cast<int32_t*>(p) + k * b.cap;
    b.qg[k] = gq[k];
  }
  return b;
}

static __device__ __forceinline__ int bq_get(const BlockBfs& b, int q, int i) {
  return i < b.cap ? b.qs[q][i] : b.qg[q][i];
}

static __device__ __forceinline__ void bq_put(const BlockBfs& b, int q, int i, int v) {
  if (i < b.cap) b.qs[q][i] = v;
  else b.qg[q][i] = v;
}

// Claim vertex w in a visited bitmap: true for exactly one caller.
static __device__ __forceinline__ bool bvis_claim(uint32_t* bm, int w) {
  const uint32_t bit = 1u << (w & 31);
  if (*reinterpret_cast<volatile uint32_t*>(&bm[w >> 5]) & bit) return false;
  return (atomicOr(&bm[w >> 5], bit) & bit) == 0u;
}

// Smallest entry of queue q (first `size` entries), in every thread.
static __device__ int block_queue_min(const BlockBfs& b, int q, int size) {
  if (threadIdx.x == 0) b.cnt[6] = INT_MAX;
  __syncthreads();
  int m = INT_MAX;
  for (int i = threadIdx.x; i < size; i += blockDim.x) m = min(m, bq_get(b, q, i));
  m = __reduce_min_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m != INT_MAX) atomicMin(&b.cnt[6], m);
  __syncthreads();
  const int r = *reinterpret_cast<volatile int*>(&b.cnt[6]);
  __syncthreads();
  return r;
}

struct BlockBfsOut {
  int la, lb;        // last non-empty level of A and of B (B: valid if !dropped)
  int t;             // smallest vertex of A's last level
  long long reached; // vertices reached by A
  bool dropped;      // B was dropped because t != srcB
};

// Searches A from srcA and (srcB >= 0) B from srcB, level-synchronous, in
// the calling block; every thread of the block calls it.
static __device__ BlockBfsOut block_bfs2(const BlockBfs& b, int srcA, int srcB) {
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, wbase = tid - lane;
  const int words = (b.n + 31) >> 5;
  for (int i = tid; i < words; i += T) {
    b.vis[0][i] = 0u;
    b.vis[1][i] = 0u;
  }
  if (tid < 7) b.cnt[tid] = 0;
  __syncthreads();
  if (tid == 0) {
    b.vis[0][srcA >> 5] |= 1u << (srcA & 31);
    bq_put(b, 0, 0, srcA);
    b.cnt[0] = 1;
    if (srcB >= 0) {
      b.vis[1][srcB >> 5] |= 1u << (srcB & 31);
      bq_put(b, 2, 0, srcB);
      b.cnt[3] = 1;
    }
  }
  __syncthreads();
  BlockBfsOut o{0, 0, -1, 0, false};
  bool liveB = srcB >= 0, doneA = false;
  int lastsa = 1;
  for (int level = 0;; ++level) {
    const int sa = *reinterpret_cast<volatile int*>(&b.cnt[level % 3]);
    int sb = liveB ? *reinterpret_cast<volatile int*>(&b.cnt[3 + level % 3]) : 0;
    if (sa == 0 && !doneA) {  // A has ended: its last level is known
      doneA = true;
      o.t = block_queue_min(b, o.la & 1, lastsa);
      if (liveB && o.t != srcB) {
        liveB = false;
        o.dropped = true;
        sb = 0;
      }
    }
    if (sa == 0 && sb == 0) break;
    o.reached += sa;
    if (sa) {
      o.la = level;
      lastsa = sa;
    }
    if (sb) o.lb = level;
    if (tid == 0) {
      b.cnt[(level + 2) % 3] = 0;
      b.cnt[3 + (level + 2) % 3] = 0;
    }
    const int qa = level & 1, qb = 2 + (level & 1);
    int* cntA = &b.cnt[(level + 1) % 3];
    int* cntB = &b.cnt[3 + (level + 1) % 3];
    const int total = sa + sb;
    // Two frontier vertices per lane per round, so that their loads overlap.
    for (int base = wbase; base < total; base += 2 * T) {  // warp-uniform bound
      int u[2], e0[2], deg[2];
      bool isB[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int idx = base + h * T + lane;
        isB[h] = idx >= sa;
        u[h] = -1;
        if (idx < total) u[h] = isB[h] ? bq_get(b, qb, idx - sa) : bq_get(b, qa, idx);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        e0[h] = 0;
        deg[h] = 0;
        if (u[h] >= 0) {
          e0[h] = __ldg(&b.rp[u[h]]);
          deg[h] = __ldg(&b.rp[u[h] + 1]) - e0[h];
        }
      }
      const int maxdeg = __reduce_max_sync(0xffffffffu, max(deg[0], deg[1]));
      for (int k0 = 0; k0 < maxdeg; k0 += 8) {
        int w[2][8];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int j = 0; j < 8; ++j) w[h][j] = (k0 + j < deg[h]) ? __ldg(&b.col[e0[h] + k0 + j]) : -1;
        bool push[2][8];
        int mA = 0, mB = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t* vis = b.vis[isB[h] ? 1 : 0];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            push[h][j] = w[h][j] >= 0 && bvis_claim(vis, w[h][j]);
            if (push[h][j]) {
              if (isB[h]) ++mB;
              else ++mA;
            }
          }
        }
        int incA = mA, incB = mB;
#pragma unroll
        for (int o2 = 1; o2 < 32; o2 <<= 1) {
          const int ta = __shfl_up_sync(0xffffffffu, incA, o2);
          const int tb = __shfl_up_sync(0xffffffffu, incB, o2);
          if (lane >= o2) {
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
        int posA = __shfl_sync(0xffffffffu, bA, 0) + incA - mA;
        int posB = __shfl_sync(0xffffffffu, bB, 0) + incB - mB;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            if (push[h][j]) {
              if (isB[h]) bq_put(b, qb ^ 1, posB++, w[h][j]);
              else bq_put(b, qa ^ 1, posA++, w[h][j]);
            }
          }
        }
      }
    }
    __syncthreads();
  }
  return o;  // the loop ends only after A has ended, so o.t is set
}

// 2BFS of a connected graph in one block.  Returns false (in every thread)
// if vertex 0 does not reach all n vertices; then nothing is written.
static __device__ bool block_pseudo_diameter(const BlockBfs& b, int* pdiam, int* t_out) {
  if (b.n <= 0) return false;
  const int guess = b.n - 1;
  const BlockBfsOut o = block_bfs2(b, 0, guess);
  if (o.reached != b.n) return false;
  *t_out = o.t;
  if (o.t == guess && !o.dropped) {
    *pdiam = o.lb;
  } else {
    const BlockBfsOut o2 = block_bfs2(b, o.t, -1);
    *pdiam = o2.la;
  }
  return true;
}

}  // namespace mpcg
