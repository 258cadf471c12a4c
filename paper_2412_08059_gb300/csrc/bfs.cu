// bfs.cu -- sparsity-graph features of Sec. 6: breadth-first search, 2BFS
// pseudo-diameter and, for disconnected graphs, connected components.
//
// BFS is level-synchronous in one cooperative launch: the frontier of level
// L is a queue; each thread expands one frontier vertex with a warp-uniform
// trip count (the warp's largest degree), claims unvisited neighbours with
// atomicCAS on dist, and appends them with one atomicAdd per warp
// (ballot + popc).  Distances are exact and independent of scheduling.
//
// 2BFS readings: s = vertex 0 (the smallest vertex of its component); the
// farthest vertex t is the smallest index at maximal distance, found with an
// atomicMax over the key (dist, ~index).  If the first BFS does not reach
// every vertex, components are labelled by their smallest vertex (label
// propagation with pointer jumping) and 2BFS runs in every component at once
// from multi-source frontiers; l~ is the largest second-BFS level.
#include "internal.h"

namespace mpcg {

enum BfsSources { kSrcSingle = 0, kSrcFromCtl = 1, kSrcRoots = 2, kSrcRootFar = 3 };
enum BfsGate { kAlways = 0, kIfConnected = 1, kIfDisconnected = 2 };
enum BfsRole { kRoleFirst = 0, kRoleSecond = 1, kRoleComponentFirst = 2, kRolePlain = 3 };

struct BfsArgs {
  Ctl* ctl;
  const int32_t* rp;
  const int32_t* col;
  int n;
  int32_t* dist;
  int32_t *fq0, *fq1;
  const int32_t* label;
  unsigned long long* ckey;
  int sources, src, gate, role, slot;
};

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Append `v` (when `want`) to queue q with counter *cnt: one atomic per warp.
// Must be called by all 32 lanes.
__device__ __forceinline__ void warp_append(bool want, int v, int32_t* q, int* cnt) {
  const unsigned mask = __ballot_sync(0xffffffffu, want);
  if (mask == 0) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(cnt, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (want) q[base + __popc(mask & ((1u << lane) - 1u))] = v;
}

__global__ void __launch_bounds__(kCgThreads) k_bfs(BfsArgs a) {
  __shared__ unsigned long long smax[32];
  Ctl* ctl = a.ctl;
  if (volatile_status(ctl) != 0) return;
  if (a.gate == kIfConnected && !ctl->connected) return;
  if (a.gate == kIfDisconnected && ctl->connected) return;
  const int n = a.n;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int T = gridDim.x * blockDim.x;
  unsigned long long round = 0;

  for (int v = tid; v < n; v += T) a.dist[v] = -1;
  if (tid == 0) {
    ctl->qsize[0] = 0;
    ctl->qsize[1] = 0;
    ctl->qsize[2] = 0;
  }
  if (!grid_barrier(ctl, a.slot, round)) return;

  // Sources at level 0.
  if (a.sources == kSrcSingle || a.sources == kSrcFromCtl) {
    if (tid == 0) {
      const int s = a.sources == kSrcSingle ? a.src : ctl->far_t;
      a.dist[s] = 0;
      a.fq0[0] = s;
      ctl->qsize[0] = 1;
    }
  } else {
    for (int base = blockIdx.x * blockDim.x; base < n; base += T) {  // warp-uniform bound
      const int v = base + threadIdx.x;
      bool root = v < n && a.label[v] == v;
      int s = v;
      if (root && a.sources == kSrcRootFar) s = far_key_vertex(a.ckey[v]);
      if (root) a.dist[s] = 0;
      warp_append(root, s, a.fq0, &ctl->qsize[0]);
    }
  }
  if (!grid_barrier(ctl, a.slot, round)) return;

  int level = 0;
  long long reached = 0;
  for (;;) {
    const int32_t* in = (level & 1) ? a.fq1 : a.fq0;
    int32_t* out = (level & 1) ? a.fq0 : a.fq1;
    const int size = *reinterpret_cast<volatile int*>(&ctl->qsize[level % 3]);
    if (size == 0) break;
    reached += size;
    if (tid == 0) ctl->qsize[(level + 2) % 3] = 0;
    int* cnt = &ctl->qsize[(level + 1) % 3];
    for (int base = blockIdx.x * blockDim.x; base < size; base += T) {
      const int idx = base + threadIdx.x;
      int u = -1, e0 = 0, deg = 0;
      if (idx < size) {
        u = in[idx];
        e0 = a.rp[u];
        deg = a.rp[u + 1] - e0;
      }
      const int maxdeg = __reduce_max_sync(0xffffffffu, deg);
      // Neighbours in groups of 8: all column loads of a group, then all
      // claims (atomicCAS on dist), then the appends -- three dependent
      // round trips per group instead of per neighbour.
      for (int k0 = 0; k0 < maxdeg; k0 += 8) {
        int w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) w[j] = (k0 + j < deg) ? a.col[e0 + k0 + j] : -1;
        bool push[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
          push[j] = w[j] >= 0 && w[j] != u && atomicCAS(&a.dist[w[j]], -1, level + 1) == -1;
        // One reservation per warp for all of its pushes of this group.
        int mine = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) mine += push[j] ? 1 : 0;
        const int lane = threadIdx.x & 31;
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (total > 0) {
          int base0 = 0;
          if (lane == 0) base0 = atomicAdd(cnt, total);
          int pos = __shfl_sync(0xffffffffu, base0, 0) + incl - mine;
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (push[j]) out[pos++] = w[j];
        }
      }
    }
    ++level;
    if (!grid_barrier(ctl, a.slot, round)) return;
  }
  const int maxlevel = level - 1;  // levels 0 .. level-1 were non-empty

  if (a.role == kRoleFirst) {
    unsigned long long best = 0;
    for (int v = tid; v < n; v += T) {
      const int d = a.dist[v];
      if (d >= 0) {
        const unsigned long long k = far_key(d, v);
        best = k > best ? k : best;
      }
    }
    best = warp_max_u64(best);
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x < 32) {
      unsigned long long b2 = threadIdx.x < (blockDim.x >> 5) ? smax[threadIdx.x] : 0ull;
      b2 = warp_max_u64(b2);
      if (threadIdx.x == 0 && b2) atomicMax(&ctl->key, b2);
    }
    if (tid == 0) ctl->reached = (int)reached;
  } else if (a.role == kRoleComponentFirst) {
    for (int v = tid; v < n; v += T) {
      const int d = a.dist[v];
      if (d >= 0) atomicMax(&a.ckey[a.label[v]], far_key(d, v));
    }
  } else if (a.role == kRoleSecond) {
    if (tid == 0) ctl->pdiam = maxlevel > 0 ? maxlevel : 0;
  }
}

// Decides between the connected and the per-component paths.
__global__ void k_pd_mid(Ctl* c) {
  if (c->status) return;
  c->connected = c->reached == c->n;
  c->far_t = far_key_vertex(c->key);
}

// Connected components: label[v] = smallest vertex of v's component.
// Rounds of (hook: for every edge with differing labels, lower the larger
// label's entry to the smaller label) and (pointer jumping to the root),
// until a hook round changes nothing.  Labels only decrease and always name
// a vertex of the same component, so the root of a component is its
// smallest vertex.
__global__ void __launch_bounds__(kCgThreads) k_cc(BfsArgs a) {
  __shared__ int sflag;
  Ctl* ctl = a.ctl;
  if (volatile_status(ctl) != 0) return;
  if (ctl->connected) return;
  const int n = a.n;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int T = gridDim.x * blockDim.x;
  int32_t* label = const_cast<int32_t*>(a.label);
  unsigned long long round = 0;
  for (int v = tid; v < n; v += T) {
    label[v] = v;
    a.ckey[v] = 0ull;
  }
  if (!grid_barrier(ctl, a.slot, round)) return;
  for (int r = 0;; ++r) {
    if (threadIdx.x == 0) sflag = 0;
    __syncthreads();
    int changed = 0;
    for (int u = tid; u < n; u += T) {
      const int e1 = a.rp[u + 1];
      for (int e = a.rp[u]; e < e1; ++e) {
        const int v = a.col[e];
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
    if (changed) sflag = 1;
    __syncthreads();
    if (threadIdx.x == 0 && sflag) atomicExch(&ctl->ccflag[r & 1], 1);
    if (!grid_barrier(ctl, a.slot, round)) return;
    if (tid == 0) ctl->ccflag[(r + 1) & 1] = 0;
    for (int v = tid; v < n; v += T) {
      int l = label[v];
      for (int ll = label[l]; ll != l; ll = label[l]) l = ll;
      label[v] = l;
    }
    if (!grid_barrier(ctl, a.slot, round)) return;
    if (*reinterpret_cast<volatile int*>(&ctl->ccflag[r & 1]) == 0) break;
  }
}

__global__ void k_pd_end(Ctl* c, const unsigned long long* ckey) {
  if (c->status) return;
  if (!c->connected) c->far_t = far_key_vertex(ckey[0]);
}

__global__ void k_copy_pdiam(const Ctl* c, int32_t* out) {
  const bool ok = c->status == 0;
  out[0] = ok ? c->pdiam : -1;
  out[1] = ok ? c->far_t : -1;
}

static BfsArgs bfs_args(const Launch& L, int32_t* dist, int sources, int src, int gate, int role,
                        int slot) {
  BfsArgs a{};
  a.ctl = L.ws.ctl;
  a.rp = L.A->row_ptr;
  a.col = L.A->col;
  a.n = L.d.n;
  a.dist = dist;
  a.fq0 = L.ws.fq0;
  a.fq1 = L.ws.fq1;
  a.label = L.ws.label;
  a.ckey = L.ws.ckey;
  a.sources = sources;
  a.src = src;
  a.gate = gate;
  a.role = role;
  a.slot = slot;
  return a;
}

const void* bfs_kernel() { return (const void*)k_bfs; }
const void* cc_kernel() { return (const void*)k_cc; }

static cudaError_t coop(const void* k, BfsArgs& a, const Launch& L) {
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(k, dim3(L.grid), dim3(kCgThreads), args, 0, L.st);
}

cudaError_t launch_pseudo_diameter(const Launch& L, int s) {
  cudaError_t e;
  BfsArgs a1 = bfs_args(L, L.ws.dist, kSrcSingle, 0, kAlways, kRoleFirst, s);
  if ((e = coop((const void*)k_bfs, a1, L)) != cudaSuccess) return e;
  k_pd_mid<<<1, 1, 0, L.st>>>(L.ws.ctl);
  BfsArgs a2 = bfs_args(L, L.ws.dist2, kSrcFromCtl, 0, kIfConnected, kRoleSecond, s + 1);
  if ((e = coop((const void*)k_bfs, a2, L)) != cudaSuccess) return e;
  BfsArgs a3 = bfs_args(L, L.ws.dist, kSrcSingle, 0, kIfDisconnected, kRolePlain, s + 2);
  if ((e = coop((const void*)k_cc, a3, L)) != cudaSuccess) return e;
  BfsArgs a4 = bfs_args(L, L.ws.dist, kSrcRoots, 0, kIfDisconnected, kRoleComponentFirst, s + 3);
  if ((e = coop((const void*)k_bfs, a4, L)) != cudaSuccess) return e;
  BfsArgs a5 = bfs_args(L, L.ws.dist2, kSrcRootFar, 0, kIfDisconnected, kRoleSecond, s + 4);
  if ((e = coop((const void*)k_bfs, a5, L)) != cudaSuccess) return e;
  k_pd_end<<<1, 1, 0, L.st>>>(L.ws.ctl, L.ws.ckey);
  return cudaGetLastError();
}

cudaError_t launch_bfs_only(const Launch& L, int src, int32_t* dist, int slot) {
  BfsArgs a = bfs_args(L, dist, kSrcSingle, src, kAlways, kRoleFirst, slot);
  return coop((const void*)k_bfs, a, L);
}

cudaError_t launch_copy_pdiam(const Launch& L, int32_t* out) {
  k_copy_pdiam<<<1, 1, 0, L.st>>>(L.ws.ctl, out);
  return cudaGetLastError();
}

}  // namespace mpcg
