// bfs.cu -- standalone kernels for the sparsity-graph features of Sec. 6
// (the routines are in bfs_core.cuh): the 2BFS pseudo-diameter, with the
// per-component rule, in one cooperative launch, and a plain BFS.
#include "bfs_core.cuh"
#include "internal.h"

namespace mpcg {

__global__ void __launch_bounds__(kCgThreads, 1) k_pdiam(BfsGraph g, int32_t* d1, int32_t* d2,
                                                      int slot) {
  if (volatile_status(g.ctl) != 0) return;
  GridSync sync{g.ctl, slot, 0ull};
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  pseudo_diameter_run(g, d1, d2, tid, gridDim.x * blockDim.x, sync);
}

__global__ void __launch_bounds__(kCgThreads, 1) k_bfs1(BfsGraph g, int32_t* dist, int src,
                                                     int slot) {
  if (volatile_status(g.ctl) != 0) return;
  GridSync sync{g.ctl, slot, 0ull};
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  bfs_run(g, dist, kSrcSingle, src, kRoleFirst, tid, gridDim.x * blockDim.x, sync);
}

__global__ void k_copy_pdiam(const Ctl* c, int32_t* out) {
  const bool ok = c->status == 0;
  out[0] = ok ? c->pdiam : -1;
  out[1] = ok ? c->far_t : -1;
}

BfsGraph bfs_graph(const Launch& L) {
  BfsGraph g{};
  g.ctl = L.ws.ctl;
  g.rp = L.A->row_ptr;
  g.col = L.A->col;
  g.n = L.d.n;
  g.fq0 = L.ws.fq0;
  g.fq1 = L.ws.fq1;
  g.fq2 = L.ws.fq2;
  g.fq3 = L.ws.fq3;
  g.label = L.ws.label;
  g.ckey = L.ws.ckey;
  return g;
}

const void* bfs_kernel() { return (const void*)k_pdiam; }

cudaError_t launch_pseudo_diameter(const Launch& L, int slot) {
  BfsGraph g = bfs_graph(L);
  int32_t* d1 = L.ws.dist;
  int32_t* d2 = L.ws.dist2;
  void* args[] = {&g, &d1, &d2, &slot};
  return cudaLaunchCooperativeKernel((const void*)k_pdiam, dim3(L.grid), dim3(kCgThreads), args, 0,
                                    L.st);
}

cudaError_t launch_bfs_only(const Launch& L, int src, int32_t* dist, int slot) {
  BfsGraph g = bfs_graph(L);
  void* args[] = {&g, &dist, &src, &slot};
  return cudaLaunchCooperativeKernel((const void*)k_bfs1, dim3(L.grid), dim3(kCgThreads), args, 0,
                                    L.st);
}

cudaError_t launch_copy_pdiam(const Launch& L, int32_t* out) {
  k_copy_pdiam<<<1, 1, 0, L.st>>>(L.ws.ctl, out);
  return cudaGetLastError();
}

}  // namespace mpcg
