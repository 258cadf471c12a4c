// batch.cu -- many independent systems in one persistent launch (a batching
// pattern; the paper solves one system at a time).
//
// The grid (one block per SM, cooperative) is split into teams of 1, 2, 4,
// ..., 128 blocks.  A host-side planner puts every system in the queue of a
// team-size class (larger systems, larger teams; largest first) and gives
// each class a number of teams in proportion to its estimated work.  The
// leader of a team takes the next system from its class queue, or, when
// that queue is empty, from a queue of a smaller class; the team then runs
// the whole method on it and writes its result record:
//   set-up (CSR check, b~ = float32(b), sliced layout, ||b||),
//   Algorithm II features (2BFS of Sec. 6, k0 single-precision iterations
//   and v of Eq. 13, kNN of Sec. 11) or the fixed eps1 of Algorithm I,
//   single-precision CG to eps1, promotion, double-precision CG to eps2 with
//   the true-residual check.
// Teams synchronise with a bounded barrier over their own blocks (a block
// barrier for one-block teams).  Scalars are computed from team-wide sums
// that every block of the team forms in the same order, so all blocks take
// the same decisions.  The arithmetic is that of the single-system kernels:
// SpMV rows summed in stored order with fused multiply-adds, float-float
// dot products in single precision, alpha and beta rounded once to float.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <queue>
#include <utility>
#include <vector>

#include "stage.cuh"
#include "team_core.cuh"

namespace mpcg {

// Set-up of a system: CSR check, b~ = float32(b), sliced layout, ||b||; x = 0
// when b = 0.  Returns false if the launch aborted.
static __device__ bool sys_prep(Team& t, const BatchSys& s, const BatchArgs& a, int& red) {
  Ctl* ctl = s.w.ctl;
  const bool lead0 = t.rank == 0 && threadIdx.x == 0;
  sys_init(t, s, a);
  if (!team_sync(t)) return false;
  sys_rows(t, s);
  if (!team_sync(t)) return false;
  if (sys_status(s) == 0) {
    if (t.rank == 0) block_scan_slices(s.w.slice_w, s.w.slice_ptr, s.nslices);
    if (!team_sync(t)) return false;
    sys_fill(t, s, true);
    // ||b||_2 in double
    double p = 0.0;
    for (int i = team_tid(t); i < s.n; i += team_threads(t)) p = __fma_rn(s.b[i], s.b[i], p);
    double bb;
    if (!team_sum_d(t, p, s.w.partials, red, bb)) return false;  // includes the fill barrier
    if (lead0) {
      const double bn = sqrt(bb);
      ctl->t_prep = globaltimer();
      ctl->bnorm64 = bn;
      if (!isfinite(bn)) set_status(ctl, MPCG_ERR_NAN);
      else if (bn == 0.0) ctl->trivial = 1;
    }
    if (!team_sync(t)) return false;
  }
  if (sys_status(s) == 0 && *reinterpret_cast<volatile int*>(&ctl->trivial)) {
    for (int i = team_tid(t); i < s.n; i += team_threads(t)) s.x[i] = 0.0;  // b = 0: x = 0
  }
  return team_sync(t);
}

// First launch of a mixed-precision batch: set-up, then Algorithm II's
// features (2BFS, the k0 iterations and v, the kNN label) or the fixed eps1
// of Algorithm I, and the single-precision stage.  Returns false if the
// launch aborted.
static __device__ bool sys_stage1(Team& t, const BatchSys& s, const BatchArgs& a) {
  Ctl* ctl = s.w.ctl;
  int red = 0;
  if (!sys_prep(t, s, a, red)) return false;
  if (sys_status(s) != 0 || ctl->trivial) return true;
  bool done;
  if (a.auto_eps1) {
    if (!team_pseudo_diameter(t, s, a.smem_bytes)) return false;
    if (!team_sync(t)) return false;
    if (!sys_cg32<true>(t, s, kCgK0, red, kNoBudget, &done)) return false;
    if (!team_sync(t)) return false;
    if (sys_status(s) == 0 && t.rank == 0 && threadIdx.x < 32) {
      const double chi[4] = {(double)s.n, (double)s.nnz, (double)ctl->pdiam, ctl->v};
      const int cls = knn_warp(a.knn, chi);
      if (threadIdx.x == 0) {
        if (cls < 0) {
          set_status(ctl, MPCG_ERR_INVALID_ARG);
        } else {
          ctl->cls = cls;
          ctl->eps1 = pow10_neg(cls);
        }
        ctl->t_features = globaltimer();
      }
    }
    if (!team_sync(t)) return false;
    if (sys_status(s) == 0 && !sys_cg32<true>(t, s, kCgContinue, red, kNoBudget, &done)) return false;
  } else {
    if (!sys_cg32<true>(t, s, kCgToEps1, red, kNoBudget, &done)) return false;
  }
  return team_sync(t);
}

// The whole method for one system in one launch (set-up, features or the
// fixed eps1, both stages, the result record), single-precision SpMV from
// global memory; with a.part == 2 only the double-precision stage after
// sys_stage1 and the result record.  Returns false if the launch aborted.
// Its set-up repeats sys_prep's steps inline on purpose: this kernel's code
// sets the schedule of its FP64 loops (see k_batch), and this form is the
// one measured at 305 ms for the FP64-only 512-system batch.
static __device__ bool sys_solve(Team& t, const BatchSys& s, const BatchArgs& a) {
  Ctl* ctl = s.w.ctl;
  const bool lead0 = t.rank == 0 && threadIdx.x == 0;
  int red = 0;
  if (a.part == 2) {
    bool done;
    if (sys_status(s) == 0 && !*reinterpret_cast<volatile int*>(&ctl->trivial) &&
        !sys_cg64(t, s, 0, red, kNoBudget, false, &done))
      return false;
    if (!team_sync(t)) return false;
    sys_finalize(t, s);
    return true;
  }
  sys_init(t, s, a);
  if (!team_sync(t)) return false;
  sys_rows(t, s);
  if (!team_sync(t)) return false;
  if (sys_status(s) == 0) {
    if (t.rank == 0) block_scan_slices(s.w.slice_w, s.w.slice_ptr, s.nslices);
    if (!team_sync(t)) return false;
    sys_fill(t, s, false);
    // ||b||_2 in double
    double p = 0.0;
    for (int i = team_tid(t); i < s.n; i += team_threads(t)) p = __fma_rn(s.b[i], s.b[i], p);
    double bb;
    if (!team_sum_d(t, p, s.w.partials, red, bb)) return false;  // includes the fill barrier
    if (lead0) {
      const double bn = sqrt(bb);
      ctl->t_prep = globaltimer();
      ctl->bnorm64 = bn;
      if (!isfinite(bn)) set_status(ctl, MPCG_ERR_NAN);
      else if (bn == 0.0) ctl->trivial = 1;
    }
    if (!team_sync(t)) return false;
  }
  const bool trivial = ctl->trivial != 0;
  if (sys_status(s) == 0 && trivial) {  // b = 0: x = 0 solves A x = b exactly
    for (int i = team_tid(t); i < s.n; i += team_threads(t)) s.x[i] = 0.0;
  } else if (sys_status(s) == 0 && a.o.fp64_only) {  // pure FP64 CG from x0 = 0
    bool done;
    if (!sys_cg64(t, s, 1, red, kNoBudget, false, &done)) return false;
  } else if (sys_status(s) == 0) {
    if (a.auto_eps1) {
      // Algorithm II: l~ by 2BFS, v over the first k0 iterations, eps1 by kNN
      if (!team_pseudo_diameter(t, s, a.smem_bytes)) return false;
      if (!team_sync(t)) return false;
      bool done;
      if (!sys_cg32<false>(t, s, kCgK0, red, kNoBudget, &done)) return false;
      if (!team_sync(t)) return false;
      if (sys_status(s) == 0 && t.rank == 0 && threadIdx.x < 32) {
        const double chi[4] = {(double)s.n, (double)s.nnz, (double)ctl->pdiam, ctl->v};
        const int cls = knn_warp(a.knn, chi);
        if (threadIdx.x == 0) {
          if (cls < 0) {
            set_status(ctl, MPCG_ERR_INVALID_ARG);
          } else {
            ctl->cls = cls;
            ctl->eps1 = pow10_neg(cls);
          }
          ctl->t_features = globaltimer();
        }
      }
      if (!team_sync(t)) return false;
      if (sys_status(s) == 0 && !sys_cg32<false>(t, s, kCgContinue, red, kNoBudget, &done)) return false;
    } else {
      bool done;
      if (!sys_cg32<false>(t, s, kCgToEps1, red, kNoBudget, &done)) return false;
    }
    if (!team_sync(t)) return false;
    bool done;
    if (sys_status(s) == 0 && !sys_cg64(t, s, 0, red, kNoBudget, false, &done)) return false;
  }
  if (!team_sync(t)) return false;
  sys_finalize(t, s);
  return true;
}

// The persistent team loop of one launch: kPart 1 runs sys_stage1 on every
// system, kPart 2 sys_solve.  Two kernels, so that the code of one stage
// does not change the register allocation of the other's loops (measured:
// with both stages in one kernel, whatever else the kernel held moved the
// FP64 stage by up to 50 %).
template <int kPart>
__global__ void __launch_bounds__(kBatchThreads, 1) k_batch(BatchArgs a) {
  __shared__ TeamShared S;
  Team t;
  t.h = a.h;
  t.team = a.team_of_block[blockIdx.x];
  t.rank = a.rank_of_block[blockIdx.x];
  t.size = a.team_size[t.team];
  t.bar = &a.h->bar[t.team];
  t.round = 0;
  t.timeout_ns = (long long)(a.o.timeout_ms > 0 ? a.o.timeout_ms : 20000) * 1000000ll;
  t.S = &S;
  const int cls = a.team_class[t.team];
  for (;;) {
    // A team barrier sees the abort flag only when it has to wait, so the
    // leader also checks it before taking the next system.
    if (t.rank == 0 && threadIdx.x == 0)
      a.h->next[t.team] =
          *reinterpret_cast<volatile int*>(&a.h->abort) ? -1 : batch_take(a.h, a.order, cls);
    if (!team_sync(t)) return;
    const int idx = *reinterpret_cast<volatile int*>(&a.h->next[t.team]);
    if (idx < 0) return;
    if constexpr (kPart == 1) {
      if (!sys_stage1(t, a.sys[idx], a)) return;
    } else {
      if (!sys_solve(t, a.sys[idx], a)) return;
    }
    if (!team_sync(t)) return;  // every block has read next[team]
  }
}

// ---------------------------------------------------------------------------------------
// Host: the plan (teams and queues) and the launch.
// ---------------------------------------------------------------------------------------
// Plan of one launch: teams (blocks, sizes, classes) and the class queues.
// Team-size class of a system: the smallest team (1, 2, 4, ..., 128 blocks)
// with at most rows_per_block rows per block.
int size_class(int n, int rows_per_block) {
  int c = 0;
  while (c < kTeamClasses - 1 && (long long)n > (long long)rows_per_block << c) ++c;
  return c;
}

// Work estimate of a system: entries touched per iteration times an
// iteration count that grows like sqrt(n) (CG on discretised operators).
double work_of(int n, int nnz) { return ((double)nnz + 6.0 * n) * sqrt((double)n); }

int team_smem(const void* kernel, int stage1) {
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTeamSmem) !=
      cudaSuccess)
    return -1;
  return stage1 ? kTeamSmem : kScanSmem;
}

Plan make_plan(int nsys, const int* n, const double* work, int grid, int rows_per_block,
               const int32_t* rows_sys) {
  if (rows_per_block <= 0) rows_per_block = kRowsPerBlock;
  Plan P;
  std::vector<int> cls(nsys);
  std::vector<double> w(nsys);
  double cw[kTeamClasses] = {0};
  int cnt[kTeamClasses] = {0};
  for (int i = 0; i < nsys; ++i) {
    const int rpb = rows_sys && rows_sys[i] > 0 ? rows_sys[i] : rows_per_block;
    cls[i] = size_class(n[i], rpb);
    w[i] = work[i];
  }
  // Demote the largest classes while one team of every non-empty class does
  // not fit in the grid.
  for (;;) {
    int need = 0, top = -1;
    for (int i = 0; i < nsys; ++i) top = std::max(top, cls[i]);
    bool present[kTeamClasses] = {false};
    for (int i = 0; i < nsys; ++i) present[cls[i]] = true;
    for (int c = 0; c < kTeamClasses; ++c)
      if (present[c]) need += 1 << c;
    if (need <= grid || top <= 0) break;
    for (int i = 0; i < nsys; ++i)
      if (cls[i] == top) cls[i] = top - 1;
  }
  for (int i = 0; i < nsys; ++i) {
    cw[cls[i]] += w[i];
    cnt[cls[i]] += 1;
  }
  // Teams per class: one each, then one more team at a time to the class
  // with the most work per block, while blocks remain and the class (with
  // the smaller ones it can take from) has systems for it.
  int teams[kTeamClasses] = {0};
  int used = 0;
  for (int c = 0; c < kTeamClasses; ++c)
    if (cnt[c]) {
      teams[c] = 1;
      used += 1 << c;
    }
  for (;;) {
    int best = -1;
    double best_load = -1.0;
    for (int c = 0; c < kTeamClasses; ++c) {
      if (!cnt[c] || used + (1 << c) > grid) continue;
      int avail = 0;
      for (int cc = 0; cc <= c; ++cc) avail += cnt[cc];
      if (teams[c] >= avail) continue;
      const double load = cw[c] / (double)(teams[c] << c);
      if (load > best_load) {
        best_load = load;
        best = c;
      }
    }
    if (best < 0) break;
    teams[best] += 1;
    used += 1 << best;
  }
  // Block layout: largest teams first; blocks left over become one-block
  // teams of class 0.
  P.team_of_block.assign(grid, 0);
  P.rank_of_block.assign(grid, 0);
  int b = 0;
  for (int c = kTeamClasses - 1; c >= 0; --c) {
    for (int k = 0; k < teams[c]; ++k) {
      const int tm = (int)P.team_size.size();
      P.team_size.push_back(1 << c);
      P.team_class.push_back(c);
      for (int r = 0; r < (1 << c); ++r) {
        P.team_of_block[b] = tm;
        P.rank_of_block[b] = r;
        ++b;
      }
    }
  }
  for (; b < grid; ++b) {
    P.team_of_block[b] = (int)P.team_size.size();
    P.rank_of_block[b] = 0;
    P.team_size.push_back(1);
    P.team_class.push_back(0);
  }
  // Queues: class by class, largest work first.
  int base = 0;
  for (int c = 0; c < kTeamClasses; ++c) {
    std::vector<int> q;
    for (int i = 0; i < nsys; ++i)
      if (cls[i] == c) q.push_back(i);
    std::stable_sort(q.begin(), q.end(), [&](int x, int y) { return w[x] > w[y]; });
    P.qbase[c] = base;
    P.qlen[c] = (int)q.size();
    for (int i : q) P.order.push_back(i);
    base += (int)q.size();
  }
  return P;
}

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace bytes ahead of the per-system regions.
size_t batch_header_bytes(int nsys) {
  return a256(sizeof(BatchHdr)) + a256(sizeof(BatchSys) * (size_t)nsys) +
         a256(sizeof(int) * (size_t)nsys) + 4 * a256(sizeof(int) * kMaxGrid);
}

// Every record starts as MPCG_ERR_TIMEOUT: a system that the launch leaves
// unfinished after a team barrier timed out (the launch aborts) reports that
// instead of the record's earlier contents.
__global__ void k_pre_records(mpcg_result_t* res, int nsys) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsys) return;
  mpcg_result_t r;
  memset(&r, 0, sizeof(r));
  r.status = MPCG_ERR_TIMEOUT;
  r.cls = -1;
  res[i] = r;
}

int batch_grid(int requested, int smem) {
  return persistent_grid((const void*)k_batch<1>, kBatchThreads, requested, (size_t)smem);
}

}  // namespace

}  // namespace mpcg

using namespace mpcg;

extern "C" size_t mpcg_batch_workspace_bytes(int32_t nsys, const int32_t* n, const int32_t* nnz,
                                             const mpcg_options_t* opts) {
  if (nsys <= 0 || !n || !nnz) return 0;
  size_t total = batch_header_bytes(nsys);
  for (int32_t i = 0; i < nsys; ++i) {
    const size_t w = mpcg_workspace_bytes(n[i], nnz[i], opts);
    if (!w) return 0;
    total += a256(w);
  }
  return total;
}

extern "C" int32_t mpcg_batch_plan(int32_t nsys, const int32_t* n, const int32_t* nnz,
                                   const mpcg_options_t* opts, int32_t grid_blocks,
                                   int32_t* team_blocks_out) {
  if (nsys <= 0 || !n || !nnz || !opts || !team_blocks_out || grid_blocks < 0)
    return MPCG_ERR_INVALID_ARG;
  std::vector<int> nv(nsys);
  std::vector<double> work(nsys);
  for (int32_t i = 0; i < nsys; ++i) {
    if (n[i] <= 0 || nnz[i] < 0) return MPCG_ERR_INVALID_ARG;
    nv[i] = n[i];
    work[i] = work_of(n[i], nnz[i]);
  }
  int grid = grid_blocks;
  if (grid == 0) {  // the grid mpcg_solve_batch would launch with these options
    const int smem = team_smem((const void*)k_batch<1>, 1);
    grid = smem < 0 ? 0 : batch_grid(opts->grid_blocks, smem);
    if (grid <= 0) return MPCG_ERR_CUDA;
  }
  const Plan P = make_plan(nsys, nv.data(), work.data(), grid, opts->team_rows, opts->team_rows_sys);
  for (int c = 0; c < kTeamClasses; ++c)
    for (int k = 0; k < P.qlen[c]; ++k) team_blocks_out[P.order[P.qbase[c] + k]] = 1 << c;
  return MPCG_OK;
}

extern "C" int32_t mpcg_solve_batch(int32_t nsys, const mpcg_csr_t* A, const double* const* b,
                                    double* const* x, const mpcg_sample_t* sample,
                                    const mpcg_options_t* opts, void* ws, size_t ws_bytes,
                                    mpcg_result_t* res, mpcg_stream_t stream) {
  if (nsys <= 0 || !A || !b || !x || !res || !options_ok(opts)) return MPCG_ERR_INVALID_ARG;
  if (opts->stage1_only) return MPCG_ERR_UNIMPLEMENTED;
  const int auto_eps1 = !opts->fp64_only && !(opts->eps1 > 0.0);
  if (auto_eps1 && !sample_ok(sample)) return MPCG_ERR_INVALID_ARG;
  if (auto_eps1 && opts->bfs_starts > 1) return MPCG_ERR_UNIMPLEMENTED;  // one 2BFS run in teams
  if (opts->precond || opts->stop_true_residual)  // plain CG, recursive stop test in teams
    return MPCG_ERR_UNIMPLEMENTED;
  if (!ws || ((uintptr_t)ws & 255u)) return MPCG_ERR_WORKSPACE;
  std::vector<int> nv(nsys), mv(nsys);
  for (int32_t i = 0; i < nsys; ++i) {
    const mpcg_csr_t& a = A[i];
    if (a.n <= 0 || a.nnz < 0 || !a.row_ptr || (a.nnz > 0 && (!a.col || !a.val)) || !b[i] || !x[i])
      return MPCG_ERR_INVALID_ARG;
    nv[i] = a.n;
    mv[i] = a.nnz;
  }
  if (mpcg_batch_workspace_bytes(nsys, nv.data(), mv.data(), opts) > ws_bytes)
    return MPCG_ERR_WORKSPACE;
  const int smem = team_smem((const void*)k_batch<1>, 1);
  const int smem2 = team_smem((const void*)k_batch<2>, 0);
  if (smem < 0 || smem2 < 0) return MPCG_ERR_CUDA;
  const int grid = batch_grid(opts->grid_blocks, smem);
  if (grid <= 0) return MPCG_ERR_CUDA;
  std::vector<double> work(nsys);
  for (int32_t i = 0; i < nsys; ++i) work[i] = work_of(nv[i], mv[i]);
  const Plan P = make_plan(nsys, nv.data(), work.data(), grid, opts->team_rows, opts->team_rows_sys);

  // Header blob: [BatchHdr | BatchSys[nsys] | order | team_of_block |
  // rank_of_block | team_size | team_class], then the systems' regions.
  const size_t hdr = batch_header_bytes(nsys);
  std::vector<char> blob(hdr, 0);
  char* dev = (char*)ws;
  size_t off = 0;
  BatchHdr* H = (BatchHdr*)(blob.data() + off);
  BatchHdr* Hd = (BatchHdr*)(dev + off);
  off += a256(sizeof(BatchHdr));
  BatchSys* Sy = (BatchSys*)(blob.data() + off);
  BatchSys* Syd = (BatchSys*)(dev + off);
  off += a256(sizeof(BatchSys) * (size_t)nsys);
  auto put = [&](const std::vector<int>& v, size_t cap) -> const int* {
    memcpy(blob.data() + off, v.data(), sizeof(int) * v.size());
    const int* d = (const int*)(dev + off);
    off += a256(sizeof(int) * cap);
    return d;
  };
  const int* order_d = put(P.order, nsys);
  const int* tob_d = put(P.team_of_block, kMaxGrid);
  const int* rob_d = put(P.rank_of_block, kMaxGrid);
  const int* tsz_d = put(P.team_size, kMaxGrid);
  const int* tcl_d = put(P.team_class, kMaxGrid);
  for (int c = 0; c < kTeamClasses; ++c) {
    H->qbase[c] = P.qbase[c];
    H->qlen[c] = P.qlen[c];
  }
  size_t sys_off = hdr;
  for (int32_t i = 0; i < nsys; ++i) {
    Dims d;
    dims_for(nv[i], mv[i], &d);
    BatchSys& y = Sy[i];
    y.A = A[i];
    y.b = b[i];
    y.x = x[i];
    y.res = res + i;
    carve(d, dev + sys_off, &y.w);
    y.n = d.n;
    y.nnz = d.nnz;
    y.nslices = d.nslices;
    y.wcap = d.wcap;
    y.eps2 = opts->eps2;
    sys_off += a256(carve(d, nullptr, nullptr));
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (stage_to_device(dev, blob.data(), hdr, st) != cudaSuccess) return MPCG_ERR_CUDA;
  k_pre_records<<<(nsys + 255) / 256, 256, 0, st>>>(res, nsys);
  if (cudaGetLastError() != cudaSuccess) return MPCG_ERR_CUDA;
  BatchArgs a{};
  a.h = Hd;
  a.sys = Syd;
  a.order = order_d;
  a.team_of_block = tob_d;
  a.rank_of_block = rob_d;
  a.team_size = tsz_d;
  a.team_class = tcl_d;
  a.o = *opts;
  a.auto_eps1 = auto_eps1;
  if (auto_eps1) a.knn = knn_spec(*sample, *opts);
  void* args[] = {&a};
  if (!opts->fp64_only) {  // set-up, features and the single-precision stage
    a.smem_bytes = smem;
    if (cudaLaunchCooperativeKernel((const void*)k_batch<1>, dim3(grid), dim3(kBatchThreads), args,
                                    (size_t)smem, st) != cudaSuccess)
      return MPCG_ERR_CUDA;
    // fresh barriers and queues for the second launch; an abort stays set
    if (cudaMemsetAsync(Hd, 0, offsetof(BatchHdr, qbase), st) != cudaSuccess) return MPCG_ERR_CUDA;
  }
  a.smem_bytes = smem2;
  a.part = opts->fp64_only ? 0 : 2;
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_batch<2>, dim3(grid),
                                                    dim3(kBatchThreads), args, (size_t)smem2, st);
  return e == cudaSuccess ? MPCG_OK : MPCG_ERR_CUDA;
}

namespace {

// Busy times (ns) of one system measured on teams of 2^c blocks: set-up and
// stage 1 (the first launch of a mixed batch), and stage 2; < 0 unmeasured.
struct SysTimes {
  double s1[kTeamClasses], s2[kTeamClasses];
  int n1[kTeamClasses], n2[kTeamClasses];  // measurements averaged into each entry
};

// Busy time on a team of 2^c blocks: the measurement there, else the nearest
// measured size scaled by the block ratio (perfect scaling).
double busy_at(const double* v, int c) {
  if (v[c] >= 0.0) return v[c];
  for (int d = 1; d < kTeamClasses; ++d) {
    if (c - d >= 0 && v[c - d] >= 0.0) return v[c - d] / (double)(1 << d);
    if (c + d < kTeamClasses && v[c + d] >= 0.0) return v[c + d] * (double)(1 << d);
  }
  return 0.0;
}

// Simulated span (ns) of one launch under plan P: every team starts at 0 and
// takes the next system of its own class queue, then of the smaller classes
// (as batch_take does), until all queues are empty.  stage: 1 = the first
// launch of a mixed batch, 2 = the second, 0 = one launch with both.
double simulate_launch(const Plan& P, const std::vector<SysTimes>& T, int stage) {
  using Ev = std::pair<double, int>;
  std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> q;
  for (int tm = 0; tm < (int)P.team_class.size(); ++tm) q.push({0.0, tm});
  int head[kTeamClasses] = {0};
  double span = 0.0;
  while (!q.empty()) {
    const Ev e = q.top();
    q.pop();
    const int c = P.team_class[e.second];
    int sys = -1;
    for (int cc = c; cc >= 0 && sys < 0; --cc)
      if (head[cc] < P.qlen[cc]) sys = P.order[P.qbase[cc] + head[cc]++];
    if (sys < 0) {
      span = std::max(span, e.first);
      continue;
    }
    const SysTimes& t = T[sys];
    const double d = stage == 1 ? busy_at(t.s1, c)
                     : stage == 2 ? busy_at(t.s2, c)
                                  : busy_at(t.s1, c) + busy_at(t.s2, c);
    q.push({e.first + d, e.second});
  }
  return span;
}

// Per-system team granularity: starting from the best uniform candidate,
// each system in turn (largest block-time first; at most kTuneMoves of them,
// which bounds the host time for large batches) moves to another candidate
// when that shortens the simulated batch (the planner re-run on the new
// choice, then each launch simulated); two passes.
constexpr int kTuneMoves = 256;
std::vector<int32_t> per_system_rows(const std::vector<SysTimes>& T, const std::vector<double>& order_key,
                                     const int* nv, const std::vector<double>& work, int grid,
                                     const int* cand, int K, int best, bool two_launch) {
  const int nsys = (int)T.size();
  std::vector<int32_t> rows(nsys, cand[best]);
  auto span = [&]() {
    const Plan P = make_plan(nsys, nv, work.data(), grid, cand[best], rows.data());
    return two_launch ? simulate_launch(P, T, 1) + simulate_launch(P, T, 2) : simulate_launch(P, T, 0);
  };
  std::vector<int> idx(nsys);
  for (int i = 0; i < nsys; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return order_key[a] > order_key[b]; });
  if ((int)idx.size() > kTuneMoves) idx.resize(kTuneMoves);
  double cur = span();
  for (int pass = 0; pass < 2; ++pass)
    for (int i : idx)
      for (int k = 0; k < K; ++k) {
        if (cand[k] == rows[i]) continue;
        const int32_t old = rows[i];
        rows[i] = cand[k];
        const double m = span();
        if (m < cur * (1.0 - 1e-4)) cur = m;
        else rows[i] = old;
      }
  return rows;
}

}  // namespace

extern "C" int32_t mpcg_batch_tune(int32_t nsys, const mpcg_csr_t* A, const double* const* b,
                                   double* const* x, const mpcg_sample_t* sample,
                                   const mpcg_options_t* opts, void* ws, size_t ws_bytes,
                                   mpcg_result_t* res, mpcg_stream_t stream,
                                   int32_t* team_rows_out, int32_t* team_rows_sys_out,
                                   float* ms_out) {
  if (!opts || !team_rows_out || nsys <= 0 || !A || !res) return MPCG_ERR_INVALID_ARG;
  static const int kCand[MPCG_TUNE_CANDIDATES] = {8192, 16384, 32768, 65536};
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return MPCG_ERR_CUDA;
  }
  if (ms_out)
    for (int k = 0; k < MPCG_TUNE_RUNS; ++k) ms_out[k] = -1.0f;
  // One timed batch call; the records copied to `rec`.
  std::vector<mpcg_result_t> rec(nsys);
  auto timed = [&](const mpcg_options_t& o, float* ms) -> int32_t {
    if (cudaEventRecord(e0, st) != cudaSuccess) return MPCG_ERR_CUDA;
    const int32_t s = mpcg_solve_batch(nsys, A, b, x, sample, &o, ws, ws_bytes, res, st);
    if (s != MPCG_OK) return s;
    if (cudaEventRecord(e1, st) != cudaSuccess ||
        cudaMemcpyAsync(rec.data(), res, sizeof(mpcg_result_t) * (size_t)nsys, cudaMemcpyDefault,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
      return MPCG_ERR_CUDA;
    return MPCG_OK;
  };
  std::vector<int> nv(nsys);
  std::vector<double> work(nsys);
  for (int i = 0; i < nsys; ++i) {
    nv[i] = A[i].n;
    work[i] = work_of(A[i].n, A[i].nnz);
  }
  const int smem = team_smem((const void*)k_batch<1>, 1);
  const int grid = smem < 0 ? 0 : batch_grid(opts->grid_blocks, smem);
  int32_t status = grid > 0 ? MPCG_OK : MPCG_ERR_CUDA;
  int best = -1;
  float best_ms = 0.0f;
  std::vector<SysTimes> T(nsys);
  for (SysTimes& t : T)
    for (int c = 0; c < kTeamClasses; ++c) {
      t.s1[c] = t.s2[c] = -1.0;
      t.n1[c] = t.n2[c] = 0;
    }
  std::vector<double> key(nsys, 0.0);  // block-time under the best uniform candidate
  for (int k = 0; k < MPCG_TUNE_CANDIDATES && status == MPCG_OK; ++k) {
    mpcg_options_t o = *opts;
    o.team_rows = kCand[k];
    o.team_rows_sys = nullptr;
    float ms = -1.0f;
    status = timed(o, &ms);
    if (status != MPCG_OK) break;
    if (ms_out) ms_out[k] = ms;
    const bool better = best < 0 || ms < best_ms;
    if (better) {
      best = k;
      best_ms = ms;
    }
    for (int i = 0; i < nsys; ++i) {
      const mpcg_result_t& r = rec[i];
      int c = 0;
      while (c < kTeamClasses - 1 && (1 << c) < r.team_blocks) ++c;
      const long long a = (long long)(r.t_fp32_ns - r.t_start_ns);
      const long long b2 = (long long)(r.t_end_ns - r.t_stage2_ns);
      const double s1 = (double)(a > 0 ? a : 0), s2 = (double)(b2 > 0 ? b2 : 0);
      SysTimes& t = T[i];
      t.s1[c] = (t.n1[c] * std::max(t.s1[c], 0.0) + s1) / (t.n1[c] + 1);
      t.s2[c] = (t.n2[c] * std::max(t.s2[c], 0.0) + s2) / (t.n2[c] + 1);
      ++t.n1[c];
      ++t.n2[c];
      if (better) key[i] = (double)(1 << c) * (s1 + s2);
    }
  }
  if (status == MPCG_OK) {
    *team_rows_out = kCand[best];
    if (team_rows_sys_out) {
      std::vector<int32_t> rows = per_system_rows(T, key, nv.data(), work, grid, kCand,
                                                  MPCG_TUNE_CANDIDATES, best, !opts->fp64_only);
      mpcg_options_t o = *opts;
      o.team_rows = kCand[best];
      o.team_rows_sys = rows.data();
      float ms = -1.0f;
      status = timed(o, &ms);
      if (status == MPCG_OK) {
        if (ms_out) ms_out[MPCG_TUNE_CANDIDATES] = ms;
        // keep the per-system choice only if it measured faster
        for (int i = 0; i < nsys; ++i) team_rows_sys_out[i] = ms < best_ms ? rows[i] : kCand[best];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return status;
}
