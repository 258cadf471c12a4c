// serve.cu -- continuous batching over a slot table (a serving pattern; the
// paper solves one system at a time).
//
// A server holds up to max_slots admitted systems.  Each system keeps its
// own workspace in a device pool (sliced matrix, Krylov vectors, control
// block) for as long as it is admitted; admission takes a slot and a pool
// block of the system's workspace size (first fit), so requests are
// admitted by device-memory footprint.  mpcg_batch_step runs one persistent
// team launch over the admitted systems: every system advances through a
// phase machine by at most `max_iters` CG iterations per stage,
//   new -> (set-up, features and kNN, or the fixed eps1) -> single-precision
//   stage -> double-precision stage -> done (result record written),
// so the single- and double-precision stages of different requests run
// side by side, and requests admitted between steps join the next one.  The
// host retires finished systems (freeing their slot and pool block) and
// admits new ones between steps.
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "stage.cuh"
#include "team_core.cuh"

namespace mpcg {

enum Phase { kPhNew = 0, kPhStage1 = 1, kPhStage2Start = 2, kPhStage2 = 3, kPhDone = 4 };

struct ServeArgs {
  BatchArgs b;
  int* phase;  // [max_slots]
  int budget;
  int part;    // phases this launch advances (slot_advance)
};

// Set-up of a new system (as in the batched solve).  Returns false if the
// launch aborted.
__device__ bool slot_setup(Team& t, const BatchSys& s, const BatchArgs& a, int& red, bool narrow) {
  Ctl* ctl = s.w.ctl;
  sys_init(t, s, a);
  if (!team_sync(t)) return false;
  sys_rows(t, s);
  if (!team_sync(t)) return false;
  if (sys_status(s) != 0) return true;
  if (t.rank == 0) block_scan_slices(s.w.slice_w, s.w.slice_ptr, s.nslices);
  if (!team_sync(t)) return false;
  sys_fill(t, s, narrow);
  double p = 0.0;
  for (int i = team_tid(t); i < s.n; i += team_threads(t)) p = __fma_rn(s.b[i], s.b[i], p);
  double bb;
  if (!team_sum_d(t, p, s.w.partials, red, bb)) return false;
  if (t.rank == 0 && threadIdx.x == 0) {
    const double bn = sqrt(bb);
    ctl->t_prep = globaltimer();
    ctl->bnorm64 = bn;
    if (!isfinite(bn)) set_status(ctl, MPCG_ERR_NAN);
    else if (bn == 0.0) ctl->trivial = 1;
  }
  return team_sync(t);
}

// Algorithm II features: 2BFS, the k0 iterations and the kNN vote.
template <bool kStage>
__device__ bool slot_features(Team& t, const BatchSys& s, const BatchArgs& a, int& red) {
  Ctl* ctl = s.w.ctl;
  if (!team_pseudo_diameter(t, s, a.smem_bytes)) return false;
  if (!team_sync(t)) return false;
  bool done;
  if (!sys_cg32<kStage>(t, s, kCgK0, red, kNoBudget, &done)) return false;
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
  return team_sync(t);
}

// Advance one system by one step.  part 0: every phase; part 1: set-up,
// features and the single-precision stage only (a system that ends the stage
// stops at kPhStage2Start); part 2: the double-precision stage only (the two
// launches of a step with the serve_split option).
// kStage: the single-precision SpMV staged in shared memory.  Returns false
// if the launch aborted.
template <bool kStage>
__device__ bool slot_advance(Team& t, const BatchSys& s, int* phase_p, const BatchArgs& a,
                             int budget, int part) {
  Ctl* ctl = s.w.ctl;
  int ph = *reinterpret_cast<volatile int*>(phase_p);
  if (ph == kPhDone || ph < 0 || ph > kPhDone) return true;
  if ((part == 1 && ph >= kPhStage2Start) || (part == 2 && ph < kPhStage2Start)) return true;
  int red = 0;
  bool done = true;
  if (ph == kPhNew) {
    if (!slot_setup(t, s, a, red, kStage)) return false;
    if (sys_status(s) != 0) {
      ph = kPhDone;
    } else if (*reinterpret_cast<volatile int*>(&ctl->trivial)) {  // b = 0: x = 0
      for (int i = team_tid(t); i < s.n; i += team_threads(t)) s.x[i] = 0.0;
      ph = kPhDone;
    } else if (a.o.fp64_only) {
      ph = kPhStage2Start;
    } else if (a.auto_eps1) {
      if (!slot_features<kStage>(t, s, a, red)) return false;
      ph = sys_status(s) != 0 ? kPhDone : kPhStage1;
    } else {
      if (!sys_cg32<kStage>(t, s, kCgToEps1, red, budget, &done)) return false;
      if (!team_sync(t)) return false;
      ph = sys_status(s) != 0 ? kPhDone : (done ? kPhStage2Start : kPhStage1);
    }
  } else if (ph == kPhStage1) {
    if (!sys_cg32<kStage>(t, s, kCgContinue, red, budget, &done)) return false;
    if (!team_sync(t)) return false;
    ph = sys_status(s) != 0 ? kPhDone : (done ? kPhStage2Start : kPhStage1);
  }
  if ((ph == kPhStage2Start || ph == kPhStage2) && part != 1) {
    const bool resume = ph == kPhStage2;
    if (!sys_cg64(t, s, a.o.fp64_only ? 1 : 0, red, budget, resume, &done)) return false;
    if (!team_sync(t)) return false;
    ph = (done || sys_status(s) != 0) ? kPhDone : kPhStage2;
  }
  if (!team_sync(t)) return false;
  if (ph == kPhDone) sys_finalize(t, s);
  if (t.rank == 0 && threadIdx.x == 0) *reinterpret_cast<volatile int*>(phase_p) = ph;
  return true;
}

// One step over the admitted systems.  By default one launch of k_serve<2>
// with part 0 advances every phase.  With the serve_split option a
// mixed-precision server runs two launches per step:
//   * k_serve<1>: set-up, features and the single-precision stage, with the
//     SpMV staged in shared memory;
//   * k_serve<2> with part 2: the double-precision stage.
// Measured on the serving mix at 300 requests/s, the split has cheaper FP32
// iterations, but a step then costs both launches in sequence. The median
// latency rose from 19 to 30 ms, so the split is off by default.
template <int kPart>
__global__ void __launch_bounds__(kBatchThreads, 1) k_serve(ServeArgs sa) {
  __shared__ TeamShared S;
  const BatchArgs& a = sa.b;
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
    if (t.rank == 0 && threadIdx.x == 0) a.h->next[t.team] = batch_take(a.h, a.order, cls);
    if (!team_sync(t)) return;
    const int idx = *reinterpret_cast<volatile int*>(&a.h->next[t.team]);
    if (idx < 0) return;
    if (!slot_advance<kPart == 1>(t, a.sys[idx], sa.phase + idx, a, sa.budget, sa.part)) return;
    if (!team_sync(t)) return;
  }
}

// After a step (same stream): if the step aborted (a team barrier timed out),
// every system of the step that is not done ends as timed out, with its
// result record written.  A team that aborted may have left a system's
// vectors part-way through an update that its saved state does not
// describe, and which teams did is not recorded, so every unfinished system
// of the step fails.  A kernel of its own, so that the step kernel's code is
// not changed by it (its schedule moved by 5-8 % with such code inside).
__global__ void k_serve_abort(const BatchHdr* h, const BatchSys* sys, const int* order, int count,
                              int* phase) {
  if (threadIdx.x != 0 || !*reinterpret_cast<const volatile int*>(&h->abort)) return;
  Team t0{};  // rank 0: sys_finalize writes from thread 0 of rank 0
  for (int j = 0; j < count; ++j) {
    const int i = order[j];
    if (phase[i] == kPhDone) continue;
    set_status(sys[i].w.ctl, MPCG_ERR_TIMEOUT);
    sys_finalize(t0, sys[i]);
    phase[i] = kPhDone;
  }
}

// ---------------------------------------------------------------------------------------
// Host: the server (slot table, device pool, per-step plan and launch).
// ---------------------------------------------------------------------------------------
namespace {

size_t s256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device layout: [BatchHdr | BatchSys[max] | order[max] | team_of_block |
// rank_of_block | team_size | team_class (kMaxGrid each)] (mirrored on the
// host and copied at every step), [phase[max]], then the pool.
size_t tables_bytes(int max_slots) {
  return s256(sizeof(BatchHdr)) + s256(sizeof(BatchSys) * (size_t)max_slots) +
         s256(sizeof(int) * (size_t)max_slots) + 4 * s256(sizeof(int) * kMaxGrid);
}
size_t fixed_bytes(int max_slots) {
  return tables_bytes(max_slots) + s256(sizeof(int) * (size_t)max_slots);
}

}  // namespace

}  // namespace mpcg

using namespace mpcg;

// The server: host-side state.  Not thread-safe.
struct mpcg_server {
  char* dev;              // workspace base (device)
  int max_slots;
  size_t pool_off, pool_bytes;
  std::vector<char> mirror;  // host copy of the tables region, staged each step
  BatchSys* sys_h;           // inside mirror
  int* phase_d;
  std::vector<int> active;       // 1 if admitted and not retired
  std::vector<int> fresh;        // admitted since the last step: phase reset pending
  std::vector<size_t> blk_off, blk_size;
  std::map<size_t, size_t> free_blocks;  // pool offset -> size
  mpcg_options_t o;
  KnnSpec knn;
  int auto_eps1;
  int grid;
  int smem, smem2;  // dynamic shared memory of the two launches of a step
};

namespace {

bool pool_alloc(mpcg_server* s, size_t bytes, size_t* off) {
  for (auto it = s->free_blocks.begin(); it != s->free_blocks.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t at = it->first + bytes;
      s->free_blocks.erase(it);
      if (rest) s->free_blocks[at] = rest;
      return true;
    }
  }
  return false;
}

void pool_free(mpcg_server* s, size_t off, size_t bytes) {
  auto it = s->free_blocks.emplace(off, bytes).first;
  auto next = std::next(it);
  if (next != s->free_blocks.end() && it->first + it->second == next->first) {
    it->second += next->second;
    s->free_blocks.erase(next);
  }
  if (it != s->free_blocks.begin()) {
    auto prev = std::prev(it);
    if (prev->first + prev->second == it->first) {
      prev->second += it->second;
      s->free_blocks.erase(it);
    }
  }
}

}  // namespace

extern "C" size_t mpcg_server_workspace_bytes(int32_t max_slots, size_t pool_bytes) {
  if (max_slots <= 0) return 0;
  return fixed_bytes(max_slots) + s256(pool_bytes);
}

extern "C" int32_t mpcg_server_create(void* ws, size_t ws_bytes, int32_t max_slots,
                                      const mpcg_sample_t* sample, const mpcg_options_t* opts,
                                      mpcg_server_t** out) {
  if (!out || max_slots <= 0 || !options_ok(opts) || opts->stage1_only) return MPCG_ERR_INVALID_ARG;
  const int auto_eps1 = !opts->fp64_only && !(opts->eps1 > 0.0);
  if (auto_eps1 && !sample_ok(sample)) return MPCG_ERR_INVALID_ARG;
  if (auto_eps1 && opts->bfs_starts > 1) return MPCG_ERR_UNIMPLEMENTED;  // one 2BFS run in teams
  if (opts->precond || opts->stop_true_residual)  // plain CG, recursive stop test in teams
    return MPCG_ERR_UNIMPLEMENTED;
  if (!ws || ((uintptr_t)ws & 255u) || ws_bytes <= fixed_bytes(max_slots)) return MPCG_ERR_WORKSPACE;
  const int smem = team_smem((const void*)k_serve<1>, 1);
  const int smem2 = team_smem((const void*)k_serve<2>, 1);
  if (smem < 0 || smem2 < 0) return MPCG_ERR_CUDA;
  const int grid = persistent_grid((const void*)k_serve<1>, kBatchThreads, opts->grid_blocks,
                                   (size_t)smem);
  if (grid <= 0) return MPCG_ERR_CUDA;
  mpcg_server* s = new mpcg_server();
  s->dev = (char*)ws;
  s->max_slots = max_slots;
  s->pool_off = fixed_bytes(max_slots);
  s->pool_bytes = (ws_bytes - s->pool_off) & ~(size_t)255;
  s->mirror.assign(tables_bytes(max_slots), 0);
  s->sys_h = (BatchSys*)(s->mirror.data() + s256(sizeof(BatchHdr)));
  s->phase_d = (int*)(s->dev + tables_bytes(max_slots));
  s->active.assign(max_slots, 0);
  s->fresh.assign(max_slots, 0);
  s->blk_off.assign(max_slots, 0);
  s->blk_size.assign(max_slots, 0);
  if (s->pool_bytes) s->free_blocks[0] = s->pool_bytes;
  s->o = *opts;
  s->auto_eps1 = auto_eps1;
  if (auto_eps1) s->knn = knn_spec(*sample, *opts);
  s->grid = grid;
  s->smem = smem;
  s->smem2 = smem2;
  *out = s;
  return MPCG_OK;
}

extern "C" void mpcg_server_destroy(mpcg_server_t* s) { delete s; }

extern "C" int32_t mpcg_server_admit(mpcg_server_t* s, const mpcg_csr_t* A, const double* b,
                                     double* x, double eps2, mpcg_result_t* res, int32_t* slot) {
  if (!s || !A || !b || !x || !res || !slot || !(eps2 >= 0.0)) return MPCG_ERR_INVALID_ARG;
  if (A->n <= 0 || A->nnz < 0 || !A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))
    return MPCG_ERR_INVALID_ARG;
  Dims d;
  if (!dims_for(A->n, A->nnz, &d)) return MPCG_ERR_INVALID_ARG;
  int k = -1;
  for (int i = 0; i < s->max_slots; ++i)
    if (!s->active[i]) {
      k = i;
      break;
    }
  if (k < 0) return MPCG_ERR_WORKSPACE;  // no free slot
  const size_t need = s256(carve(d, nullptr, nullptr));
  size_t off = 0;
  if (!pool_alloc(s, need, &off)) return MPCG_ERR_WORKSPACE;  // no room in the pool
  BatchSys& y = s->sys_h[k];
  memset(&y, 0, sizeof(y));
  y.A = *A;
  y.b = b;
  y.x = x;
  y.res = res;
  carve(d, s->dev + s->pool_off + off, &y.w);
  y.n = d.n;
  y.nnz = d.nnz;
  y.nslices = d.nslices;
  y.wcap = d.wcap;
  y.eps2 = eps2;
  s->active[k] = 1;
  s->fresh[k] = 1;
  s->blk_off[k] = off;
  s->blk_size[k] = need;
  *slot = k;
  return MPCG_OK;
}

extern "C" int32_t mpcg_server_retire(mpcg_server_t* s, int32_t slot) {
  if (!s || slot < 0 || slot >= s->max_slots || !s->active[slot]) return MPCG_ERR_INVALID_ARG;
  s->active[slot] = 0;
  s->fresh[slot] = 0;
  pool_free(s, s->blk_off[slot], s->blk_size[slot]);
  return MPCG_OK;
}

extern "C" int32_t mpcg_batch_step_launches(const mpcg_server_t* s) {
  if (!s) return -1;
  const int stage = (int)((s->mirror.size() + kStageChunk - 1) / kStageChunk);
  const bool split = s->o.serve_split && !s->o.fp64_only;
  return stage + (split ? 2 : 1) + 1;
}

extern "C" int32_t mpcg_batch_step(mpcg_server_t* s, int32_t max_iters, int32_t* slot_phase,
                                   mpcg_stream_t stream) {
  if (!s || max_iters <= 0) return MPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int> ids, nv;
  std::vector<double> work;
  for (int i = 0; i < s->max_slots; ++i) {
    if (!s->active[i]) continue;
    ids.push_back(i);
    nv.push_back(s->sys_h[i].n);
    work.push_back((double)s->sys_h[i].nnz + 6.0 * s->sys_h[i].n);  // cost of one iteration
  }
  for (int i = 0; i < s->max_slots; ++i)
    if (s->fresh[i]) {
      if (cudaMemsetAsync(s->phase_d + i, 0, sizeof(int), st) != cudaSuccess) return MPCG_ERR_CUDA;
      s->fresh[i] = 0;
    }
  if (!ids.empty()) {
    const Plan P = make_plan((int)ids.size(), nv.data(), work.data(), s->grid, s->o.team_rows);
    char* m = s->mirror.data();
    BatchHdr* H = (BatchHdr*)m;
    memset(H, 0, sizeof(BatchHdr));
    for (int c = 0; c < kTeamClasses; ++c) {
      H->qbase[c] = P.qbase[c];
      H->qlen[c] = P.qlen[c];
    }
    size_t off = s256(sizeof(BatchHdr)) + s256(sizeof(BatchSys) * (size_t)s->max_slots);
    auto put = [&](const std::vector<int>& v, size_t cap) -> const int* {
      memset(m + off, 0, sizeof(int) * cap);
      memcpy(m + off, v.data(), sizeof(int) * v.size());
      const int* dptr = (const int*)(s->dev + off);
      off += s256(sizeof(int) * cap);
      return dptr;
    };
    std::vector<int> order(P.order.size());
    for (size_t j = 0; j < P.order.size(); ++j) order[j] = ids[P.order[j]];  // slot numbers
    BatchArgs a{};
    a.h = (BatchHdr*)s->dev;
    a.sys = (const BatchSys*)(s->dev + s256(sizeof(BatchHdr)));
    a.order = put(order, s->max_slots);
    a.team_of_block = put(P.team_of_block, kMaxGrid);
    a.rank_of_block = put(P.rank_of_block, kMaxGrid);
    a.team_size = put(P.team_size, kMaxGrid);
    a.team_class = put(P.team_class, kMaxGrid);
    a.o = s->o;
    a.auto_eps1 = s->auto_eps1;
    a.knn = s->knn;
    if (stage_to_device(s->dev, m, s->mirror.size(), st) != cudaSuccess) return MPCG_ERR_CUDA;
    ServeArgs sa{};
    sa.phase = s->phase_d;
    sa.budget = max_iters;
    void* args[] = {&sa};
    const bool split = s->o.serve_split && !s->o.fp64_only;
    if (split) {  // set-up, features, single-precision stage
      a.smem_bytes = s->smem;
      sa.b = a;
      sa.part = 1;
      if (cudaLaunchCooperativeKernel((const void*)k_serve<1>, dim3(s->grid), dim3(kBatchThreads),
                                      args, (size_t)s->smem, st) != cudaSuccess)
        return MPCG_ERR_CUDA;
      // fresh barriers and queues for the second launch; an abort stays set
      if (cudaMemsetAsync(s->dev, 0, offsetof(BatchHdr, qbase), st) != cudaSuccess)
        return MPCG_ERR_CUDA;
    }
    a.smem_bytes = s->smem2;
    sa.b = a;
    sa.part = split ? 2 : 0;
    if (cudaLaunchCooperativeKernel((const void*)k_serve<2>, dim3(s->grid), dim3(kBatchThreads),
                                    args, (size_t)s->smem2, st) != cudaSuccess)
      return MPCG_ERR_CUDA;
    k_serve_abort<<<1, 32, 0, st>>>(a.h, a.sys, a.order, (int)ids.size(), s->phase_d);
    if (cudaGetLastError() != cudaSuccess) return MPCG_ERR_CUDA;
  }
  if (slot_phase &&
      cudaMemcpyAsync(slot_phase, s->phase_d, sizeof(int) * (size_t)s->max_slots,
                      cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MPCG_ERR_CUDA;
  return MPCG_OK;
}
