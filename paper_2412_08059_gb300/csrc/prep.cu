// prep.cu -- per-call set-up: control block, CSR validation, the sliced
// layout with its float32 copy of the values (Algorithm I/II step
// "A~ = float32(A), b~ = float32(b)"), ||b|| and the result record.
#include <math.h>

#include "internal.h"

namespace mpcg {

bool dims_for(int n, int nnz, Dims* d) {
  if (n <= 0 || nnz < 0) return false;
  d->n = n;
  d->nnz = nnz;
  d->nslices = (n + kSlice - 1) / kSlice;
  // Entries per row kept in the sliced arrays: enough for every row of the
  // stencil and graph families (<= 1.25x the mean + 2), at most 64.
  long long mean_up = ((long long)nnz + n - 1) / n;
  long long wc = (5 * mean_up + 3) / 4 + 2;
  if (wc < 4) wc = 4;
  if (wc > 64) wc = 64;
  d->wcap = (int)wc;
  d->pcap = (long long)d->nslices * kSlice * d->wcap;
  return d->pcap < (1ll << 31);
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t carve(const Dims& d, char* base, Ws* ws) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  };
  const size_t n = (size_t)d.n, S = (size_t)d.nslices, P = (size_t)d.pcap;
  Ws w{};
  w.ctl = (Ctl*)take(sizeof(Ctl));
  w.partials = (double*)take(sizeof(double) * 4 * kMaxGrid);
  w.slice_w = (uint32_t*)take(sizeof(uint32_t) * S);
  w.slice_ptr = (int32_t*)take(sizeof(int32_t) * (S + 1));
  w.scol = (int32_t*)take(sizeof(int32_t) * P);
  w.sv32 = (float*)take(sizeof(float) * P);
  w.sv64 = (double*)take(sizeof(double) * P);
  w.b32 = (float*)take(sizeof(float) * n);
  w.x32 = (float*)take(sizeof(float) * n);
  w.r32 = (float*)take(sizeof(float) * n);
  w.d32a = (float*)take(sizeof(float) * n);
  w.d32b = (float*)take(sizeof(float) * n);
  w.q32 = (float*)take(sizeof(float) * n);
  w.r64 = (double*)take(sizeof(double) * n);
  w.d64 = (double*)take(sizeof(double) * n);
  w.q64 = (double*)take(sizeof(double) * n);
  w.dist = (int32_t*)take(sizeof(int32_t) * n);
  w.dist2 = (int32_t*)take(sizeof(int32_t) * n);
  w.fq0 = (int32_t*)take(sizeof(int32_t) * n);
  w.fq1 = (int32_t*)take(sizeof(int32_t) * n);
  w.fq2 = (int32_t*)take(sizeof(int32_t) * n);
  w.fq3 = (int32_t*)take(sizeof(int32_t) * n);
  w.label = (int32_t*)take(sizeof(int32_t) * n);
  w.ckey = (unsigned long long*)take(sizeof(unsigned long long) * n);
  w.snap = (float*)take(sizeof(float) * 6 * n);
  // team kernels (batched solve, server): a 16-bit copy of the columns for
  // the staged single-precision SpMV
  w.scol16 = (int16_t*)take(sizeof(int16_t) * P);
  w.bytes = off;
  if (ws) *ws = w;
  return off;
}

int persistent_grid(const void* kernel, int threads, int requested, size_t dyn_smem) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, dyn_smem) !=
      cudaSuccess)
    return 0;
  if (per_sm > 1) per_sm = 1;  // fewer barrier arrivals: one block per SM
  int full = sms * per_sm;
  if (full > kMaxGrid) full = kMaxGrid;
  if (requested > 0 && requested < full) return requested;
  return full;
}

// ---------------------------------------------------------------------------------------
__global__ void k_init(Ctl* c, int n, int nnz, int nslices, int wcap, mpcg_options_t o) {
  c->t_start = globaltimer();
  c->n = n;
  c->nnz = nnz;
  c->nslices = nslices;
  c->wcap = wcap;
  c->k0 = o.k0 > 0 ? o.k0 : 0;
  c->max1 = o.max_it_fp32 > 0 ? o.max_it_fp32 : n;
  long long m2 = o.max_it_fp64 > 0 ? (long long)o.max_it_fp64 : 10ll * n;
  c->max2 = m2 > 0x7fffffffll ? 0x7fffffff : (int)m2;
  c->max_restarts = o.max_true_restarts > 0 ? o.max_true_restarts : 0;
  c->tol_relative = o.tol_relative ? 1 : 0;
  c->acc32 = o.acc32 ? 1 : 0;
  c->colwide = o.spmv_variant == 1 ? 1 : 0;  // 32-bit columns asked for
  c->eps1 = o.eps1;
  c->eps2 = o.eps2;
  c->timeout_ns = (long long)(o.timeout_ms > 0 ? o.timeout_ms : 20000) * 1000000ll;
  c->cls = -1;
  c->first = 1;
  c->x32_src = -1;
  c->bfs_starts = o.bfs_starts > 1 ? o.bfs_starts : 1;
  c->rz = 0.0;
  c->cancel = reinterpret_cast<const volatile int*>(o.cancel);
}

// Jacobi preconditioner M = diag(A) (the PCG form of Sec. 5), one thread per
// row: dinv64 = 1 / a_ii and dinv32 = 1 / float32(a_ii), each a correctly
// rounded division in its precision.  A row without a stored diagonal, or
// with a_ii zero or not finite, makes M singular: MPCG_ERR_INVALID_ARG.
__global__ void k_jacobi(Ctl* c, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                         const double* __restrict__ val, int n, double* dinv64, float* dinv32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = 0.0;
  int found = 0;
  for (int e = rp[i]; e < rp[i + 1]; ++e)
    if (col[e] == i) {
      a = val[e];
      found = 1;
    }
  if (!found || !(a != 0.0) || !isfinite(a)) {
    set_status(c, MPCG_ERR_INVALID_ARG);
    a = 1.0;
  }
  dinv64[i] = __ddiv_rn(1.0, a);
  dinv32[i] = __fdiv_rn(1.0f, __double2float_rn(a));
}

size_t precond_bytes(int n, int precond) {
  if (!precond || n <= 0) return 0;
  auto a = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return a(sizeof(double) * (size_t)n) + a(sizeof(float) * (size_t)n) + a(sizeof(float) * (size_t)n);
}

cudaError_t launch_jacobi(const Launch& L) {
  const int n = L.d.n;
  k_jacobi<<<(n + 255) / 256, 256, 0, L.st>>>(L.ws.ctl, L.A->row_ptr, L.A->col, L.A->val, n,
                                              L.dinv64, L.dinv32);
  return cudaGetLastError();
}

// One thread per row (padded to whole slices): checks the CSR rules, writes
// b~ = float32(b), and the width and overflow flag of every slice.  Also
// notes whether some entry kept in the sliced arrays (the first wcap of its
// row) lies more than 32767 columns from the diagonal: the fill then stores
// int32 columns, otherwise int16 offsets (a quarter of the FP32 stage's
// matrix bytes less, a sixth of the FP64 stage's).
__global__ void k_rows(Ctl* c, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                       const double* __restrict__ b, float* __restrict__ b32,
                       uint32_t* __restrict__ slice_w, int n, int nnz, int nslices, int wcap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = i >> 5;
  if (s >= nslices) return;  // whole warps exit together
  int len = 0, ok = 1, wide = 0;
  if (i < n) {
    int a = rp[i], e = rp[i + 1];
    if (a < 0 || e < a || e > nnz) {
      ok = 0;
    } else {
      len = e - a;
      int prev = -1;
      for (int k = a; k < e; ++k) {
        int cc = col[k];
        if (cc < 0 || cc >= n || cc <= prev) { ok = 0; break; }
        if (k - a < wcap && (cc - i > 32767 || i - cc > 32768)) wide = 1;
        prev = cc;
      }
    }
    if (i == 0 && a != 0) ok = 0;
    if (i == n - 1 && e != nnz) ok = 0;
    if (b) b32[i] = (float)b[i];
  }
  if (!ok) {
    set_status(c, MPCG_ERR_INVALID_ARG);
    len = 0;
  }
  int w = len < wcap ? len : wcap;
  int wmax = __reduce_max_sync(0xffffffffu, w);
  int any_ovf = __any_sync(0xffffffffu, len > wcap);
  if ((threadIdx.x & 31) == 0) slice_w[s] = (uint32_t)wmax | (any_ovf ? kOverflowBit : 0u);
  if (__any_sync(0xffffffffu, wide) && (threadIdx.x & 31) == 0) atomicExch(&c->colwide, 1);
}

// Exclusive scan of 32 * width over the slices: one block, tiles of
// kScanTile slices loaded coalesced into shared memory, a running carry.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;
__global__ void k_scan(const uint32_t* __restrict__ slice_w, int32_t* __restrict__ slice_ptr,
                       int nslices) {
  __shared__ int32_t tile[kScanTile];
  __shared__ long long part[kScanThreads];
  __shared__ long long carry_s;
  const int t = threadIdx.x;
  if (t == 0) carry_s = 0;
  __syncthreads();
  for (int base = 0; base < nslices; base += kScanTile) {
    for (int j = t; j < kScanTile; j += kScanThreads) {
      const int s = base + j;
      tile[j] = s < nslices ? (int32_t)(kSlice * (slice_w[s] & ~kOverflowBit)) : 0;
    }
    __syncthreads();
    long long loc = 0;
    for (int j = 0; j < kScanPer; ++j) loc += tile[t * kScanPer + j];
    part[t] = loc;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {  // Hillis-Steele inclusive scan
      const long long v = t >= o ? part[t - o] : 0;
      __syncthreads();
      part[t] += v;
      __syncthreads();
    }
    long long run = carry_s + part[t] - loc;
    for (int j = 0; j < kScanPer; ++j) {
      const int v = tile[t * kScanPer + j];
      tile[t * kScanPer + j] = (int32_t)run;
      run += v;
    }
    __syncthreads();
    for (int j = t; j < kScanTile; j += kScanThreads) {
      const int s = base + j;
      if (s < nslices) slice_ptr[s] = tile[j];
    }
    if (t == kScanThreads - 1) carry_s += part[kScanThreads - 1];
    __syncthreads();
  }
  if (t == 0) slice_ptr[nslices] = (int32_t)carry_s;
}

// Fill the sliced arrays: entry k of row i of slice s sits at
// slice_ptr[s] + 32 k + (i mod 32), in the row's stored order.  Rows shorter
// than the slice width are padded with value 0 and their own column; the
// rows past n that fill the last slice, with value 0 and column n - 1 (0 in
// the int32 form).  Columns are int16 offsets from the row (Ctl::col16) when
// k_rows found that every one fits, int32 otherwise; the same entries are
// summed in the same order either way.
__global__ void k_fill(Ctl* c, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                       const double* __restrict__ val, const uint32_t* __restrict__ slice_w,
                       const int32_t* __restrict__ slice_ptr, int32_t* __restrict__ scol,
                       float* __restrict__ sv32, double* __restrict__ sv64, int n, int nslices) {
  if (volatile_status(c) != 0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = i >> 5, lane = i & 31;
  if (s >= nslices) return;
  const bool c16 = c->colwide == 0;
  if (i == 0) {
    c->col16 = c16 ? 1 : 0;
    c->colbits = c16 ? 16 : 32;
  }
  int16_t* scol16 = reinterpret_cast<int16_t*>(scol);
  const int w = (int)(slice_w[s] & ~kOverflowBit);
  const int base = slice_ptr[s] + lane;
  int a = 0, len = 0;
  if (i < n) {
    a = rp[i];
    len = rp[i + 1] - a;
  }
  for (int k = 0; k < w; ++k) {
    const int e = base + kSlice * k;
    double v = 0.0;
    int cc = i < n ? i : (c16 ? n - 1 : 0);
    if (k < len) {
      v = val[a + k];
      cc = col[a + k];
    }
    if (c16) scol16[e] = (int16_t)(cc - i);
    else scol[e] = cc;
    sv64[e] = v;
    sv32[e] = (float)v;
  }
}

// ||b||_2 in double: per-block partial sums, then a fixed-order final sum.
constexpr int kNormBlocks = 512;
__global__ void k_bnorm_partial(const double* __restrict__ b, int n, double* __restrict__ part) {
  __shared__ double sm[33];
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    s = fma(b[i], b[i], s);
  s = warp_sum(s);
  s = block_sum_warp_values(s, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_bnorm_final(Ctl* c, const double* __restrict__ part, int nb) {
  __shared__ double sm[33];
  double s = block_sum_global(part, nb, sm);
  if (threadIdx.x == 0) {
    double bn = sqrt(s);
    c->t_prep = globaltimer();
    c->bnorm64 = bn;
    if (!isfinite(bn)) set_status(c, MPCG_ERR_NAN);
    else if (bn == 0.0) c->trivial = 1;
  }
}

cudaError_t launch_init(const Launch& L, const mpcg_options_t& o, int fp64_only) {
  cudaError_t e = cudaMemsetAsync(L.ws.ctl, 0, sizeof(Ctl), L.st);
  if (e != cudaSuccess) return e;
  mpcg_options_t oo = o;
  if (fp64_only) oo.eps1 = 0.0;
  k_init<<<1, 1, 0, L.st>>>(L.ws.ctl, L.d.n, L.d.nnz, L.d.nslices, L.d.wcap, oo);
  return cudaGetLastError();
}

cudaError_t launch_prep(const Launch& L, const double* b) {
  const Dims& d = L.d;
  const int threads = 256;
  const int blocks = (int)(((long long)d.nslices * kSlice + threads - 1) / threads);
  k_rows<<<blocks, threads, 0, L.st>>>(L.ws.ctl, L.A->row_ptr, L.A->col, b, L.ws.b32,
                                       L.ws.slice_w, d.n, d.nnz, d.nslices, d.wcap);
  k_scan<<<1, kScanThreads, 0, L.st>>>(L.ws.slice_w, L.ws.slice_ptr, d.nslices);
  k_fill<<<blocks, threads, 0, L.st>>>(L.ws.ctl, L.A->row_ptr, L.A->col, L.A->val, L.ws.slice_w,
                                       L.ws.slice_ptr, L.ws.scol, L.ws.sv32, L.ws.sv64, d.n,
                                       d.nslices);
  if (b) {
    int nb = (d.n + 255) / 256;
    if (nb > kNormBlocks) nb = kNormBlocks;
    k_bnorm_partial<<<nb, 256, 0, L.st>>>(b, d.n, L.ws.partials);
    k_bnorm_final<<<1, 1024, 0, L.st>>>(L.ws.ctl, L.ws.partials, nb);
  }
  return cudaGetLastError();
}

__global__ void k_finalize(const Ctl* c, mpcg_result_t* res, mpcg_features_t* feat) {
  int st = c->status;
  if (st == 0) st = c->warn_restart ? MPCG_WARN_TRUE_RESID_RESTARTED
                                    : (c->warn_eps1 ? MPCG_WARN_EPS1_NOT_REACHED : MPCG_OK);
  const unsigned long long now = globaltimer();
  if (res) {
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
    res->t_end_ns = now;
    res->t_prep_ns = t0;
    res->t_stage2_ns = c->t_s2 ? c->t_s2 : res->t_fp32_ns;
    res->spmv_cols = c->colbits;
    res->team_blocks = 0;
  }
  if (feat) {
    feat->n = (double)c->n;
    feat->m = (double)c->nnz;
    feat->pdiam = (double)c->pdiam;
    feat->v = c->v;
    feat->k0_done = c->k0_done;
    feat->status = st;
  }
}

cudaError_t launch_finalize(const Launch& L, mpcg_result_t* res, mpcg_features_t* feat) {
  k_finalize<<<1, 1, 0, L.st>>>(L.ws.ctl, res, feat);
  return cudaGetLastError();
}

}  // namespace mpcg
