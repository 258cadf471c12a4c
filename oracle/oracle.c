/*
 * oracle.c -- plain CPU oracle for restarted mixed-precision CG
 * (Prolubnikov, arXiv 2412.08059).  TEST INFRASTRUCTURE ONLY: see oracle.h.
 *
 * One thread, no blocking, no fusion, no reordering beyond what the paper's
 * steps state.  Every loop runs in index order.  Build with
 * -ffp-contract=off so that a*b+c is two roundings unless fma() is written.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* eps1 = 10^-t for the classes t of Sec. 11.1 (written as decimal literals,
 * so the value is the correctly rounded double of 10^-t). */
static const double kPow10Neg[16] = {1e0,  1e-1,  1e-2,  1e-3,  1e-4,  1e-5,
                                     1e-6, 1e-7,  1e-8,  1e-9,  1e-10, 1e-11,
                                     1e-12, 1e-13, 1e-14, 1e-15};

/* ------------------------------------------------------------------------ */
/* SpMV y = A x.  Reading: each row is summed in stored (column) order by a   */
/* chain of fused multiply-adds that starts from +0.                          */
/* ------------------------------------------------------------------------ */
void orc_spmv64(const orc_csr* A, const double* x, double* y) {
  for (int32_t i = 0; i < A->n; ++i) {
    double acc = 0.0;
    for (int32_t e = A->row_ptr[i]; e < A->row_ptr[i + 1]; ++e)
      acc = fma(A->val[e], x[A->col[e]], acc);
    y[i] = acc;
  }
}

void orc_spmv32(int32_t n, const int32_t* row_ptr, const int32_t* col,
                const float* val32, const float* x, float* y) {
  for (int32_t i = 0; i < n; ++i) {
    float acc = 0.0f;
    for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
      acc = fmaf(val32[e], x[col[e]], acc);
    y[i] = acc;
  }
}

/* Dot product in double: sum_i a_i b_i, sequential. */
double orc_dot64(int32_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int32_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Dot product of two FP32 vectors, accumulated in double (Remark 3 of Sec. 9:
 * the residual norms of the single-precision stage are computed in double).
 * The product of two floats is exact in double, so only the sum rounds. */
double orc_dot32(int32_t n, const float* a, const float* b) {
  double s = 0.0;
  for (int32_t i = 0; i < n; ++i) s += (double)a[i] * (double)b[i];
  return s;
}

/* The other reading of the single-precision stage's inner products: both
 * the products and the running sum rounded to float, in index order.  The
 * float result is returned widened (exactly) to double. */
double orc_dot32_f(int32_t n, const float* a, const float* b) {
  float s = 0.0f;
  for (int32_t i = 0; i < n; ++i) {
    const float p = a[i] * b[i];
    s = s + p;
  }
  return (double)s;
}

/* Stop measure of the CG loop test (Sec. 3): ||r||, or ||r||/||b|| when the
 * relative reading is selected.  r is the recursively updated residual. */
static double stop_measure(double rr, double bnorm, int32_t rel) {
  return rel ? sqrt(rr) / bnorm : sqrt(rr);
}

/* ------------------------------------------------------------------------ */
/* Single-precision CG state (Sec. 3 on float32(A), float32(b)).            */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t n;
  const int32_t *rp, *ci;
  const float* v32;
  float *x, *r, *d, *q;
  double rr; /* r^T r in double */
  /* Jacobi preconditioning (the PCG form of Sec. 5; NULL: plain CG):
   * dinv = 1 / diag(A~) in float, z = dinv r, rz = r^T z in double. */
  const float* dinv;
  float* z;
  double rz;
  int acc32;  /* inner products summed in float (orc_dot32_f) instead of double */
} cg32_t;

/* Inner product of the single-precision stage in the selected reading. */
static double sdot(const cg32_t* s, const float* a, const float* b) {
  return s->acc32 ? orc_dot32_f(s->n, a, b) : orc_dot32(s->n, a, b);
}

enum { IT_OK = 0, IT_BREAKDOWN = 1, IT_NAN = 2 };

static int cg32_alloc(cg32_t* s, const orc_csr* A, const float* v32, const float* dinv,
                      int acc32) {
  s->n = A->n;
  s->acc32 = acc32;
  s->rp = A->row_ptr;
  s->ci = A->col;
  s->v32 = v32;
  s->dinv = dinv;
  s->rz = 0.0;
  size_t bytes = sizeof(float) * (size_t)(A->n > 0 ? A->n : 1);
  s->x = (float*)malloc(bytes);
  s->r = (float*)malloc(bytes);
  s->d = (float*)malloc(bytes);
  s->q = (float*)malloc(bytes);
  s->z = (float*)malloc(bytes);
  if (s->x && s->r && s->d && s->q && s->z) return 1;
  free(s->x); free(s->r); free(s->d); free(s->q); free(s->z);
  return 0;
}
static void cg32_free(cg32_t* s) {
  free(s->x); free(s->r); free(s->d); free(s->q); free(s->z);
}

/* CG line 1: x0 = 0, r0 = b - A x0, d0 = r0 (PCG: z0 = M^-1 r0, d0 = z0). */
static void cg32_start(cg32_t* s, const float* b32) {
  for (int32_t i = 0; i < s->n; ++i) s->x[i] = 0.0f;
  orc_spmv32(s->n, s->rp, s->ci, s->v32, s->x, s->q);
  for (int32_t i = 0; i < s->n; ++i) s->r[i] = b32[i] - s->q[i];
  if (s->dinv) {
    for (int32_t i = 0; i < s->n; ++i) s->z[i] = s->dinv[i] * s->r[i];
    for (int32_t i = 0; i < s->n; ++i) s->d[i] = s->z[i];
    s->rz = sdot(s, s->r, s->z);
  } else {
    for (int32_t i = 0; i < s->n; ++i) s->d[i] = s->r[i];
  }
  s->rr = sdot(s, s->r, s->r);
}

/* One CG iteration (the loop body of Sec. 3) in single precision.
 * alpha and beta are the double ratios rounded once to float. */
static int cg32_iter(cg32_t* s) {
  const int32_t n = s->n;
  orc_spmv32(n, s->rp, s->ci, s->v32, s->d, s->q);         /* q = A d      */
  double dq = sdot(s, s->d, s->q);                           /* d^T A d      */
  if (!isfinite(dq)) return IT_NAN;
  if (!(dq > 0.0)) return IT_BREAKDOWN;
  const double num = s->dinv ? s->rz : s->rr;                /* PCG: r^T z   */
  float alpha = (float)(num / dq);                           /* alpha_i      */
  for (int32_t i = 0; i < n; ++i) s->x[i] = fmaf(alpha, s->d[i], s->x[i]);
  for (int32_t i = 0; i < n; ++i) s->r[i] = fmaf(-alpha, s->q[i], s->r[i]);
  double rr_new = sdot(s, s->r, s->r);
  if (!isfinite(rr_new)) return IT_NAN;
  if (s->dinv) {                                             /* z = M^-1 r   */
    for (int32_t i = 0; i < n; ++i) s->z[i] = s->dinv[i] * s->r[i];
    double rz_new = sdot(s, s->r, s->z);
    if (!isfinite(rz_new)) return IT_NAN;
    float beta = (float)(rz_new / s->rz);
    for (int32_t i = 0; i < n; ++i) s->d[i] = fmaf(beta, s->d[i], s->z[i]);
    s->rz = rz_new;
  } else {
    float beta = (float)(rr_new / s->rr);                    /* beta_{i+1}   */
    for (int32_t i = 0; i < n; ++i) s->d[i] = fmaf(beta, s->d[i], s->r[i]);
  }
  s->rr = rr_new;
  return IT_OK;
}

/* ------------------------------------------------------------------------ */
/* Double-precision CG state (Sec. 3).                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_csr* A;
  double *x, *r, *d, *q; /* x is caller memory */
  double rr;
  const double* dinv;    /* Jacobi: 1 / diag(A); NULL: plain CG */
  double *z, rz;
} cg64_t;

static int cg64_alloc(cg64_t* s, const orc_csr* A, double* x, const double* dinv) {
  s->A = A;
  s->x = x;
  s->dinv = dinv;
  s->rz = 0.0;
  size_t bytes = sizeof(double) * (size_t)(A->n > 0 ? A->n : 1);
  s->r = (double*)malloc(bytes);
  s->d = (double*)malloc(bytes);
  s->q = (double*)malloc(bytes);
  s->z = (double*)malloc(bytes);
  if (s->r && s->d && s->q && s->z) return 1;
  free(s->r); free(s->d); free(s->q); free(s->z);
  s->r = s->d = s->q = s->z = NULL;
  return 0;
}
static void cg64_free(cg64_t* s) { free(s->r); free(s->d); free(s->q); free(s->z); }

/* CG line 1 from the current x: r0 = b - A x0 in double, d0 = r0
 * (PCG: z0 = M^-1 r0, d0 = z0). */
static void cg64_start(cg64_t* s, const double* b) {
  const int32_t n = s->A->n;
  orc_spmv64(s->A, s->x, s->q);
  for (int32_t i = 0; i < n; ++i) s->r[i] = b[i] - s->q[i];
  if (s->dinv) {
    for (int32_t i = 0; i < n; ++i) s->z[i] = s->dinv[i] * s->r[i];
    for (int32_t i = 0; i < n; ++i) s->d[i] = s->z[i];
    s->rz = orc_dot64(n, s->r, s->z);
  } else {
    for (int32_t i = 0; i < n; ++i) s->d[i] = s->r[i];
  }
  s->rr = orc_dot64(n, s->r, s->r);
}

static int cg64_iter(cg64_t* s) {
  const int32_t n = s->A->n;
  orc_spmv64(s->A, s->d, s->q);
  double dq = orc_dot64(n, s->d, s->q);
  if (!isfinite(dq)) return IT_NAN;
  if (!(dq > 0.0)) return IT_BREAKDOWN;
  double alpha = (s->dinv ? s->rz : s->rr) / dq;
  for (int32_t i = 0; i < n; ++i) s->x[i] = fma(alpha, s->d[i], s->x[i]);
  for (int32_t i = 0; i < n; ++i) s->r[i] = fma(-alpha, s->q[i], s->r[i]);
  double rr_new = orc_dot64(n, s->r, s->r);
  if (!isfinite(rr_new)) return IT_NAN;
  if (s->dinv) {
    for (int32_t i = 0; i < n; ++i) s->z[i] = s->dinv[i] * s->r[i];
    double rz_new = orc_dot64(n, s->r, s->z);
    if (!isfinite(rz_new)) return IT_NAN;
    double beta = rz_new / s->rz;
    for (int32_t i = 0; i < n; ++i) s->d[i] = fma(beta, s->d[i], s->z[i]);
    s->rz = rz_new;
  } else {
    double beta = rr_new / s->rr;
    for (int32_t i = 0; i < n; ++i) s->d[i] = fma(beta, s->d[i], s->r[i]);
  }
  s->rr = rr_new;
  return IT_OK;
}

/* Builder's rule for the stop test on the true residual.  The paper does
 * not say how a stage ends whose tolerance its precision cannot reach on the
 * true residual; Sec. 7 (Fig. 2) shows ||b - A x|| ceasing to fall while the
 * recursively updated residual keeps falling.  This implementation takes a
 * stage as stagnated once the recursive r has fallen 1e3 times below
 * ||b - A x|| (the factor 1e3 is its own choice, not the paper's) and ends
 * it as it would end at its iteration cap.  Compared on squares:
 * r^T r <= 1e-6 ||b - A x||^2. */
#define STAGNATION_RR 1e-6

/* Paper-literal stop measure (the loop test of Sec. 3 is on ||A x_i - b||):
 * ||b - A x||^2 of the current iterate in the stage's precision -- the
 * product by the stage's matrix and the difference rounded in that
 * precision, the squares summed in double as for the other norms.  NAN if
 * the scratch vector cannot be had. */
static double true_rr32(const cg32_t* s, const float* b32) {
  float* t = (float*)malloc(sizeof(float) * (size_t)(s->n > 0 ? s->n : 1));
  if (!t) return NAN;
  orc_spmv32(s->n, s->rp, s->ci, s->v32, s->x, t);
  for (int32_t i = 0; i < s->n; ++i) t[i] = b32[i] - t[i];
  const double rr = sdot(s, t, t);
  free(t);
  return rr;
}
static double true_rr64(const cg64_t* s, const double* b) {
  const int32_t n = s->A->n;
  double* t = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!t) return NAN;
  orc_spmv64(s->A, s->x, t);
  for (int32_t i = 0; i < n; ++i) t[i] = b[i] - t[i];
  const double rr = orc_dot64(n, t, t);
  free(t);
  return rr;
}

/* Jacobi preconditioner M = diag(A) (Sec. 5): dinv64[i] = 1 / a_ii and
 * dinv32[i] = 1 / float32(a_ii), each a correctly rounded division in its
 * precision.  0 if a row has no stored diagonal or a_ii is zero or not
 * finite (M is then not invertible). */
static int jacobi_dinv(const orc_csr* A, double* dinv64, float* dinv32) {
  for (int32_t i = 0; i < A->n; ++i) {
    double a = 0.0;
    int found = 0;
    for (int32_t e = A->row_ptr[i]; e < A->row_ptr[i + 1]; ++e)
      if (A->col[e] == i) { a = A->val[e]; found = 1; }
    if (!found || !(a != 0.0) || !isfinite(a)) return 0;
    if (dinv64) dinv64[i] = 1.0 / a;
    if (dinv32) dinv32[i] = 1.0f / (float)a;
  }
  return 1;
}

static int32_t it_status(int st) {
  return st == IT_NAN ? ORC_ERR_NAN : (st == IT_BREAKDOWN ? ORC_ERR_BREAKDOWN : ORC_OK);
}

static int csr_ok(const orc_csr* A) {
  if (!A || A->n <= 0 || A->nnz < 0 || !A->row_ptr || !A->col || !A->val) return 0;
  if (A->row_ptr[0] != 0 || A->row_ptr[A->n] != A->nnz) return 0;
  for (int32_t i = 0; i < A->n; ++i)
    if (A->row_ptr[i + 1] < A->row_ptr[i]) return 0;
  for (int32_t e = 0; e < A->nnz; ++e)
    if (A->col[e] < 0 || A->col[e] >= A->n) return 0;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Plain CG drivers (Sec. 3).                                                */
/* ------------------------------------------------------------------------ */
int32_t orc_cg64(const orc_csr* A, const double* b, double* x, double eps,
                 int32_t tol_relative, int32_t max_it, int32_t precond, int32_t true_res,
                 int32_t* iters, double* res_hist) {
  *iters = 0;
  if (!csr_ok(A)) return ORC_ERR_INVALID_ARG;
  double bnorm = sqrt(orc_dot64(A->n, b, b));
  if (!isfinite(bnorm)) return ORC_ERR_NAN;
  double* dinv = NULL;
  if (precond) {
    dinv = (double*)malloc(sizeof(double) * (size_t)A->n);
    if (!dinv || !jacobi_dinv(A, dinv, NULL)) { free(dinv); return ORC_ERR_INVALID_ARG; }
  }
  cg64_t s;
  if (!cg64_alloc(&s, A, x, dinv)) { cg64_free(&s); free(dinv); return ORC_ERR_INVALID_ARG; }
  cg64_start(&s, b);
  int32_t st = ORC_OK, it = 0;
  for (;;) {
    const double trr = true_res ? true_rr64(&s, b) : s.rr;
    double m = stop_measure(trr, bnorm, tol_relative);
    if (res_hist) res_hist[it] = m;
    if (isnan(m)) { st = ORC_ERR_NAN; break; }
    if (m <= eps) break;
    if (it >= max_it || (true_res && s.rr <= STAGNATION_RR * trr)) {
      st = ORC_ERR_NOT_CONVERGED;
      break;
    }
    int r = cg64_iter(&s);
    if (r != IT_OK) { st = it_status(r); break; }
    ++it;
  }
  *iters = it;
  cg64_free(&s);
  free(dinv);
  return st;
}

int32_t orc_cg32(const orc_csr* A, const double* b, float* x, double eps,
                 int32_t tol_relative, int32_t max_it, int32_t precond, int32_t true_res,
                 int32_t acc32, int32_t* iters, double* res_hist) {
  *iters = 0;
  if (!csr_ok(A)) return ORC_ERR_INVALID_ARG;
  const int32_t n = A->n;
  float* v32 = (float*)malloc(sizeof(float) * (size_t)(A->nnz > 0 ? A->nnz : 1));
  float* b32 = (float*)malloc(sizeof(float) * (size_t)n);
  float* dinv = precond ? (float*)malloc(sizeof(float) * (size_t)n) : NULL;
  cg32_t s;
  int32_t st = ORC_OK, it = 0;
  if (v32 && b32) {
    for (int32_t e = 0; e < A->nnz; ++e) v32[e] = (float)A->val[e];
    for (int32_t i = 0; i < n; ++i) b32[i] = (float)b[i];
  }
  int ok = v32 && b32 && (!precond || (dinv && jacobi_dinv(A, NULL, dinv))) &&
           cg32_alloc(&s, A, v32, dinv, acc32);
  if (ok) {
    double bnorm = sqrt(sdot(&s, b32, b32));
    cg32_start(&s, b32);
    for (;;) {
      const double trr = true_res ? true_rr32(&s, b32) : s.rr;
      double m = stop_measure(trr, bnorm, tol_relative);
      if (res_hist) res_hist[it] = m;
      if (isnan(m)) { st = ORC_ERR_NAN; break; }
      if (m <= eps) break;
      if (it >= max_it || (true_res && s.rr <= STAGNATION_RR * trr)) {
        st = ORC_ERR_NOT_CONVERGED;
        break;
      }
      int r = cg32_iter(&s);
      if (r != IT_OK) { st = it_status(r); break; }
      ++it;
    }
    for (int32_t i = 0; i < n; ++i) x[i] = s.x[i];
    cg32_free(&s);
  } else {
    st = ORC_ERR_INVALID_ARG;
  }
  free(v32);
  free(b32);
  free(dinv);
  *iters = it;
  return st;
}

/* ------------------------------------------------------------------------ */
/* Sparsity graph (Sec. 4): vertex i ~ row i; edge (i,j) for every stored    */
/* off-diagonal entry.  The self-loop of the diagonal is ignored.            */
/* ------------------------------------------------------------------------ */

/* Breadth-first search from src; dist[v] = hops, -1 when unreached. */
int32_t orc_bfs(const orc_csr* A, int32_t src, int32_t* dist) {
  const int32_t n = A->n;
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!queue) return -1;
  for (int32_t i = 0; i < n; ++i) dist[i] = -1;
  int32_t head = 0, tail = 0;
  dist[src] = 0;
  queue[tail++] = src;
  while (head < tail) {
    int32_t u = queue[head++];
    for (int32_t e = A->row_ptr[u]; e < A->row_ptr[u + 1]; ++e) {
      int32_t w = A->col[e];
      if (w == u || dist[w] >= 0) continue;
      dist[w] = dist[u] + 1;
      queue[tail++] = w;
    }
  }
  free(queue);
  return tail;
}

/* Connected components; label[v] = smallest vertex of v's component. */
int32_t orc_components(const orc_csr* A, int32_t* label) {
  const int32_t n = A->n;
  int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!dist) return -1;
  for (int32_t i = 0; i < n; ++i) label[i] = -1;
  int32_t count = 0;
  for (int32_t s = 0; s < n; ++s) {
    if (label[s] >= 0) continue;
    orc_bfs(A, s, dist);
    for (int32_t v = 0; v < n; ++v)
      if (dist[v] >= 0) label[v] = s;
    ++count;
  }
  free(dist);
  return count;
}

/* 2BFS pseudo-diameter (Sec. 6).  Readings: the start vertex s of a
 * component is its smallest vertex; the farthest vertex t is the smallest
 * index among the vertices at maximal distance.  A disconnected graph gets
 * the maximum of the per-component values (paragraph on disconnected
 * graphs); an isolated vertex contributes 0.  t_out (nullable) receives t of
 * the component of vertex 0. */
int32_t orc_pseudo_diameter(const orc_csr* A, int32_t* t_out) {
  const int32_t n = A->n;
  int32_t* done = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  int32_t* d1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* d2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!done || !d1 || !d2) { free(done); free(d1); free(d2); return -1; }
  int32_t ell = 0;
  for (int32_t s = 0; s < n; ++s) {
    if (done[s]) continue;
    orc_bfs(A, s, d1);                       /* BFS from s */
    int32_t far = -1, t = s;
    for (int32_t v = 0; v < n; ++v) {        /* ascending v: first max = smallest index */
      if (d1[v] > far) { far = d1[v]; t = v; }
    }
    orc_bfs(A, t, d2);                       /* BFS from t */
    int32_t ecc = 0;
    for (int32_t v = 0; v < n; ++v)
      if (d2[v] > ecc) ecc = d2[v];
    if (ecc > ell) ell = ecc;
    if (s == 0 && t_out) *t_out = t;
    for (int32_t v = 0; v < n; ++v)
      if (d1[v] >= 0) done[v] = 1;
  }
  free(done); free(d1); free(d2);
  return ell;
}

/* Repeated 2BFS (the remark of Sec. 6: running 2BFS from several start
 * vertices and keeping the largest pseudo-diameter).  Reading: run 0 is
 * orc_pseudo_diameter above; run r = 1 .. R-1 starts from s_r = floor(r n /
 * R) and is one 2BFS inside the component of s_r (BFS from s_r, t_r = the
 * smallest vertex at maximal distance, BFS from t_r, its largest distance).
 * l~ is the largest value of the R runs.  R <= 1 is the single run. */
int32_t orc_pseudo_diameter_rep(const orc_csr* A, int32_t R, int32_t* t_out) {
  int32_t ell = orc_pseudo_diameter(A, t_out);
  if (ell < 0 || R <= 1) return ell;
  const int32_t n = A->n;
  int32_t* d1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* d2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!d1 || !d2) { free(d1); free(d2); return -1; }
  for (int32_t r = 1; r < R; ++r) {
    const int32_t s = (int32_t)(((int64_t)r * n) / R);
    orc_bfs(A, s, d1);
    int32_t far = -1, t = s;
    for (int32_t v = 0; v < n; ++v)
      if (d1[v] > far) { far = d1[v]; t = v; }
    orc_bfs(A, t, d2);
    for (int32_t v = 0; v < n; ++v)
      if (d2[v] > ell) ell = d2[v];
  }
  free(d1); free(d2);
  return ell;
}

/* ------------------------------------------------------------------------ */
/* kNN classification (Sec. 11).                                             */
/* ------------------------------------------------------------------------ */

/* Min-max scaling of one feature component with the sample's min and max
 * (Sec. 11.1).  The query is not clamped; a constant component maps to 0. */
static double scale_comp(double v, double lo, double hi) {
  return hi > lo ? (v - lo) / (hi - lo) : 0.0;
}

typedef struct { double d2; int32_t i; } knn_pair;

static int knn_cmp(const void* a, const void* b) {
  const knn_pair* x = (const knn_pair*)a;
  const knn_pair* y = (const knn_pair*)b;
  if (x->d2 < y->d2) return -1;
  if (x->d2 > y->d2) return 1;
  return (x->i > y->i) - (x->i < y->i);
}

/* Reading: the k nearest are the first k after sorting by (squared
 * distance, sample index); this is what the procedure of Sec. 11.2 keeps,
 * since it replaces a kept neighbour only on a strictly smaller distance.
 * Vote: Eq. (23) weights 1/rho with rho the Euclidean distance, summed in
 * selection order; Eq. (22) counts.  If a selected neighbour is at distance
 * 0, only the zero-distance neighbours vote, by count.  Ties of the vote go
 * to the smallest t (the larger eps1). */
int32_t orc_knn(const double chi[4], const orc_sample* S, int32_t k,
                int32_t weighted, uint32_t feat_mask, int32_t* nbr,
                double* score) {
  if (!S || S->count <= 0 || k <= 0 || !S->feat || !S->cls) return -1;
  for (int c = 0; c < 4; ++c)
    if (((feat_mask >> c) & 1u) && !isfinite(chi[c])) return -1;
  if (k > S->count) k = S->count;
  double q[4];
  for (int c = 0; c < 4; ++c) q[c] = scale_comp(chi[c], S->fmin[c], S->fmax[c]);
  knn_pair* p = (knn_pair*)malloc(sizeof(knn_pair) * (size_t)S->count);
  if (!p) return -1;
  for (int32_t i = 0; i < S->count; ++i) {
    double d2 = 0.0;
    for (int c = 0; c < 4; ++c) {
      if (!((feat_mask >> c) & 1u)) continue;
      double diff = q[c] - scale_comp(S->feat[4 * (size_t)i + c], S->fmin[c], S->fmax[c]);
      d2 = d2 + diff * diff;
    }
    p[i].d2 = d2;
    p[i].i = i;
  }
  qsort(p, (size_t)S->count, sizeof(knn_pair), knn_cmp);
  double sc[16];
  int present[16];
  for (int t = 0; t < 16; ++t) { sc[t] = 0.0; present[t] = 0; }
  int zero = (p[0].d2 == 0.0);
  int32_t result = -1;
  for (int32_t j = 0; j < k; ++j) {
    int32_t t = S->cls[p[j].i];
    if (t < 0 || t > 15) { free(p); return -1; }
    if (nbr) nbr[j] = p[j].i;
    if (zero) {
      if (p[j].d2 == 0.0) { sc[t] += 1.0; present[t] = 1; }
    } else {
      sc[t] += weighted ? 1.0 / sqrt(p[j].d2) : 1.0;
      present[t] = 1;
    }
  }
  double best = -1.0;
  for (int t = 0; t < 16; ++t) {
    if (present[t] && sc[t] > best) { best = sc[t]; result = t; }
  }
  if (score)
    for (int t = 0; t < 16; ++t) score[t] = sc[t];
  free(p);
  return result;
}

/* ------------------------------------------------------------------------ */
/* Algorithm I / Algorithm II.                                               */
/* ------------------------------------------------------------------------ */
orc_opts orc_opts_default(void) {
  orc_opts o;
  o.eps1 = -1.0;
  o.eps2 = 1e-10;
  o.k0 = 10;
  o.knn_k = 5;
  o.weighted = 1;
  o.tol_relative = 1;
  o.max_it_fp32 = 0;
  o.max_it_fp64 = 0;
  o.max_true_restarts = 2;
  o.feat_mask = 0xFu;
  o.bfs_starts = 1;
  o.precond = 0;
  o.stop_true_residual = 0;
  o.acc32 = 0;
  return o;
}

static int32_t cap_or(int32_t given, int64_t dflt) {
  if (given > 0) return given;
  return dflt > 0x7fffffff ? 0x7fffffff : (int32_t)dflt;
}

double orc_true_rel_resid(const orc_csr* A, const double* b, const double* x) {
  const int32_t n = A->n;
  double* q = (double*)malloc(sizeof(double) * (size_t)n);
  if (!q) return NAN;
  orc_spmv64(A, x, q);
  for (int32_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
  double rn = sqrt(orc_dot64(n, q, q));
  double bn = sqrt(orc_dot64(n, b, b));
  free(q);
  return bn > 0.0 ? rn / bn : rn;
}

/* Shared front of Algorithm II: float32(A), float32(b), x~0 = 0 and k0
 * single-precision iterations that define v (Eq. 13).  Reading: the loop
 * ends early when the residual reaches eps2 or 0, and v averages the ratios
 * completed; the ratio uses norms computed in double (Remark 3). */
static int32_t k0_phase(cg32_t* s, const float* b32, double bnorm32, const orc_opts* o,
                        int32_t max1, int32_t* n1, int32_t* k0_done, double* v,
                        int* broke) {
  double sum = 0.0;
  int32_t done = 0;
  *broke = 0;
  while (done < o->k0 && *n1 < max1) {
    const double trr = o->stop_true_residual ? true_rr32(s, b32) : s->rr;
    double m = stop_measure(trr, bnorm32, o->tol_relative);
    if (isnan(m)) return ORC_ERR_NAN;
    if (m <= o->eps2 || s->rr == 0.0) break;
    if (o->stop_true_residual && s->rr <= STAGNATION_RR * trr) break;
    double rr_prev = s->rr;
    int r = cg32_iter(s);
    if (r == IT_NAN) return ORC_ERR_NAN;
    if (r == IT_BREAKDOWN) { *broke = 1; break; }
    ++*n1;
    sum += sqrt(s->rr) / sqrt(rr_prev);
    ++done;
  }
  *k0_done = done;
  *v = done > 0 ? sum / (double)done : 0.0;
  return ORC_OK;
}

int32_t orc_features(const orc_csr* A, const double* b, const orc_opts* o,
                     double feat[4], int32_t* k0_done) {
  if (!csr_ok(A) || !b || !o) return ORC_ERR_INVALID_ARG;
  const int32_t n = A->n;
  float* v32 = (float*)malloc(sizeof(float) * (size_t)(A->nnz > 0 ? A->nnz : 1));
  float* b32 = (float*)malloc(sizeof(float) * (size_t)n);
  cg32_t s;
  float* dinv = o->precond ? (float*)malloc(sizeof(float) * (size_t)n) : NULL;
  if (!v32 || !b32 || (o->precond && (!dinv || !jacobi_dinv(A, NULL, dinv)))) {
    free(v32); free(b32); free(dinv);
    return ORC_ERR_INVALID_ARG;
  }
  for (int32_t e = 0; e < A->nnz; ++e) v32[e] = (float)A->val[e];
  for (int32_t i = 0; i < n; ++i) b32[i] = (float)b[i];
  if (!cg32_alloc(&s, A, v32, dinv, o->acc32)) { free(v32); free(b32); free(dinv); return ORC_ERR_INVALID_ARG; }
  double bnorm32 = sqrt(sdot(&s, b32, b32));
  cg32_start(&s, b32);
  int32_t n1 = 0, broke = 0;
  double v = 0.0;
  int32_t st = ORC_OK;
  if (bnorm32 > 0.0 || !o->tol_relative)
    st = k0_phase(&s, b32, bnorm32, o, cap_or(o->max_it_fp32, n), &n1, k0_done, &v, &broke);
  else
    *k0_done = 0;
  feat[0] = (double)n;
  feat[1] = (double)A->nnz;
  feat[2] = (double)orc_pseudo_diameter_rep(A, o->bfs_starts, NULL);
  feat[3] = v;
  cg32_free(&s);
  free(v32);
  free(b32);
  free(dinv);
  return st;
}

int32_t orc_solve(const orc_csr* A, const double* b, double* x,
                  const orc_sample* S, const orc_opts* o, orc_result* res) {
  memset(res, 0, sizeof(*res));
  res->cls = -1;
  if (!csr_ok(A) || !b || !x || !o) return res->status = ORC_ERR_INVALID_ARG;
  const int32_t n = A->n;
  const int auto_eps1 = !(o->eps1 > 0.0);
  if (auto_eps1 && (!S || S->count <= 0)) return res->status = ORC_ERR_INVALID_ARG;
  const int32_t max1 = cap_or(o->max_it_fp32, n);
  const int32_t max2 = cap_or(o->max_it_fp64, 10 * (int64_t)n);
  const int rel = o->tol_relative;

  double bnorm = sqrt(orc_dot64(n, b, b));
  if (!isfinite(bnorm)) return res->status = ORC_ERR_NAN;
  if (bnorm == 0.0) { /* x = 0 solves A x = 0 exactly */
    for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
    res->eps1 = o->eps1;
    return res->status = ORC_OK;
  }

  /* Algorithm I/II step: A~ = float32(A), b~ = float32(b), x~0 = 0. */
  float* v32 = (float*)malloc(sizeof(float) * (size_t)(A->nnz > 0 ? A->nnz : 1));
  float* b32 = (float*)malloc(sizeof(float) * (size_t)n);
  cg32_t s;
  cg64_t s64;
  /* Jacobi preconditioning in both stages (the PCG form of Sec. 5) */
  float* dinv32 = o->precond ? (float*)malloc(sizeof(float) * (size_t)n) : NULL;
  double* dinv64 = o->precond ? (double*)malloc(sizeof(double) * (size_t)n) : NULL;
  if (!v32 || !b32 || (o->precond && (!dinv32 || !dinv64 || !jacobi_dinv(A, dinv64, dinv32)))) {
    free(v32); free(b32); free(dinv32); free(dinv64);
    return res->status = ORC_ERR_INVALID_ARG;
  }
  for (int32_t e = 0; e < A->nnz; ++e) v32[e] = (float)A->val[e];
  for (int32_t i = 0; i < n; ++i) b32[i] = (float)b[i];
  if (!cg32_alloc(&s, A, v32, dinv32, o->acc32)) {
    free(v32); free(b32); free(dinv32); free(dinv64);
    return res->status = ORC_ERR_INVALID_ARG;
  }
  double bnorm32 = sqrt(sdot(&s, b32, b32));
  int32_t status = ORC_OK;
  int warn_eps1 = 0, warn_restart = 0, broke = 0;
  int32_t n1 = 0, n2 = 0;
  double eps1 = o->eps1;
  if (!isfinite(bnorm32)) { status = ORC_ERR_NAN; goto done32; }
  cg32_start(&s, b32);

  if (auto_eps1) {
    /* Algorithm II: k0 FP32 iterations -> v; 2BFS -> l~; kNN -> eps1. */
    int32_t k0_done = 0;
    double v = 0.0;
    status = k0_phase(&s, b32, bnorm32, o, max1, &n1, &k0_done, &v, &broke);
    if (status != ORC_OK) goto done32;
    res->k0_done = k0_done;
    res->v = v;
    res->pdiam = (double)orc_pseudo_diameter_rep(A, o->bfs_starts, NULL);
    res->feat[0] = (double)n;
    res->feat[1] = (double)A->nnz;
    res->feat[2] = res->pdiam;
    res->feat[3] = v;
    int32_t t = orc_knn(res->feat, S, o->knn_k, o->weighted, o->feat_mask, NULL, NULL);
    if (t < 0) { status = ORC_ERR_INVALID_ARG; goto done32; }
    res->cls = t;
    eps1 = kPow10Neg[t];
  }
  res->eps1 = eps1;

  /* Stage 1: FP32 CG to eps1, continuing from the current iterate. */
  const int tres = o->stop_true_residual;
  while (!broke) {
    const double trr = tres ? true_rr32(&s, b32) : s.rr;
    double m = stop_measure(trr, bnorm32, rel);
    if (isnan(m)) { status = ORC_ERR_NAN; goto done32; }
    if (m <= eps1 || n1 >= max1 || (tres && s.rr <= STAGNATION_RR * trr)) break;
    int r = cg32_iter(&s);
    if (r == IT_NAN) { status = ORC_ERR_NAN; goto done32; }
    if (r == IT_BREAKDOWN) { broke = 1; break; }
    ++n1;
  }
  if (stop_measure(tres ? true_rr32(&s, b32) : s.rr, bnorm32, rel) > eps1) warn_eps1 = 1;

  /* Promote: x0 = float64(x~); restart FP64 CG with r0 = b - A x0. */
  for (int32_t i = 0; i < n; ++i) x[i] = (double)s.x[i];
  if (!cg64_alloc(&s64, A, x, dinv64)) { cg64_free(&s64); status = ORC_ERR_INVALID_ARG; goto done32; }
  for (int32_t restart = 0;; ++restart) {
    cg64_start(&s64, b);
    for (;;) {
      const double trr = tres ? true_rr64(&s64, b) : s64.rr;
      double m = stop_measure(trr, bnorm, rel);
      if (isnan(m)) { status = ORC_ERR_NAN; goto done64; }
      if (m <= o->eps2) break;
      if (n2 >= max2 || (tres && s64.rr <= STAGNATION_RR * trr)) {
        status = ORC_ERR_NOT_CONVERGED;
        goto done64;
      }
      int r = cg64_iter(&s64);
      if (r != IT_OK) { status = it_status(r); goto done64; }
      ++n2;
    }
    /* Reading: if the true residual misses eps2, restart from x, at most
     * max_true_restarts times; if it still misses eps2 after the last one,
     * the stage has not met its tolerance (eps2 bounds the final residual of
     * Algorithm I), which is reported as for the iteration cap.  (With the
     * paper-literal stop test the loop above already ended on it.) */
    double tr = orc_true_rel_resid(A, b, x);
    double tm = rel ? tr : tr * bnorm;
    res->true_rel_resid = tr;
    if (!(tm > o->eps2)) break;
    if (restart >= o->max_true_restarts) { status = ORC_ERR_NOT_CONVERGED; goto done64; }
    warn_restart = 1;
    res->restarts = restart + 1;
  }
  status = warn_restart ? ORC_WARN_TRUE_RESID_RESTARTED
                        : (warn_eps1 ? ORC_WARN_EPS1_NOT_REACHED : ORC_OK);
done64:
  cg64_free(&s64);
done32:
  res->n1 = n1;
  res->n2 = n2;
  if (status < 0 && status != ORC_ERR_NOT_CONVERGED) res->true_rel_resid = NAN;
  else if (status == ORC_ERR_NOT_CONVERGED) res->true_rel_resid = orc_true_rel_resid(A, b, x);
  cg32_free(&s);
  free(v32);
  free(b32);
  free(dinv32);
  free(dinv64);
  return res->status = status;
}
