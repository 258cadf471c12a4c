/*
 * oracle.h -- plain, slow, single-threaded CPU oracle for the restarted
 * mixed-precision conjugate gradient method of Prolubnikov, "Parameter
 * Optimization for Restarted Mixed-Precision Iterative Sparse Solver"
 * (arXiv 2412.08059).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library (libmpcg); neither includes
 * or links the other.  It is written from the paper's text:
 *
 *   CG                 Sec. 3 (the CG procedure), unpreconditioned; optionally
 *                      the loop test on ||A x_i - b|| as printed, with the
 *                      stagnation of Sec. 7 (Fig. 2) ending a stage
 *   PCG                Sec. 5 (CG with the Jacobi preconditioner)
 *   Algorithm I        Sec. 1 (two stages: FP32 to eps1, promote, FP64 to eps2)
 *   Algorithm II       Sec. 9 (k0 FP32 iterations, features, kNN, continue)
 *   decay rate v       Sec. 9, Eq. (13) and Remark 3
 *   2BFS               Sec. 6 (the 2BFS procedure) and its paragraph on
 *                      disconnected graphs
 *   kNN                Sec. 11.2 (selection), Sec. 11.4 Eqs. (22)/(23) (vote),
 *                      squared Euclidean distance of Sec. 11.5
 *   min-max scaling    Sec. 11.1
 *
 * Readings of points the paper leaves open are stated next to the code that
 * takes them.  Floating point: the FP64 path is IEEE double, the FP32 path
 * is IEEE single.  Build with -ffp-contract=off; every fused multiply-add is
 * written out as fma()/fmaf().
 *
 * All arrays are caller-owned host memory.  CSR: row_ptr[n+1], col[nnz]
 * (sorted within each row, diagonal stored), val[nnz].
 */
#ifndef MPCG_ORACLE_H
#define MPCG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t n, nnz;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* val;
} orc_csr;

/* Labelled kNN sample S = {(psi_i, y_i)} of Sec. 11.1/11.2: raw (unscaled)
 * feature rows feat[count][4] = (n, m, pseudo-diameter, v), class labels t
 * (eps1 = 10^-t), and the per-component min/max used for min-max scaling. */
typedef struct {
  const double* feat;
  const int8_t* cls;
  int32_t count;
  double fmin[4], fmax[4];
} orc_sample;

typedef struct {
  double eps1;          /* > 0: Algorithm I with this eps1; <= 0: Algorithm II */
  double eps2;          /* final tolerance */
  int32_t k0;           /* FP32 iterations that define v (Eq. 13) */
  int32_t knn_k;        /* neighbours */
  int32_t weighted;     /* 1: Eq. (23) distance-weighted vote; 0: Eq. (22) */
  int32_t tol_relative; /* 1: ||r||/||b|| <= eps; 0: ||r|| <= eps (paper-literal) */
  int32_t max_it_fp32;  /* cap on N1 (<= 0: n) */
  int32_t max_it_fp64;  /* cap on N2 (<= 0: 10 n) */
  int32_t max_true_restarts; /* extra FP64 restarts when the true residual misses eps2;
                                still missing it after the last: ORC_ERR_NOT_CONVERGED */
  uint32_t feat_mask;   /* bit c set: feature c used in the distance */
  int32_t bfs_starts;   /* 2BFS runs for l~ (Sec. 6 remark; <= 1: the single run) */
  int32_t precond;      /* 1: Jacobi-preconditioned CG in both stages (Sec. 5); 0: plain */
  int32_t stop_true_residual; /* 1: every stop test on ||b - A x|| (the loop test of Sec. 3
                                 as printed), and a stage that has stagnated (recursive r
                                 1e3 times below it) ends as at its cap; 0: on the recursive r
                                 (default) */
  int32_t acc32;        /* 1: every inner product of the single-precision stage is summed
                           in float, sequentially (orc_dot32_f); 0: in double (default,
                           the reading of Sec. 9, Remark 3) */
} orc_opts;

typedef struct {
  int32_t status;       /* 0 ok; >0 warning; <0 error (same codes as the paper-side enum below) */
  int32_t n1, n2, cls, k0_done;
  double eps1, true_rel_resid, pdiam, v;
  double feat[4];
  int32_t restarts;     /* FP64 restarts taken because the true residual missed eps2 */
} orc_result;

enum {
  ORC_OK = 0,
  ORC_WARN_EPS1_NOT_REACHED = 1,
  ORC_WARN_TRUE_RESID_RESTARTED = 2,
  ORC_ERR_INVALID_ARG = -1,
  ORC_ERR_BREAKDOWN = -3,
  ORC_ERR_NAN = -4,
  ORC_ERR_NOT_CONVERGED = -5
};

/* ---- kernels of one CG iteration (Sec. 3) ---- */
void orc_spmv64(const orc_csr* A, const double* x, double* y);
void orc_spmv32(int32_t n, const int32_t* row_ptr, const int32_t* col,
                const float* val32, const float* x, float* y);
double orc_dot64(int32_t n, const double* a, const double* b);
double orc_dot32(int32_t n, const float* a, const float* b);
double orc_dot32_f(int32_t n, const float* a, const float* b);

/* ---- plain CG in one precision from x0 (Sec. 3) ----
 * Runs while the stop measure exceeds eps and it < max_it.  x is in/out.
 * The stop measure uses the recursive r, or with true_res the residual
 * b - A x of the iterate in the stage's precision (the loop test as printed);
 * with true_res a run whose recursive r has fallen 1e3 times below it has
 * stagnated and ends as NOT_CONVERGED.
 * res_hist (nullable, max_it+1 entries) receives the stop measure at the
 * head of every iteration.  Returns status; *iters = iterations performed. */
int32_t orc_cg64(const orc_csr* A, const double* b, double* x, double eps,
                 int32_t tol_relative, int32_t max_it, int32_t precond, int32_t true_res,
                 int32_t* iters, double* res_hist);
int32_t orc_cg32(const orc_csr* A, const double* b, float* x, double eps,
                 int32_t tol_relative, int32_t max_it, int32_t precond, int32_t true_res,
                 int32_t acc32, int32_t* iters, double* res_hist);

/* ---- sparsity-graph features (Sec. 6) ---- */
int32_t orc_bfs(const orc_csr* A, int32_t src, int32_t* dist);  /* returns #reached */
int32_t orc_pseudo_diameter(const orc_csr* A, int32_t* t_out);    /* 2BFS, per component */
int32_t orc_pseudo_diameter_rep(const orc_csr* A, int32_t R, int32_t* t_out); /* R runs, max */
int32_t orc_components(const orc_csr* A, int32_t* label);         /* label = min vertex; returns #components */

/* ---- kNN (Sec. 11) ----
 * Returns the class t; nbr (nullable, k entries) receives the selected sample
 * indices in selection order; score (nullable, 16 entries) the class scores. */
int32_t orc_knn(const double chi[4], const orc_sample* S, int32_t k,
                int32_t weighted, uint32_t feat_mask, int32_t* nbr,
                double* score);

/* ---- the method: Algorithm I (eps1 > 0) or Algorithm II (eps1 <= 0) ---- */
orc_opts orc_opts_default(void);
int32_t orc_solve(const orc_csr* A, const double* b, double* x,
                  const orc_sample* S, const orc_opts* o, orc_result* res);

/* Features only (Algorithm II steps 1-3 plus 2BFS): feat = (n, m, l~, v). */
int32_t orc_features(const orc_csr* A, const double* b, const orc_opts* o,
                     double feat[4], int32_t* k0_done);

/* True relative residual ||b - A x||_2 / ||b||_2 in FP64. */
double orc_true_rel_resid(const orc_csr* A, const double* b, const double* x);

#ifdef __cplusplus
}
#endif
#endif
