/*
 * vest_oracle.h -- plain FP64 CPU oracle for the VeST coordinate-descent path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this library.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Conventions (all host memory, all 0-based):
 *   - Observed entries Omega in COO, structure-of-arrays: idx[n*nnz + a] is the
 *     mode-n index of entry a; x[a] is its value.
 *   - Factor A^(n) is I_n x J_n, row-major.  Mask arrays: 1 = pruned.
 *   - Core G has prod_n J_n entries; linear index with j_1 fastest
 *     (lin = j_1 + J_1*(j_2 + J_2*(j_3 + ...))).
 *   - Every floating-point quantity is double.
 */
#ifndef VEST_ORACLE_H
#define VEST_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_ORDER 10

enum { OR_REG_LF = 0, OR_REG_L1 = 1 };
enum { OR_OK = 0, OR_ERR_INVALID = 1, OR_ERR_NOMEM = 3, OR_ERR_NUMERIC = 7 };

typedef struct {
  int32_t N;
  int64_t I[OR_MAX_ORDER];
  int64_t nnz;
  const int32_t* idx; /* [N][nnz] */
  const double* x;    /* [nnz] */
} or_tensor;

typedef struct {
  int32_t N;
  int64_t I[OR_MAX_ORDER];
  int32_t J[OR_MAX_ORDER];
  double* A[OR_MAX_ORDER];      /* I_n x J_n row-major */
  uint8_t* Amask[OR_MAX_ORDER]; /* I_n x J_n, 1 = pruned; may be NULL */
  double* G;                    /* prod J, j_1 fastest */
  uint8_t* Gmask;               /* may be NULL */
} or_model;

typedef struct {
  int32_t reg;            /* OR_REG_LF or OR_REG_L1 */
  double lambda;          /* > 0 */
  double init_pr;         /* INIT_PR, paper default 0.01 */
  double max_pr;          /* MAX_PR, paper default 0.1 */
  double elbow_thresh;    /* paper: 0.05 */
  double target_sparsity; /* >= 0: manual mode (VeST_man); < 0: auto (VeST_auto) */
  double conv_tol;        /* relative RE change counted as converged */
  int32_t max_iter;       /* <= 256 */
  int32_t fixed_pr_mode;  /* 1: use fixed_pr at every pruning step */
  double fixed_pr;
  int32_t count_mode;     /* 0: k = floor(pr * #unpruned); 1: k = floor(pr * size) */
  int32_t normalize;      /* 1: final column normalisation */
  int32_t revive_on_stop; /* VeST_auto only: when the elbow rule stops pruning, the elements
                             pruned by the last pruning step are unpruned again (Section 3.1) */
  int32_t resume;         /* 1: continue the run recorded in the report passed in (iters done,
                             histories, stop_iter) on the model as it stands */
  int32_t elbow_rise;     /* VeST_auto, 1: the elbow also needs RE_t > RE_{t-1} (Section 3.1
                             describes the stop as the error climbing fast) */
} or_params;

typedef struct {
  int32_t iters;
  int32_t stop_iter;      /* iteration at which pruning stopped (0 = never) */
  double re_hist[256];
  double obj_hist[256];
  double pr_hist[256];    /* pruning rate applied at iteration t (0 = none) */
  double sparsity_hist[256];
  double final_sparsity;
} or_report;

/* Eq. 7 */
double or_entry(const or_model* m, const int32_t* i);
int or_reconstruct(const or_tensor* t, const or_model* m, double* out);
/* Eq. 1, Eq. 2, Eq. 4: out = {sum r^2, sum x^2, reg term, objective, RE} */
int or_loss(const or_tensor* t, const or_model* m, int32_t reg, double lambda, double* out);
/* Omega^(n)_{i_n} lists: stable counting sort of Omega by i_n */
int or_build_index(const or_tensor* t, int32_t mode, int64_t* row_ptr, int32_t* perm);
/* Eq. 11 */
void or_delta(const or_model* m, int32_t mode, const int32_t* i, double* delta);
/* Algorithm 4 for one row of A^(mode) (Eq. 9 / Eq. 13) */
int or_update_row(const or_tensor* t, or_model* m, int32_t mode, int64_t row,
                  const int64_t* row_ptr, const int32_t* perm, int32_t reg, double lambda);
/* Algorithm 4 over all rows of one mode, or all modes in order when mode < 0 */
int or_sweep_factors(const or_tensor* t, or_model* m, int32_t reg, double lambda, int32_t mode);
/* Eq. 12 / Eq. 14, sequential over core entries in linear order */
int or_sweep_core(const or_tensor* t, or_model* m, int32_t reg, double lambda);
/* Definition 1-2, Eq. 3-6, Algorithm 3 (scores only) */
int or_responsibility(const or_tensor* t, const or_model* m, double* const* delta_factor,
                      double* delta_core, double* const* resp_factor, double* resp_core);
/* Pruning with the marking table (Section 3.3, the pruning step of Algorithm 3) */
int or_prune(or_model* m, double* const* delta_factor, const double* delta_core, double pr,
             int32_t count_mode, int32_t threshold_mode, double tau, int64_t* n_pruned);
/* Algorithm 2, final loop: unit-norm columns, core rescaled */
int or_normalize(or_model* m);
/* fraction of exactly-zero elements over |G| + sum_n I_n J_n */
double or_sparsity(const or_model* m);
/* VeST_auto stop statistic (Section 3.3): (RE_t + RE_{t-2} - 2 RE_{t-1}) / pr_t */
double or_elbow_stat(double re_t, double re_t1, double re_t2, double pr_t);
/* Algorithm 2 */
int or_autosearch(const or_tensor* t, or_model* m, const or_params* p, or_report* rep);

#ifdef __cplusplus
}
#endif
#endif
