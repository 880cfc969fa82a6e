/*
 * vest_oracle.c -- plain, slow, obviously correct FP64 CPU oracle for the VeST
 * (Park, Jang, Sael, "VeST: Very Sparse Tucker Factorization of Large-Scale
 * Tensors") coordinate-descent hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call it; the product
 * path never does.  It shares no code with the CUDA library.
 *
 * Every function follows the paper's definitions in the paper's order, with
 * plain loops and no blocking or fusion.  Where the paper is garbled or
 * silent, the reading taken is stated at the function.
 */
#include "vest_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static int64_t core_size(const or_model* m) {
  int64_t s = 1;
  for (int n = 0; n < m->N; ++n) s *= m->J[n];
  return s;
}

/* Linear core index -> (j_1, ..., j_N), j_1 fastest (the mode-n
 * matricisation convention of Section 2.1). */
static void core_unravel(const or_model* m, int64_t lin, int32_t* j) {
  for (int n = 0; n < m->N; ++n) {
    j[n] = (int32_t)(lin % m->J[n]);
    lin /= m->J[n];
  }
}

static void entry_index(const or_tensor* t, int64_t a, int32_t* i) {
  for (int n = 0; n < t->N; ++n) i[n] = t->idx[(int64_t)n * t->nnz + a];
}

static double fac(const or_model* m, int n, int64_t row, int32_t col) {
  return m->A[n][row * m->J[n] + col];
}

static int valid(const or_tensor* t, const or_model* m) {
  if (!m || m->N < 1 || m->N > OR_MAX_ORDER) return 0;
  if (t) {
    if (t->N != m->N || t->nnz < 0) return 0;
    for (int n = 0; n < m->N; ++n)
      if (t->I[n] != m->I[n]) return 0;
  }
  for (int n = 0; n < m->N; ++n)
    if (m->J[n] < 1 || m->I[n] < 1) return 0;
  return 1;
}

/* Eq. 7: B(alpha) = sum over every core element beta of
 * G_beta * prod_n a^(n)_{i_n j_n}. */
double or_entry(const or_model* m, const int32_t* i) {
  int32_t j[OR_MAX_ORDER];
  double b = 0.0;
  const int64_t gs = core_size(m);
  for (int64_t lin = 0; lin < gs; ++lin) {
    core_unravel(m, lin, j);
    double p = m->G[lin];
    for (int n = 0; n < m->N; ++n) p *= fac(m, n, i[n], j[n]);
    b += p;
  }
  return b;
}

int or_reconstruct(const or_tensor* t, const or_model* m, double* out) {
  if (!valid(t, m)) return OR_ERR_INVALID;
  int32_t i[OR_MAX_ORDER];
  for (int64_t a = 0; a < t->nnz; ++a) {
    entry_index(t, a, i);
    out[a] = or_entry(m, i);
  }
  return OR_OK;
}

/* Eq. 1 (L_F) and Eq. 2 (L_1); RE of Eq. 4 with ||X||_F taken over the
 * observed entries only (the only values that exist). */
int or_loss(const or_tensor* t, const or_model* m, int32_t reg, double lambda, double* out) {
  if (!valid(t, m)) return OR_ERR_INVALID;
  int32_t i[OR_MAX_ORDER];
  double sq = 0.0, xx = 0.0;
  for (int64_t a = 0; a < t->nnz; ++a) {
    entry_index(t, a, i);
    const double r = t->x[a] - or_entry(m, i);
    sq += r * r;
    xx += t->x[a] * t->x[a];
  }
  double rg = 0.0;
  const int64_t gs = core_size(m);
  for (int64_t b = 0; b < gs; ++b) rg += (reg == OR_REG_L1) ? fabs(m->G[b]) : m->G[b] * m->G[b];
  for (int n = 0; n < m->N; ++n) {
    const int64_t sz = m->I[n] * m->J[n];
    for (int64_t e = 0; e < sz; ++e)
      rg += (reg == OR_REG_L1) ? fabs(m->A[n][e]) : m->A[n][e] * m->A[n][e];
  }
  rg *= lambda;
  out[0] = sq;
  out[1] = xx;
  out[2] = rg;
  out[3] = sq + rg;
  out[4] = (xx > 0.0) ? sqrt(sq) / sqrt(xx) : 0.0;
  return OR_OK;
}

/* Omega^(n)_{i} of the symbol table: the observed entries whose mode-n index
 * is i.  A stable counting sort: row_ptr[i]..row_ptr[i+1] delimit row i, and
 * within a row the entries keep their COO order. */
int or_build_index(const or_tensor* t, int32_t mode, int64_t* row_ptr, int32_t* perm) {
  if (!t || mode < 0 || mode >= t->N) return OR_ERR_INVALID;
  const int64_t rows = t->I[mode];
  const int32_t* key = t->idx + (int64_t)mode * t->nnz;
  for (int64_t r = 0; r <= rows; ++r) row_ptr[r] = 0;
  for (int64_t a = 0; a < t->nnz; ++a) {
    if (key[a] < 0 || key[a] >= rows) return OR_ERR_INVALID;
    row_ptr[key[a] + 1] += 1;
  }
  for (int64_t r = 0; r < rows; ++r) row_ptr[r + 1] += row_ptr[r];
  int64_t* next = (int64_t*)malloc((size_t)(rows > 0 ? rows : 1) * sizeof(int64_t));
  if (!next) return OR_ERR_NOMEM;
  memcpy(next, row_ptr, (size_t)rows * sizeof(int64_t));
  for (int64_t a = 0; a < t->nnz; ++a) perm[next[key[a]]++] = (int32_t)a;
  free(next);
  return OR_OK;
}

/* Eq. 11: delta^(n)_alpha(j) = sum over core elements beta with beta_n = j of
 * G_beta * prod_{k != n} a^(k)_{i_k j_k}. */
void or_delta(const or_model* m, int32_t mode, const int32_t* i, double* delta) {
  int32_t j[OR_MAX_ORDER];
  for (int32_t q = 0; q < m->J[mode]; ++q) delta[q] = 0.0;
  const int64_t gs = core_size(m);
  for (int64_t lin = 0; lin < gs; ++lin) {
    core_unravel(m, lin, j);
    double p = m->G[lin];
    for (int k = 0; k < m->N; ++k)
      if (k != mode) p *= fac(m, k, i[k], j[k]);
    delta[j[mode]] += p;
  }
}

/* Soft-threshold minimiser shared by the two L_1 rules (Eq. 13, Eq. 14) as
 * read here: the coordinate objective is (d/2) a^2 + g a + lambda |a|, with g
 * the derivative of the squared-error part at a = 0 and d its curvature.
 * a = (lambda - g)/d if g > lambda; -(lambda + g)/d if g < -lambda; else 0. */
static double l1_rule(double g, double d, double lambda) {
  if (g > lambda) return (lambda - g) / d;
  if (g < -lambda) return -(lambda + g) / d;
  return 0.0;
}

/* Algorithm 4 for row `row` of A^(mode).
 *   - for each unpruned j = 1..J_n in ascending order (pruned ones skipped),
 *   - accumulate sum_alpha X_alpha delta_alpha(j) and the vector v_j of Eq. 10
 *     over alpha in Omega^(n)_i (in the index's order),
 *   - update a_ij by Eq. 9 (L_F) or Eq. 13 (L_1) from the current row values
 *     (the entries already updated in this pass are used: Gauss-Seidel).
 * delta_alpha does not involve A^(mode), so it is evaluated once per alpha
 * before the j loop; the sums over alpha are taken in the same order for
 * every j, which is what re-evaluating it inside the loop would give.
 * Eq. 13 as printed drops a sign and a factor 2 in g; the reading used is
 * g = -2 (c_j - sum_{t != j} v_j(t) a_t), d = 2 v_j(j), which is the one
 * consistent with its case split and with g_c of Eq. 14. */
int or_update_row(const or_tensor* t, or_model* m, int32_t mode, int64_t row,
                  const int64_t* row_ptr, const int32_t* perm, int32_t reg, double lambda) {
  if (!valid(t, m) || mode < 0 || mode >= m->N || row < 0 || row >= m->I[mode]) return OR_ERR_INVALID;
  const int32_t Jn = m->J[mode];
  const int64_t beg = row_ptr[row], len = row_ptr[row + 1] - row_ptr[row];
  double* D = (double*)malloc((size_t)(len > 0 ? len : 1) * (size_t)Jn * sizeof(double));
  double* v = (double*)malloc((size_t)Jn * sizeof(double));
  if (!D || !v) {
    free(D);
    free(v);
    return OR_ERR_NOMEM;
  }
  int32_t i[OR_MAX_ORDER];
  for (int64_t q = 0; q < len; ++q) {
    entry_index(t, perm[beg + q], i);
    or_delta(m, mode, i, D + q * Jn);
  }
  double* arow = m->A[mode] + row * Jn;
  const uint8_t* mrow = m->Amask[mode] ? m->Amask[mode] + row * Jn : NULL;
  for (int32_t j = 0; j < Jn; ++j) {
    if (mrow && mrow[j]) continue; /* pruned: excluded from the update */
    double c = 0.0;
    for (int32_t s = 0; s < Jn; ++s) v[s] = 0.0;
    for (int64_t q = 0; q < len; ++q) {
      const double* dq = D + q * Jn;
      c += t->x[perm[beg + q]] * dq[j];
      for (int32_t s = 0; s < Jn; ++s) v[s] += dq[s] * dq[j];
    }
    double other = 0.0;
    for (int32_t s = 0; s < Jn; ++s)
      if (s != j) other += v[s] * arow[s];
    if (reg == OR_REG_L1)
      arow[j] = l1_rule(-2.0 * (c - other), 2.0 * v[j], lambda);
    else
      arow[j] = (c - other) / (v[j] + lambda);
  }
  free(D);
  free(v);
  return OR_OK;
}

int or_sweep_factors(const or_tensor* t, or_model* m, int32_t reg, double lambda, int32_t mode) {
  if (!valid(t, m) || mode >= m->N || !(lambda > 0.0)) return OR_ERR_INVALID;
  const int32_t first = mode < 0 ? 0 : mode, last = mode < 0 ? m->N - 1 : mode;
  for (int32_t n = first; n <= last; ++n) {
    int64_t* row_ptr = (int64_t*)malloc((size_t)(m->I[n] + 1) * sizeof(int64_t));
    int32_t* perm = (int32_t*)malloc((size_t)(t->nnz > 0 ? t->nnz : 1) * sizeof(int32_t));
    if (!row_ptr || !perm) {
      free(row_ptr);
      free(perm);
      return OR_ERR_NOMEM;
    }
    int rc = or_build_index(t, n, row_ptr, perm);
    for (int64_t r = 0; rc == OR_OK && r < m->I[n]; ++r)
      rc = or_update_row(t, m, n, r, row_ptr, perm, reg, lambda);
    free(row_ptr);
    free(perm);
    if (rc != OR_OK) return rc;
  }
  return OR_OK;
}

/* Eq. 12 (L_F) / Eq. 14 (L_1), one core element at a time in linear order
 * (the core elements depend on each other, Section 3.5), pruned ones skipped.
 * The sum over alpha of (X_alpha - sum_{gamma != beta} G_gamma P_alpha(gamma))
 * is evaluated as r_alpha + G_beta P_alpha(beta) with r = X - B kept current
 * after every update (the same bookkeeping Algorithm 3 uses with B(alpha));
 * P_alpha(beta) = prod_n a^(n)_{i_n beta_n}. */
int or_sweep_core(const or_tensor* t, or_model* m, int32_t reg, double lambda) {
  if (!valid(t, m) || !(lambda > 0.0)) return OR_ERR_INVALID;
  const int64_t nnz = t->nnz, gs = core_size(m);
  double* r = (double*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
  double* P = (double*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
  if (!r || !P) {
    free(r);
    free(P);
    return OR_ERR_NOMEM;
  }
  int32_t i[OR_MAX_ORDER], j[OR_MAX_ORDER];
  for (int64_t a = 0; a < nnz; ++a) {
    entry_index(t, a, i);
    r[a] = t->x[a] - or_entry(m, i);
  }
  for (int64_t lin = 0; lin < gs; ++lin) {
    if (m->Gmask && m->Gmask[lin]) continue;
    core_unravel(m, lin, j);
    double num = 0.0, den = 0.0;
    const double g_old = m->G[lin];
    for (int64_t a = 0; a < nnz; ++a) {
      entry_index(t, a, i);
      double p = 1.0;
      for (int n = 0; n < m->N; ++n) p *= fac(m, n, i[n], j[n]);
      P[a] = p;
      num += (r[a] + g_old * p) * p;
      den += p * p;
    }
    double g_new;
    if (reg == OR_REG_L1)
      g_new = l1_rule(-2.0 * num, 2.0 * den, lambda);
    else
      g_new = num / (lambda + den);
    m->G[lin] = g_new;
    const double dg = g_new - g_old;
    if (dg != 0.0)
      for (int64_t a = 0; a < nnz; ++a) r[a] -= dg * P[a];
  }
  free(r);
  free(P);
  return OR_OK;
}

/* Definitions 1-2 and Algorithm 3 (scores).  For an element e, the increase
 * of the squared error when e is set to zero is
 *   Delta(e) = sum_alpha (2 r_alpha + B_e(alpha)) B_e(alpha),
 * r = X - B, with B_e(alpha) = a_ij delta_alpha(j) for a factor element
 * (Eq. 6 and Eq. 8, sum over Omega^(n)_i) and G_gamma P_alpha(gamma) for a core
 * element (Eq. 5 expanded the same way; Algorithm 3 prints the core sum
 * without its square, Eq. 5 is followed).  Then RE(e)^2 = RE^2 + Delta/||X||^2
 * and Resp(e) = (RE(e) - RE)/RE (Eq. 3). */
int or_responsibility(const or_tensor* t, const or_model* m, double* const* delta_factor,
                      double* delta_core, double* const* resp_factor, double* resp_core) {
  if (!valid(t, m)) return OR_ERR_INVALID;
  const int64_t nnz = t->nnz, gs = core_size(m);
  double* r = (double*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
  if (!r) return OR_ERR_NOMEM;
  int32_t i[OR_MAX_ORDER], j[OR_MAX_ORDER];
  double sq = 0.0, xx = 0.0;
  for (int64_t a = 0; a < nnz; ++a) {
    entry_index(t, a, i);
    r[a] = t->x[a] - or_entry(m, i);
    sq += r[a] * r[a];
    xx += t->x[a] * t->x[a];
  }
  const double re2 = xx > 0.0 ? sq / xx : 0.0, re = sqrt(re2);
  int rc = OR_OK;
  /* core elements */
  for (int64_t lin = 0; lin < gs; ++lin) {
    core_unravel(m, lin, j);
    double d = 0.0;
    for (int64_t a = 0; a < nnz; ++a) {
      entry_index(t, a, i);
      double p = m->G[lin];
      for (int n = 0; n < m->N; ++n) p *= fac(m, n, i[n], j[n]);
      d += (2.0 * r[a] + p) * p;
    }
    if (delta_core) delta_core[lin] = d;
    if (resp_core) resp_core[lin] = re > 0.0 ? (sqrt(fmax(re2 + d / xx, 0.0)) - re) / re : 0.0;
  }
  /* factor elements, row by row over Omega^(n)_i */
  for (int32_t n = 0; n < m->N && rc == OR_OK; ++n) {
    const int32_t Jn = m->J[n];
    int64_t* row_ptr = (int64_t*)malloc((size_t)(m->I[n] + 1) * sizeof(int64_t));
    int32_t* perm = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    double* delta = (double*)malloc((size_t)Jn * sizeof(double));
    if (!row_ptr || !perm || !delta) rc = OR_ERR_NOMEM;
    if (rc == OR_OK) rc = or_build_index(t, n, row_ptr, perm);
    double* acc = (double*)malloc((size_t)Jn * sizeof(double));
    if (!acc) rc = OR_ERR_NOMEM;
    for (int64_t row = 0; rc == OR_OK && row < m->I[n]; ++row) {
      for (int32_t q = 0; q < Jn; ++q) acc[q] = 0.0;
      for (int64_t p = row_ptr[row]; p < row_ptr[row + 1]; ++p) {
        const int64_t a = perm[p];
        entry_index(t, a, i);
        or_delta(m, n, i, delta);
        for (int32_t q = 0; q < Jn; ++q) {
          const double be = fac(m, n, row, q) * delta[q]; /* Eq. 8 */
          acc[q] += (2.0 * r[a] + be) * be;
        }
      }
      for (int32_t q = 0; q < Jn; ++q) {
        if (delta_factor) delta_factor[n][row * Jn + q] = acc[q];
        if (resp_factor)
          resp_factor[n][row * Jn + q] =
              re > 0.0 ? (sqrt(fmax(re2 + acc[q] / xx, 0.0)) - re) / re : 0.0;
      }
    }
    free(acc);
    free(row_ptr);
    free(perm);
    free(delta);
  }
  free(r);
  return rc;
}

typedef struct {
  double key;
  int64_t index;
} or_cand;

/* Ascending responsibility; equal scores fall back to the element's linear
 * index (row-major i*J + j for a factor, the core linear index for G). */
static int cand_cmp(const void* pa, const void* pb) {
  const or_cand* a = (const or_cand*)pa;
  const or_cand* b = (const or_cand*)pb;
  if (a->key < b->key) return -1;
  if (a->key > b->key) return 1;
  return (a->index > b->index) - (a->index < b->index);
}

/* Section 3.3 pruning: per matrix (each A^(n), and G separately), sort the
 * unpruned elements by responsibility ascending and prune the smallest
 * k = floor(pr * #unpruned) (count_mode 0) or floor(pr * size) (count_mode 1,
 * the printed pr|G|), capped at #unpruned; a pruned element is set to zero
 * and marked.  Resp is increasing in Delta for a fixed RE, so Delta is the
 * sort key.  threshold_mode prunes every unpruned element with Delta < tau. */
int or_prune(or_model* m, double* const* delta_factor, const double* delta_core, double pr,
             int32_t count_mode, int32_t threshold_mode, double tau, int64_t* n_pruned) {
  if (!valid(NULL, m) || !(pr >= 0.0) || pr > 1.0) return OR_ERR_INVALID;
  for (int32_t seg = 0; seg <= m->N; ++seg) {
    const int is_core = (seg == m->N);
    const int64_t size = is_core ? core_size(m) : m->I[seg] * m->J[seg];
    double* val = is_core ? m->G : m->A[seg];
    uint8_t* mask = is_core ? m->Gmask : m->Amask[seg];
    const double* dl = is_core ? delta_core : delta_factor[seg];
    if (!mask) return OR_ERR_INVALID;
    or_cand* c = (or_cand*)malloc((size_t)(size > 0 ? size : 1) * sizeof(or_cand));
    if (!c) return OR_ERR_NOMEM;
    int64_t nc = 0;
    for (int64_t e = 0; e < size; ++e) {
      if (mask[e]) continue;
      if (isnan(dl[e])) {
        free(c);
        return OR_ERR_NUMERIC;
      }
      c[nc].key = dl[e] == 0.0 ? 0.0 : dl[e];
      c[nc].index = e;
      ++nc;
    }
    int64_t k = 0;
    if (threshold_mode) {
      for (int64_t q = 0; q < nc; ++q)
        if (c[q].key < tau) {
          mask[c[q].index] = 1;
          val[c[q].index] = 0.0;
          ++k;
        }
    } else {
      k = (int64_t)floor(pr * (double)(count_mode ? size : nc));
      if (k > nc) k = nc;
      qsort(c, (size_t)nc, sizeof(or_cand), cand_cmp);
      for (int64_t q = 0; q < k; ++q) {
        mask[c[q].index] = 1;
        val[c[q].index] = 0.0;
      }
    }
    if (n_pruned) n_pruned[seg] = k;
    free(c);
  }
  return OR_OK;
}

/* Algorithm 2, final loop: A^(n) = U^(n) B^(n) with unit columns in U and the
 * column norms on the diagonal of B; A^(n) <- U^(n); G <- G x_n B^(n).  A
 * column of norm 0 stays 0 and its B entry is 0 (its core slice contributed
 * nothing and becomes 0). */
int or_normalize(or_model* m) {
  if (!valid(NULL, m)) return OR_ERR_INVALID;
  int32_t j[OR_MAX_ORDER];
  const int64_t gs = core_size(m);
  for (int32_t n = 0; n < m->N; ++n) {
    const int32_t Jn = m->J[n];
    double* b = (double*)calloc((size_t)Jn, sizeof(double));
    if (!b) return OR_ERR_NOMEM;
    for (int32_t q = 0; q < Jn; ++q) {
      double s = 0.0;
      for (int64_t row = 0; row < m->I[n]; ++row) s += fac(m, n, row, q) * fac(m, n, row, q);
      b[q] = sqrt(s);
      if (b[q] > 0.0)
        for (int64_t row = 0; row < m->I[n]; ++row) m->A[n][row * Jn + q] /= b[q];
    }
    for (int64_t lin = 0; lin < gs; ++lin) {
      core_unravel(m, lin, j);
      m->G[lin] *= b[j[n]];
    }
    free(b);
  }
  return OR_OK;
}

double or_sparsity(const or_model* m) {
  int64_t zeros = 0, total = 0;
  const int64_t gs = core_size(m);
  for (int64_t b = 0; b < gs; ++b) zeros += (m->G[b] == 0.0);
  total += gs;
  for (int32_t n = 0; n < m->N; ++n) {
    const int64_t sz = m->I[n] * m->J[n];
    for (int64_t e = 0; e < sz; ++e) zeros += (m->A[n][e] == 0.0);
    total += sz;
  }
  return total > 0 ? (double)zeros / (double)total : 0.0;
}

double or_elbow_stat(double re_t, double re_t1, double re_t2, double pr_t) {
  return (re_t + re_t2 - 2.0 * re_t1) / pr_t;
}

/* Algorithm 2.  Iteration t = 1, 2, ...: update the factor matrices
 * (Algorithm 4), the core (Eq. 12 / 14), compute RE (Eq. 4), then prune if
 * should_prune().  Readings where the paper is silent:
 *   - pr_t = min(INIT_PR * t, MAX_PR), t counted from 1 (pr = 0 at t = 0
 *     would prune nothing), or fixed_pr when fixed_pr_mode is set;
 *   - VeST_man stops pruning once the sparsity reaches the target;
 *   - VeST_auto stops pruning, for good, the first time t >= 3 and
 *     (RE_t + RE_{t-2} - 2 RE_{t-1}) / pr_t exceeds the threshold; with
 *     elbow_rise also RE_t > RE_{t-1} is required, reading Section 3.1's
 *     description of the stop (the error climbing fast) into the rule: a
 *     falling RE with a large second difference, as in the first sweeps from
 *     a random start, is then no elbow;
 *   - the loop ends at max_iter, or once pruning has stopped and
 *     |RE_{t-1} - RE_t| <= conv_tol * RE_{t-1};
 *   - revive_on_stop (VeST_auto only; the paper describes it and leaves it
 *     out of its runs): when the elbow rule fires, the masks go back to what
 *     they were before the last pruning step, so the elements that step
 *     removed are unpruned; they hold 0 until the next sweep refits them;
 *   - resume: the loop continues from iteration rep->iters + 1 with the
 *     report's histories, and pruning continues unless rep->stop_iter is set.
 *     A run of K iterations without normalisation, resumed to max_iter,
 *     equals one run to max_iter (the revive step only sees prunes made
 *     after the resume). */
int or_autosearch(const or_tensor* t, or_model* m, const or_params* p, or_report* rep) {
  if (!valid(t, m) || !p || !rep || p->max_iter < 1 || p->max_iter > 256) return OR_ERR_INVALID;
  if (p->resume && (rep->iters < 0 || rep->iters > 256)) return OR_ERR_INVALID;
  if (!p->resume) memset(rep, 0, sizeof(*rep));
  const int64_t gs = core_size(m);
  double* df[OR_MAX_ORDER] = {0};
  double* dc = (double*)malloc((size_t)gs * sizeof(double));
  int rc = dc ? OR_OK : OR_ERR_NOMEM;
  for (int32_t n = 0; n < m->N && rc == OR_OK; ++n) {
    df[n] = (double*)malloc((size_t)(m->I[n] * m->J[n]) * sizeof(double));
    if (!df[n]) rc = OR_ERR_NOMEM;
  }
  int pruning = p->resume ? rep->stop_iter == 0 : 1, saved = 0;
  const int revive = p->revive_on_stop && p->target_sparsity < 0.0;
  uint8_t* keep[OR_MAX_ORDER + 1] = {0}; /* masks before the last pruning step */
  for (int32_t n = 0; revive && n <= m->N && rc == OR_OK; ++n) {
    const int64_t sz = n < m->N ? m->I[n] * m->J[n] : gs;
    keep[n] = (uint8_t*)calloc((size_t)(sz > 0 ? sz : 1), 1);
    if (!keep[n]) rc = OR_ERR_NOMEM;
  }
  double out[5];
  for (int32_t it = p->resume ? rep->iters + 1 : 1; rc == OR_OK && it <= p->max_iter; ++it) {
    rc = or_sweep_factors(t, m, p->reg, p->lambda, -1);
    if (rc == OR_OK) rc = or_sweep_core(t, m, p->reg, p->lambda);
    if (rc == OR_OK) rc = or_loss(t, m, p->reg, p->lambda, out);
    if (rc != OR_OK) break;
    const int h = it - 1;
    rep->iters = it;
    rep->re_hist[h] = out[4];
    rep->obj_hist[h] = out[3];
    if (pruning) {
      const double pr = p->fixed_pr_mode ? p->fixed_pr : fmin(p->init_pr * it, p->max_pr);
      if (p->target_sparsity >= 0.0) {
        if (or_sparsity(m) >= p->target_sparsity) pruning = 0;
      } else if (it >= 3 && (!p->elbow_rise || out[4] > rep->re_hist[h - 1]) &&
                 or_elbow_stat(out[4], rep->re_hist[h - 1], rep->re_hist[h - 2], pr) > p->elbow_thresh) {
        pruning = 0;
      }
      if (!pruning) {
        rep->stop_iter = it;
        if (revive && saved) {
          for (int32_t n = 0; n <= m->N; ++n) {
            uint8_t* mk = n < m->N ? m->Amask[n] : m->Gmask;
            if (mk) memcpy(mk, keep[n], (size_t)(n < m->N ? m->I[n] * m->J[n] : gs));
          }
        }
      } else {
        for (int32_t n = 0; revive && n <= m->N; ++n) {
          const int64_t sz = n < m->N ? m->I[n] * m->J[n] : gs;
          const uint8_t* mk = n < m->N ? m->Amask[n] : m->Gmask;
          if (mk) memcpy(keep[n], mk, (size_t)sz); else memset(keep[n], 0, (size_t)(sz > 0 ? sz : 1));
        }
        saved = revive;
        rc = or_responsibility(t, m, df, dc, NULL, NULL);
        if (rc == OR_OK) rc = or_prune(m, df, dc, pr, p->count_mode, 0, 0.0, NULL);
        rep->pr_hist[h] = pr;
      }
    }
    rep->sparsity_hist[h] = or_sparsity(m);
    if (!pruning && it > 1 &&
        fabs(rep->re_hist[h - 1] - rep->re_hist[h]) <= p->conv_tol * rep->re_hist[h - 1])
      break;
  }
  if (rc == OR_OK && p->normalize) rc = or_normalize(m);
  rep->final_sparsity = or_sparsity(m);
  free(dc);
  for (int32_t n = 0; n < m->N; ++n) free(df[n]);
  for (int32_t n = 0; n <= m->N; ++n) free(keep[n]);
  return rc;
}
