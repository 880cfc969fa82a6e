/*
 * vest.h -- C ABI of the GB300 VeST coordinate-descent library (libvest.so).
 *
 * The library implements the per-iteration hot path of VeST (Park, Jang,
 * Sael, "VeST: Very Sparse Tucker Factorization of Large-Scale Tensors"):
 * element-wise coordinate-descent (CD) updates of the factor matrices and of
 * the core tensor of a partially observed Tucker model, the responsibility
 * scores with pruning, the loss the auto-search watches, and the auto-search
 * loop itself (Algorithm 2).  Every compute call runs hand-written CUDA
 * kernels for sm_103a; there is no CPU fallback.
 *
 * General conventions
 *   - Indices are 0-based.  "Device" means memory the GPU can address
 *     (cudaMalloc / torch CUDA tensors).  The caller owns every buffer; the
 *     library allocates no device memory.  Calls that need temporary device
 *     memory take a caller-provided workspace (`ws`) or scratch buffer whose
 *     size is given by the matching *_bytes() query.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls enqueue work on it and return without synchronising,
 *     except vest_autosearch(), which reads loss scalars back each iteration.
 *   - Errors: every call returns a vest_status; nothing throws across the ABI.
 *     On failure nothing is enqueued unless stated, and vest_last_error()
 *     returns a thread-local message.  Asynchronous kernel faults surface as
 *     VEST_ERR_CUDA at a later call.
 *   - Determinism: no floating-point atomics; reductions run in a fixed order,
 *     so equal inputs give bitwise-equal outputs on the same device model.
 *   - One stream per scratch buffer: two calls that share a scratch buffer must
 *     not overlap on the GPU.
 *
 * Data model
 *   - Observed tensor X on Omega (symbol table, Section 2): COO, one int32
 *     index row per mode, values in F64 or F32.
 *   - Model: factor A^(n) is I_n x J_n row-major; core G has prod_n J_n
 *     entries with linear index j_1 fastest (lin = j_1 + J_1 (j_2 + J_2 (...))),
 *     the mode-n matricisation convention of Section 2.1.  Masks are the
 *     marking table of Section 3.3: one byte per element, 1 = pruned (value 0,
 *     never updated again).  The tensor values, factors and core share one
 *     dtype.
 *   - Limits: 2 <= order <= VEST_MAX_ORDER, 1 <= J_n <= VEST_MAX_RANK,
 *     nnz < 2^31, I_n < 2^31, lambda > 0.
 */
#ifndef VEST_H
#define VEST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VEST_MAX_ORDER 10
#define VEST_MAX_RANK 32

typedef enum {
  VEST_OK = 0,
  VEST_ERR_INVALID = 1,     /* bad argument: shape, dtype, null pointer, lambda <= 0 ... */
  VEST_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed */
  VEST_ERR_NOMEM = 3,       /* host allocation failed */
  VEST_ERR_WORKSPACE = 4,   /* workspace / scratch smaller than the *_bytes() query */
  VEST_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  VEST_ERR_UNSUPPORTED = 6, /* valid request outside what this build implements */
  VEST_ERR_NUMERIC = 7      /* NaN or Inf met where a finite value is required */
} vest_status;

typedef enum { VEST_F64 = 0, VEST_F32 = 1 } vest_dtype;
typedef enum { VEST_REG_LF = 0, VEST_REG_L1 = 1 } vest_reg;

/* Observed entries Omega of an N-order tensor X (Section 2, Eq. 1).
 * idx: device int32 [order][nnz], row n holds the mode-n index of every entry.
 * val: device [nnz] of val_dtype.  Entries should be distinct positions. */
typedef struct {
  int32_t order;
  int32_t val_dtype; /* vest_dtype */
  int64_t dims[VEST_MAX_ORDER];
  int64_t nnz;
  const int32_t* idx;
  const void* val;
} vest_tensor;

/* Tucker model being fitted: core G and factors A^(n) (Section 2.2).
 * All pointers are device memory of `dtype` (masks: uint8).  Masks may not
 * be NULL: a model with nothing pruned has all-zero masks. */
typedef struct {
  int32_t order;
  int32_t dtype; /* vest_dtype; equal to the tensor's val_dtype */
  int64_t dims[VEST_MAX_ORDER];
  int32_t ranks[VEST_MAX_ORDER];
  void* factor[VEST_MAX_ORDER];          /* I_n x J_n row-major */
  uint8_t* factor_mask[VEST_MAX_ORDER];  /* I_n x J_n */
  void* core;                            /* prod J_n, j_1 fastest */
  uint8_t* core_mask;                    /* prod J_n */
} vest_model;

/* Opaque host handle of the mode-n index.  Its device arrays live in the
 * workspace given to vest_build_index(); the workspace must outlive it. */
typedef struct vest_index vest_index;

/* Device views of one mode of an index (for inspection and tests). */
typedef struct {
  const int64_t* row_ptr; /* [I_n + 1]: Omega^(n)_i = positions row_ptr[i] .. row_ptr[i+1]-1 */
  const int32_t* perm;    /* [nnz]: position p holds COO entry perm[p] */
  const int32_t* oidx;    /* [(order-1)][nnz]: the other modes' indices (ascending mode order) */
  const void* val;        /* [nnz]: values in index order */
  const int64_t* nzptr;   /* [R_n + 1]: start of every non-empty row, then nnz */
  const int32_t* nzrow;   /* [R_n]: ids of the non-empty rows */
  const int32_t* nrows_nonempty; /* device scalar R_n */
} vest_mode_view;

/* Auto-search parameters (Algorithm 2, Section 3.3). */
typedef struct {
  int32_t reg;            /* vest_reg */
  double lambda;          /* > 0 */
  double init_pr;         /* INIT_PR (paper default 0.01) */
  double max_pr;          /* MAX_PR (paper default 0.1) */
  double elbow_thresh;    /* VeST_auto threshold (paper: 0.05) */
  double target_sparsity; /* >= 0: VeST_man target s; < 0: VeST_auto */
  double conv_tol;        /* converged when |RE_{t-1} - RE_t| <= conv_tol * RE_{t-1} */
  int32_t max_iter;       /* 1 .. 256 */
  int32_t fixed_pr_mode;  /* 1: prune fixed_pr at every pruning step */
  double fixed_pr;
  int32_t count_mode;     /* 0: k = floor(pr * #unpruned); 1: k = floor(pr * size) */
  int32_t normalize;      /* 1: final column normalisation (end of Algorithm 2) */
  int32_t revive_on_stop; /* VeST_auto only, 1: when the elbow rule stops pruning, unprune
                             the elements the last pruning step removed (Section 3.1) */
  int32_t resume;         /* 1: continue the run recorded in the report passed in (a checkpoint:
                             iters done, histories, stop_iter) on the model as it stands */
  int32_t elbow_rise;     /* VeST_auto, 1: the elbow also needs RE_t > RE_{t-1} (Section 3.1
                             describes the stop as the error climbing fast) */
} vest_params;

typedef struct {
  int32_t iters;
  int32_t stop_iter;      /* iteration at which pruning stopped (0 = never) */
  double re_hist[256];
  double obj_hist[256];
  double pr_hist[256];    /* pruning rate applied at iteration t (0 = none) */
  double sparsity_hist[256];
  double final_sparsity;
} vest_report;

/* Version string and the calling thread's last error message. */
const char* vest_version(void);
const char* vest_last_error(void);
/* Number of CUDA kernels this library has launched in this process (all
 * threads, all devices): a diagnostic for profiling and launch budgets. */
uint64_t vest_launch_count(void);

/* Device-side status.  Kernels never trap: a wait with a bounded number of polls
 * that runs out (the tensor-core completion wait of the FP32 factor sweep, which
 * a healthy GPU never exhausts) abandons the rest of its work, raises a bit
 * here and returns, and the results of that call are not valid.  This call
 * synchronises the device, writes the bits raised since the last clear to
 * *flags (nullable; bit 0: a factor-sweep wait gave up, bit 1: a loss wait gave up
 * -- the loss kernel behind vest_loss, vest_iteration and the core sweep), clears them when
 * clear != 0, and returns VEST_ERR_TIMEOUT when any was set, else VEST_OK. */
vest_status vest_device_status(uint32_t* flags, int32_t clear);

/* Peak-rate probes (measurement support, no counterpart in the paper): runs one
 * self-timed probe on `stream` and writes its rate to *rate (host double):
 *   kind 0  FP32 FMA throughput, TFLOP/s (independent FMA chains, every lane of every SM)
 *   kind 1  FP64 FMA throughput, TFLOP/s
 *   kind 2  tcgen05 TF32 MMA throughput with A in tensor memory, TFLOP/s (M = 128, N = 256,
 *           K = 8, the operand placement of the FP32 factor sweep)
 *   kind 3  L2 random-gather throughput of 16-byte reads, TB/s, from a table of up to
 *           32 MiB kept in `buffer` (device, at least 4 MiB, contents overwritten)
 * Each probe runs twice and the second run is timed with CUDA events; the call
 * synchronises on its last event.  Clocks are left as they are: compare a rate
 * with the SM clock seen while it ran. */
vest_status vest_probe_peak(int32_t kind, double* rate, void* buffer, size_t buffer_bytes, void* stream);

/* ---- a1: mode-n index (the sets Omega^(n)_{i_n} of the symbol table, used by
 * Algorithm 3 and Algorithm 4).  For every mode n the observed entries are
 * stably sorted by i_n (ties keep COO order) with a device radix sort; the
 * result is a CSR structure per mode plus the other modes' indices and the
 * values permuted into that order.  The index copies everything it needs:
 * the tensor's arrays may be freed after the call completes on the stream.
 * The call checks every index against dims on the device and synchronises
 * `stream` once to read that check (VEST_ERR_INVALID if one is out of range). */
size_t vest_index_workspace_bytes(const vest_tensor* t);
vest_status vest_build_index(const vest_tensor* t, void* ws, size_t ws_bytes, vest_index** out,
                             void* stream);
vest_status vest_index_destroy(vest_index* ix);
vest_status vest_index_mode(const vest_index* ix, int32_t mode, vest_mode_view* out);

/* Scratch needed by the compute calls below for this index and model shape. */
size_t vest_scratch_bytes(const vest_index* ix, const vest_model* m);
/* The same figure from the tensor's description alone (no index needed yet), for callers
 * that budget device memory before building anything: equals vest_scratch_bytes() for
 * the index vest_build_index(t) makes.  Only the shape fields of t (order, dims, nnz,
 * val_dtype) and of m (order, dtype, dims, ranks) are read; their pointers may be
 * NULL.  Returns 0 on invalid arguments. */
size_t vest_scratch_bytes_for(const vest_tensor* t, const vest_model* m);

/* ---- a2-a4: factor sweep (Algorithm 4; Lemma 1, Eq. 9-11 for L_F; Lemma 3,
 * Eq. 13 for L_1).  For mode n (mode >= 0) or every mode in order 0..N-1
 * (mode = -1): every row i of A^(n) is updated element by element, j
 * ascending, pruned elements skipped, each new value the exact minimiser of
 * the objective in that coordinate given the current others.  A row with no
 * observed entry becomes 0 (the minimiser).  Updates A^(n) in place. */
vest_status vest_sweep_factors(const vest_index* ix, vest_model* m, int32_t reg, double lambda,
                               int32_t mode, void* scratch, size_t scratch_bytes, void* stream);

/* The factor sweep with the kernel for Eq. 11 chosen by the caller (an autotuner, for one):
 *   VEST_DELTA_AUTO    the tensor cores (split-TF32 tcgen05 MMA, FP32 models) where they
 *                      apply, the FMA kernels elsewhere; what vest_sweep_factors does
 *   VEST_DELTA_FMA     the FMA kernels everywhere
 *   VEST_DELTA_TENSOR  the tensor cores, or VEST_ERR_UNSUPPORTED (before anything is
 *                      enqueued) where they do not apply: FP64 models, a rank above 16, or
 *                      more than one other mode left after the one or two "A" modes
 * All paths compute the same update to within FP32 rounding (FP64 models: bit-identical,
 * the FMA kernels).  The environment variable VEST_TENSOR_CORES=0 turns AUTO into FMA. */
typedef enum { VEST_DELTA_AUTO = 0, VEST_DELTA_FMA = 1, VEST_DELTA_TENSOR = 2 } vest_delta_path;
vest_status vest_sweep_factors_ex(const vest_index* ix, vest_model* m, int32_t reg, double lambda, int32_t mode,
                                  int32_t path, void* scratch, size_t scratch_bytes, void* stream);

/* ---- a5: core sweep (Lemma 2, Eq. 12 for L_F; Lemma 4, Eq. 14 for L_1).
 * Sequential CD over the unpruned core elements in linear order; results
 * equal, in exact arithmetic, one element at a time (Section 3.5). */
vest_status vest_sweep_core(const vest_index* ix, vest_model* m, int32_t reg, double lambda,
                            void* scratch, size_t scratch_bytes, void* stream);

/* ---- a6: loss (Eq. 1 / Eq. 2, RE of Eq. 4 over Omega).  out: device
 * double[5] = {sum_Omega r^2, sum_Omega X^2, regulariser term, objective, RE},
 * r = X - B (Eq. 7).  resid: optional device [nnz] of the model dtype that
 * receives r in COO order (NULL to skip). */
vest_status vest_loss(const vest_index* ix, const vest_model* m, int32_t reg, double lambda,
                      double* out, void* resid, void* scratch, size_t scratch_bytes, void* stream);

/* ---- a7: responsibility (Definitions 1-2, Eq. 3-6, Algorithm 3).
 * delta_factor[n] (device double, I_n x J_n) and delta_core (device double,
 * prod J_n) receive Delta(e) = sum_alpha (2 r_alpha + B_e(alpha)) B_e(alpha),
 * the increase of the squared error when element e is set to zero;
 * resp_factor / resp_core (nullable, device double) receive
 * Resp(e) = (sqrt(RE^2 + Delta/||X||^2) - RE) / RE.  Pass delta_factor /
 * resp_factor as arrays of `order` device pointers (host array). */
vest_status vest_responsibility(const vest_index* ix, const vest_model* m, double* const* delta_factor,
                                double* delta_core, double* const* resp_factor, double* resp_core,
                                void* scratch, size_t scratch_bytes, void* stream);

/* ---- a8: prune (Section 3.3; the pruning step of Algorithm 3).  For each A^(n) and
 * for G separately, among unpruned elements select the k smallest Delta
 * (ties: smaller linear index first; -0 == +0), k = floor(pr * #unpruned)
 * (count_mode 0) or floor(pr * size) (count_mode 1), capped at #unpruned; or,
 * with threshold_mode = 1, every unpruned element with Delta < tau.  Selected
 * elements get mask 1 and value 0.  n_pruned: device int64[order + 1]
 * (nullable) receives the count per segment (factors in mode order, then G).
 * A NaN Delta among the candidates leaves the model unchanged for that
 * segment and sets n_pruned[segment] = -1. */
vest_status vest_prune(vest_model* m, double* const* delta_factor, const double* delta_core, double pr,
                       int32_t count_mode, int32_t threshold_mode, double tau, int64_t* n_pruned,
                       void* scratch, size_t scratch_bytes, void* stream);

/* ---- Value Pruning keys (Section 4.1, competitors: VeST_man with s = 0, then
 * value pruning at ratio 0.6).  Writes |element| in FP64 for every element
 * of every segment: key_factor[n] is device double[I_n * J_n] row-major like
 * A^(n), key_core device double[prod J_n] like G.  Passing them to vest_prune
 * with pr = 0.6 and count_mode = 1 prunes, in each segment, the 60 % of its
 * elements with the smallest magnitude (ties by linear index).  Buffers are
 * caller-owned; NULL outputs give VEST_ERR_INVALID.  Never synchronises. */
vest_status vest_value_keys(const vest_model* m, double* const* key_factor, double* key_core, void* stream);

/* ---- a9: normalisation (the final step of Algorithm 2): A^(n) = U^(n) B^(n) with
 * unit-norm columns, A^(n) <- U^(n), G <- G x_n B^(n); zero columns stay 0. */
vest_status vest_normalize(vest_model* m, void* scratch, size_t scratch_bytes, void* stream);

/* Number of exactly-zero elements per segment (factors in mode order, then G)
 * into device int64[order + 1]; sparsity = sum / (|G| + sum_n I_n J_n). */
vest_status vest_count_zeros(const vest_model* m, int64_t* out, void* scratch, size_t scratch_bytes,
                             void* stream);

/* ---- a9: auto-search (Algorithm 2, Section 3.3): iterations of factor sweep,
 * core sweep, RE, and, while should_prune(), responsibility + prune with
 * pr_t = min(init_pr * t, max_pr) (t = 1, 2, ...) or fixed_pr.  VeST_man
 * stops pruning once the sparsity reaches target_sparsity; VeST_auto stops
 * the first time t >= 3 and (RE_t + RE_{t-2} - 2 RE_{t-1}) / pr_t > elbow_thresh
 * (and, with elbow_rise, RE_t > RE_{t-1}).
 * With revive_on_stop (VeST_auto), the masks return to their state before
 * the last pruning step when the elbow rule fires; the revived elements hold 0
 * until the next sweep refits them.  With resume, the loop continues from
 * iteration report->iters + 1 with the report's histories (report->iters in
 * [0, 256], else VEST_ERR_INVALID) and keeps pruning unless report->stop_iter
 * is set: a run of K iterations with normalize = 0, resumed to max_iter from
 * its model and report, gives bitwise the same model and report as one run to
 * max_iter (a revive only restores prunes made after the resume).  Ends at max_iter or when RE has converged
 * after pruning stopped; then normalises if asked.  Synchronises `stream` once
 * per iteration to read RE.  report: host memory.  scratch: at least
 * vest_autosearch_scratch_bytes() (vest_scratch_bytes() plus 8 bytes per model
 * element for the Delta scores and, with revive_on_stop, 1 byte per element for
 * the saved masks); a smaller buffer gives VEST_ERR_WORKSPACE. */
size_t vest_autosearch_scratch_bytes(const vest_index* ix, const vest_model* m);
vest_status vest_autosearch(const vest_index* ix, vest_model* m, const vest_params* p, vest_report* report,
                            void* scratch, size_t scratch_bytes, void* stream);

/* ---- a2-a8 in one call: one iteration of the loop of Algorithm 2: factor
 * sweep over every mode (skipped when factor_sweep is 0, for callers that
 * sweep the modes themselves), core sweep, loss of the swept model, and, when
 * delta_factor is not NULL, the responsibility of every element (Eq. 5/6) and
 * the prune with rate pr (count_mode as in vest_prune; pr = 0 prunes nothing).
 * The residual that the core sweep keeps current serves the loss and the
 * responsibility, so neither recomputes B: the results equal vest_sweep_factors
 * (-1), vest_sweep_core, vest_loss, vest_responsibility and vest_prune in turn,
 * up to rounding.  loss: device double[5] as in vest_loss, the model after the
 * sweeps and before the prune.  delta_factor / delta_core: device outputs as in
 * vest_responsibility (both NULL to stop after the loss).  n_pruned: NULL or
 * device int64[order + 1] as in vest_prune.  scratch: vest_scratch_bytes().
 * Never synchronises. */
vest_status vest_iteration(const vest_index* ix, vest_model* m, int32_t reg, double lambda, double pr,
                           int32_t count_mode, int32_t factor_sweep, double* loss, double* const* delta_factor,
                           double* delta_core, int64_t* n_pruned, void* scratch, size_t scratch_bytes, void* stream);

/* ---- vest_loss without a scratch buffer.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when they
 * need the loss, such as a host runtime that owns the device heap and forbids
 * other allocations, or a service whose memory budget is fixed at start-up.
 * It computes exactly what vest_loss() computes (out: device double[5];
 * resid: optional device [nnz] in COO order) and allocates nothing: its
 * scratch is a fixed 1 MiB array inside libvest, present on every device that
 * loads the library until the process exits.
 *   - Limit: the permuted mode-0 core (prod_n J_n rounded up to the rank bucket,
 *     in the model dtype) plus about 12 KB of partial sums must fit in 1 MiB;
 *     larger models get VEST_ERR_WORKSPACE and should use vest_loss().
 *   - The first call on a device looks up the array's device address (one
 *     cudaGetSymbolAddress with that device current) and keeps it for that
 *     device's CUDA context; make that first call before any stream capture.
 *     If the context is replaced (cudaDeviceReset, then new work), the next
 *     call sees the new context and looks the address up again.
 *   - Input checks are those of vest_loss(): both accept the same inputs.
 *   - Every call on a device shares the one array and overwrites what the
 *     previous call left there (nothing in it needs to start at zero: each
 *     call writes every value it reads).  Calls that overlap on the GPU race
 *     on it: serialise them, e.g. on one stream. */
vest_status vest_loss_noalloc(const vest_index* ix, const vest_model* m, int32_t reg, double lambda, double* out,
                              void* resid, void* stream);

/* Completion queries: B(alpha) (Eq. 7) for m query positions q_idx (device
 * int32 [order][m]) into out (device, model dtype, [m]).  A tuple with an index
 * outside [0, I_n) reads nothing and gives NaN. */
vest_status vest_reconstruct(const vest_model* m, const int32_t* q_idx, int64_t count, void* out,
                             void* stream);

#ifdef __cplusplus
}
#endif
#endif
