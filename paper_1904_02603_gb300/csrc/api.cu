// C ABI of libvest: argument checks, scratch planning, dtype dispatch and the
// host loop of the auto-search (Algorithm 2).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <utility>

#include "delta.cuh"

namespace vest {

size_t core_scratch_bytes(const vest_model* m, int64_t nnz, int64_t cap0, size_t* y_bytes, size_t* gram_bytes,
                          size_t* part_bytes);
size_t loss_part_bytes();
size_t normalize_scratch_bytes();
size_t prune_scratch_bytes(int64_t maxseg, size_t* keys_bytes, size_t* vals_bytes, size_t* tmp_bytes);
template <typename T>
int sweep_task_size(int Jn, int P, int64_t core_elems, int* use_smem_core);

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

void count_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }
vest_status fail(vest_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}
vest_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return VEST_ERR_CUDA;
}

int num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 148;
  return n;
}

vest_status max_dynamic_smem(const void* kern, size_t* out) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> cache;
  int dev = 0;
  VEST_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find({dev, kern});
    if (it != cache.end()) {
      *out = it->second;
      return VEST_OK;
    }
  }
  int optin = 0;
  VEST_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa{};
  VEST_CUDA(cudaFuncGetAttributes(&fa, kern));
  const size_t cap = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
  std::lock_guard<std::mutex> lock(mu);
  cache[{dev, kern}] = cap;
  *out = cap;
  return VEST_OK;
}

static size_t dtype_size(int dt) { return dt == VEST_F64 ? 8 : 4; }

// Shape fields of a model: order, dtype, ranks, dims and the size limits.
static vest_status check_model_shape(const vest_model* m) {
  if (!m) return fail(VEST_ERR_INVALID, "model is NULL");
  if (m->order < 2 || m->order > VEST_MAX_ORDER) return fail(VEST_ERR_INVALID, "order must be in [2, 10]");
  if (m->dtype != VEST_F64 && m->dtype != VEST_F32) return fail(VEST_ERR_INVALID, "model dtype must be F64 or F32");
  int64_t gs = 1;
  for (int n = 0; n < m->order; ++n) {
    if (m->ranks[n] < 1 || m->ranks[n] > VEST_MAX_RANK) return fail(VEST_ERR_INVALID, "rank must be in [1, 32]");
    if (m->dims[n] < 1 || m->dims[n] >= (int64_t(1) << 31)) return fail(VEST_ERR_INVALID, "dims must be in [1, 2^31)");
    if (m->dims[n] * m->ranks[n] >= (int64_t(1) << 31)) return fail(VEST_ERR_INVALID, "factor too large");
    gs *= m->ranks[n];
  }
  if (gs >= (int64_t(1) << 24)) return fail(VEST_ERR_UNSUPPORTED, "core larger than 2^24 elements");
  return VEST_OK;
}

static vest_status check_model(const vest_model* m) {
  VEST_TRY(check_model_shape(m));
  for (int n = 0; n < m->order; ++n)
    if (!m->factor[n] || !m->factor_mask[n]) return fail(VEST_ERR_INVALID, "factor or mask pointer is NULL");
  if (!m->core || !m->core_mask) return fail(VEST_ERR_INVALID, "core or core mask pointer is NULL");
  return VEST_OK;
}

vest_status check_pair(const vest_index* ix, const vest_model* m) {
  if (!ix) return fail(VEST_ERR_INVALID, "index is NULL");
  VEST_TRY(check_model(m));
  if (ix->order != m->order) return fail(VEST_ERR_INVALID, "index and model order differ");
  if (ix->val_dtype != m->dtype) return fail(VEST_ERR_INVALID, "tensor and model dtypes differ");
  for (int n = 0; n < m->order; ++n)
    if (ix->dims[n] != m->dims[n]) return fail(VEST_ERR_INVALID, "index and model dims differ");
  return VEST_OK;
}

static vest_status check_lambda(double lambda) {
  if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(VEST_ERR_INVALID, "lambda must be finite and > 0");
  return VEST_OK;
}

template <typename T>
static void sweep_need(const vest_index* ix, const vest_model* m, int64_t* max_ntasks, size_t* spill, size_t* gperm) {
  *max_ntasks = 1;
  *spill = 0;
  *gperm = 0;
  for (int n = 0; n < m->order; ++n) {
    const ModeRoles r = mode_roles(m->ranks, m->order, n);
    const int JN = jn_bucket(r.Jn);
    const int64_t core_elems = r.n_outer * r.Jf * JN;
    *gperm = std::max(*gperm, align_up((size_t)core_elems * sizeof(T)) + align_up((size_t)r.n_outer));
    for (int kind = 0; kind < 2; ++kind) {
      const int P = kind == 0 ? r.Jn + r.Jn * (r.Jn + 1) / 2 : 2 * r.Jn;
      int us = 0;
      const int task = sweep_task_size<T>(r.Jn, P, core_elems, &us);
      const int64_t nt = std::max<int64_t>(1, ceil_div(ix->nnz, task));
      *max_ntasks = std::max(*max_ntasks, nt);
      *spill = std::max(*spill, (size_t)nt * 2 * P * 8);
    }
  }
}

ScratchPlan plan_scratch(const vest_index* ix, const vest_model* m) {
  ScratchPlan p{};
  const size_t sT = dtype_size(m->dtype);
  int64_t nt;
  size_t spill, gperm;
  if (m->dtype == VEST_F64) sweep_need<double>(ix, m, &nt, &spill, &gperm);
  else sweep_need<float>(ix, m, &nt, &spill, &gperm);
  int64_t maxseg = 1;
  for (int n = 0; n < m->order; ++n) maxseg = std::max<int64_t>(maxseg, m->dims[n] * m->ranks[n]);
  int64_t gs = 1;
  for (int n = 0; n < m->order; ++n) gs *= m->ranks[n];
  maxseg = std::max(maxseg, gs);
  size_t o = 0;
  p.off_status = o; o += 256;
  p.off_gperm = o; p.gperm_bytes = align_up(gperm); o += p.gperm_bytes;
  p.off_spill = o; p.spill_bytes = align_up(spill); o += p.spill_bytes;
  p.off_spanning = o; o += align_up((size_t)nt * 4);
  p.ntasks = nt;
  p.off_resid = o; o += align_up((size_t)std::max<int64_t>(ix->nnz, 1) * sT);
  p.off_resid_coo = o; o += align_up((size_t)std::max<int64_t>(ix->nnz, 1) * sT);
  p.part_bytes = align_up(std::max(loss_part_bytes(), normalize_scratch_bytes()));
  p.off_part = o; o += p.part_bytes;
  p.off_small = o; o += 128 * 1024;
  size_t kb, vb, tb;
  prune_scratch_bytes(maxseg, &kb, &vb, &tb);
  p.off_prune_keys = o; o += kb;
  p.off_prune_vals = o; o += vb;
  p.off_prune_tmp = o; o += tb;
  size_t yb, gb, cpb;
  const int64_t cap0 = std::min<int64_t>(ix->dims[0], std::max<int64_t>(ix->nnz, 1));
  p.off_core = o; o += align_up(core_scratch_bytes(m, ix->nnz, cap0, &yb, &gb, &cpb));
  size_t rb = 0;  // the update's outputs per row (J + J(J+1)/2) exceed the responsibility's (2J)
  for (int n = 0; n < m->order; ++n) {
    const int64_t capn = std::min<int64_t>(ix->dims[n], std::max<int64_t>(ix->nnz, 1));
    const int J = m->ranks[n];
    rb = std::max(rb, (size_t)capn * (size_t)(J + J * (J + 1) / 2) * 8);
  }
  p.off_rowbuf = o; p.rowbuf_bytes = align_up(rb); o += p.rowbuf_bytes;
  p.total = o;
  return p;
}

// offsets (in doubles) inside the small scratch region
constexpr size_t kSmallStats = 9400;   // 5 doubles: responsibility's loss statistics
constexpr size_t kSmallLoss = 9410;    // 5 doubles: auto-search loss
constexpr size_t kSmallZeros = 9420;   // order+1 int64: zero counts

static vest_status check_scratch(const vest_index* ix, const vest_model* m, void* scratch, size_t bytes, ScratchPlan* plan) {
  *plan = plan_scratch(ix, m);
  if (!scratch) return fail(VEST_ERR_INVALID, "scratch is NULL");
  if (bytes < plan->total) return fail(VEST_ERR_WORKSPACE, "scratch smaller than vest_scratch_bytes()");
  return VEST_OK;
}

}  // namespace vest

using namespace vest;

extern "C" {

const char* vest_version(void) { return "vest-gb300 0.2 (sm_103a)"; }

vest_status vest_device_status(uint32_t* flags, int32_t clear) {
  uint32_t f = 0, fl = 0;
  VEST_TRY(sweep_device_status(&f, clear != 0));  // synchronises the device first
  VEST_TRY(loss_device_status(&fl, clear != 0));
  f |= fl;
  if (flags) *flags = f;
  if (f) return fail(VEST_ERR_TIMEOUT, "a bounded device wait gave up since the last clear (flags " + std::to_string(f) + ")");
  return VEST_OK;
}
const char* vest_last_error(void) { return g_last_error.c_str(); }
uint64_t vest_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

size_t vest_index_workspace_bytes(const vest_tensor* t) {
  if (!t || t->order < 2 || t->order > VEST_MAX_ORDER || t->nnz < 0) return 0;
  return index_workspace_bytes(t);
}

vest_status vest_build_index(const vest_tensor* t, void* ws, size_t ws_bytes, vest_index** out, void* stream) {
  if (!t || !out) return fail(VEST_ERR_INVALID, "tensor or out is NULL");
  *out = nullptr;
  if (t->order < 2 || t->order > VEST_MAX_ORDER) return fail(VEST_ERR_INVALID, "order must be in [2, 10]");
  if (t->val_dtype != VEST_F64 && t->val_dtype != VEST_F32) return fail(VEST_ERR_INVALID, "value dtype must be F64 or F32");
  if (t->nnz < 0 || t->nnz >= (int64_t(1) << 31)) return fail(VEST_ERR_INVALID, "nnz must be in [0, 2^31)");
  for (int n = 0; n < t->order; ++n)
    if (t->dims[n] < 1 || t->dims[n] >= (int64_t(1) << 31)) return fail(VEST_ERR_INVALID, "dims must be in [1, 2^31)");
  if (t->nnz > 0 && (!t->idx || !t->val)) return fail(VEST_ERR_INVALID, "idx or val is NULL");
  if (!ws) return fail(VEST_ERR_INVALID, "workspace is NULL");
  vest_index* ix = new (std::nothrow) vest_index();
  if (!ix) return fail(VEST_ERR_NOMEM, "host allocation of the index handle failed");
  const vest_status st = build_index_impl(t, ws, ws_bytes, ix, as_stream(stream));
  if (st != VEST_OK) {
    delete ix;
    return st;
  }
  *out = ix;
  return VEST_OK;
}

vest_status vest_index_destroy(vest_index* ix) {
  delete ix;
  return VEST_OK;
}

vest_status vest_index_mode(const vest_index* ix, int32_t mode, vest_mode_view* out) {
  if (!ix || !out || mode < 0 || mode >= ix->order) return fail(VEST_ERR_INVALID, "bad index, mode or out");
  const ModeIndex& mi = ix->mode[mode];
  out->row_ptr = mi.row_ptr;
  out->perm = mi.perm;
  out->oidx = mi.oidx;
  out->val = mi.val;
  out->nzptr = mi.nzptr;
  out->nzrow = mi.nzrow;
  out->nrows_nonempty = mi.nnzrows;
  return VEST_OK;
}

size_t vest_scratch_bytes(const vest_index* ix, const vest_model* m) {
  if (check_pair(ix, m) != VEST_OK) return 0;
  return plan_scratch(ix, m).total;
}

size_t vest_scratch_bytes_for(const vest_tensor* t, const vest_model* m) {
  // the scratch plan reads only the tensor's shape, entry count and dtype: a host-side
  // description stands in for the index that vest_build_index would make
  if (!t || t->order < 2 || t->order > VEST_MAX_ORDER || t->nnz < 0) return 0;
  vest_index d{};
  d.order = t->order;
  d.val_dtype = t->val_dtype;
  d.nnz = t->nnz;
  for (int n = 0; n < t->order; ++n) {
    d.dims[n] = t->dims[n];
    d.mode[n].cap = std::min<int64_t>(t->dims[n], std::max<int64_t>(t->nnz, 1));
  }
  if (check_model_shape(m) != VEST_OK || d.order != m->order || d.val_dtype != m->dtype) return 0;
  for (int n = 0; n < m->order; ++n)
    if (d.dims[n] != m->dims[n]) return 0;
  return plan_scratch(&d, m).total;
}

vest_status vest_sweep_factors(const vest_index* ix, vest_model* m, int32_t reg, double lambda, int32_t mode,
                               void* scratch, size_t scratch_bytes, void* stream) {
  return vest_sweep_factors_ex(ix, m, reg, lambda, mode, VEST_DELTA_AUTO, scratch, scratch_bytes, stream);
}

vest_status vest_sweep_factors_ex(const vest_index* ix, vest_model* m, int32_t reg, double lambda, int32_t mode,
                                  int32_t path, void* scratch, size_t scratch_bytes, void* stream) {
  if (path < VEST_DELTA_AUTO || path > VEST_DELTA_TENSOR) return fail(VEST_ERR_INVALID, "unknown delta path");
  VEST_TRY(check_pair(ix, m));
  VEST_TRY(check_lambda(lambda));
  if (reg != VEST_REG_LF && reg != VEST_REG_L1) return fail(VEST_ERR_INVALID, "unknown regulariser");
  if (mode < -1 || mode >= m->order) return fail(VEST_ERR_INVALID, "mode out of range");
  ScratchPlan plan;
  VEST_TRY(check_scratch(ix, m, scratch, scratch_bytes, &plan));
  const cudaStream_t s = as_stream(stream);
  char* sc = static_cast<char*>(scratch);
  const int first = mode < 0 ? 0 : mode, last = mode < 0 ? m->order - 1 : mode;
  if (path == VEST_DELTA_TENSOR)
    for (int n = first; n <= last; ++n)
      if (!sweep_tc_applies(m, n))
        return fail(VEST_ERR_UNSUPPORTED, "the tensor-core delta does not apply to mode " + std::to_string(n) +
                                              " (FP64, a rank above 16, or more than one other mode left after "
                                              "the A modes)");
  for (int n = first; n <= last; ++n) {
    if (m->dtype == VEST_F64) VEST_TRY(sweep_factors_mode<double>(ix, m, reg, lambda, n, sc, plan, s, path));
    else VEST_TRY(sweep_factors_mode<float>(ix, m, reg, lambda, n, sc, plan, s, path));
  }
  return VEST_OK;
}

vest_status vest_sweep_core(const vest_index* ix, vest_model* m, int32_t reg, double lambda, void* scratch,
                            size_t scratch_bytes, void* stream) {
  VEST_TRY(check_pair(ix, m));
  VEST_TRY(check_lambda(lambda));
  if (reg != VEST_REG_LF && reg != VEST_REG_L1) return fail(VEST_ERR_INVALID, "unknown regulariser");
  ScratchPlan plan;
  VEST_TRY(check_scratch(ix, m, scratch, scratch_bytes, &plan));
  char* sc = static_cast<char*>(scratch);
  if (m->dtype == VEST_F64) return sweep_core_impl<double>(ix, m, reg, lambda, sc, plan, as_stream(stream));
  return sweep_core_impl<float>(ix, m, reg, lambda, sc, plan, as_stream(stream));
}

vest_status vest_loss(const vest_index* ix, const vest_model* m, int32_t reg, double lambda, double* out, void* resid,
                      void* scratch, size_t scratch_bytes, void* stream) {
  VEST_TRY(check_pair(ix, m));
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return fail(VEST_ERR_INVALID, "lambda must be finite and >= 0");
  if (reg != VEST_REG_LF && reg != VEST_REG_L1) return fail(VEST_ERR_INVALID, "unknown regulariser");
  if (!out) return fail(VEST_ERR_INVALID, "out is NULL");
  ScratchPlan plan;
  VEST_TRY(check_scratch(ix, m, scratch, scratch_bytes, &plan));
  char* sc = static_cast<char*>(scratch);
  if (m->dtype == VEST_F64)
    return loss_impl<double>(ix, m, reg, lambda, out, nullptr, static_cast<double*>(resid), sc, plan, as_stream(stream));
  return loss_impl<float>(ix, m, reg, lambda, out, nullptr, static_cast<float*>(resid), sc, plan, as_stream(stream));
}

vest_status vest_responsibility(const vest_index* ix, const vest_model* m, double* const* delta_factor,
                                double* delta_core, double* const* resp_factor, double* resp_core, void* scratch,
                                size_t scratch_bytes, void* stream) {
  VEST_TRY(check_pair(ix, m));
  if (!delta_factor || !delta_core) return fail(VEST_ERR_INVALID, "delta outputs are NULL");
  for (int n = 0; n < m->order; ++n) {
    if (!delta_factor[n]) return fail(VEST_ERR_INVALID, "delta_factor entry is NULL");
    if (resp_factor && !resp_factor[n]) return fail(VEST_ERR_INVALID, "resp_factor entry is NULL");
  }
  ScratchPlan plan;
  VEST_TRY(check_scratch(ix, m, scratch, scratch_bytes, &plan));
  char* sc = static_cast<char*>(scratch);
  const cudaStream_t s = as_stream(stream);
  double* stats = reinterpret_cast<double*>(sc + plan.off_small) + kSmallStats;
  if (m->dtype == VEST_F64) {
    double* r0 = reinterpret_cast<double*>(sc + plan.off_resid);
    double* rc = reinterpret_cast<double*>(sc + plan.off_resid_coo);
    VEST_TRY(loss_impl<double>(ix, m, VEST_REG_LF, 1.0, stats, r0, rc, sc, plan, s));
    VEST_TRY(responsibility_factors<double>(ix, m, stats, delta_factor, resp_factor, sc, plan, s));
    return core_responsibility<double>(ix, m, r0, stats, delta_core, resp_core, sc, plan, s);
  }
  float* r0 = reinterpret_cast<float*>(sc + plan.off_resid);
  float* rc = reinterpret_cast<float*>(sc + plan.off_resid_coo);
  VEST_TRY(loss_impl<float>(ix, m, VEST_REG_LF, 1.0, stats, r0, rc, sc, plan, s));
  VEST_TRY(responsibility_factors<float>(ix, m, stats, delta_factor, resp_factor, sc, plan, s));
  return core_responsibility<float>(ix, m, r0, stats, delta_core, resp_core, sc, plan, s);
}

// One iteration of Algorithm 2 in two halves.  The first sweeps (factors unless told
// otherwise, then the core) and leaves the residual of the swept model in the scratch,
// writing its loss; the second takes the responsibility from that residual (and diag M
// from the core sweep's block Grams) and prunes.  Nothing may change the model between them.
static vest_status iteration_sweeps(const vest_index* ix, vest_model* m, int32_t reg, double lambda,
                                    int32_t factor_sweep, double* loss, void* scratch, size_t scratch_bytes,
                                    const ScratchPlan& plan, void* stream) {
  char* sc = static_cast<char*>(scratch);
  const cudaStream_t s = as_stream(stream);
  if (factor_sweep) VEST_TRY(vest_sweep_factors(ix, m, reg, lambda, -1, scratch, scratch_bytes, stream));
  if (m->dtype == VEST_F64) return sweep_core_impl<double>(ix, m, reg, lambda, sc, plan, s, loss);
  return sweep_core_impl<float>(ix, m, reg, lambda, sc, plan, s, loss);
}

static vest_status iteration_prune(const vest_index* ix, vest_model* m, const double* loss, double pr,
                                   int32_t count_mode, double* const* delta_factor, double* delta_core,
                                   int64_t* n_pruned, char* sc, const ScratchPlan& plan, cudaStream_t s) {
  if (m->dtype == VEST_F64) {
    const double* r0 = reinterpret_cast<const double*>(sc + plan.off_resid);
    VEST_TRY(responsibility_factors<double>(ix, m, loss, delta_factor, nullptr, sc, plan, s));
    VEST_TRY(core_responsibility<double>(ix, m, r0, loss, delta_core, nullptr, sc, plan, s, true));
    return prune_impl<double>(m, delta_factor, delta_core, pr, count_mode, 0, 0.0, n_pruned, sc, plan, s);
  }
  const float* r0 = reinterpret_cast<const float*>(sc + plan.off_resid);
  VEST_TRY(responsibility_factors<float>(ix, m, loss, delta_factor, nullptr, sc, plan, s));
  VEST_TRY(core_responsibility<float>(ix, m, r0, loss, delta_core, nullptr, sc, plan, s, true));
  return prune_impl<float>(m, delta_factor, delta_core, pr, count_mode, 0, 0.0, n_pruned, sc, plan, s);
}

vest_status vest_iteration(const vest_index* ix, vest_model* m, int32_t reg, double lambda, double pr,
                           int32_t count_mode, int32_t factor_sweep, double* loss, double* const* delta_factor,
                           double* delta_core, int64_t* n_pruned, void* scratch, size_t scratch_bytes, void* stream) {
  VEST_TRY(check_pair(ix, m));
  VEST_TRY(check_lambda(lambda));
  if (reg != VEST_REG_LF && reg != VEST_REG_L1) return fail(VEST_ERR_INVALID, "unknown regulariser");
  if (!loss) return fail(VEST_ERR_INVALID, "loss is NULL");
  if (!(pr >= 0.0) || pr > 1.0) return fail(VEST_ERR_INVALID, "pr must be in [0, 1]");
  const bool resp = delta_factor != nullptr;
  if (resp != (delta_core != nullptr)) return fail(VEST_ERR_INVALID, "delta_factor and delta_core: both or neither");
  if (resp)
    for (int n = 0; n < m->order; ++n)
      if (!delta_factor[n]) return fail(VEST_ERR_INVALID, "delta_factor entry is NULL");
  ScratchPlan plan;
  VEST_TRY(check_scratch(ix, m, scratch, scratch_bytes, &plan));
  VEST_TRY(iteration_sweeps(ix, m, reg, lambda, factor_sweep, loss, scratch, scratch_bytes, plan, stream));
  if (!resp) return VEST_OK;
  return iteration_prune(ix, m, loss, pr, count_mode, delta_factor, delta_core, n_pruned,
                         static_cast<char*>(scratch), plan, as_stream(stream));
}

static vest_status prune_checked(vest_model* m, double* const* delta_factor, const double* delta_core, double pr,
                                 int32_t count_mode, int32_t threshold_mode, double tau, int64_t* n_pruned, char* sc,
                                 const ScratchPlan& plan, cudaStream_t s) {
  if (m->dtype == VEST_F64)
    return prune_impl<double>(m, delta_factor, delta_core, pr, count_mode, threshold_mode, tau, n_pruned, sc, plan, s);
  return prune_impl<float>(m, delta_factor, delta_core, pr, count_mode, threshold_mode, tau, n_pruned, sc, plan, s);
}

vest_status vest_prune(vest_model* m, double* const* delta_factor, const double* delta_core, double pr,
                       int32_t count_mode, int32_t threshold_mode, double tau, int64_t* n_pruned, void* scratch,
                       size_t scratch_bytes, void* stream) {
  VEST_TRY(check_model(m));
  if (!delta_factor || !delta_core) return fail(VEST_ERR_INVALID, "delta inputs are NULL");
  for (int n = 0; n < m->order; ++n)
    if (!delta_factor[n]) return fail(VEST_ERR_INVALID, "delta_factor entry is NULL");
  if (!threshold_mode && (!(pr >= 0.0) || pr > 1.0)) return fail(VEST_ERR_INVALID, "pr must be in [0, 1]");
  if (threshold_mode && std::isnan(tau)) return fail(VEST_ERR_INVALID, "tau is NaN");
  // the prune needs only the model shape: plan with a shape-only index stand-in
  vest_index shape{};
  shape.order = m->order;
  shape.val_dtype = m->dtype;
  shape.nnz = 0;
  for (int n = 0; n < m->order; ++n) shape.dims[n] = m->dims[n];
  const ScratchPlan plan = plan_scratch(&shape, m);
  if (!scratch) return fail(VEST_ERR_INVALID, "scratch is NULL");
  // any scratch sized for this model by vest_scratch_bytes() is large enough
  if (scratch_bytes < plan.total) return fail(VEST_ERR_WORKSPACE, "scratch too small for the prune");
  ScratchPlan p2 = plan;
  return prune_checked(m, delta_factor, delta_core, pr, count_mode, threshold_mode, tau, n_pruned,
                       static_cast<char*>(scratch), p2, as_stream(stream));
}

vest_status vest_value_keys(const vest_model* m, double* const* key_factor, double* key_core, void* stream) {
  VEST_TRY(check_model(m));
  if (!key_factor || !key_core) return fail(VEST_ERR_INVALID, "key outputs are NULL");
  for (int n = 0; n < m->order; ++n)
    if (!key_factor[n]) return fail(VEST_ERR_INVALID, "key_factor entry is NULL");
  if (m->dtype == VEST_F64) return value_keys_impl<double>(m, key_factor, key_core, as_stream(stream));
  return value_keys_impl<float>(m, key_factor, key_core, as_stream(stream));
}

vest_status vest_normalize(vest_model* m, void* scratch, size_t scratch_bytes, void* stream) {
  VEST_TRY(check_model(m));
  if (!scratch || scratch_bytes < normalize_scratch_bytes()) return fail(VEST_ERR_WORKSPACE, "scratch too small");
  if (m->dtype == VEST_F64) return normalize_impl<double>(m, static_cast<char*>(scratch), as_stream(stream));
  return normalize_impl<float>(m, static_cast<char*>(scratch), as_stream(stream));
}

vest_status vest_count_zeros(const vest_model* m, int64_t* out, void* scratch, size_t scratch_bytes, void* stream) {
  (void)scratch_bytes;
  VEST_TRY(check_model(m));
  if (!out) return fail(VEST_ERR_INVALID, "out is NULL");
  if (m->dtype == VEST_F64) return count_zeros_impl<double>(m, out, static_cast<char*>(scratch), as_stream(stream));
  return count_zeros_impl<float>(m, out, static_cast<char*>(scratch), as_stream(stream));
}

vest_status vest_reconstruct(const vest_model* m, const int32_t* q_idx, int64_t count, void* out, void* stream) {
  VEST_TRY(check_model(m));
  if (count < 0) return fail(VEST_ERR_INVALID, "count < 0");
  if (count > 0 && (!q_idx || !out)) return fail(VEST_ERR_INVALID, "q_idx or out is NULL");
  if (m->dtype == VEST_F64) return reconstruct_impl<double>(m, q_idx, count, static_cast<double*>(out), as_stream(stream));
  return reconstruct_impl<float>(m, q_idx, count, static_cast<float*>(out), as_stream(stream));
}

size_t vest_autosearch_scratch_bytes(const vest_index* ix, const vest_model* m) {
  if (check_pair(ix, m) != VEST_OK) return 0;
  int64_t total_elems = 1;
  for (int n = 0; n < m->order; ++n) total_elems *= m->ranks[n];
  for (int n = 0; n < m->order; ++n) total_elems += m->dims[n] * m->ranks[n];
  return plan_scratch(ix, m).total + align_up((size_t)total_elems * 8) + align_up((size_t)total_elems);
}

vest_status vest_autosearch(const vest_index* ix, vest_model* m, const vest_params* p, vest_report* rep, void* scratch,
                            size_t scratch_bytes, void* stream) {
  VEST_TRY(check_pair(ix, m));
  if (!p || !rep) return fail(VEST_ERR_INVALID, "params or report is NULL");
  VEST_TRY(check_lambda(p->lambda));
  if (p->max_iter < 1 || p->max_iter > 256) return fail(VEST_ERR_INVALID, "max_iter must be in [1, 256]");
  if (p->reg != VEST_REG_LF && p->reg != VEST_REG_L1) return fail(VEST_ERR_INVALID, "unknown regulariser");
  ScratchPlan plan;
  VEST_TRY(check_scratch(ix, m, scratch, scratch_bytes, &plan));
  const cudaStream_t s = as_stream(stream);
  char* sc = static_cast<char*>(scratch);
  if (p->resume && (rep->iters < 0 || rep->iters > 256)) return fail(VEST_ERR_INVALID, "resumed report: iters must be in [0, 256]");
  if (!p->resume) std::memset(rep, 0, sizeof(*rep));
  double* loss = reinterpret_cast<double*>(sc + plan.off_small) + kSmallLoss;
  int64_t* zeros = reinterpret_cast<int64_t*>(reinterpret_cast<double*>(sc + plan.off_small) + kSmallZeros);
  // the Delta scores of every element follow the planned regions of the scratch
  int64_t total_elems = 1;
  for (int n = 0; n < m->order; ++n) total_elems *= m->ranks[n];
  const int64_t gs = total_elems;
  for (int n = 0; n < m->order; ++n) total_elems += m->dims[n] * m->ranks[n];
  const bool revive = p->revive_on_stop != 0 && p->target_sparsity < 0.0;
  const size_t need = plan.total + align_up((size_t)total_elems * 8) + (revive ? align_up((size_t)total_elems) : 0);
  if (scratch_bytes < need) return fail(VEST_ERR_WORKSPACE, "auto-search scratch smaller than vest_autosearch_scratch_bytes()");
  // the masks before the latest pruning step (revive_on_stop), segment after segment
  uint8_t* saved = reinterpret_cast<uint8_t*>(sc + plan.total + align_up((size_t)total_elems * 8));
  auto copy_masks = [&](bool save) -> vest_status {
    uint8_t* at = saved;
    for (int n = 0; n <= m->order; ++n) {
      const size_t sz = n < m->order ? (size_t)(m->dims[n] * m->ranks[n]) : (size_t)gs;
      uint8_t* mk = n < m->order ? m->factor_mask[n] : m->core_mask;
      VEST_CUDA(cudaMemcpyAsync(save ? at : mk, save ? mk : at, sz, cudaMemcpyDeviceToDevice, s));
      at += sz;
    }
    return VEST_OK;
  };
  bool have_saved = false;
  double* dbase = reinterpret_cast<double*>(sc + plan.total);
  double* dfac[VEST_MAX_ORDER];
  double* dptr = dbase;
  for (int n = 0; n < m->order; ++n) {
    dfac[n] = dptr;
    dptr += m->dims[n] * m->ranks[n];
  }
  double* dcore = dptr;
  const double total_size = (double)total_elems;
  auto sparsity = [&](double* out_sp) -> vest_status {
    VEST_TRY(vest_count_zeros(m, zeros, sc, scratch_bytes, stream));
    int64_t hz[VEST_MAX_ORDER + 1];
    VEST_CUDA(cudaMemcpyAsync(hz, zeros, (size_t)(m->order + 1) * 8, cudaMemcpyDeviceToHost, s));
    VEST_CUDA(cudaStreamSynchronize(s));
    int64_t z = 0;
    for (int n = 0; n <= m->order; ++n) z += hz[n];
    *out_sp = (double)z / total_size;
    return VEST_OK;
  };
  bool pruning = p->resume ? rep->stop_iter == 0 : true;
  for (int it = p->resume ? rep->iters + 1 : 1; it <= p->max_iter; ++it) {
    // the sweeps leave the residual of the swept model in the scratch: the loss and, when
    // this iteration prunes, the responsibility read it instead of recomputing B
    VEST_TRY(iteration_sweeps(ix, m, p->reg, p->lambda, 1, loss, scratch, scratch_bytes, plan, stream));
    double hl[5];
    VEST_CUDA(cudaMemcpyAsync(hl, loss, sizeof(hl), cudaMemcpyDeviceToHost, s));
    VEST_CUDA(cudaStreamSynchronize(s));
    if (!std::isfinite(hl[3])) return fail(VEST_ERR_NUMERIC, "objective is not finite");
    const int h = it - 1;
    rep->iters = it;
    rep->re_hist[h] = hl[4];
    rep->obj_hist[h] = hl[3];
    if (pruning) {
      const double pr = p->fixed_pr_mode ? p->fixed_pr : std::min(p->init_pr * it, p->max_pr);
      if (p->target_sparsity >= 0.0) {
        double sp;
        VEST_TRY(sparsity(&sp));
        if (sp >= p->target_sparsity) pruning = false;
      } else if (it >= 3 && (!p->elbow_rise || hl[4] > rep->re_hist[h - 1]) &&
                 (hl[4] + rep->re_hist[h - 2] - 2.0 * rep->re_hist[h - 1]) / pr > p->elbow_thresh) {
        pruning = false;
      }
      if (!pruning) {
        rep->stop_iter = it;
        if (revive && have_saved) VEST_TRY(copy_masks(false));
      } else {
        if (revive) VEST_TRY(copy_masks(true));
        have_saved = revive;
        VEST_TRY(iteration_prune(ix, m, loss, pr, p->count_mode, dfac, dcore, nullptr, sc, plan, s));
        rep->pr_hist[h] = pr;
      }
    }
    double sp;
    VEST_TRY(sparsity(&sp));
    rep->sparsity_hist[h] = sp;
    if (!pruning && it > 1 && std::fabs(rep->re_hist[h - 1] - rep->re_hist[h]) <= p->conv_tol * rep->re_hist[h - 1]) break;
  }
  if (p->normalize) VEST_TRY(vest_normalize(m, scratch, scratch_bytes, stream));
  double sp;
  VEST_TRY(sparsity(&sp));
  rep->final_sparsity = sp;
  return VEST_OK;
}

}  // extern "C"
