// vest_loss_noalloc: the loss of vest_loss() without a caller-provided scratch
// buffer.  Its scratch is a fixed array in the library's device memory, so the
// call allocates nothing: no cudaMalloc, no cudaFree, no allocating library
// routine.  The array exists once per device that loads the library and lives
// until the process exits.
#include <cmath>
#include <mutex>

#include "delta.cuh"

namespace vest {

size_t loss_part_bytes();

constexpr size_t kNoAllocBytes = size_t(1) << 20;  // 1 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
char* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the array for the current device.  The symbol's name is a
// host-side stand-in, not a device address, so the address is looked up once
// per device with that device current and cached.
vest_status noalloc_base(char** out) {
  int dev = 0;
  VEST_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(VEST_ERR_UNSUPPORTED, "device ordinal beyond 63");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    VEST_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<char*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return VEST_OK;
}
}  // namespace

}  // namespace vest

using namespace vest;

extern "C" vest_status vest_loss_noalloc(const vest_index* ix, const vest_model* m, int32_t reg, double lambda,
                                         double* out, void* resid, void* stream) {
  if (!ix || !m || !out) return fail(VEST_ERR_INVALID, "index, model or out is NULL");
  if (ix->order != m->order || ix->val_dtype != m->dtype) return fail(VEST_ERR_INVALID, "index and model disagree");
  if (m->order < 2 || m->order > VEST_MAX_ORDER) return fail(VEST_ERR_INVALID, "order must be in [2, 10]");
  if (m->dtype != VEST_F64 && m->dtype != VEST_F32) return fail(VEST_ERR_INVALID, "model dtype must be F64 or F32");
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return fail(VEST_ERR_INVALID, "lambda must be finite and >= 0");
  if (reg != VEST_REG_LF && reg != VEST_REG_L1) return fail(VEST_ERR_INVALID, "unknown regulariser");
  for (int n = 0; n < m->order; ++n) {
    if (ix->dims[n] != m->dims[n]) return fail(VEST_ERR_INVALID, "index and model dims differ");
    if (m->ranks[n] < 1 || m->ranks[n] > VEST_MAX_RANK) return fail(VEST_ERR_INVALID, "rank must be in [1, 32]");
    if (!m->factor[n]) return fail(VEST_ERR_INVALID, "factor pointer is NULL");
  }
  if (!m->core) return fail(VEST_ERR_INVALID, "core pointer is NULL");
  // layout inside the fixed array: permuted mode-0 core | nonzero flags | per-block partial sums
  const ModeRoles r = mode_roles(m->ranks, m->order, 0);
  const size_t sT = m->dtype == VEST_F64 ? 8 : 4;
  const int64_t core_elems = r.n_outer * r.Jf * jn_bucket(r.Jn);
  ScratchPlan plan{};
  plan.off_gperm = 0;
  plan.gperm_bytes = align_up((size_t)core_elems * sT) + align_up((size_t)r.n_outer);
  plan.off_part = plan.gperm_bytes;
  plan.part_bytes = align_up(loss_part_bytes());
  plan.total = plan.off_part + plan.part_bytes;
  if (plan.total > kNoAllocBytes)
    return fail(VEST_ERR_WORKSPACE, "model too large for the 1 MiB fixed scratch of vest_loss_noalloc (needs " +
                                         std::to_string(plan.total) + " bytes); use vest_loss with a scratch buffer");
  char* base = nullptr;
  VEST_TRY(noalloc_base(&base));
  const cudaStream_t s = as_stream(stream);
  if (m->dtype == VEST_F64)
    return loss_impl<double>(ix, m, reg, lambda, out, nullptr, static_cast<double*>(resid), base, plan, s);
  return loss_impl<float>(ix, m, reg, lambda, out, nullptr, static_cast<float*>(resid), base, plan, s);
}
