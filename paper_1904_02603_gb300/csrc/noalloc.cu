// vest_loss_noalloc: the loss of vest_loss() without a caller-provided scratch
// buffer.  Its scratch is a fixed array in the library's device memory, so the
// call allocates nothing: no cudaMalloc, no cudaFree, no allocating library
// routine.  The array exists once per device that loads the library and lives
// until the process exits.
#include <dlfcn.h>

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
unsigned long long g_noalloc_ctx[kMaxDevices] = {0};

// Identity of the calling thread's current CUDA context, from the driver library the
// runtime has already loaded (looked up by name, so libvest needs no link-time driver
// dependency).  cuCtxGetId gives an id that is never reused within the process; without
// it the context handle itself serves.  0 when neither can be read.
using CtxGetCurrentFn = int (*)(void**);
using CtxGetIdFn = int (*)(void*, unsigned long long*);
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* h = dlopen("libcuda.so.1", RTLD_LAZY | RTLD_NOLOAD);
    if (!h) return;
    get_current = reinterpret_cast<CtxGetCurrentFn>(dlsym(h, "cuCtxGetCurrent"));
    get_id = reinterpret_cast<CtxGetIdFn>(dlsym(h, "cuCtxGetId"));
  });
  if (!get_current) return 0;
  void* ctx = nullptr;
  if (get_current(&ctx) != 0 || !ctx) return 0;
  unsigned long long id = 0;
  if (get_id && get_id(ctx, &id) == 0) return id + 1;
  return reinterpret_cast<unsigned long long>(ctx);
}

// Device address of the array for the current device.  The symbol's name is a
// host-side stand-in, not a device address, so the address is looked up with that
// device current and kept for the device's context.  When the context changes (after a
// cudaDeviceReset, say) the array lives at a new address and the lookup runs again.
vest_status noalloc_base(char** out) {
  int dev = 0;
  VEST_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(VEST_ERR_UNSUPPORTED, "device ordinal beyond 63");
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev] || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
    void* p = nullptr;
    VEST_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));  // binds the device's context to this thread
    g_noalloc_ptr[dev] = static_cast<char*>(p);
    g_noalloc_ctx[dev] = ctx != 0 ? ctx : current_context_id();
  }
  *out = g_noalloc_ptr[dev];
  return VEST_OK;
}
}  // namespace

}  // namespace vest

using namespace vest;

extern "C" vest_status vest_loss_noalloc(const vest_index* ix, const vest_model* m, int32_t reg, double lambda,
                                         double* out, void* resid, void* stream) {
  // the same checks as vest_loss, so both entry points accept exactly the same inputs
  VEST_TRY(check_pair(ix, m));
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return fail(VEST_ERR_INVALID, "lambda must be finite and >= 0");
  if (reg != VEST_REG_LF && reg != VEST_REG_L1) return fail(VEST_ERR_INVALID, "unknown regulariser");
  if (!out) return fail(VEST_ERR_INVALID, "out is NULL");
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
