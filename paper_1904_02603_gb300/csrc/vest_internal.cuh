// Internal declarations shared by the libvest translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "vest.h"

namespace vest {

constexpr int kMaxOrder = VEST_MAX_ORDER;
constexpr int kMaxRank = VEST_MAX_RANK;

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
vest_status fail(vest_status st, const std::string& msg);
vest_status cuda_fail(cudaError_t e, const char* what);

#define VEST_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e__ = (call);                             \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call); \
  } while (0)

// Every kernel launch site is followed by VEST_LAUNCH (or VEST_LAUNCH_N when
// one check covers n launches): it checks the launch and counts it.
void count_launches(int n);

#define VEST_LAUNCH_N(what, n)                                 \
  do {                                                         \
    count_launches(n);                                         \
    cudaError_t e__ = cudaGetLastError();                      \
    if (e__ != cudaSuccess) return cuda_fail(e__, what);       \
  } while (0)
#define VEST_LAUNCH(what) VEST_LAUNCH_N(what, 1)

#define VEST_TRY(...)                   \
  do {                                  \
    vest_status s__ = (__VA_ARGS__);    \
    if (s__ != VEST_OK) return s__;     \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ------------------------------------------------------------------ index
struct ModeIndex {
  int64_t* row_ptr;  // [I_n + 1]
  int32_t* perm;     // [nnz]
  int32_t* oidx;     // [(N-1)][nnz], other modes ascending
  void* val;         // [nnz]
  int64_t* nzptr;    // [cap + 1]
  int32_t* nzrow;    // [cap]
  int32_t* nnzrows;  // device scalar R_n
  int32_t* gran;     // [ceil(nnz/32) + 1]: non-empty-row number k holding position 32 g
  int32_t* rowk;     // [nnz]: non-empty-row number of every position
  int64_t cap;       // min(I_n, nnz)
};

}  // namespace vest

struct vest_index {
  int32_t order;
  int32_t val_dtype;
  int64_t dims[VEST_MAX_ORDER];
  int64_t nnz;
  vest::ModeIndex mode[VEST_MAX_ORDER];
  size_t ws_bytes;
};

namespace vest {

// x rounded to the nearest value with a 24-bit significand, ties to even (IEEE 754
// round-to-nearest at single precision), by integer operations on the FP64 bit pattern:
// the result equals (double)(float)x wherever that is a normal float.  Outside that range
// (zero, float subnormals, overflow, inf, NaN) the conversion itself is used.
__device__ __forceinline__ double round_to_single(double x) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
  const int e = (int)((bits >> 52) & 0x7FF);
  if (e < 1023 - 126 || e >= 1023 + 127) return (double)(float)x;
  const unsigned long long lsb = (bits >> 29) & 1ull;
  return __longlong_as_double(static_cast<long long>((bits + 0x0FFFFFFFull + lsb) & ~0x1FFFFFFFull));
}

// ------------------------------------------------------------------ device views
template <typename T>
struct DevModel {
  int32_t N;
  int32_t J[kMaxOrder];
  int64_t I[kMaxOrder];
  T* A[kMaxOrder];
  uint8_t* mask[kMaxOrder];
  T* G;
  uint8_t* Gmask;
  int64_t gsize;
};

template <typename T>
inline DevModel<T> dev_model(const vest_model* m) {
  DevModel<T> d{};
  d.N = m->order;
  d.gsize = 1;
  for (int n = 0; n < m->order; ++n) {
    d.J[n] = m->ranks[n];
    d.I[n] = m->dims[n];
    d.A[n] = static_cast<T*>(m->factor[n]);
    d.mask[n] = m->factor_mask[n];
    d.gsize *= m->ranks[n];
  }
  d.G = static_cast<T*>(m->core);
  d.Gmask = m->core_mask;
  return d;
}

// Per-mode CSR view handed to kernels.
template <typename T>
struct DevMode {
  const int64_t* nzptr;
  const int32_t* nzrow;
  const int32_t* nnzrows;
  const int32_t* gran;
  const int32_t* rowk;
  const int32_t* oidx;  // [(N-1)][nnz]
  const T* val;
  const int32_t* perm;
  int64_t nnz;
};

template <typename T>
inline DevMode<T> dev_mode(const vest_index* ix, int n) {
  DevMode<T> d;
  const ModeIndex& mi = ix->mode[n];
  d.nzptr = mi.nzptr;
  d.nzrow = mi.nzrow;
  d.nnzrows = mi.nnzrows;
  d.gran = mi.gran;
  d.rowk = mi.rowk;
  d.oidx = mi.oidx;
  d.val = static_cast<const T*>(mi.val);
  d.perm = mi.perm;
  d.nnz = ix->nnz;
  return d;
}

// ------------------------------------------------------------------ scratch layout
// Scratch is carved into fixed regions; every compute call validates the size.
struct ScratchPlan {
  size_t total;
  size_t off_status, off_gperm, off_spill, off_spanning, off_resid, off_resid_coo, off_part, off_small;
  size_t off_prune_keys, off_prune_vals, off_prune_tmp;
  size_t off_core;  // core-sweep region: per-piece gram statistics, block Grams, partial sums
  size_t off_rowbuf;  // factor sweep: FP64 sums of every non-empty row of one mode
  size_t gperm_bytes, spill_bytes, part_bytes, rowbuf_bytes;
  int task;        // alpha per task in the factor sweep
  int64_t ntasks;  // factor-sweep tasks per mode
};

ScratchPlan plan_scratch(const vest_index* ix, const vest_model* m);

// ------------------------------------------------------------------ helpers
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

int num_sms();

// Largest dynamic shared memory `kern` may take: the device's opt-in maximum per CTA (227 KB
// on sm_103) less the kernel's static shared memory; looked up once per kernel and device.
vest_status max_dynamic_smem(const void* kern, size_t* out);

// Lets `kern` launch with dynamic shared memory up to that maximum; `need` is what the coming
// launch asks for (checked against it).  The attribute is set to the one fixed maximum, never
// to `need`: host threads that launch the same kernel with different sizes at the same time
// then cannot narrow the bound under each other's launches.
template <typename K>
inline vest_status allow_smem(K kern, size_t need) {
  size_t cap = 0;
  VEST_TRY(max_dynamic_smem(reinterpret_cast<const void*>(kern), &cap));
  if (need > cap) return fail(VEST_ERR_UNSUPPORTED, "a kernel needs more shared memory than a CTA may have");
  VEST_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
  return VEST_OK;
}

// Argument checks shared by every entry point that takes an index and a model:
// order, dtype, ranks, dims, pointers and the size limits of the library.
vest_status check_pair(const vest_index* ix, const vest_model* m);

// Generic device scans (exclusive) used by the index build and the prune.
vest_status exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp, cudaStream_t s);
vest_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s);
size_t scan_tmp_elems(int64_t n);

// Stable LSD radix sort of (key, value) pairs; `bits` low bits of the key are significant.
template <typename K>
vest_status radix_sort_pairs(K* keys, int32_t* vals, K* keys_alt, int32_t* vals_alt, int64_t n, int bits,
                             int32_t* hist, int32_t* scan_tmp, bool* result_in_alt, cudaStream_t s);
size_t radix_hist_elems(int64_t n);

// Status bits the factor-sweep kernels raise instead of trapping (bit 0: a bounded wait
// on the tensor cores gave up); reads them after a device synchronise, clears on request.
vest_status sweep_device_status(uint32_t* flags, bool clear);
// The same for the tensor-core loss kernel (bit 1); no synchronise of its own.
vest_status loss_device_status(uint32_t* flags, bool clear);

// Whether the tensor-core delta of the FP32 factor sweep serves mode n of this model.
bool sweep_tc_applies(const vest_model* m, int n);

// Operations implemented in their own translation units.
template <typename T>
vest_status sweep_factors_mode(const vest_index* ix, const vest_model* m, int reg, double lambda, int mode,
                               char* scratch, const ScratchPlan& plan, cudaStream_t s, int path = VEST_DELTA_AUTO);
template <typename T>
vest_status responsibility_factors(const vest_index* ix, const vest_model* m, const double* stats,
                                   double* const* delta_factor, double* const* resp_factor, char* scratch,
                                   const ScratchPlan& plan, cudaStream_t s);
template <typename T>
vest_status loss_impl(const vest_index* ix, const vest_model* m, int reg, double lambda, double* out,
                      T* resid_csr0, T* resid_coo, char* scratch, const ScratchPlan& plan, cudaStream_t s);
// With final_loss set, the core sweep also applies the last block's change to the residual,
// stores the residual in COO order and writes the five loss values of the swept model
// there (device, FP64): the residual then serves the responsibility without a new pass.
template <typename T>
vest_status sweep_core_impl(const vest_index* ix, const vest_model* m, int reg, double lambda, char* scratch,
                            const ScratchPlan& plan, cudaStream_t s, double* final_loss = nullptr);
template <typename T>
vest_status loss_finish(const vest_model* m, int reg, double lambda, int nl, double* out, char* scratch,
                        const ScratchPlan& plan, cudaStream_t s);
int loss_ctas();
// grams_valid: a core sweep with the current factors ran last, so its block Grams hold diag M.
template <typename T>
vest_status core_responsibility(const vest_index* ix, const vest_model* m, const T* resid_csr0,
                                const double* stats, double* delta_core, double* resp_core, char* scratch,
                                const ScratchPlan& plan, cudaStream_t s, bool grams_valid = false);
template <typename T>
vest_status prune_impl(const vest_model* m, double* const* delta_factor, const double* delta_core, double pr,
                       int count_mode, int threshold_mode, double tau, int64_t* n_pruned, char* scratch,
                       const ScratchPlan& plan, cudaStream_t s);
template <typename T>
vest_status value_keys_impl(const vest_model* m, double* const* key_factor, double* key_core, cudaStream_t s);
template <typename T>
vest_status normalize_impl(const vest_model* m, char* scratch, cudaStream_t s);
template <typename T>
vest_status count_zeros_impl(const vest_model* m, int64_t* out, char* scratch, cudaStream_t s);
template <typename T>
vest_status reconstruct_impl(const vest_model* m, const int32_t* q_idx, int64_t count, T* out, cudaStream_t s);

vest_status build_index_impl(const vest_tensor* t, void* ws, size_t ws_bytes, vest_index* ix, cudaStream_t s);
size_t index_workspace_bytes(const vest_tensor* t);

}  // namespace vest
