// Pruning with the marking table (Section 3.4; last step of Algorithm 3).
// Per segment (each A^(n), then G): every unpruned element gets an
// order-preserving 64-bit key of its Delta (-0 read as +0), pruned ones the
// largest key; a stable radix sort of (key, linear index) puts the candidates
// in (Delta, index) order; the first k = floor(pr * #candidates) (or
// floor(pr * size)) are marked and zeroed.  Integer work only after the key
// map, so the selected set is exact.
#include <algorithm>

#include "vest_internal.cuh"

namespace vest {

__device__ __forceinline__ uint64_t delta_key(double d) {
  if (d == 0.0) d = 0.0;  // -0 -> +0
  const uint64_t u = (uint64_t)__double_as_longlong(d);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void prune_keys_kernel(const double* __restrict__ delta, const uint8_t* __restrict__ mask, int64_t size,
                                  uint64_t* __restrict__ keys, int32_t* __restrict__ vals, int32_t* __restrict__ nan_flag,
                                  unsigned long long* __restrict__ ncand) {
  unsigned long long c = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < size; e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = ~0ull;
    if (!mask[e]) {
      const double d = delta[e];
      if (isnan(d)) *nan_flag = 1;
      k = delta_key(d);
      ++c;
    }
    keys[e] = k;
    vals[e] = (int32_t)e;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(ncand, c);
}

template <typename T>
__global__ void prune_mark_kernel(const int32_t* __restrict__ order, int64_t size, const unsigned long long* __restrict__ ncand,
                                  const int32_t* __restrict__ nan_flag, double pr, int count_mode, uint8_t* __restrict__ mask,
                                  T* __restrict__ val, int64_t* __restrict__ n_pruned) {
  if (*nan_flag) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && n_pruned) *n_pruned = -1;
    return;
  }
  const int64_t nc = (int64_t)*ncand;
  int64_t k = (int64_t)floor(pr * (double)(count_mode ? size : nc));
  if (k > nc) k = nc;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < k; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = order[p];
    mask[e] = 1;
    val[e] = T(0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && n_pruned) *n_pruned = k;
}

template <typename T>
__global__ void prune_threshold_kernel(const double* __restrict__ delta, int64_t size, double tau, uint8_t* __restrict__ mask,
                                       T* __restrict__ val, unsigned long long* __restrict__ cnt) {
  unsigned long long c = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < size; e += (int64_t)gridDim.x * blockDim.x) {
    if (!mask[e] && delta[e] < tau) {
      mask[e] = 1;
      val[e] = T(0);
      ++c;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

__global__ void copy_count_kernel(const unsigned long long* __restrict__ c, int64_t* __restrict__ out) { *out = (int64_t)*c; }

template <typename T>
vest_status prune_impl(const vest_model* m, double* const* delta_factor, const double* delta_core, double pr,
                       int count_mode, int threshold_mode, double tau, int64_t* n_pruned, char* scratch,
                       const ScratchPlan& plan, cudaStream_t s) {
  const DevModel<T> M = dev_model<T>(m);
  int64_t maxseg = M.gsize;
  for (int n = 0; n < M.N; ++n) maxseg = std::max<int64_t>(maxseg, M.I[n] * M.J[n]);
  char* base = scratch + plan.off_prune_keys;
  uint64_t* ka = reinterpret_cast<uint64_t*>(base);
  uint64_t* kb = ka + maxseg;
  int32_t* va = reinterpret_cast<int32_t*>(scratch + plan.off_prune_vals);
  int32_t* vb = va + maxseg;
  char* tmp = scratch + plan.off_prune_tmp;
  int32_t* flags = reinterpret_cast<int32_t*>(tmp);                       // [0]: nan flag
  unsigned long long* ncand = reinterpret_cast<unsigned long long*>(tmp + 64);
  int32_t* hist = reinterpret_cast<int32_t*>(tmp + 256);
  int32_t* scan_tmp = hist + radix_hist_elems(maxseg);
  for (int seg = 0; seg <= M.N; ++seg) {
    const bool core = seg == M.N;
    const int64_t size = core ? M.gsize : M.I[seg] * M.J[seg];
    uint8_t* mask = core ? M.Gmask : M.mask[seg];
    T* val = core ? M.G : M.A[seg];
    const double* dl = core ? delta_core : delta_factor[seg];
    int64_t* np = n_pruned ? n_pruned + seg : nullptr;
    const int grid = std::max(1, std::min<int>((int)ceil_div(size, 256), num_sms() * 8));
    VEST_CUDA(cudaMemsetAsync(tmp, 0, 256, s));
    if (threshold_mode) {
      prune_threshold_kernel<T><<<grid, 256, 0, s>>>(dl, size, tau, mask, val, ncand);
      VEST_LAUNCH("prune_threshold");
      if (np) {
        copy_count_kernel<<<1, 1, 0, s>>>(ncand, np);
        VEST_LAUNCH("copy_count");
      }
      continue;
    }
    prune_keys_kernel<<<grid, 256, 0, s>>>(dl, mask, size, ka, va, flags, ncand);
    VEST_LAUNCH("prune_keys");
    bool in_alt = false;
    VEST_TRY(radix_sort_pairs<uint64_t>(ka, va, kb, vb, size, 64, hist, scan_tmp, &in_alt, s));
    prune_mark_kernel<T><<<grid, 256, 0, s>>>(in_alt ? vb : va, size, ncand, flags, pr, count_mode, mask, val, np);
    VEST_LAUNCH("prune_mark");
  }
  return VEST_OK;
}

size_t prune_scratch_bytes(int64_t maxseg, size_t* keys_bytes, size_t* vals_bytes, size_t* tmp_bytes) {
  *keys_bytes = align_up((size_t)std::max<int64_t>(maxseg, 1) * 16);
  *vals_bytes = align_up((size_t)std::max<int64_t>(maxseg, 1) * 8);
  *tmp_bytes = align_up(256 + radix_hist_elems(maxseg) * 4 + scan_tmp_elems((int64_t)radix_hist_elems(maxseg)) * 8);
  return *keys_bytes + *vals_bytes + *tmp_bytes;
}

template vest_status prune_impl<float>(const vest_model*, double* const*, const double*, double, int, int, double,
                                       int64_t*, char*, const ScratchPlan&, cudaStream_t);
template vest_status prune_impl<double>(const vest_model*, double* const*, const double*, double, int, int, double,
                                        int64_t*, char*, const ScratchPlan&, cudaStream_t);

}  // namespace vest
