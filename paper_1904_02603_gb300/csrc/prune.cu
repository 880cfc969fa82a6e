// Pruning with the marking table (Section 3.3; the pruning step of Algorithm 3).
// Per segment (each A^(n), then G) the unpruned elements are ordered by
// (Delta, linear index) and the first k = floor(pr * #candidates) (or
// floor(pr * size)) are marked and zeroed.  The k-th pair is found by a radix
// select on the 96-bit composite (order-preserving 64-bit key of Delta, with
// -0 read as +0; 32-bit index): nine histogram passes of 11-bit digits, most
// significant first, each narrowing the prefix of the k-th pair; the last CTA
// of a pass (atomic ticket) picks the digit.  A final pass marks every
// candidate whose pair is not above the selected one.  Integer work only after
// the key map, so the selected set is exact.
#include <algorithm>

#include "vest_internal.cuh"

namespace vest {

constexpr int kSelBits = 11;
constexpr int kSelBins = 1 << kSelBits;
constexpr int kSelPasses = 9;  // 96 bits: 8 x 11 + 8

struct SelectState {
  unsigned long long pkey;  // selected prefix: key bits
  unsigned int pidx;        // selected prefix: index bits
  unsigned int ticket;
  long long krem;           // rank of the k-th pair inside the current prefix (1-based)
  long long k;
  unsigned long long ncand;
  int done;                 // 1: nothing (more) to select
  int nan;
  unsigned int hist[kSelBins];
};

// Every segment of one prune in one launch: blockIdx.y is the segment, each with its own
// select state (the segments are independent, so 4 launches a pass become one).
struct PruneSegs {
  const double* delta[kMaxOrder + 1];
  uint8_t* mask[kMaxOrder + 1];
  void* val[kMaxOrder + 1];
  int64_t size[kMaxOrder + 1];
  int64_t* np[kMaxOrder + 1];
};

__device__ __forceinline__ uint64_t delta_key(double d) {
  if (d == 0.0) d = 0.0;  // -0 -> +0
  const uint64_t u = (uint64_t)__double_as_longlong(d);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// bits [lo, hi) of the composite key * 2^32 + idx
__device__ __forceinline__ unsigned sel_digit(uint64_t key, uint32_t idx, int lo, int hi) {
  const unsigned mask = (1u << (hi - lo)) - 1u;
  if (lo >= 32) return (unsigned)(key >> (lo - 32)) & mask;
  if (hi <= 32) return (idx >> lo) & mask;
  return (unsigned)((key << (32 - lo)) | (uint64_t)(idx >> lo)) & mask;
}

// the composite agrees with the prefix on every bit >= hi
__device__ __forceinline__ bool sel_match(uint64_t key, uint32_t idx, uint64_t pkey, uint32_t pidx, int hi) {
  if (hi >= 96) return true;
  if (hi >= 32) return (key >> (hi - 32)) == (pkey >> (hi - 32));
  return key == pkey && (idx >> hi) == (pidx >> hi);
}

__host__ __device__ constexpr int sel_hi(int pass) { return 96 - kSelBits * pass; }
__host__ __device__ constexpr int sel_lo(int pass) { return sel_hi(pass) - kSelBits > 0 ? sel_hi(pass) - kSelBits : 0; }

// One histogram pass of segment blockIdx.y.  Pass 0 also counts the candidates and looks for
// NaN; its last CTA turns pr into k.  The last CTA of every pass picks the digit of the k-th
// pair and clears the histogram for the next pass.
__global__ void __launch_bounds__(256) prune_select_kernel(PruneSegs ps, int pass, double pr, int count_mode,
                                                           SelectState* st_all) {
  const int seg = blockIdx.y;
  const double* __restrict__ delta = ps.delta[seg];
  const uint8_t* __restrict__ mask = ps.mask[seg];
  const int64_t size = ps.size[seg];
  int64_t* __restrict__ n_pruned = ps.np[seg];
  SelectState* st = st_all + seg;
  __shared__ unsigned sh[kSelBins];
  __shared__ unsigned long long s_cand;
  __shared__ int s_nan, s_last;
  __shared__ unsigned s_part[256];
  if (pass > 0 && st->done) return;  // uniform: written by the previous launch
  const int hi = sel_hi(pass), lo = sel_lo(pass);
  const uint64_t pkey = st->pkey;
  const uint32_t pidx = st->pidx;
  for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) sh[b] = 0;
  if (threadIdx.x == 0) {
    s_cand = 0;
    s_nan = 0;
  }
  __syncthreads();
  unsigned long long c = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < size; e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = ~0ull;
    if (!mask[e]) {
      const double d = delta[e];
      if (pass == 0) {
        ++c;
        if (isnan(d)) s_nan = 1;
      }
      key = delta_key(d);
    }
    if (sel_match(key, (uint32_t)e, pkey, pidx, hi)) atomicAdd(&sh[sel_digit(key, (uint32_t)e, lo, hi)], 1u);
  }
  if (pass == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s_cand, c);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kSelBins; b += blockDim.x)
    if (sh[b]) atomicAdd(&st->hist[b], sh[b]);
  if (threadIdx.x == 0) {
    if (pass == 0) {
      if (s_cand) atomicAdd(&st->ncand, s_cand);
      if (s_nan) atomicExch(&st->nan, 1);
    }
    __threadfence();
    s_last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last CTA: every other CTA's histogram and counts are visible
  if (threadIdx.x == 0) {
    st->ticket = 0;
    if (pass == 0) {
      const long long nc = (long long)*(volatile unsigned long long*)&st->ncand;
      long long k = (long long)floor(pr * (double)(count_mode ? size : nc));
      if (k > nc) k = nc;
      if (k < 0) k = 0;
      st->k = k;
      st->krem = k;
      if (*(volatile int*)&st->nan) {
        st->done = 1;
        if (n_pruned) *n_pruned = -1;
      } else if (k == 0) {
        st->done = 1;
        if (n_pruned) *n_pruned = 0;
      }
    }
  }
  __syncthreads();
  const int done = *(volatile int*)&st->done;
  // per-thread chunk of 8 bins, block-wide exclusive scan of the chunk sums
  constexpr int kPer = kSelBins / 256;
  unsigned loc[kPer];
  unsigned tot = 0;
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    loc[i] = *(volatile unsigned*)&st->hist[threadIdx.x * kPer + i];
    tot += loc[i];
  }
  s_part[threadIdx.x] = tot;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    const unsigned v = threadIdx.x >= o ? s_part[threadIdx.x - o] : 0u;
    __syncthreads();
    s_part[threadIdx.x] += v;
    __syncthreads();
  }
  if (!done) {
    const long long krem = *(volatile long long*)&st->krem;
    long long cum = (long long)(s_part[threadIdx.x] - tot);  // exclusive
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      if (cum < krem && krem <= cum + (long long)loc[i]) {
        const unsigned b = (unsigned)(threadIdx.x * kPer + i);
        // prefix |= b << lo within the 96-bit composite
        if (lo >= 32) {
          st->pkey = pkey | ((uint64_t)b << (lo - 32));
        } else if (hi <= 32) {
          st->pidx = pidx | (b << lo);
        } else {
          st->pkey = pkey | ((uint64_t)b >> (32 - lo));
          st->pidx = pidx | (b << lo);
        }
        st->krem = krem - cum;
      }
      cum += loc[i];
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) st->hist[b] = 0;
}

// Marks every candidate whose (key, index) is not above the selected pair: exactly k
// (segment blockIdx.y).
template <typename T>
__global__ void prune_mark_kernel(PruneSegs ps, const SelectState* st_all) {
  const int seg = blockIdx.y;
  const double* __restrict__ delta = ps.delta[seg];
  uint8_t* __restrict__ mask = ps.mask[seg];
  T* __restrict__ val = static_cast<T*>(ps.val[seg]);
  const int64_t size = ps.size[seg];
  int64_t* __restrict__ n_pruned = ps.np[seg];
  const SelectState* st = st_all + seg;
  if (st->done) return;
  const uint64_t pkey = st->pkey;
  const uint32_t pidx = st->pidx;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < size; e += (int64_t)gridDim.x * blockDim.x) {
    if (mask[e]) continue;
    const uint64_t key = delta_key(delta[e]);
    if (key < pkey || (key == pkey && (uint32_t)e <= pidx)) {
      mask[e] = 1;
      val[e] = T(0);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && n_pruned) *n_pruned = st->k;
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
  char* tmp = scratch + plan.off_prune_tmp;
  SelectState* st = reinterpret_cast<SelectState*>(tmp);
  unsigned long long* cnt =
      reinterpret_cast<unsigned long long*>(tmp + align_up((size_t)(kMaxOrder + 1) * sizeof(SelectState)));
  if (!threshold_mode) {
    PruneSegs ps{};
    int grid = 1;
    for (int seg = 0; seg <= M.N; ++seg) {
      const bool core = seg == M.N;
      const int64_t size = core ? M.gsize : M.I[seg] * M.J[seg];
      if (size > 0xFFFFFFFFll) return fail(VEST_ERR_UNSUPPORTED, "prune: a segment holds 2^32 elements or more");
      ps.delta[seg] = core ? delta_core : delta_factor[seg];
      ps.mask[seg] = core ? M.Gmask : M.mask[seg];
      ps.val[seg] = core ? M.G : M.A[seg];
      ps.size[seg] = size;
      ps.np[seg] = n_pruned ? n_pruned + seg : nullptr;
      grid = std::max(grid, std::max(1, std::min<int>((int)ceil_div(size, 256), num_sms() * 4)));
    }
    const dim3 g((unsigned)grid, (unsigned)(M.N + 1));
    VEST_CUDA(cudaMemsetAsync(st, 0, (size_t)(M.N + 1) * sizeof(SelectState), s));
    for (int pass = 0; pass < kSelPasses; ++pass) {
      prune_select_kernel<<<g, 256, 0, s>>>(ps, pass, pr, count_mode, st);
      VEST_LAUNCH("prune_select");
    }
    prune_mark_kernel<T><<<g, 256, 0, s>>>(ps, st);
    VEST_LAUNCH("prune_mark");
    return VEST_OK;
  }
  for (int seg = 0; seg <= M.N; ++seg) {
    const bool core = seg == M.N;
    const int64_t size = core ? M.gsize : M.I[seg] * M.J[seg];
    uint8_t* mask = core ? M.Gmask : M.mask[seg];
    T* val = core ? M.G : M.A[seg];
    const double* dl = core ? delta_core : delta_factor[seg];
    int64_t* np = n_pruned ? n_pruned + seg : nullptr;
    const int grid = std::max(1, std::min<int>((int)ceil_div(size, 256), num_sms() * 4));
    if (size > 0xFFFFFFFFll) return fail(VEST_ERR_UNSUPPORTED, "prune: a segment holds 2^32 elements or more");
    VEST_CUDA(cudaMemsetAsync(cnt, 0, sizeof(*cnt), s));
    prune_threshold_kernel<T><<<grid, 256, 0, s>>>(dl, size, tau, mask, val, cnt);
    VEST_LAUNCH("prune_threshold");
    if (np) {
      copy_count_kernel<<<1, 1, 0, s>>>(cnt, np);
      VEST_LAUNCH("copy_count");
    }
  }
  return VEST_OK;
}

// |value| in FP64 as the pruning key of every element: the Value Pruning baseline of the
// evaluation (Section 4.1, competitors) selects through the same (key, index) order as
// the responsibility prune.
template <typename T>
__global__ void value_keys_kernel(const T* __restrict__ v, int64_t size, double* __restrict__ key) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < size; e += (int64_t)gridDim.x * blockDim.x)
    key[e] = fabs((double)v[e]);
}

template <typename T>
vest_status value_keys_impl(const vest_model* m, double* const* key_factor, double* key_core, cudaStream_t s) {
  const DevModel<T> M = dev_model<T>(m);
  for (int seg = 0; seg <= M.N; ++seg) {
    const bool core = seg == M.N;
    const int64_t size = core ? M.gsize : M.I[seg] * M.J[seg];
    const int grid = std::max(1, std::min<int>((int)ceil_div(size, 256), num_sms() * 4));
    value_keys_kernel<T><<<grid, 256, 0, s>>>(core ? M.G : M.A[seg], size, core ? key_core : key_factor[seg]);
    VEST_LAUNCH("value_keys");
  }
  return VEST_OK;
}

size_t prune_scratch_bytes(int64_t maxseg, size_t* keys_bytes, size_t* vals_bytes, size_t* tmp_bytes) {
  (void)maxseg;
  *keys_bytes = 0;
  *vals_bytes = 0;
  *tmp_bytes = align_up((size_t)(kMaxOrder + 1) * sizeof(SelectState)) + 256;
  return *keys_bytes + *vals_bytes + *tmp_bytes;
}

template vest_status value_keys_impl<float>(const vest_model*, double* const*, double*, cudaStream_t);
template vest_status value_keys_impl<double>(const vest_model*, double* const*, double*, cudaStream_t);
template vest_status prune_impl<float>(const vest_model*, double* const*, const double*, double, int, int, double,
                                       int64_t*, char*, const ScratchPlan&, cudaStream_t);
template vest_status prune_impl<double>(const vest_model*, double* const*, const double*, double, int, int, double,
                                        int64_t*, char*, const ScratchPlan&, cudaStream_t);

}  // namespace vest
