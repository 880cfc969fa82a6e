// Mode-n index build: a stable device LSD radix sort of the observed entries by
// i_n, then the CSR pointers, the non-empty-row list and the other modes'
// indices and values gathered into that order.  These are the sets
// Omega^(n)_{i_n} that Algorithm 3 and Algorithm 4 iterate over.
#include <algorithm>
#include <cstring>

#include "vest_internal.cuh"

namespace vest {

// ============================================================== scans
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048

size_t scan_tmp_elems(int64_t n) { return (size_t)std::max<int64_t>(ceil_div(n, kScanTile), 1) + 32; }

template <typename V>
__device__ V block_exclusive_scan(V x, V* total, V* sh /* >= 32 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  V inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    V y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  if (warp == 0) {
    V w = lane < nw ? sh[lane] : V(0);
    V wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      V y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < nw) sh[lane] = wi - w;  // exclusive warp offsets
    if (lane == nw - 1) sh[32] = wi;   // block total
  }
  __syncthreads();
  V res = inc - x + sh[warp];
  *total = sh[32];
  __syncthreads();
  return res;
}

template <typename V>
__global__ void scan_reduce_kernel(const V* __restrict__ in, int64_t n, V* __restrict__ bsum) {
  __shared__ V sh[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  V acc = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t k = base + (int64_t)i * kScanThreads + threadIdx.x;
    if (k < n) acc += in[k];
  }
  V total;
  block_exclusive_scan<V>(acc, &total, sh);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// Single-block exclusive scan of bsum[0..nb) in place.
template <typename V>
__global__ void scan_spine_kernel(V* bsum, int64_t nb) {
  __shared__ V sh[33];
  V carry = 0;
  for (int64_t c = 0; c < nb; c += blockDim.x) {
    int64_t k = c + threadIdx.x;
    V x = k < nb ? bsum[k] : V(0);
    V total;
    V ex = block_exclusive_scan<V>(x, &total, sh);
    if (k < nb) bsum[k] = ex + carry;
    carry += total;
  }
}

template <typename V>
__global__ void scan_down_kernel(const V* in, V* out, int64_t n, const V* __restrict__ boff) {
  __shared__ V tile[kScanTile];
  __shared__ V sh[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t k = base + (int64_t)i * kScanThreads + threadIdx.x;
    tile[i * kScanThreads + threadIdx.x] = k < n ? in[k] : V(0);
  }
  __syncthreads();
  V loc[kScanItems];
  V sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    loc[i] = tile[threadIdx.x * kScanItems + i];
    sum += loc[i];
  }
  V total;
  V run = block_exclusive_scan<V>(sum, &total, sh) + boff[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    tile[threadIdx.x * kScanItems + i] = run;
    run += loc[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t k = base + (int64_t)i * kScanThreads + threadIdx.x;
    if (k < n) out[k] = tile[i * kScanThreads + threadIdx.x];
  }
}

template <typename V>
static vest_status exclusive_scan(const V* in, V* out, int64_t n, V* tmp, cudaStream_t s) {
  if (n <= 0) return VEST_OK;
  const int64_t nb = ceil_div(n, kScanTile);
  scan_reduce_kernel<V><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp);
  scan_spine_kernel<V><<<1, 1024, 0, s>>>(tmp, nb);
  scan_down_kernel<V><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, tmp);
  VEST_LAUNCH_N("exclusive_scan", 3);
  return VEST_OK;
}

vest_status exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp, cudaStream_t s) {
  return exclusive_scan<int32_t>(in, out, n, tmp, s);
}
vest_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s) {
  return exclusive_scan<int64_t>(in, out, n, tmp, s);
}

// ============================================================== radix sort
// Stable LSD radix sort, 8-bit digits.  Tile = 8 warps x 16 rounds x 32 items;
// within a tile, items are ranked per warp with __match_any_sync (warp w owns
// a contiguous 512-item slice), then offset by the per-warp digit counts and
// the global (digit-major, tile-minor) exclusive scan of tile histograms.
constexpr int kRsThreads = 256;
constexpr int kRsRounds = 16;
constexpr int kRsWarpItems = 32 * kRsRounds;          // 512
constexpr int kRsTile = kRsThreads * kRsRounds;       // 4096

size_t radix_hist_elems(int64_t n) { return (size_t)256 * (size_t)std::max<int64_t>(ceil_div(n, kRsTile), 1); }

template <typename K>
__global__ void radix_hist_kernel(const K* __restrict__ keys, int64_t n, int shift, int32_t* __restrict__ hist,
                                  int64_t ntiles) {
  __shared__ int32_t h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll 4
  for (int r = 0; r < kRsRounds; ++r) {
    int64_t k = base + (int64_t)r * kRsThreads + threadIdx.x;
    if (k < n) atomicAdd(&h[(int)((keys[k] >> shift) & 255u)], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

template <typename K>
__global__ void __launch_bounds__(kRsThreads) radix_scatter_kernel(const K* __restrict__ keys_in,
                                                                   const int32_t* __restrict__ vals_in,
                                                                   K* __restrict__ keys_out,
                                                                   int32_t* __restrict__ vals_out, int64_t n,
                                                                   int shift, const int32_t* __restrict__ offs,
                                                                   int64_t ntiles) {
  __shared__ int32_t wcnt[kRsThreads / 32][256];
  __shared__ int32_t toff[256];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  for (int i = tid; i < (kRsThreads / 32) * 256; i += kRsThreads) (&wcnt[0][0])[i] = 0;
  for (int d = tid; d < 256; d += kRsThreads) toff[d] = offs[(int64_t)d * ntiles + blockIdx.x];
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile + (int64_t)w * kRsWarpItems;
  const unsigned lt = (1u << lane) - 1u;
  K key[kRsRounds];
  int32_t val[kRsRounds];
  int dg[kRsRounds];
  int rk[kRsRounds];
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    const int64_t k = base + r * 32 + lane;
    const bool valid = k < n;
    key[r] = valid ? keys_in[k] : K(0);
    val[r] = valid ? vals_in[k] : 0;
    const int d = valid ? (int)((key[r] >> shift) & 255u) : 256;
    dg[r] = d;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int before = valid ? wcnt[w][d] : 0;
    rk[r] = before + __popc(peers & lt);
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wcnt[w][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  if (tid < 256) {
    int run = 0;
#pragma unroll
    for (int w2 = 0; w2 < kRsThreads / 32; ++w2) {
      int c = wcnt[w2][tid];
      wcnt[w2][tid] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    if (dg[r] < 256) {
      const int64_t pos = (int64_t)toff[dg[r]] + wcnt[w][dg[r]] + rk[r];
      keys_out[pos] = key[r];
      vals_out[pos] = val[r];
    }
  }
}

template <typename K>
vest_status radix_sort_pairs(K* keys, int32_t* vals, K* keys_alt, int32_t* vals_alt, int64_t n, int bits,
                             int32_t* hist, int32_t* scan_tmp, bool* result_in_alt, cudaStream_t s) {
  *result_in_alt = false;
  if (n <= 0 || bits <= 0) return VEST_OK;
  const int64_t ntiles = ceil_div(n, kRsTile);
  K* kin = keys;
  int32_t* vin = vals;
  K* kout = keys_alt;
  int32_t* vout = vals_alt;
  for (int shift = 0; shift < bits; shift += 8) {
    radix_hist_kernel<K><<<(unsigned)ntiles, kRsThreads, 0, s>>>(kin, n, shift, hist, ntiles);
    VEST_LAUNCH("radix_hist");
    VEST_TRY(exclusive_scan_i32(hist, hist, 256 * ntiles, scan_tmp, s));
    radix_scatter_kernel<K><<<(unsigned)ntiles, kRsThreads, 0, s>>>(kin, vin, kout, vout, n, shift, hist, ntiles);
    VEST_LAUNCH("radix_scatter");
    std::swap(kin, kout);
    std::swap(vin, vout);
    *result_in_alt = !*result_in_alt;
  }
  return VEST_OK;
}

template vest_status radix_sort_pairs<uint32_t>(uint32_t*, int32_t*, uint32_t*, int32_t*, int64_t, int, int32_t*,
                                                int32_t*, bool*, cudaStream_t);
template vest_status radix_sort_pairs<uint64_t>(uint64_t*, int32_t*, uint64_t*, int32_t*, int64_t, int, int32_t*,
                                                int32_t*, bool*, cudaStream_t);

// ============================================================== CSR build
__global__ void iota_kernel(int32_t* v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (int32_t)i;
}

// row_ptr[r] = number of sorted keys < r, for r in [0, rows].
__global__ void row_ptr_kernel(const uint32_t* __restrict__ skey, int64_t n, int64_t rows, int64_t* __restrict__ row_ptr) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= rows; r += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if ((int64_t)skey[mid] < r) lo = mid + 1;
      else hi = mid;
    }
    row_ptr[r] = lo;
  }
}

__global__ void row_start_flags_kernel(const uint32_t* __restrict__ skey, int64_t n, int32_t* __restrict__ flags) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    flags[p] = (p == 0 || skey[p] != skey[p - 1]) ? 1 : 0;
}

// rowk[p] = number of row starts at or before p, minus one
__global__ void rowk_kernel(const int32_t* __restrict__ flags, const int32_t* __restrict__ pos, int64_t n,
                            int32_t* __restrict__ rowk) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    rowk[p] = pos[p] + flags[p] - 1;
}

__global__ void nzrows_kernel(const uint32_t* __restrict__ skey, int64_t n, const int32_t* __restrict__ flags,
                              const int32_t* __restrict__ pos, int64_t* __restrict__ nzptr, int32_t* __restrict__ nzrow,
                              int32_t* __restrict__ count) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    if (flags[p]) {
      nzptr[pos[p]] = p;
      nzrow[pos[p]] = (int32_t)skey[p];
    }
    if (p == n - 1) {
      const int32_t R = pos[p] + flags[p];
      *count = R;
      nzptr[R] = n;
    }
  }
}

// gran[g] = k such that nzptr[k] <= 32 g < nzptr[k + 1] (the non-empty row holding position 32 g)
__global__ void granule_kernel(const int64_t* __restrict__ nzptr, const int32_t* __restrict__ count, int64_t ng,
                               int32_t* __restrict__ gran) {
  const int64_t R = *count;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = g * 32;
    int64_t lo = 0, hi = R - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (nzptr[mid] <= p) lo = mid;
      else hi = mid - 1;
    }
    gran[g] = (int32_t)lo;
  }
}

__global__ void empty_index_kernel(int64_t* nzptr, int32_t* count) {
  nzptr[0] = 0;
  *count = 0;
}

// oidx[k'][p] = idx[k][perm[p]] for the other modes k (ascending), val_n[p] = val[perm[p]].
template <typename T>
__global__ void gather_kernel(const int32_t* __restrict__ idx, const T* __restrict__ val, const int32_t* __restrict__ perm,
                              int64_t n, int N, int mode, int32_t* __restrict__ oidx, T* __restrict__ vout) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = perm[p];
    int q = 0;
    for (int k = 0; k < N; ++k) {
      if (k == mode) continue;
      oidx[(int64_t)q * n + p] = idx[(int64_t)k * n + a];
      ++q;
    }
    vout[p] = val[a];
  }
}

__global__ void check_range_kernel(const int32_t* __restrict__ idx, int64_t n, int64_t rows, int32_t* __restrict__ bad) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    if (idx[p] < 0 || (int64_t)idx[p] >= rows) *bad = 1;
}

// ------------------------------------------------------------ workspace layout
namespace {
struct IndexLayout {
  size_t mode_off[kMaxOrder];
  size_t row_ptr, perm, oidx, val, nzptr, nzrow, cnt;  // offsets inside a mode region
  size_t mode_bytes[kMaxOrder];
  size_t tmp_off, tmp_keys_a, tmp_keys_b, tmp_vals_a, tmp_vals_b, tmp_hist, tmp_scan, tmp_flags, tmp_pos, tmp_bad;
  size_t total;
};

IndexLayout layout(const vest_tensor* t) {
  IndexLayout L{};
  const int64_t n = t->nnz;
  const size_t sv = t->val_dtype == VEST_F64 ? 8 : 4;
  size_t off = 0;
  for (int m = 0; m < t->order; ++m) {
    const int64_t cap = std::min<int64_t>(t->dims[m], n);
    L.mode_off[m] = off;
    size_t o = 0;
    o += align_up((size_t)(t->dims[m] + 1) * 8);       // row_ptr
    o += align_up((size_t)std::max<int64_t>(n, 1) * 4);  // perm
    o += align_up((size_t)std::max<int64_t>(n, 1) * 4 * (size_t)(t->order - 1));  // oidx
    o += align_up((size_t)std::max<int64_t>(n, 1) * sv);                           // val
    o += align_up((size_t)(cap + 1) * 8);                                          // nzptr
    o += align_up((size_t)std::max<int64_t>(cap, 1) * 4);                          // nzrow
    o += align_up(4);                                                              // count
    o += align_up((size_t)(ceil_div(std::max<int64_t>(n, 1), 32) + 1) * 4);       // granule rows
    o += align_up((size_t)std::max<int64_t>(n, 1) * 4);                           // row of every position
    L.mode_bytes[m] = o;
    off += o;
  }
  L.tmp_off = off;
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  size_t o = off;
  L.tmp_keys_a = o; o += align_up(nn * 4);
  L.tmp_keys_b = o; o += align_up(nn * 4);
  L.tmp_vals_a = o; o += align_up(nn * 4);
  L.tmp_vals_b = o; o += align_up(nn * 4);
  L.tmp_hist = o; o += align_up(radix_hist_elems(n) * 4);
  L.tmp_scan = o; o += align_up(scan_tmp_elems((int64_t)std::max(radix_hist_elems(n), nn)) * 8);
  L.tmp_flags = o; o += align_up(nn * 4);
  L.tmp_pos = o; o += align_up(nn * 4);
  L.tmp_bad = o; o += align_up(4);
  L.total = o;
  return L;
}
}  // namespace

size_t index_workspace_bytes(const vest_tensor* t) { return layout(t).total; }

static int bit_length(int64_t v) {
  int b = 0;
  while (v > 0) {
    ++b;
    v >>= 1;
  }
  return b;
}

vest_status build_index_impl(const vest_tensor* t, void* ws, size_t ws_bytes, vest_index* ix, cudaStream_t s) {
  const IndexLayout L = layout(t);
  if (ws_bytes < L.total) return fail(VEST_ERR_WORKSPACE, "index workspace too small");
  char* base = static_cast<char*>(ws);
  const int64_t n = t->nnz;
  const int N = t->order;
  ix->order = N;
  ix->val_dtype = t->val_dtype;
  ix->nnz = n;
  ix->ws_bytes = L.total;
  for (int m = 0; m < N; ++m) ix->dims[m] = t->dims[m];

  uint32_t* keys_a = reinterpret_cast<uint32_t*>(base + L.tmp_keys_a);
  uint32_t* keys_b = reinterpret_cast<uint32_t*>(base + L.tmp_keys_b);
  int32_t* vals_a = reinterpret_cast<int32_t*>(base + L.tmp_vals_a);
  int32_t* vals_b = reinterpret_cast<int32_t*>(base + L.tmp_vals_b);
  int32_t* hist = reinterpret_cast<int32_t*>(base + L.tmp_hist);
  int32_t* scan_tmp = reinterpret_cast<int32_t*>(base + L.tmp_scan);
  int32_t* flags = reinterpret_cast<int32_t*>(base + L.tmp_flags);
  int32_t* pos = reinterpret_cast<int32_t*>(base + L.tmp_pos);
  int32_t* bad = reinterpret_cast<int32_t*>(base + L.tmp_bad);
  const int grid = std::max(1, std::min<int>((int)ceil_div(std::max<int64_t>(n, 1), 256), num_sms() * 8));

  // index range check, read back once: out-of-range indices are a caller error
  if (n > 0) {
    VEST_CUDA(cudaMemsetAsync(bad, 0, 4, s));
    for (int m = 0; m < N; ++m) {
      check_range_kernel<<<grid, 256, 0, s>>>(t->idx + (int64_t)m * n, n, t->dims[m], bad);
      VEST_LAUNCH("check_range");
    }
    int32_t hbad = 0;
    VEST_CUDA(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, s));
    VEST_CUDA(cudaStreamSynchronize(s));
    if (hbad) return fail(VEST_ERR_INVALID, "tensor index out of range");
  }

  for (int m = 0; m < N; ++m) {
    char* mb = base + L.mode_off[m];
    ModeIndex& mi = ix->mode[m];
    const int64_t cap = std::min<int64_t>(t->dims[m], n);
    size_t o = 0;
    mi.row_ptr = reinterpret_cast<int64_t*>(mb + o); o += align_up((size_t)(t->dims[m] + 1) * 8);
    mi.perm = reinterpret_cast<int32_t*>(mb + o); o += align_up((size_t)std::max<int64_t>(n, 1) * 4);
    mi.oidx = reinterpret_cast<int32_t*>(mb + o); o += align_up((size_t)std::max<int64_t>(n, 1) * 4 * (size_t)(N - 1));
    mi.val = mb + o; o += align_up((size_t)std::max<int64_t>(n, 1) * (t->val_dtype == VEST_F64 ? 8 : 4));
    mi.nzptr = reinterpret_cast<int64_t*>(mb + o); o += align_up((size_t)(cap + 1) * 8);
    mi.nzrow = reinterpret_cast<int32_t*>(mb + o); o += align_up((size_t)std::max<int64_t>(cap, 1) * 4);
    mi.nnzrows = reinterpret_cast<int32_t*>(mb + o); o += align_up(4);
    mi.gran = reinterpret_cast<int32_t*>(mb + o); o += align_up((size_t)(ceil_div(std::max<int64_t>(n, 1), 32) + 1) * 4);
    mi.rowk = reinterpret_cast<int32_t*>(mb + o);
    mi.cap = cap;
    if (n == 0) {
      VEST_CUDA(cudaMemsetAsync(mi.row_ptr, 0, (size_t)(t->dims[m] + 1) * 8, s));
      empty_index_kernel<<<1, 1, 0, s>>>(mi.nzptr, mi.nnzrows);
      VEST_LAUNCH("empty_index");
      continue;
    }
    VEST_CUDA(cudaMemcpyAsync(keys_a, t->idx + (int64_t)m * n, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    iota_kernel<<<grid, 256, 0, s>>>(vals_a, n);
    VEST_LAUNCH("iota");
    bool in_alt = false;
    VEST_TRY(radix_sort_pairs<uint32_t>(keys_a, vals_a, keys_b, vals_b, n, bit_length(t->dims[m] - 1), hist,
                                        scan_tmp, &in_alt, s));
    const uint32_t* skey = in_alt ? keys_b : keys_a;
    const int32_t* sval = in_alt ? vals_b : vals_a;
    VEST_CUDA(cudaMemcpyAsync(mi.perm, sval, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    const int rgrid = std::max(1, std::min<int>((int)ceil_div(t->dims[m] + 1, 256), num_sms() * 8));
    row_ptr_kernel<<<rgrid, 256, 0, s>>>(skey, n, t->dims[m], mi.row_ptr);
    VEST_LAUNCH("row_ptr");
    row_start_flags_kernel<<<grid, 256, 0, s>>>(skey, n, flags);
    VEST_LAUNCH("row_flags");
    VEST_TRY(exclusive_scan_i32(flags, pos, n, scan_tmp, s));
    nzrows_kernel<<<grid, 256, 0, s>>>(skey, n, flags, pos, mi.nzptr, mi.nzrow, mi.nnzrows);
    VEST_LAUNCH("nzrows");
    rowk_kernel<<<grid, 256, 0, s>>>(flags, pos, n, mi.rowk);
    VEST_LAUNCH("rowk");
    const int64_t ng = ceil_div(n, 32);
    granule_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ng, 256), num_sms() * 8)), 256, 0, s>>>(
        mi.nzptr, mi.nnzrows, ng, mi.gran);
    VEST_LAUNCH("granule");
    if (t->val_dtype == VEST_F64)
      gather_kernel<double><<<grid, 256, 0, s>>>(t->idx, static_cast<const double*>(t->val), mi.perm, n, N, m,
                                                 mi.oidx, static_cast<double*>(mi.val));
    else
      gather_kernel<float><<<grid, 256, 0, s>>>(t->idx, static_cast<const float*>(t->val), mi.perm, n, N, m,
                                                mi.oidx, static_cast<float*>(mi.val));
    VEST_LAUNCH("gather");
  }
  return VEST_OK;
}

}  // namespace vest
