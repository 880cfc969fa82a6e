// Core sweep (Lemma 2, Eq. 12; Lemma 4, Eq. 14) and the core part of the
// responsibility (Eq. 5, Algorithm 3).
//
// The core elements are updated one at a time in linear order (j_1 fastest),
// as the paper requires (Section 3.5).  On the GPU this is blocked
// Gauss-Seidel, equal to the one-at-a-time sweep in exact arithmetic:
//   - a block is b = J_0 * m consecutive core elements, (j_0, j_1) in
//     J_0 x [q0, q0 + m) for one suffix s = (j_2, ..., j_{N-1});
//     P_alpha(j_0, j_1) = a0[i_0, j_0] * a1[i_1, j_1] * c_alpha(s), with
//     c_alpha(s) = prod_{n>=2} a_n[i_n, s_n];
//   - the block Grams M_b = sum_alpha P_alpha P_alpha^T depend on the factors
//     only, which the core sweep does not change, so all of them are formed
//     first.  Entries are grouped by their mode-0 row piece (row within a task):
//     a gram pass writes per piece Y(s, q, q') = sum c(s)^2 a1[q] a1[q'], a tiled
//     reduction over pieces forms Z(s) = sum_piece sym(a0 a0^T) (x) Y(s), and a
//     merge expands Z into each packed M_b in FP64;
//   - then per block in order: one pass over the mode-0 CSR applies the
//     previous block's Delta to r and forms g_k = sum_alpha r_alpha P_alpha(k)
//     (per row segment h(q) = sum r w(q), g += a0 (x) h); one warp performs the
//     b updates in order with sum_alpha r P(k) = g_k - sum_{l<k} Delta_l M_lk;
//   - optionally a last light pass applies the last block's Delta, so r is the
//     residual of the swept model (loss and responsibility then reuse it).
// The core responsibility needs g and diag(M) of every element for a fixed r:
// one stats pass per group of suffixes forms both, or g alone right after a core
// sweep with the same factors, whose block Grams hold diag(M).
// Sums: per piece in the storage type; across pieces and tasks FP32 with Kahan
// compensation (or FP64); across thread blocks FP64 in a fixed order.
#include <algorithm>

#include "delta.cuh"

namespace vest {

constexpr int kCoreTask = 256;
constexpr int kCoreMaxB = 128;
constexpr int kCoreMaxM = 10;
constexpr int kGramKSplit = 64;     // fixed: reduction order does not depend on the device
// Fixed CTA counts (the order of every sum is then the same on any device), chosen as
// whole waves on 152 SMs: the stats pass holds 2 CTAs per SM (304 = one wave; each CTA ends
// with an FP64 combination of its warps, which issues at the FP64 rate, so fewer CTAs pay it
// fewer times), the g pass 4 (608 = one wave of grid-strided CTAs; 64 registers a thread).
constexpr int kCorePassCtas = 304;
constexpr int kGPassCtas = 608;

struct CoreBlock {
  int64_t s;  // suffix linear index over modes >= 2
  int q0, m;  // j_1 range
  int b;      // J_0 * m
};

// Running sums across tasks: Kahan-compensated for FP32, plain for FP64.
template <typename T>
struct CoreAcc;
template <>
struct CoreAcc<float> {
  static __device__ void add(float& s, float& c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  static __device__ double value(float s, float c) { return (double)s - (double)c; }
};
template <>
struct CoreAcc<double> {
  static __device__ void add(double& s, double&, double v) { s += v; }
  static __device__ double value(double s, double) { return s; }
};

__host__ __device__ __forceinline__ int sym_index(int x, int y, int n) {
  const int lo = x < y ? x : y, hi = x < y ? y : x;
  return lo * n - (lo * (lo - 1)) / 2 + (hi - lo);
}

__device__ __forceinline__ void sym_decode(int u, int n, int& a, int& b) {
  int k = 0;
  while (u >= n - k) {
    u -= n - k;
    ++k;
  }
  a = k;
  b = k + u;
}

// entry e of a packed upper b x b matrix -> (k, l), k <= l
__device__ __forceinline__ void entry_kl(int e, int b, int& k, int& l) { sym_decode(e, b, k, l); }

// c_alpha(s) for the `count` consecutive suffixes starting at s0 (mode 2 fastest)
template <typename T>
__device__ __forceinline__ void suffix_weights(const DevModel<T>& M, const int32_t* __restrict__ oidx, int64_t nnz,
                                               int64_t p, int64_t s0, int count, T* out, int stride) {
  if (M.N == 2) {
    for (int i = 0; i < count; ++i) out[i * stride] = T(1);
    return;
  }
  if (M.N == 3) {
    const T* row = M.A[2] + (int64_t)oidx[nnz + p] * M.J[2] + s0;
    for (int i = 0; i < count; ++i) out[i * stride] = row[i];
    return;
  }
  const T* rows[kMaxOrder];
  int dig[kMaxOrder];
  int64_t rem = s0;
  for (int n = 2; n < M.N; ++n) {
    rows[n] = M.A[n] + (int64_t)oidx[(int64_t)(n - 1) * nnz + p] * M.J[n];
    dig[n] = (int)(rem % M.J[n]);
    rem /= M.J[n];
  }
  for (int i = 0; i < count; ++i) {
    T c = T(1);
    for (int n = 2; n < M.N; ++n) c *= rows[n][dig[n]];
    out[i * stride] = c;
    for (int n = 2; n < M.N; ++n) {
      if (++dig[n] < M.J[n]) break;
      dig[n] = 0;
    }
  }
}

// dst[i] = src[i] for i < len: 8- or 16-byte pair loads where `pair` says src is 2-element
// aligned, a scalar tail for odd len.  The staging loops of the Gram and stats passes gather
// whole factor rows this way: the gathers, not the arithmetic, fill the L1 data pipe there.
template <typename T>
__device__ __forceinline__ void copy_row(const T* __restrict__ src, int len, bool pair, T* dst) {
  int q = 0;
  if (pair) {
    for (; q + 1 < len; q += 2) {
      T x, y;
      load2<T>(src + q, x, y);
      dst[q] = x;
      dst[q + 1] = y;
    }
  }
  for (; q < len; ++q) dst[q] = src[q];
}

// Whether rows of A^(n) starting at column c0 are 2-element aligned for copy_row.
template <typename T>
__device__ __forceinline__ bool rows_paired(const DevModel<T>& M, int n, int64_t c0) {
  return M.J[n] % 2 == 0 && c0 % 2 == 0 && reinterpret_cast<uintptr_t>(M.A[n]) % (2 * sizeof(T)) == 0;
}

// ================================================================== gram pass
constexpr int kGramSgB = 16;  // suffixes per gram group at most (registers per lane: 2 x 16)

struct GramArgs {
  int J0, J1;
  int q0, mq, nY;
  int64_t s0;
  int Sg, P;
  int64_t nnz, ntasks;
  void* Y;         // [slots][P]
  int32_t* srow;   // [slots]: compacted mode-0 row of the slot, -1 if unused
};

// Gram pass for one j_1 chunk [q0, q0 + mq) and one group of Sg suffixes: for every row
// piece (the part of a mode-0 row inside one 256-entry task, slot = row + task)
//   Y(s, q, q') = sum over the piece of c(s)^2 a1[q0 + q] a1[q0 + q'],  q <= q',
// stored at Y[slot][s * nY + packed(q, q')].  Each warp takes whole tasks (warp-strided) and
// walks them 32 entries at a time: the lanes stage one entry each (row, c(s)^2 of the group
// zero-padded to SGB, the a1 values of the chunk); then every lane runs through the entries
// in order for its pairs (q, q') = packed index lane, lane + 32 and all SGB >= Sg suffixes
// (the padding adds zeros), and writes the piece's sums at a row change and at the end of
// the task.
template <typename T, int SGB>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) core_gram_pass_kernel(DevModel<T> M, DevMode<T> csr, GramArgs a) {
  constexpr int V = 16 / (int)sizeof(T);  // values per 16-byte shared-memory load
  static_assert(SGB % V == 0, "SGB must fill whole 16-byte loads");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int mq = a.mq, nY = a.nY, Sg = a.Sg, P = a.P;
  const int ld = (SGB + mq + V - 1) / V * V;  // staged entry: c(s)^2 (SGB), a1 chunk
  T* st = reinterpret_cast<T*>(smem_raw) + (size_t)warp * 32 * ld;
  int* sk = reinterpret_cast<int*>(reinterpret_cast<T*>(smem_raw) + (size_t)nwarps * 32 * ld) + warp * 32;
  T* Y = static_cast<T*>(a.Y);
  int qa[2], qb[2];
  bool on[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int pr = lane + 32 * i;
    on[i] = pr < nY;
    int x = 0, y = 0;
    if (on[i]) sym_decode(pr, mq, x, y);
    qa[i] = x;
    qb[i] = y;
  }
  T acc[2][SGB];
  const bool pair1 = rows_paired(M, 1, a.q0), pair2 = M.N == 3 && rows_paired(M, 2, a.s0);
  auto flush = [&](int64_t slot, int row) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
      if (on[i])
#pragma unroll
        for (int s = 0; s < SGB; ++s)
          if (s < Sg) Y[slot * P + s * nY + lane + 32 * i] = acc[i][s];
    if (lane == 0) a.srow[slot] = row;
  };
  const int64_t gw = (int64_t)blockIdx.x * nwarps + warp, nw = (int64_t)gridDim.x * nwarps;
  for (int64_t task = gw; task < a.ntasks; task += nw) {
    const int64_t t0 = task * kCoreTask, t1 = min(t0 + (int64_t)kCoreTask, a.nnz);
    int cur = -1;
    for (int64_t c0 = t0; c0 < t1; c0 += 32) {
      const int64_t p = c0 + lane;
      __syncwarp();
      if (p < t1) {
        sk[lane] = csr.rowk[p];
        T* se = st + lane * ld;
        if (M.N == 3) copy_row<T>(M.A[2] + (int64_t)csr.oidx[a.nnz + p] * M.J[2] + a.s0, Sg, pair2, se);
        else suffix_weights<T>(M, csr.oidx, a.nnz, p, a.s0, Sg, se, 1);
        for (int s = 0; s < Sg; ++s) se[s] *= se[s];
        for (int s = Sg; s < SGB; ++s) se[s] = T(0);
        copy_row<T>(M.A[1] + (int64_t)csr.oidx[p] * a.J1 + a.q0, mq, pair1, se + SGB);
      }
      __syncwarp();
      const int n = (int)min((int64_t)32, t1 - c0);
      for (int e = 0; e < n; ++e) {
        const int k = sk[e];
        const T* se = st + e * ld;
        if (k != cur) {
          if (cur >= 0) flush(cur + task, cur);
          cur = k;
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int s = 0; s < SGB; ++s) acc[i][s] = T(0);
        }
        T cv[SGB];
#pragma unroll
        for (int s4 = 0; s4 < SGB; s4 += V) {
          if constexpr (sizeof(T) == 4) {
            const float4 v = *reinterpret_cast<const float4*>(se + s4);
            cv[s4] = v.x;
            cv[s4 + 1] = v.y;
            cv[s4 + 2] = v.z;
            cv[s4 + 3] = v.w;
          } else {
            const double2 v = *reinterpret_cast<const double2*>(se + s4);
            cv[s4] = v.x;
            cv[s4 + 1] = v.y;
          }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const T kq = se[SGB + qa[i]] * se[SGB + qb[i]];
#pragma unroll
          for (int s = 0; s < SGB; ++s) acc[i][s] += cv[s] * kq;
        }
      }
    }
    if (cur >= 0) flush(cur + task, cur);
  }
}

// X of every slot: Xs[slot][xi] = a0[ja] a0[jb] for the packed upper pair xi = (ja, jb)
// of the slot's mode-0 row (0 for unused slots).  The slots are the same for every gram
// group, so this runs once per core sweep.
template <typename T>
__global__ void core_gram_x_kernel(DevModel<T> M, DevMode<T> csr, const int32_t* __restrict__ srow, int64_t nslots,
                                   int J0, int nX, T* __restrict__ Xs) {
  const int64_t n = nslots * nX;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t slot = e / nX;
    const int xi = (int)(e % nX);
    const int32_t k = srow[slot];
    T v = T(0);
    if (k >= 0) {
      int ja, jb;
      sym_decode(xi, J0, ja, jb);
      const T* a0 = M.A[0] + (int64_t)csr.nzrow[k] * J0;
      v = a0[ja] * a0[jb];
    }
    Xs[e] = v;
  }
}

// Z[ks][xi][p] = sum over the slots of split ks of Xs[slot][xi] * Y[slot][p].  CTA tile
// 64 (xi) x 64 (p), 4 x 4 outputs per thread; slots staged CS at a time through registers
// (the next chunk's loads are in flight while the current one is multiplied); each chunk
// is summed in the storage type and added to the running sums with Kahan compensation.
struct GemmArgs {
  int J0, nX, P;
  int64_t nslots;
  const void* Xs;
  const void* Y;
  const int32_t* srow;
  double* part;  // [ks][nX][P]
};

template <typename T>
__global__ void __launch_bounds__(256, 2) core_gram_gemm_kernel(GemmArgs a) {
  constexpr int CS = sizeof(T) == 4 ? 32 : 16;  // slots per chunk
  constexpr int NX = CS * 64 / 256;             // staged X (and Y) values per thread
  __shared__ __align__(16) T sX[CS][64];
  __shared__ __align__(16) T sY[CS][64];
  const T* Xs = static_cast<const T*>(a.Xs);
  const T* Y = static_cast<const T*>(a.Y);
  const int tiles_p = (a.P + 63) / 64;
  const int tx0 = (blockIdx.x / tiles_p) * 64, tp0 = (blockIdx.x % tiles_p) * 64;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int64_t per = ceil_div(a.nslots, (int64_t)gridDim.y);
  const int64_t sl0 = blockIdx.y * per, sl1 = min(a.nslots, sl0 + per);
  T xr[NX], yr[NX];
  auto load = [&](int64_t c0) {
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      const int e = threadIdx.x + 256 * i, cs = e >> 6, l = e & 63;
      const int64_t slot = c0 + cs;
      const bool in = slot < sl1 && a.srow[slot] >= 0;
      xr[i] = (in && tx0 + l < a.nX) ? Xs[slot * a.nX + tx0 + l] : T(0);
      yr[i] = (in && tp0 + l < a.P) ? Y[slot * a.P + tp0 + l] : T(0);
    }
  };
  T run_s[4][4], run_c[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) run_s[i][j] = run_c[i][j] = T(0);
  if (sl0 < sl1) load(sl0);
  for (int64_t c0 = sl0; c0 < sl1; c0 += CS) {
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      const int e = threadIdx.x + 256 * i, cs = e >> 6, l = e & 63;
      sX[cs][l] = xr[i];
      sY[cs][l] = yr[i];
    }
    __syncthreads();
    if (c0 + CS < sl1) load(c0 + CS);
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
#pragma unroll 8
    for (int cs = 0; cs < CS; ++cs) {
      T xv[4], yv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xv[i] = sX[cs][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) yv[j] = sY[cs][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += xv[i] * yv[j];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) CoreAcc<T>::add(run_s[i][j], run_c[i][j], acc[i][j]);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int xi = tx0 + ty * 4 + i, p = tp0 + tx * 4 + j;
      if (xi < a.nX && p < a.P)
        a.part[((size_t)blockIdx.y * a.nX + xi) * a.P + p] = CoreAcc<T>::value(run_s[i][j], run_c[i][j]);
    }
}

// Packed M of block (s0 + sidx, q chunk qc) in FP64 from the split partials; sidx = blockIdx.y,
// so one launch merges every suffix of the group.
__global__ void core_gram_merge_kernel(const double* __restrict__ part, int ksplit, int nX, int P, int J0, int mq,
                                       int nY, int64_t s0, int nq0, int qc, int64_t nmmax, double* __restrict__ gram_all) {
  const int b = J0 * mq, nm = b * (b + 1) / 2;
  const int sidx = blockIdx.y;
  double* gram = gram_all + ((s0 + sidx) * nq0 + qc) * nmmax;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nm; e += gridDim.x * blockDim.x) {
    int k, l;
    entry_kl(e, b, k, l);
    const int xi = sym_index(k % J0, l % J0, J0);
    const int p = sidx * nY + sym_index(k / J0, l / J0, mq);
    double c4[4] = {0, 0, 0, 0};
    int c = 0;
    for (; c + 3 < ksplit; c += 4) {
#pragma unroll
      for (int k = 0; k < 4; ++k) c4[k] += part[((size_t)(c + k) * nX + xi) * P + p];
    }
    for (; c < ksplit; ++c) c4[0] += part[((size_t)c * nX + xi) * P + p];
    gram[e] = (c4[0] + c4[1]) + (c4[2] + c4[3]);
  }
}

// ================================================================== g pass (one block)
// v[q] = row[q] for q < len (len <= kCoreMaxM), 0 beyond.  In pairs when `pair` is set: the
// row start is 2-element aligned and, for odd len, the row goes on past row[len - 1].
template <typename T>
__device__ __forceinline__ void row_part(const T* row, int len, int pair, T (&v)[kCoreMaxM]) {
  if (pair) {
#pragma unroll
    for (int q = 0; q < kCoreMaxM; q += 2)
      if (q < len) load2<T>(row + q, v[q], v[q + 1]);
  } else {
#pragma unroll
    for (int q = 0; q < kCoreMaxM; ++q)
      if (q < len) v[q] = row[q];
  }
#pragma unroll
  for (int q = 0; q < kCoreMaxM; ++q)
    if (q >= len) v[q] = T(0);
}

struct GPassArgs {
  int J0, J1;
  CoreBlock cur, prev;
  int has_prev;
  int pair_a1;  // mode-1 rows read two elements at a time (J1, both q0 even; aligned factor)
  int pair_u;   // u rows read two elements at a time (aligned U)
  int64_t nnz;
  double* part;  // [ctas][b]
};

// u(k, q) = sum_j0 Delta_prev(j0, q) a0[row_k, j0] for every non-empty mode-0 row k.
template <typename T>
__global__ void core_u_kernel(DevModel<T> M, const int32_t* __restrict__ nzrow, const int32_t* __restrict__ nnzrows,
                              const double* __restrict__ dprev, int J0, int mp, T* __restrict__ U) {
  // Delta in the storage type, converted once here rather than once per product (a conversion
  // from FP64 issues at the FP64 rate)
  __shared__ T sd[kCoreMaxB];
  for (int i = threadIdx.x; i < J0 * mp; i += blockDim.x) sd[i] = (T)dprev[i];
  __syncthreads();
  const int64_t R = *nnzrows;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < R; k += (int64_t)gridDim.x * blockDim.x) {
    const T* a0 = M.A[0] + (int64_t)nzrow[k] * J0;
    for (int q = 0; q < mp; ++q) {
      T u = T(0);
      for (int j = 0; j < J0; ++j) u += sd[q * J0 + j] * a0[j];
      U[k * kCoreMaxM + q] = u;
    }
  }
}

// A0c[k] = a0 row of the k-th non-empty mode-0 row (the core sweep leaves A^(0) unchanged).
template <typename T>
__global__ void core_a0c_kernel(DevModel<T> M, const int32_t* __restrict__ nzrow, const int32_t* __restrict__ nnzrows,
                                int J0, T* __restrict__ A0c) {
  const int64_t n = (int64_t)*nnzrows * J0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    A0c[e] = M.A[0][(int64_t)nzrow[e / J0] * J0 + e % J0];
}

// One streaming pass per block.  Each warp takes 32 consecutive entries at a
// time: it applies the previous block's Delta to r (r -= c' a1 . u(row)), forms
// h(q) = r a1[q0 + q] c, adds h over each row segment inside the warp, and every
// segment head adds a0[row] (x) h into the warp's g accumulators (lane l holds
// elements l, l + 32, ...; Kahan across heads).  g is linear in the rows, so row
// segments cut by chunk edges need no fix-up.  All gathers of a chunk (a1, the
// suffix weights, u, and the head lanes' a0 rows from A0c) are issued together
// after the coalesced index loads; a1 and u rows are read in pairs where aligned.
// The pass is bound by the L1 data pipe, so a chunk of one row only (most chunks:
// about 1.3 rows per chunk on the Zipf workload) sums h by reduce-scatter, 17
// shuffles, instead of the segmented scan's 5 (m + 1).
template <typename T>
__global__ void __launch_bounds__(256, 4) core_g_pass_kernel(DevModel<T> M, DevMode<T> csr, T* r, const T* __restrict__ U,
                                                          const T* __restrict__ A0c, GPassArgs a) {
  constexpr int kPer = kCoreMaxB / 32;
  __shared__ T sh[8][kCoreMaxM];
  __shared__ double sw[8][kCoreMaxB];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int J0 = a.J0, m = a.cur.m, b = a.cur.b, mp = a.has_prev ? a.prev.m : 0;
  T* sa = reinterpret_cast<T*>(smem_raw) + (size_t)warp * 32 * J0;  // a0 row of each head lane
  const bool same_q = a.has_prev && a.prev.q0 == a.cur.q0;
  T as[kPer], ac[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) as[i] = ac[i] = T(0);
  const int64_t nchunks = ceil_div(a.nnz, 32);
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp, nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  // the coalesced loads of a chunk (row, mode-1 index, mode-2 index when N = 3, r) are
  // issued one chunk ahead
  const bool n3 = M.N == 3;
  int nk = 0, ni1 = 0, ni2 = 0;
  T nrv = T(0);
  auto prefetch = [&](int64_t ch) {
    const int64_t p = ch * 32 + lane;
    if (ch < nchunks && p < a.nnz) {
      nk = csr.rowk[p];
      ni1 = csr.oidx[p];
      if (n3) ni2 = csr.oidx[a.nnz + p];
      nrv = r[p];
    }
  };
  prefetch(gw);
  for (int64_t ch = gw; ch < nchunks; ch += nw) {
    const int64_t p = ch * 32 + lane;
    const bool valid = p < a.nnz;
    const int k = valid ? nk : -1 - lane;
    const int i1 = ni1, i2 = ni2;
    const T rv0 = nrv;
    prefetch(ch + nw);
    const int kup = __shfl_up_sync(0xffffffffu, k, 1);
    const bool head = valid && (lane == 0 || kup != k);
    T h[kCoreMaxM];
#pragma unroll
    for (int q = 0; q < kCoreMaxM; ++q) h[q] = T(0);
    __syncwarp();
    if (head) {
      const T* a0 = A0c + (int64_t)k * J0;
      for (int j = 0; j < J0; ++j) sa[lane * J0 + j] = a0[j];
    }
    if (valid) {
      const T* a1 = M.A[1] + (int64_t)i1 * a.J1;
      T rv = rv0;
      T v[kCoreMaxM];
      row_part<T>(a1 + a.cur.q0, m, a.pair_a1, v);
      if (a.has_prev) {
        T cp;
        if (n3) cp = M.A[2][(int64_t)i2 * M.J[2] + a.prev.s];
        else suffix_weights<T>(M, csr.oidx, a.nnz, p, a.prev.s, 1, &cp, 1);
        const T* u = U + (int64_t)k * kCoreMaxM;
        T acc = T(0);
        if (same_q) {
          if (a.pair_u) {
#pragma unroll
            for (int q = 0; q < kCoreMaxM; q += 2)
              if (q < mp) {
                T u0, u1;
                load2<T>(u + q, u0, u1);
                acc += v[q] * u0;
                if (q + 1 < mp) acc += v[q + 1] * u1;
              }
          } else {
#pragma unroll
            for (int q = 0; q < kCoreMaxM; ++q)
              if (q < mp) acc += v[q] * u[q];
          }
        } else {
          const T* w = a1 + a.prev.q0;
#pragma unroll
          for (int q = 0; q < kCoreMaxM; ++q)
            if (q < mp) acc += w[q] * u[q];
        }
        rv -= cp * acc;
        r[p] = rv;
      }
      T c;
      if (n3) c = M.A[2][(int64_t)i2 * M.J[2] + a.cur.s];
      else suffix_weights<T>(M, csr.oidx, a.nnz, p, a.cur.s, 1, &c, 1);
      const T rc = rv * c;
#pragma unroll
      for (int q = 0; q < kCoreMaxM; ++q)
        if (q < m) h[q] = rc * v[q];
    }
    if (__all_sync(0xffffffffu, k == __shfl_sync(0xffffffffu, k, 0))) {
      // one row: reduce-scatter of the 10 sums (halves at offset 16, 3 | 2 at offset 8,
      // butterfly over the last 3 at offsets 4, 2, 1); lanes 0, 8, 16, 24 hold q 0-2,
      // 3-4, 5-7, 8-9
      static_assert(kCoreMaxM == 10, "reduce-scatter split is written for 10 sums");
      const bool up = lane & 16, b3 = lane & 8;
      T k1[5], k2[3];
#pragma unroll
      for (int i = 0; i < 5; ++i) k1[i] = (up ? h[i + 5] : h[i]) + __shfl_xor_sync(0xffffffffu, up ? h[i] : h[i + 5], 16);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const T hi = i < 2 ? k1[3 + i] : T(0);
        k2[i] = (b3 ? hi : k1[i]) + __shfl_xor_sync(0xffffffffu, b3 ? k1[i] : hi, 8);
      }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 3; ++i) k2[i] += __shfl_xor_sync(0xffffffffu, k2[i], o);
      if ((lane & 7) == 0) {
        const int qb = (up ? 5 : 0) + (b3 ? 3 : 0);
#pragma unroll
        for (int i = 0; i < 3; ++i)
          if (i < (b3 ? 2 : 3)) sh[warp][qb + i] = k2[i];
      }
      __syncwarp();
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int e = lane + 32 * i;
        if (e < b) CoreAcc<T>::add(as[i], ac[i], sa[e % J0] * sh[warp][e / J0]);
      }
      __syncwarp();
      continue;
    }
    // segmented suffix sums: lane l ends with the sum over its row from l to the chunk end
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int ko = __shfl_down_sync(0xffffffffu, k, o);
#pragma unroll
      for (int q = 0; q < kCoreMaxM; ++q) {
        if (q < m) {
          const T v = __shfl_down_sync(0xffffffffu, h[q], o);
          if (lane + o < 32 && ko == k) h[q] += v;
        }
      }
    }
    unsigned heads = __ballot_sync(0xffffffffu, head);
    while (heads) {
      const int hl = __ffs(heads) - 1;
      heads &= heads - 1;
      if (lane == hl) {
#pragma unroll
        for (int q = 0; q < kCoreMaxM; ++q)
          if (q < m) sh[warp][q] = h[q];
      }
      __syncwarp();
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int e = lane + 32 * i;
        if (e < b) CoreAcc<T>::add(as[i], ac[i], sa[hl * J0 + e % J0] * sh[warp][e / J0]);
      }
      __syncwarp();
    }
  }
#pragma unroll
  for (int i = 0; i < kPer; ++i) sw[warp][lane + 32 * i] = CoreAcc<T>::value(as[i], ac[i]);
  __syncthreads();
  const int nwarps = blockDim.x >> 5;
  for (int e = threadIdx.x; e < b; e += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < nwarps; ++w) t += sw[w][e];
    a.part[(size_t)blockIdx.x * b + e] = t;
  }
}

// After the last block: r -= c_last a1 . u(row) (the last block's change), the residual
// copied to COO order, and per CTA (sum r^2, sum x^2) with per-thread Kahan sums in the
// storage type, FP64 across threads.
template <typename T>
__global__ void __launch_bounds__(256) core_final_kernel(DevModel<T> M, DevMode<T> csr, T* __restrict__ r,
                                                         T* __restrict__ rcoo, const T* __restrict__ U, CoreBlock last,
                                                         double* __restrict__ part) {
  __shared__ double red[32];
  T sq = T(0), sqc = T(0), xx = T(0), xxc = T(0);
  auto kadd = [](T& s, T& c, T v) {
    const T y = v - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  };
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < csr.nnz; p += (int64_t)gridDim.x * blockDim.x) {
    const int k = csr.rowk[p];
    const T* a1 = M.A[1] + (int64_t)csr.oidx[p] * M.J[1] + last.q0;
    T cp;
    suffix_weights<T>(M, csr.oidx, csr.nnz, p, last.s, 1, &cp, 1);
    const T* u = U + (int64_t)k * kCoreMaxM;
    T acc = T(0);
#pragma unroll
    for (int q = 0; q < kCoreMaxM; ++q)
      if (q < last.m) acc += a1[q] * u[q];
    const T rv = r[p] - cp * acc;
    r[p] = rv;
    rcoo[csr.perm[p]] = rv;
    const T x = csr.val[p];
    kadd(sq, sqc, rv * rv);
    kadd(xx, xxc, x * x);
  }
  double v1 = (double)sq - (double)sqc, v2 = (double)xx - (double)xxc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    v2 += __shfl_xor_sync(0xffffffffu, v2, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    red[w] = v1;
    red[16 + w] = v2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a += red[i];
      b += red[16 + i];
    }
    part[blockIdx.x * 2 + 0] = a;
    part[blockIdx.x * 2 + 1] = b;
  }
}

// First level of the FP64 merge of many per-CTA partials: block (x, g) sums the
// partials c of group g (a contiguous range) for outputs 32 x .. 32 x + 31, eight
// warps over c with four chains each, warps combined in order.
constexpr int kMergeGroups = 16;

__global__ void core_vec_merge1_kernel(const double* __restrict__ part, int nctas, int n, double* __restrict__ tmp) {
  __shared__ double sh[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  const int per = (nctas + gridDim.y - 1) / gridDim.y;
  const int c0 = blockIdx.y * per, c1 = min(nctas, c0 + per);
  double c4[4] = {0, 0, 0, 0};
  if (e < n) {
    int c = c0 + w, u = 0;
    for (; c + 24 < c1; c += 32) {
#pragma unroll
      for (int k = 0; k < 4; ++k) c4[k] += part[(size_t)(c + 8 * k) * n + e];
    }
    for (; c < c1; c += 8, ++u) c4[u & 3] += part[(size_t)c * n + e];
  }
  sh[w][lane] = (c4[0] + c4[1]) + (c4[2] + c4[3]);
  __syncthreads();
  if (w == 0 && e < n) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += sh[k][lane];
    tmp[(size_t)blockIdx.y * n + e] = s;
  }
}

// out[e] = sum over c of part[c][e] in FP64: block of 8 warps x 32 outputs, warp w
// sums c = w, w + 8, ... with four independent chains, warps combined in order.
__global__ void core_vec_merge_kernel(const double* __restrict__ part, int nctas, int n, double* __restrict__ out) {
  __shared__ double sh[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  double c4[4] = {0, 0, 0, 0};
  if (e < n) {
    int c = w, u = 0;
    for (; c + 24 < nctas; c += 32) {
#pragma unroll
      for (int k = 0; k < 4; ++k) c4[k] += part[(size_t)(c + 8 * k) * n + e];
    }
    for (; c < nctas; c += 8, ++u) c4[u & 3] += part[(size_t)c * n + e];
  }
  sh[w][lane] = (c4[0] + c4[1]) + (c4[2] + c4[3]);
  __syncthreads();
  if (w == 0 && e < n) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += sh[k][lane];
    out[e] = s;
  }
}

// Groups of CTAs the first merge level forms from nctas per-CTA partials.
static int merge_groups(int nctas) { return std::max(1, std::min(kMergeGroups, nctas / 8)); }

// First level only: tmp[g][e] = sum over the CTAs of group g of part[c][e] (the block solve
// adds the groups itself).
static vest_status vec_merge_groups(const double* part, int nctas, int n, double* tmp, cudaStream_t s) {
  const dim3 g1((unsigned)ceil_div(n, 32), (unsigned)merge_groups(nctas));
  core_vec_merge1_kernel<<<g1, 256, 0, s>>>(part, nctas, n, tmp);
  VEST_LAUNCH("core_vec_merge1_kernel");
  return VEST_OK;
}

// sum over c < nctas of part[c][e] -> out[e], in two FP64 levels (groups of CTAs, then
// the groups in order); tmp holds kMergeGroups x n doubles.
static vest_status vec_merge(const double* part, int nctas, int n, double* out, double* tmp, cudaStream_t s) {
  const int groups = merge_groups(nctas);
  const dim3 g1((unsigned)ceil_div(n, 32), (unsigned)groups);
  core_vec_merge1_kernel<<<g1, 256, 0, s>>>(part, nctas, n, tmp);
  VEST_LAUNCH("core_vec_merge1_kernel");
  core_vec_merge_kernel<<<(unsigned)ceil_div(n, 32), 256, 0, s>>>(tmp, groups, n, out);
  VEST_LAUNCH("core_vec_merge_kernel");
  return VEST_OK;
}

// Exact sequential updates of one block (Eq. 12 / Eq. 14): thread l holds element l's
// running sum g_l - sum_{k<l} M_kl Delta_k, its value, mask and the reciprocal of its
// denominator.  At step k thread k computes the new value alone and posts Delta_k in shared
// memory; after the step's barrier every thread l > k subtracts Delta_k M_kl.
//
// FP64 issues slowly on this part, so the block's elements are spread over four warps (one
// per SM sub-partition) rather than held four to a lane in one warp: a step's FP64 work is
// then one FMA on each sub-partition plus the owner's two, not four FMAs and the owner's work
// on one.  The new value is one FMA (the terms that stay fixed during the solve are folded in
// beforehand) and its rounding to the storage type is done on the bit pattern.  Thread counts
// and the order of every operation are fixed, so the result does not depend on the device.
// g arrives as ngroups partial vectors (the g pass's first merge level), g_l = the sum of
// gpart[i][l] over i in a fixed order (four interleaved FP64 chains, then their sum).
template <typename T>
__global__ void __launch_bounds__(kCoreMaxB) core_solve_kernel(DevModel<T> M, CoreBlock blk, int J0, int J1, int reg,
                                                               double lambda, const double* gram,
                                                               const double* __restrict__ gpart, int ngroups,
                                                               double* __restrict__ dout) {
  extern __shared__ double sgram[];
  __shared__ double s_dk[2];
  __shared__ int s_upd[2];
  const int l = threadIdx.x;
  const int b = blk.b;
  for (int e = l; e < b * (b + 1) / 2; e += blockDim.x) sgram[e] = gram[e];
  __syncthreads();
  auto lin_of = [&](int k) {
    return (int64_t)(k % J0) + (int64_t)J0 * (blk.q0 + k / J0) + (int64_t)J0 * J1 * blk.s;
  };
  const bool l1 = reg == VEST_REG_L1;
  const bool in = l < b;
  // LF: new = grad * inv + cst, cst = old M_ll inv (Eq. 12: (grad + old M_ll) / (lambda + M_ll));
  // L1: t = grad + cst, cst = old M_ll; new = (2t + lambda) / (2 M_ll) below -lambda / 2,
  // (2t - lambda) / (2 M_ll) above lambda / 2, else 0 (Eq. 14 with g = -2t)
  double grad = 0.0, gv = 0.0, iv = 0.0, cs = 0.0;
  bool fr = false;
  if (in) {
    double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;
    int i = 0;
    for (; i + 3 < ngroups; i += 4) {
      c0 += gpart[(size_t)i * b + l];
      c1 += gpart[(size_t)(i + 1) * b + l];
      c2 += gpart[(size_t)(i + 2) * b + l];
      c3 += gpart[(size_t)(i + 3) * b + l];
    }
    for (; i < ngroups; ++i) c0 += gpart[(size_t)i * b + l];
    grad = (c0 + c1) + (c2 + c3);
    gv = (double)M.G[lin_of(l)];
    fr = !M.Gmask[lin_of(l)];
    const double mll = sgram[sym_index(l, l, b)];
    iv = l1 ? 1.0 / (2.0 * mll) : 1.0 / (lambda + mll);
    cs = l1 ? gv * mll : gv * mll * iv;
  }
  const double half = 0.5 * lambda;
  for (int k = 0; k < b; ++k) {
    const bool later = in && l > k;
    const double mkl = later ? sgram[sym_index(k, l, b)] : 0.0;
    if (l == k) {
      double dk = 0.0;
      int upd = 0;
      if (fr) {
        double nv;
        if (l1) {
          const double t = grad + cs;
          nv = t < -half ? fma(t, 2.0 * iv, lambda * iv) : (t > half ? fma(t, 2.0 * iv, -lambda * iv) : 0.0);
        } else {
          nv = fma(grad, iv, cs);
        }
        const double nr = sizeof(T) == 4 ? round_to_single(nv) : nv;
        M.G[lin_of(k)] = (T)nr;
        const unsigned long long a = static_cast<unsigned long long>(__double_as_longlong(nr)),
                                 o = static_cast<unsigned long long>(__double_as_longlong(gv));
        upd = a != o && ((a | o) << 1) != 0ull;  // the value changed (either zero counts as equal)
        if (upd) dk = nr - gv;
      }
      dout[k] = dk;
      s_dk[k & 1] = dk;
      s_upd[k & 1] = upd;
    }
    // one barrier a step: the slots alternate, so step k + 1's post cannot overwrite the
    // value a thread of step k has yet to read
    __syncthreads();
    if (s_upd[k & 1] && later) grad = fma(-s_dk[k & 1], mkl, grad);
  }
}

// ================================================================== stats pass (responsibility)
// For a group of suffixes [s0, s0 + Sg) and every j_1: per piece sum r w and sum w^2
// with w = a1[j_1] c(s); then S1(j0, j1, s) += a0[j0] sum r w, S2 += a0[j0]^2 sum w^2.
struct StatsArgs {
  int J0, J1;
  int64_t s0;
  int Sg, SJ;
  int64_t nnz, ntasks;
  size_t red_off;  // byte offset in shared memory of the FP64 warp reduction
  double* part;    // [ctas][2 * J0 * SJ]
};

// Streams (pairs (j_1, s) of the group) per lane in the stats pass: the accumulators
// (kinds x J0B x streams) stay in registers with two CTAs per SM.
__host__ __device__ constexpr int stats_spl(int J0B, bool diag) {
  return diag ? (J0B <= 12 ? 2 : 1) : (J0B <= 12 ? 4 : (J0B <= 16 ? 2 : 1));
}

// Shared memory of the stats pass: per warp the staged entries and the running sums.
__host__ __device__ inline size_t stats_stage_elems(int J0, int J1, int Sg) { return (size_t)32 * (J0 + J1 + Sg + 1); }
__host__ __device__ inline size_t stats_run_elems(int J0, int spl, int kinds) { return (size_t)kinds * 2 * J0 * 32 * spl; }

// Stats pass for one group of Sg suffixes: for every core element (j0, j1, s) of the group
//   g(j0, j1, s)    = sum_alpha r a0[j0] a1[j1] c(s)
//   diag(j0, j1, s) = sum_alpha (a0[j0] a1[j1] c(s))^2   (DIAG only: right after a core
//                     sweep the block Grams hold it already).
// Each warp takes whole 256-entry tasks of the mode-0 CSR (warp-strided over the grid) and
// walks them 32 entries at a time: the lanes stage one entry each (row, r, a0 row, a1 row,
// c(s) of the group) in shared memory; then every lane runs through the 32 entries in order
// for its own pairs (j1, s), summing h1 = sum r y and h2 = sum y^2 (y = a1[j1] c(s)) while
// the row stays the same.  At a row change and at the end of the task the lane adds
// a0 (x) h1 and a0^2 (x) h2 into its task sums; at the end of the task those go into the
// warp's running sums in shared memory (Kahan).  Warps are combined in warp order in FP64,
// one partial per CTA.
template <typename T, int J0B, bool DIAG>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && J0B <= 16) ? 2 : 1)
    core_stats_kernel(DevModel<T> M, DevMode<T> csr, const T* __restrict__ r, const T* __restrict__ A0c, StatsArgs a) {
  constexpr int SPL = stats_spl(J0B, DIAG);
  constexpr int KINDS = DIAG ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int J0 = a.J0, J1 = a.J1, Sg = a.Sg, SJ = a.SJ;
  const int ld = J0 + J1 + Sg + 1;  // staged entry: a0 row (where a row starts), a1 row, c(s), r
  T* base = reinterpret_cast<T*>(smem_raw);
  const size_t stage = stats_stage_elems(J0, J1, Sg), run = stats_run_elems(J0, SPL, KINDS);
  T* st = base + (size_t)warp * stage;
  // running sums of this lane: [kind][j0][i] x (sum, comp), lane-interleaved
  T* rs = base + (size_t)nwarps * stage + (size_t)warp * run;
  int* sk = reinterpret_cast<int*>(base + (size_t)nwarps * (stage + run)) + warp * 32;
  // [2][J0][SJ] after the pass: over the staged entries, never over the running sums
  double* red = reinterpret_cast<double*>(smem_raw + a.red_off);
  for (size_t e = lane; e < run; e += 32) rs[e] = T(0);
  int qo[SPL], so[SPL];
  bool on[SPL];
#pragma unroll
  for (int i = 0; i < SPL; ++i) {
    const int pr = lane + 32 * i;
    on[i] = pr < SJ;
    qo[i] = on[i] ? pr % J1 : 0;
    so[i] = on[i] ? pr / J1 : 0;
  }
  T t1s[J0B][SPL], t2s[J0B][SPL];
  T a0r[J0B];
  T h1[SPL], h2[SPL];
  const int64_t gw = (int64_t)blockIdx.x * nwarps + warp, nw = (int64_t)gridDim.x * nwarps;
  // the coalesced loads of a chunk (row, its position in A0c, mode-1 index, mode-2 index
  // when N = 3, r) are issued one chunk ahead
  const bool n3 = M.N == 3;
  const bool pair1 = rows_paired(M, 1, 0), pair2 = n3 && rows_paired(M, 2, a.s0);
  int nk = 0, ni1 = 0, ni2 = 0;
  T nrv = T(0);
  auto prefetch = [&](int64_t p) {
    if (p >= 0 && p < a.nnz) {
      nk = csr.rowk[p];
      ni1 = csr.oidx[p];
      if (n3) ni2 = csr.oidx[a.nnz + p];
      nrv = r[p];
    }
  };
  if (gw < a.ntasks) prefetch(gw * kCoreTask + lane);
  for (int64_t task = gw; task < a.ntasks; task += nw) {
    const int64_t t0 = task * kCoreTask, t1 = min(t0 + (int64_t)kCoreTask, a.nnz);
#pragma unroll
    for (int j = 0; j < J0B; ++j)
#pragma unroll
      for (int i = 0; i < SPL; ++i) t1s[j][i] = t2s[j][i] = T(0);
    int cur = -1;
    for (int64_t c0 = t0; c0 < t1; c0 += 32) {
      const int64_t p = c0 + lane;
      const int k = nk, i1 = ni1, i2 = ni2;
      const T rv = nrv;
      // next chunk of this warp: the rest of the task, else the first chunk of its next task
      prefetch(c0 + 32 < t1 ? c0 + 32 + lane : (task + nw < a.ntasks ? (task + nw) * kCoreTask + lane : -1));
      const int kup = __shfl_up_sync(0xffffffffu, k, 1);
      __syncwarp();
      if (p < t1) {
        sk[lane] = k;
        T* se = st + lane * ld;
        // a0 is read only where a row starts inside the chunk (and at lane 0)
        if (lane == 0 || kup != k) {
          const T* a0 = A0c + (int64_t)k * J0;
          for (int j = 0; j < J0; ++j) se[j] = a0[j];
        }
        copy_row<T>(M.A[1] + (int64_t)i1 * J1, J1, pair1, se + J0);
        if (n3) {
          copy_row<T>(M.A[2] + (int64_t)i2 * M.J[2] + a.s0, Sg, pair2, se + J0 + J1);
        } else {
          suffix_weights<T>(M, csr.oidx, a.nnz, p, a.s0, Sg, se + J0 + J1, 1);
        }
        se[J0 + J1 + Sg] = rv;
      }
      __syncwarp();
      const int n = (int)min((int64_t)32, t1 - c0);
      for (int e = 0; e < n; ++e) {
        const int k = sk[e];
        const T* se = st + e * ld;
        if (k != cur) {
          if (cur >= 0) {
#pragma unroll
            for (int j = 0; j < J0B; ++j)
#pragma unroll
              for (int i = 0; i < SPL; ++i) {
                t1s[j][i] += a0r[j] * h1[i];
                if constexpr (DIAG) t2s[j][i] += a0r[j] * a0r[j] * h2[i];
              }
          }
          cur = k;
#pragma unroll
          for (int j = 0; j < J0B; ++j) a0r[j] = j < J0 ? se[j] : T(0);
#pragma unroll
          for (int i = 0; i < SPL; ++i) h1[i] = h2[i] = T(0);
        }
        const T rv = se[J0 + J1 + Sg];
#pragma unroll
        for (int i = 0; i < SPL; ++i) {
          const T y = se[J0 + qo[i]] * se[J0 + J1 + so[i]];
          h1[i] += rv * y;
          if constexpr (DIAG) h2[i] += y * y;
        }
      }
    }
    if (cur >= 0) {
#pragma unroll
      for (int j = 0; j < J0B; ++j)
#pragma unroll
        for (int i = 0; i < SPL; ++i) {
          t1s[j][i] += a0r[j] * h1[i];
          if constexpr (DIAG) t2s[j][i] += a0r[j] * a0r[j] * h2[i];
        }
    }
#pragma unroll
    for (int j = 0; j < J0B; ++j) {
      if (j < J0) {
#pragma unroll
        for (int i = 0; i < SPL; ++i) {
          T* x1 = rs + ((size_t)(0 * J0 + j) * SPL + i) * 64 + lane;
          CoreAcc<T>::add(x1[0], x1[32], t1s[j][i]);
          if constexpr (DIAG) {
            T* x2 = rs + ((size_t)(1 * J0 + j) * SPL + i) * 64 + lane;
            CoreAcc<T>::add(x2[0], x2[32], t2s[j][i]);
          }
        }
      }
    }
  }
  // warps in order, FP64: red[kind * J0 * SJ + j0 + J0 * pair]
  __syncthreads();
  const int nacc = KINDS * J0 * SJ;
  for (int w = 0; w < nwarps; ++w) {
    if (warp == w) {
      for (int j = 0; j < J0; ++j) {
#pragma unroll
        for (int i = 0; i < SPL; ++i) {
          if (on[i]) {
            const T* x1 = rs + ((size_t)(0 * J0 + j) * SPL + i) * 64 + lane;
            const int e1 = j + J0 * (lane + 32 * i);
            const double v1 = CoreAcc<T>::value(x1[0], x1[32]);
            red[e1] = w == 0 ? v1 : red[e1] + v1;
            if constexpr (DIAG) {
              const T* x2 = rs + ((size_t)(1 * J0 + j) * SPL + i) * 64 + lane;
              const int e2 = J0 * SJ + e1;
              const double v2 = CoreAcc<T>::value(x2[0], x2[32]);
              red[e2] = w == 0 ? v2 : red[e2] + v2;
            }
          }
        }
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nacc; e += blockDim.x) a.part[(size_t)blockIdx.x * nacc + e] = red[e];
}

// Delta and Resp of the group's core elements: lin = j0 + J0 (j1 + J1 s).
// diag M of the element: sums[n + e] when the stats pass formed it, else the diagonal of
// its block Gram (block (s, j1 / m), local index j0 + J0 (j1 - q0)).
struct DiagSrc {
  const double* gram;  // NULL: diag in sums
  int m, nq0;
  int64_t nmmax;
};

template <typename T>
__global__ void core_resp_kernel(DevModel<T> M, int J0, int J1, int64_t s0, int SJ, const double* __restrict__ sums,
                                 DiagSrc ds, const double* __restrict__ stats, double* __restrict__ delta,
                                 double* __restrict__ resp) {
  const double xx = stats[1], re = stats[4];
  const int n = J0 * SJ;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int64_t lin = (int64_t)J0 * J1 * s0 + e;  // e = j0 + J0 * (j1 + J1 * si)
    const double gv = (double)M.G[lin];
    double dg;
    if (ds.gram) {
      const int j0 = e % J0, j1 = (e / J0) % J1;
      const int64_t sfx = s0 + e / (J0 * J1);
      const int qc = j1 / ds.m, q0 = qc * ds.m, mq = min(ds.m, J1 - q0), b = J0 * mq;
      const int kk = j0 + J0 * (j1 - q0);
      dg = ds.gram[(sfx * ds.nq0 + qc) * ds.nmmax + sym_index(kk, kk, b)];
    } else {
      dg = sums[n + e];
    }
    const double dl = 2.0 * gv * sums[e] + gv * gv * dg;
    delta[lin] = dl;
    if (resp) resp[lin] = re > 0.0 ? (sqrt(fmax(re * re + dl / xx, 0.0)) - re) / re : 0.0;
  }
}

// ------------------------------------------------------------------ host side
struct CorePlan {
  int J0, J1, m, nq0;
  int64_t S;       // suffixes
  int64_t nblocks;
  int bmax, nmmax;
  int nX, nYmax, SgMax, Pmax;  // gram groups
  int SgStats, SJ;             // stats groups (g and diag M)
  int SgStatsG, SJG;           // stats groups (g alone, diag M from the block Grams)
  int64_t slots;
};

static int64_t stats_nacc_max(const struct CorePlan& c);

static CorePlan core_plan(const int32_t* J, int N, int64_t nnz, int64_t cap0) {
  CorePlan c{};
  c.J0 = J[0];
  c.J1 = J[1];
  c.m = std::min(std::min(std::max(1, kCoreMaxB / c.J0), c.J1), kCoreMaxM);
  c.nq0 = (c.J1 + c.m - 1) / c.m;
  c.S = 1;
  for (int n = 2; n < N; ++n) c.S *= J[n];
  c.nblocks = c.S * c.nq0;
  c.bmax = c.J0 * c.m;
  c.nmmax = c.bmax * (c.bmax + 1) / 2;
  c.nX = c.J0 * (c.J0 + 1) / 2;
  c.nYmax = c.m * (c.m + 1) / 2;
  c.SgMax = (int)std::min<int64_t>(c.S, kGramSgB);
  c.Pmax = 0;
  for (int q0 = 0; q0 < c.J1; q0 += c.m) {  // the last j_1 chunk may be narrower and take more suffixes
    const int mq = std::min(c.m, c.J1 - q0), nY = mq * (mq + 1) / 2;
    c.Pmax = std::max(c.Pmax, c.SgMax * nY);
  }
  // stats: 32 * stats_spl streams (j1, s) per group
  const int streams = 32 * stats_spl(jn_bucket(c.J0), true);
  const int sg = (int)std::max<int64_t>(1, std::min<int64_t>(c.S, streams / c.J1));
  c.SgStats = sg;
  c.SJ = sg * c.J1;
  const int streams_g = 32 * stats_spl(jn_bucket(c.J0), false);
  const int sgg = (int)std::max<int64_t>(1, std::min<int64_t>(c.S, streams_g / c.J1));
  c.SgStatsG = sgg;
  c.SJG = sgg * c.J1;
  c.slots = cap0 + ceil_div(std::max<int64_t>(nnz, 1), kCoreTask) + 1;
  return c;
}

// outputs of one stats group, at most: 2 J0 SJ with diag, J0 SJG without
static int64_t stats_nacc_max(const CorePlan& c) {
  return std::max<int64_t>((int64_t)2 * c.J0 * c.SJ, (int64_t)c.J0 * c.SJG);
}

size_t core_scratch_bytes(const vest_model* m, int64_t nnz, int64_t cap0, size_t* y_bytes, size_t* gram_bytes,
                          size_t* part_bytes) {
  const CorePlan c = core_plan(m->ranks, m->order, nnz, cap0);
  const size_t sT = m->dtype == VEST_F64 ? 8 : 4;
  // per-piece gram statistics, later reused for u and the a0 row of every non-empty mode-0 row
  // (cap0 x (kCoreMaxM + J0))
  *y_bytes = align_up(std::max((size_t)c.slots * c.Pmax, (size_t)(cap0 + 1) * (kCoreMaxM + c.J0)) * sT) +
             align_up((size_t)c.slots * 4) + align_up((size_t)c.slots * c.nX * sT);
  // the gram region also holds the responsibility sums (2 * J0 * SJ doubles)
  *gram_bytes = align_up(std::max((size_t)c.nblocks * c.nmmax, (size_t)2 * c.J0 * c.SJ) * 8);
  const size_t gemm = (size_t)kGramKSplit * c.nX * c.Pmax * 8;
  const size_t gp = (size_t)(kGPassCtas + kMergeGroups) * kCoreMaxB * 8;
  // per-CTA partials, the merge's groups and the merged sums of one stats group
  const size_t st = (size_t)(kCorePassCtas + kMergeGroups + 1) * stats_nacc_max(c) * 8;
  *part_bytes = align_up(std::max({gemm, gp, st}));
  return *y_bytes + *gram_bytes + *part_bytes;
}

// Suffix slots per lane and pair in the gram pass: the smallest of 4, 8, 12, 16 that holds Sg.
static int gram_sgb(int Sg) { return Sg <= 4 ? 4 : Sg <= 8 ? 8 : Sg <= 12 ? 12 : 16; }

template <typename T>
static size_t smem_gram(int mq, int sgb) {
  const int V = 16 / (int)sizeof(T);
  const int ld = (sgb + mq + V - 1) / V * V;
  return (size_t)8 * 32 * ld * sizeof(T) + (size_t)8 * 32 * 4;
}

template <typename T, int SGB>
static vest_status launch_gram(const DevModel<T>& M, const DevMode<T>& csr, const GramArgs& ga, int grid,
                               cudaStream_t s) {
  const size_t smem = smem_gram<T>(ga.mq, SGB);
  auto kern = core_gram_pass_kernel<T, SGB>;
  VEST_TRY(allow_smem(kern, smem));
  kern<<<grid, 256, smem, s>>>(M, csr, ga);
  VEST_LAUNCH("core_gram_pass_kernel");
  return VEST_OK;
}

// Shared memory of the stats pass; *red_off receives the offset of the FP64 warp
// reduction: inside the staging region when it fits there, else behind everything.
template <typename T>
static size_t smem_stats(int J0, int J1, int Sg, int SJ, int nwarps, bool diag, size_t* red_off = nullptr) {
  const int spl = stats_spl(jn_bucket(J0), diag), kinds = diag ? 2 : 1;
  const size_t pass = (size_t)nwarps * (stats_stage_elems(J0, J1, Sg) + stats_run_elems(J0, spl, kinds)) * sizeof(T) +
                      (size_t)nwarps * 32 * 4;
  const size_t red = (size_t)kinds * J0 * SJ * 8;
  const bool inside = red <= (size_t)nwarps * stats_stage_elems(J0, J1, Sg) * sizeof(T);
  if (red_off) *red_off = inside ? 0 : align_up(pass, 16);
  return inside ? pass : align_up(pass, 16) + red;
}

// Warps per CTA of the stats pass: 8 unless the shared memory would exceed 200 KB.
template <typename T>
static int stats_warps(int J0, int J1, int Sg, int SJ, bool diag) {
  int w = 8;
  while (w > 1 && smem_stats<T>(J0, J1, Sg, SJ, w, diag) > 200 * 1024) w /= 2;
  return w;
}

template <typename T, int J0B>
static vest_status launch_stats(const DevModel<T>& M, const DevMode<T>& csr, const T* r, const T* A0c,
                                const StatsArgs& a, bool diag, int grid, int nwarps, size_t smem, cudaStream_t s) {
  auto kern = diag ? core_stats_kernel<T, J0B, true> : core_stats_kernel<T, J0B, false>;
  VEST_TRY(allow_smem(kern, smem));
  kern<<<grid, 32 * nwarps, smem, s>>>(M, csr, r, A0c, a);
  VEST_LAUNCH("core_stats_kernel");
  return VEST_OK;
}

struct CoreBufs {
  void* Y;
  int32_t* srow;
  void* Xs;
  double* gram;
  double* part;
  double* small;
};

static CoreBufs core_bufs(const vest_index* ix, const vest_model* m, char* scratch, const ScratchPlan& plan) {
  const CorePlan c = core_plan(m->ranks, m->order, ix->nnz, ix->mode[0].cap);
  const size_t sT = m->dtype == VEST_F64 ? 8 : 4;
  CoreBufs b;
  char* base = scratch + plan.off_core;
  b.Y = base;
  b.srow = reinterpret_cast<int32_t*>(
      base + align_up(std::max((size_t)c.slots * c.Pmax, (size_t)(ix->mode[0].cap + 1) * (kCoreMaxM + c.J0)) * sT));
  b.Xs = reinterpret_cast<char*>(b.srow) + align_up((size_t)c.slots * 4);
  size_t yb, gb, pb;
  core_scratch_bytes(m, ix->nnz, ix->mode[0].cap, &yb, &gb, &pb);
  b.gram = reinterpret_cast<double*>(base + yb);
  b.part = reinterpret_cast<double*>(base + yb + gb);
  b.small = reinterpret_cast<double*>(scratch + plan.off_small);
  return b;
}

// All block Grams, packed, block bi at gram + bi * nmmax.
template <typename T>
static vest_status core_grams(const vest_index* ix, const DevModel<T>& M, const CorePlan& c, const CoreBufs& bf,
                              cudaStream_t s) {
  const DevMode<T> csr = dev_mode<T>(ix, 0);
  const int64_t ntasks = ceil_div(ix->nnz, kCoreTask);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ntasks, 8), (int64_t)num_sms() * 2));
  // every gram pass writes the same slots (one per row piece): clear them once
  VEST_CUDA(cudaMemsetAsync(bf.srow, 0xFF, (size_t)c.slots * 4, s));
  bool have_x = false;
  for (int qc = 0; qc < c.nq0; ++qc) {
    const int q0 = qc * c.m, mq = std::min(c.m, c.J1 - q0), nY = mq * (mq + 1) / 2;
    const int Sg = c.SgMax;
    for (int64_t s0 = 0; s0 < c.S; s0 += Sg) {
      const int sg = (int)std::min<int64_t>(Sg, c.S - s0);
      GramArgs ga{};
      ga.J0 = c.J0;
      ga.J1 = c.J1;
      ga.q0 = q0;
      ga.mq = mq;
      ga.nY = nY;
      ga.s0 = s0;
      ga.Sg = sg;
      ga.P = sg * nY;
      ga.nnz = ix->nnz;
      ga.ntasks = ntasks;
      ga.Y = bf.Y;
      ga.srow = bf.srow;
      if (ix->nnz > 0) {
        switch (gram_sgb(sg)) {
          case 4: VEST_TRY((launch_gram<T, 4>(M, csr, ga, grid, s))); break;
          case 8: VEST_TRY((launch_gram<T, 8>(M, csr, ga, grid, s))); break;
          case 12: VEST_TRY((launch_gram<T, 12>(M, csr, ga, grid, s))); break;
          default: VEST_TRY((launch_gram<T, 16>(M, csr, ga, grid, s))); break;
        }
      }
      if (!have_x) {
        core_gram_x_kernel<T><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(c.slots * c.nX, 256),
                                                                                (int64_t)num_sms() * 8)),
                                256, 0, s>>>(M, csr, bf.srow, c.slots, c.J0, c.nX, static_cast<T*>(bf.Xs));
        VEST_LAUNCH("core_gram_x_kernel");
        have_x = true;
      }
      GemmArgs gm{};
      gm.J0 = c.J0;
      gm.nX = c.nX;
      gm.P = ga.P;
      gm.nslots = c.slots;
      gm.Xs = bf.Xs;
      gm.Y = bf.Y;
      gm.srow = bf.srow;
      gm.part = bf.part;
      const dim3 gg((unsigned)(((c.nX + 63) / 64) * ((ga.P + 63) / 64)), kGramKSplit);
      core_gram_gemm_kernel<T><<<gg, 256, 0, s>>>(gm);
      VEST_LAUNCH("core_gram_gemm_kernel");
      const int b = c.J0 * mq, nm = b * (b + 1) / 2;
      core_gram_merge_kernel<<<dim3((unsigned)ceil_div(nm, 256), (unsigned)sg), 256, 0, s>>>(
          bf.part, kGramKSplit, c.nX, ga.P, c.J0, mq, nY, s0, c.nq0, qc, c.nmmax, bf.gram);
      VEST_LAUNCH("core_gram_merge_kernel");
    }
  }
  return VEST_OK;
}

template <typename T>
vest_status sweep_core_impl(const vest_index* ix, const vest_model* mdl, int reg, double lambda, char* scratch,
                            const ScratchPlan& plan, cudaStream_t s, double* final_loss) {
  const DevModel<T> M = dev_model<T>(mdl);
  if (M.N < 2) return fail(VEST_ERR_UNSUPPORTED, "order < 2");
  const CorePlan c = core_plan(M.J, M.N, ix->nnz, ix->mode[0].cap);
  const CoreBufs bf = core_bufs(ix, mdl, scratch, plan);
  T* r0 = reinterpret_cast<T*>(scratch + plan.off_resid);
  double* out = bf.small + 9000 + 3 * kCoreMaxB;
  double* dbuf[2] = {bf.small + 9000, bf.small + 9000 + kCoreMaxB};
  VEST_TRY(loss_impl<T>(ix, mdl, reg, lambda, out, r0, nullptr, scratch, plan, s));
  VEST_TRY(core_grams<T>(ix, M, c, bf, s));
  const DevMode<T> csr = dev_mode<T>(ix, 0);
  GPassArgs a{};
  a.J0 = c.J0;
  a.J1 = c.J1;
  a.nnz = ix->nnz;
  a.part = bf.part;
  // the per-piece gram region is free again: u and the a0 row per non-empty row
  T* U = reinterpret_cast<T*>(bf.Y);
  T* A0c = U + (size_t)(ix->mode[0].cap + 1) * kCoreMaxM;
  a.pair_u = reinterpret_cast<uintptr_t>(U) % (2 * sizeof(T)) == 0;
  const int nctas_g = kGPassCtas;
  const size_t gsm = (size_t)8 * 32 * c.J0 * sizeof(T);
  double* gpart = bf.part + (size_t)kGPassCtas * kCoreMaxB;  // the g pass's merge groups, read by the solve
  int ngroups = merge_groups(nctas_g);
  if (ix->nnz > 0) {
    core_a0c_kernel<T><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ix->mode[0].cap * c.J0, 256),
                                                                         num_sms() * 8)),
                         256, 0, s>>>(M, csr.nzrow, csr.nnzrows, c.J0, A0c);
    VEST_LAUNCH("core_a0c_kernel");
    VEST_TRY(allow_smem(core_g_pass_kernel<T>, gsm));
  }
  int64_t iblk = 0;
  for (int64_t sfx = 0; sfx < c.S; ++sfx) {
    for (int qc = 0; qc < c.nq0; ++qc, ++iblk) {
      const int q0 = qc * c.m;
      CoreBlock blk{sfx, q0, std::min(c.m, c.J1 - q0), 0};
      blk.b = c.J0 * blk.m;
      a.cur = blk;
      a.has_prev = iblk > 0;
      a.pair_a1 = c.J1 % 2 == 0 && blk.q0 % 2 == 0 && (!a.has_prev || a.prev.q0 % 2 == 0) &&
                  reinterpret_cast<uintptr_t>(M.A[1]) % (2 * sizeof(T)) == 0;
      if (ix->nnz > 0) {
        if (a.has_prev) {
          core_u_kernel<T><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ix->mode[0].cap, 256), num_sms() * 4)),
                             256, 0, s>>>(M, csr.nzrow, csr.nnzrows, dbuf[(iblk + 1) & 1], c.J0, a.prev.m, U);
          VEST_LAUNCH("core_u_kernel");
        }
        core_g_pass_kernel<T><<<nctas_g, 256, gsm, s>>>(M, csr, r0, U, A0c, a);
        VEST_LAUNCH("core_g_pass_kernel");
        VEST_TRY(vec_merge_groups(bf.part, nctas_g, blk.b, gpart, s));
      } else {
        ngroups = 0;  // no entries: g = 0
      }
      const size_t ssm = (size_t)(blk.b * (blk.b + 1) / 2) * 8;
      auto sk = core_solve_kernel<T>;
      VEST_TRY(allow_smem(sk, ssm));
      sk<<<1, kCoreMaxB, ssm, s>>>(M, blk, c.J0, c.J1, reg, lambda, bf.gram + iblk * c.nmmax, gpart, ngroups,
                                   dbuf[iblk & 1]);
      VEST_LAUNCH("core_solve_kernel");
      a.prev = blk;
    }
  }
  if (!final_loss) return VEST_OK;
  // the last block's change still has to reach r; then the loss sums and the COO copy
  const int nl = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ix->nnz, 1024), loss_ctas()));
  double* lpart = reinterpret_cast<double*>(scratch + plan.off_part);
  if (ix->nnz > 0) {
    core_u_kernel<T><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ix->mode[0].cap, 256), num_sms() * 4)),
                       256, 0, s>>>(M, csr.nzrow, csr.nnzrows, dbuf[(iblk + 1) & 1], c.J0, a.prev.m, U);
    VEST_LAUNCH("core_u_kernel");
    core_final_kernel<T><<<nl, 256, 0, s>>>(M, csr, r0, reinterpret_cast<T*>(scratch + plan.off_resid_coo), U, a.prev,
                                            lpart);
    VEST_LAUNCH("core_final_kernel");
  }
  return loss_finish<T>(mdl, reg, lambda, ix->nnz > 0 ? nl : 0, final_loss, scratch, plan, s);
}

template <typename T>
vest_status core_responsibility(const vest_index* ix, const vest_model* mdl, const T* resid_csr0, const double* stats,
                                double* delta_core, double* resp_core, char* scratch, const ScratchPlan& plan,
                                cudaStream_t s, bool grams_valid) {
  const DevModel<T> M = dev_model<T>(mdl);
  if (M.N < 2) return fail(VEST_ERR_UNSUPPORTED, "order < 2");
  const CorePlan c = core_plan(M.J, M.N, ix->nnz, ix->mode[0].cap);
  const CoreBufs bf = core_bufs(ix, mdl, scratch, plan);
  const DevMode<T> csr = dev_mode<T>(ix, 0);
  const int64_t ntasks = ceil_div(ix->nnz, kCoreTask);
  // right after a core sweep with these factors the block Grams hold diag M: the stats pass forms g alone
  const bool diag = !grams_valid;
  const int sgs = diag ? c.SgStats : c.SgStatsG;
  const DiagSrc ds{diag ? nullptr : bf.gram, c.m, c.nq0, c.nmmax};
  const int64_t nmax = stats_nacc_max(c);
  double* sums = bf.part + (size_t)(kCorePassCtas + kMergeGroups) * nmax;
  T* A0c = reinterpret_cast<T*>(bf.Y);  // the per-piece gram region is free here: a0 per non-empty row
  if (ix->nnz > 0) {
    core_a0c_kernel<T><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ix->mode[0].cap * c.J0, 256),
                                                                         num_sms() * 8)),
                         256, 0, s>>>(M, csr.nzrow, csr.nnzrows, c.J0, A0c);
    VEST_LAUNCH("core_a0c_kernel");
  }
  for (int64_t s0 = 0; s0 < c.S; s0 += sgs) {
    StatsArgs a{};
    a.J0 = c.J0;
    a.J1 = c.J1;
    a.s0 = s0;
    a.Sg = (int)std::min<int64_t>(sgs, c.S - s0);
    a.SJ = a.Sg * c.J1;
    a.nnz = ix->nnz;
    a.ntasks = ntasks;
    a.part = bf.part;
    const int nacc = (diag ? 2 : 1) * c.J0 * a.SJ;
    if (ix->nnz > 0) {
      const int nwarps = stats_warps<T>(c.J0, c.J1, a.Sg, a.SJ, diag);
      const int nctas = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ntasks, nwarps), kCorePassCtas));
      const size_t smem = smem_stats<T>(c.J0, c.J1, a.Sg, a.SJ, nwarps, diag, &a.red_off);
      switch (jn_bucket(c.J0)) {
        case 4: VEST_TRY(launch_stats<T, 4>(M, csr, resid_csr0, A0c, a, diag, nctas, nwarps, smem, s)); break;
        case 8: VEST_TRY(launch_stats<T, 8>(M, csr, resid_csr0, A0c, a, diag, nctas, nwarps, smem, s)); break;
        case 10: VEST_TRY(launch_stats<T, 10>(M, csr, resid_csr0, A0c, a, diag, nctas, nwarps, smem, s)); break;
        case 12: VEST_TRY(launch_stats<T, 12>(M, csr, resid_csr0, A0c, a, diag, nctas, nwarps, smem, s)); break;
        case 16: VEST_TRY(launch_stats<T, 16>(M, csr, resid_csr0, A0c, a, diag, nctas, nwarps, smem, s)); break;
        default: VEST_TRY(launch_stats<T, 32>(M, csr, resid_csr0, A0c, a, diag, nctas, nwarps, smem, s)); break;
      }
      VEST_TRY(vec_merge(bf.part, nctas, nacc, sums, bf.part + (size_t)kCorePassCtas * nacc, s));
    } else {
      VEST_CUDA(cudaMemsetAsync(sums, 0, (size_t)nacc * 8, s));
    }
    core_resp_kernel<T><<<(unsigned)ceil_div(c.J0 * a.SJ, 256), 256, 0, s>>>(M, c.J0, c.J1, s0, a.SJ, sums, ds, stats,
                                                                              delta_core, resp_core);
    VEST_LAUNCH("core_resp_kernel");
  }
  return VEST_OK;
}

template vest_status sweep_core_impl<float>(const vest_index*, const vest_model*, int, double, char*,
                                            const ScratchPlan&, cudaStream_t, double*);
template vest_status sweep_core_impl<double>(const vest_index*, const vest_model*, int, double, char*,
                                             const ScratchPlan&, cudaStream_t, double*);
template vest_status core_responsibility<float>(const vest_index*, const vest_model*, const float*, const double*,
                                                double*, double*, char*, const ScratchPlan&, cudaStream_t, bool);
template vest_status core_responsibility<double>(const vest_index*, const vest_model*, const double*, const double*,
                                                 double*, double*, char*, const ScratchPlan&, cudaStream_t, bool);

}  // namespace vest
