// Core sweep (Lemma 2, Eq. 12; Lemma 4, Eq. 14) and the core part of the
// responsibility (Eq. 5, Algorithm 3).
//
// The core elements are updated one at a time in linear order (j_1 fastest),
// as the paper requires (Section 3.6).  On the GPU this is blocked
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
//     (per piece h(q) = sum r w(q), g += a0 (x) h); one thread block performs
//     the b updates in order with sum_alpha r P(k) = g_k - sum_{l<k} Delta_l M_lk.
// The core responsibility needs g and diag(M) of every element for a fixed r:
// one stats pass per group of suffixes.
// Sums: per piece in the storage type; across pieces and tasks FP32 with Kahan
// compensation (or FP64); across thread blocks FP64 in a fixed order.
#include <algorithm>

#include "delta.cuh"

namespace vest {

constexpr int kCoreTask = 256;
constexpr int kCoreMaxB = 128;
constexpr int kCoreMaxM = 10;
constexpr int kGramMaxP = 576;      // per-piece gram outputs per group
constexpr int kGramKSplit = 64;     // fixed: reduction order does not depend on the device
constexpr int kCorePassCtas = 1216;  // fixed likewise (8 per SM on 152 SMs)
constexpr int kStatsEPT = 16;       // stats accumulators per thread
constexpr int kCoreKmax = 64;       // row pieces per phase-2 round

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

// ================================================================== gram pass
struct GramArgs {
  int J0, J1;
  int q0, mq, nY;
  int64_t s0;
  int Sg, P, kmax;
  int64_t nnz, ntasks;
  void* Y;         // [slots][P]
  int32_t* srow;   // [slots]: compacted mode-0 row of the slot, -1 if unused
};

// terms of the gram pass: p = sidx * nY + yi -> c(s)^2 * K(yi)
template <typename T>
struct GramTerm {
  const T* sC;  // [entry][Sg]
  const T* sK;  // [entry][nY]
  int Sg, nY;
  __device__ TermPtrs<T> prep(int p) const { return TermPtrs<T>{sC + p / nY, sK + p % nY, Sg, nY}; }
};

template <typename T>
__global__ void __launch_bounds__(kCoreTask) core_gram_pass_kernel(DevModel<T> M, DevMode<T> csr, GramArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = a.P, nY = a.nY, Sg = a.Sg, mq = a.mq;
  size_t off = 0;
  int64_t* sptr = reinterpret_cast<int64_t*>(smem_raw + off); off += (size_t)(kCoreTask + 2) * 8;
  T* sK = reinterpret_cast<T*>(smem_raw + off); off += (size_t)kCoreTask * nY * sizeof(T);
  T* sC = reinterpret_cast<T*>(smem_raw + off); off += (size_t)kCoreTask * Sg * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  T* sAcc = reinterpret_cast<T*>(smem_raw + off); off += (size_t)a.kmax * P * sizeof(T);
  T* sPart = reinterpret_cast<T*>(smem_raw + off);
  __shared__ PieceScratch pscr;
  const int R = *csr.nnzrows;
  T* Y = static_cast<T*>(a.Y);
  for (int64_t task = blockIdx.x; task < a.ntasks; task += gridDim.x) {
    const int64_t t0 = task * kCoreTask, t1 = min(t0 + (int64_t)kCoreTask, a.nnz);
    const int cnt = (int)(t1 - t0);
    int64_t k0;
    const int nrows = load_task_rows(csr.nzptr, csr.gran, R, t0, t1, sptr, &k0);
    if ((int)threadIdx.x < cnt) {
      const int64_t p = t0 + threadIdx.x;
      const T* a1 = M.A[1] + (int64_t)csr.oidx[p] * a.J1 + a.q0;
      T v[kCoreMaxM];
#pragma unroll
      for (int q = 0; q < kCoreMaxM; ++q) v[q] = q < mq ? a1[q] : T(0);
      T* k = sK + threadIdx.x * nY;
      int yi = 0;
#pragma unroll
      for (int q = 0; q < kCoreMaxM; ++q)
#pragma unroll
        for (int q2 = q; q2 < kCoreMaxM; ++q2)
          if (q2 < mq) k[yi++] = v[q] * v[q2];
      T* c = sC + threadIdx.x * Sg;
      suffix_weights<T>(M, csr.oidx, a.nnz, p, a.s0, Sg, c, 1);
      for (int i = 0; i < Sg; ++i) c[i] *= c[i];
    }
    __syncthreads();
    const GramTerm<T> f{sC, sK, Sg, nY};
    for (int r0 = 0; r0 < nrows; r0 += a.kmax) {
      const int nr = min(a.kmax, nrows - r0);
      piece_sums<T>(sptr + r0, nr, t0, t1, P, sAcc, sPart, &pscr, f);
      for (int kr = 0; kr < nr; ++kr) {
        const int64_t slot = k0 + r0 + kr + task;
        for (int pp = threadIdx.x; pp < P; pp += blockDim.x) Y[slot * P + pp] = sAcc[kr * P + pp];
        if (threadIdx.x == 0) a.srow[slot] = (int32_t)(k0 + r0 + kr);
      }
      __syncthreads();
    }
  }
}

// Z[ks][xi][p] = sum over the slots of split ks of X_slot[xi] * Y[slot][p], X = packed
// upper a0 a0^T of the slot's row.  Tile 32 (xi) x 64 (p); 32-slot chunks in FP32,
// Kahan across chunks.
struct GemmArgs {
  int J0, nX, P;
  int64_t nslots;
  const void* Y;
  const int32_t* srow;
  double* part;  // [ks][nX][P]
};

template <typename T>
__global__ void __launch_bounds__(256) core_gram_gemm_kernel(DevModel<T> M, DevMode<T> csr, GemmArgs a) {
  __shared__ T sX[32][33];
  __shared__ T sY[32][65];
  __shared__ int2 xtab[32];
  const int tiles_p = (a.P + 63) / 64;
  const int tx0 = (blockIdx.x / tiles_p) * 32, tp0 = (blockIdx.x % tiles_p) * 64;
  const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
  const int ks = blockIdx.y;
  const int64_t per = ceil_div(a.nslots, (int64_t)gridDim.y);
  const int64_t sl0 = ks * per, sl1 = min(a.nslots, sl0 + per);
  if (threadIdx.x < 32) {
    const int xi = tx0 + threadIdx.x;
    int ja = 0, jb = 0;
    if (xi < a.nX) sym_decode(xi, a.J0, ja, jb);
    xtab[threadIdx.x] = make_int2(xi < a.nX ? ja : -1, jb);
  }
  const T* Y = static_cast<const T*>(a.Y);
  T run_s[4][2], run_c[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) run_s[i][j] = run_c[i][j] = T(0);
  __syncthreads();
  for (int64_t c0 = sl0; c0 < sl1; c0 += 32) {
    // stage 32 slots: X from the slot's a0 row, Y tile
    for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
      const int cs = i >> 5, xl = i & 31;
      const int64_t slot = c0 + cs;
      T xv = T(0);
      const int2 jt = xtab[xl];
      if (slot < sl1 && jt.x >= 0) {
        const int32_t k = a.srow[slot];
        if (k >= 0) {
          const T* a0 = M.A[0] + (int64_t)csr.nzrow[k] * a.J0;
          xv = a0[jt.x] * a0[jt.y];
        }
      }
      sX[cs][xl] = xv;
    }
    for (int i = threadIdx.x; i < 32 * 64; i += blockDim.x) {
      const int cs = i >> 6, pl = i & 63;
      const int64_t slot = c0 + cs;
      const int p = tp0 + pl;
      T yv = T(0);
      if (slot < sl1 && p < a.P && a.srow[slot] >= 0) yv = Y[slot * a.P + p];
      sY[cs][pl] = yv;
    }
    __syncthreads();
    T acc[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) acc[i][j] = T(0);
#pragma unroll 8
    for (int cs = 0; cs < 32; ++cs) {
      T xv[4], yv[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) xv[i] = sX[cs][ty + 8 * i];
#pragma unroll
      for (int j = 0; j < 2; ++j) yv[j] = sY[cs][tx + 32 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[i][j] += xv[i] * yv[j];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) CoreAcc<T>::add(run_s[i][j], run_c[i][j], acc[i][j]);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int xi = tx0 + ty + 8 * i, p = tp0 + tx + 32 * j;
      if (xi < a.nX && p < a.P)
        a.part[((size_t)ks * a.nX + xi) * a.P + p] = CoreAcc<T>::value(run_s[i][j], run_c[i][j]);
    }
}

// Packed M of block (s0 + sidx, q chunk) in FP64 from the split partials.
__global__ void core_gram_merge_kernel(const double* __restrict__ part, int ksplit, int nX, int P, int J0, int mq,
                                       int nY, int sidx, double* __restrict__ gram) {
  const int b = J0 * mq, nm = b * (b + 1) / 2;
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
struct GPassArgs {
  int J0, J1;
  CoreBlock cur, prev;
  int has_prev;
  int64_t nnz;
  double* part;  // [ctas][b]
};

// u(k, q) = sum_j0 Delta_prev(j0, q) a0[row_k, j0] for every non-empty mode-0 row k.
template <typename T>
__global__ void core_u_kernel(DevModel<T> M, const int32_t* __restrict__ nzrow, const int32_t* __restrict__ nnzrows,
                              const double* __restrict__ dprev, int J0, int mp, T* __restrict__ U) {
  __shared__ double sd[kCoreMaxB];
  for (int i = threadIdx.x; i < J0 * mp; i += blockDim.x) sd[i] = dprev[i];
  __syncthreads();
  const int64_t R = *nnzrows;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < R; k += (int64_t)gridDim.x * blockDim.x) {
    const T* a0 = M.A[0] + (int64_t)nzrow[k] * J0;
    for (int q = 0; q < mp; ++q) {
      T u = T(0);
      for (int j = 0; j < J0; ++j) u += (T)sd[q * J0 + j] * a0[j];
      U[k * kCoreMaxM + q] = u;
    }
  }
}

// One streaming pass per block.  Each warp takes 32 consecutive entries at a
// time: it applies the previous block's Delta to r (r -= c' a1 . u(row)), forms
// h(q) = r a1[q0 + q] c, adds h over each row segment inside the warp, and every
// segment head adds a0[row] (x) h into the warp's g accumulators (lane l holds
// entries l, l + 32, ...; Kahan across heads).  g is linear in the rows, so row
// segments cut by chunk edges need no fix-up.
template <typename T>
__global__ void __launch_bounds__(256) core_g_pass_kernel(DevModel<T> M, DevMode<T> csr, T* r, const T* __restrict__ U,
                                                          GPassArgs a) {
  constexpr int kPer = kCoreMaxB / 32;
  __shared__ T sh[8][kCoreMaxM];
  __shared__ double sw[8][kCoreMaxB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int J0 = a.J0, m = a.cur.m, b = a.cur.b, mp = a.has_prev ? a.prev.m : 0;
  T as[kPer], ac[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) as[i] = ac[i] = T(0);
  const int64_t nchunks = ceil_div(a.nnz, 32);
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp, nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t ch = gw; ch < nchunks; ch += nw) {
    const int64_t p = ch * 32 + lane;
    const bool valid = p < a.nnz;
    const int k = valid ? csr.rowk[p] : -1 - lane;
    T h[kCoreMaxM];
#pragma unroll
    for (int q = 0; q < kCoreMaxM; ++q) h[q] = T(0);
    if (valid) {
      const T* a1 = M.A[1] + (int64_t)csr.oidx[p] * a.J1;
      T rv = r[p];
      if (a.has_prev) {
        T cp;
        suffix_weights<T>(M, csr.oidx, a.nnz, p, a.prev.s, 1, &cp, 1);
        const T* u = U + (int64_t)k * kCoreMaxM;
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < kCoreMaxM; ++q)
          if (q < mp) acc += a1[a.prev.q0 + q] * u[q];
        rv -= cp * acc;
        r[p] = rv;
      }
      T c;
      suffix_weights<T>(M, csr.oidx, a.nnz, p, a.cur.s, 1, &c, 1);
      const T rc = rv * c;
#pragma unroll
      for (int q = 0; q < kCoreMaxM; ++q)
        if (q < m) h[q] = rc * a1[a.cur.q0 + q];
    }
    // segmented suffix sums: lane l ends with the sum over its row from l to the chunk end
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int ko = __shfl_down_sync(0xffffffffu, k, o);
#pragma unroll
      for (int q = 0; q < kCoreMaxM; ++q) {
        const T v = __shfl_down_sync(0xffffffffu, h[q], o);
        if (lane + o < 32 && ko == k) h[q] += v;
      }
    }
    const int kup = __shfl_up_sync(0xffffffffu, k, 1);
    unsigned heads = __ballot_sync(0xffffffffu, valid && (lane == 0 || kup != k));
    while (heads) {
      const int hl = __ffs(heads) - 1;
      heads &= heads - 1;
      const int kk = __shfl_sync(0xffffffffu, k, hl);
      if (lane == hl) {
#pragma unroll
        for (int q = 0; q < kCoreMaxM; ++q)
          if (q < m) sh[warp][q] = h[q];
      }
      __syncwarp();
      const T* a0 = M.A[0] + (int64_t)csr.nzrow[kk] * J0;
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int e = lane + 32 * i;
        if (e < b) CoreAcc<T>::add(as[i], ac[i], a0[e % J0] * sh[warp][e / J0]);
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

// Exact sequential updates of one block (Eq. 12 / Eq. 14) by one warp: lane
// k % 32 holds the running sum_alpha r P(k) of element k; after each update
// every lane subtracts Delta_k M_kl from the elements l > k it holds.
template <typename T>
__global__ void core_solve_kernel(DevModel<T> M, CoreBlock blk, int J0, int J1, int reg, double lambda,
                                  const double* gram, const double* __restrict__ g, double* __restrict__ dout) {
  constexpr int kPer = kCoreMaxB / 32;
  extern __shared__ double sgram[];
  const int lane = threadIdx.x & 31;
  const int b = blk.b;
  for (int e = threadIdx.x; e < b * (b + 1) / 2; e += blockDim.x) sgram[e] = gram[e];
  __syncthreads();
  if (threadIdx.x >= 32) return;
  gram = sgram;
  // lane holds, for its elements l = lane + 32 i: the running sum, the current value, the mask
  double grad[kPer], gval[kPer];
  int gmask[kPer];
  auto lin_of = [&](int k) {
    return (int64_t)(k % J0) + (int64_t)J0 * (blk.q0 + k / J0) + (int64_t)J0 * J1 * blk.s;
  };
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int l = lane + 32 * i;
    grad[i] = l < b ? g[l] : 0.0;
    gval[i] = l < b ? (double)M.G[lin_of(l)] : 0.0;
    gmask[i] = l < b ? (int)M.Gmask[lin_of(l)] : 1;
  }
  for (int k = 0; k < b; ++k) {
    const int64_t lin = lin_of(k);
    double gk = 0.0, gold = 0.0;
    int mk = 1;
#pragma unroll
    for (int i = 0; i < kPer; ++i)
      if (k / 32 == i) {
        gk = grad[i];
        gold = gval[i];
        mk = gmask[i];
      }
    gk = __shfl_sync(0xffffffffu, gk, k & 31);
    gold = __shfl_sync(0xffffffffu, gold, k & 31);
    mk = __shfl_sync(0xffffffffu, mk, k & 31);
    double dk = 0.0;
    if (!mk) {
      const double mkk = gram[sym_index(k, k, b)];
      const double num = gk + gold * mkk;
      double nv;
      if (reg == VEST_REG_L1) {
        const double gcv = -2.0 * num, dc = 2.0 * mkk;
        nv = gcv > lambda ? (lambda - gcv) / dc : (gcv < -lambda ? -(lambda + gcv) / dc : 0.0);
      } else {
        nv = num / (lambda + mkk);
      }
      const T st = (T)nv;
      dk = (double)st - gold;
      if (lane == 0) M.G[lin] = st;
    }
    if (lane == 0) dout[k] = dk;
    if (dk != 0.0) {
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int l = lane + 32 * i;
        if (l > k && l < b) grad[i] -= dk * gram[sym_index(k, l, b)];
      }
    }
  }
}

// ================================================================== stats pass (responsibility)
// For a group of suffixes [s0, s0 + Sg) and every j_1: per piece sum r w and sum w^2
// with w = a1[j_1] c(s); then S1(j0, j1, s) += a0[j0] sum r w, S2 += a0[j0]^2 sum w^2.
struct StatsArgs {
  int J0, J1;
  int64_t s0;
  int Sg, SJ, P, kmax;
  int64_t nnz, ntasks;
  double* part;  // [ctas][2 * J0 * SJ]
};

template <typename T>
struct StatsTerm {
  const T* sR;
  const T* sW;
  int SJ;
  __device__ TermPtrs<T> prep(int p) const {
    if (p < SJ) return TermPtrs<T>{sR, sW + p, 1, SJ};
    return TermPtrs<T>{sW + (p - SJ), sW + (p - SJ), SJ, SJ};
  }
};

template <typename T>
__global__ void __launch_bounds__(kCoreTask) core_stats_kernel(DevModel<T> M, DevMode<T> csr, const T* __restrict__ r,
                                                               StatsArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int J0 = a.J0, SJ = a.SJ, P = a.P;
  size_t off = 0;
  int64_t* sptr = reinterpret_cast<int64_t*>(smem_raw + off); off += (size_t)(kCoreTask + 2) * 8;
  T* sA0 = reinterpret_cast<T*>(smem_raw + off); off += (size_t)kCoreTask * J0 * sizeof(T);
  T* sW = reinterpret_cast<T*>(smem_raw + off); off += (size_t)kCoreTask * SJ * sizeof(T);
  T* sR = reinterpret_cast<T*>(smem_raw + off); off += (size_t)kCoreTask * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  T* sAcc = reinterpret_cast<T*>(smem_raw + off); off += (size_t)a.kmax * P * sizeof(T);
  T* sPart = reinterpret_cast<T*>(smem_raw + off);
  __shared__ PieceScratch pscr;
  const int nacc = 2 * J0 * SJ;
  T rs[kStatsEPT], rc[kStatsEPT], tacc[kStatsEPT];
#pragma unroll
  for (int i = 0; i < kStatsEPT; ++i) rs[i] = rc[i] = T(0);
  const int R = *csr.nnzrows;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int64_t task = blockIdx.x; task < a.ntasks; task += gridDim.x) {
    const int64_t t0 = task * kCoreTask, t1 = min(t0 + (int64_t)kCoreTask, a.nnz);
    const int cnt = (int)(t1 - t0);
    int64_t k0;
    const int nrows = load_task_rows(csr.nzptr, csr.gran, R, t0, t1, sptr, &k0);
    for (int k = warp; k < nrows; k += nwarps) {
      const int64_t row = csr.nzrow[k0 + k];
      for (int j = lane; j < J0; j += 32) sA0[k * J0 + j] = M.A[0][row * J0 + j];
    }
    if ((int)threadIdx.x < cnt) {
      const int64_t p = t0 + threadIdx.x;
      const T* a1 = M.A[1] + (int64_t)csr.oidx[p] * a.J1;
      T* w = sW + threadIdx.x * SJ;
      suffix_weights<T>(M, csr.oidx, a.nnz, p, a.s0, a.Sg, w, a.J1);  // c(s) at w[s * J1]
      for (int si = 0; si < a.Sg; ++si) {
        const T c = w[si * a.J1];
        for (int q = 0; q < a.J1; ++q) w[si * a.J1 + q] = a1[q] * c;
      }
      sR[threadIdx.x] = r[p];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kStatsEPT; ++i) tacc[i] = T(0);
    const StatsTerm<T> f{sR, sW, SJ};
    for (int r0 = 0; r0 < nrows; r0 += a.kmax) {
      const int nr = min(a.kmax, nrows - r0);
      piece_sums<T>(sptr + r0, nr, t0, t1, P, sAcc, sPart, &pscr, f);
#pragma unroll
      for (int i = 0; i < kStatsEPT; ++i) {
        const int e = threadIdx.x + i * blockDim.x;
        if (e >= nacc) continue;
        const int kind = e / (J0 * SJ), rem = e % (J0 * SJ);
        const int j0 = rem % J0, sq = rem / J0;
        for (int kr = 0; kr < nr; ++kr) {
          const T av = sA0[(r0 + kr) * J0 + j0];
          tacc[i] += kind == 0 ? av * sAcc[kr * P + sq] : av * av * sAcc[kr * P + SJ + sq];
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < kStatsEPT; ++i) CoreAcc<T>::add(rs[i], rc[i], tacc[i]);
  }
#pragma unroll
  for (int i = 0; i < kStatsEPT; ++i) {
    const int e = threadIdx.x + i * blockDim.x;
    if (e < nacc) a.part[(size_t)blockIdx.x * nacc + e] = CoreAcc<T>::value(rs[i], rc[i]);
  }
}

// Delta and Resp of the group's core elements: lin = j0 + J0 (j1 + J1 s).
template <typename T>
__global__ void core_resp_kernel(DevModel<T> M, int J0, int J1, int64_t s0, int SJ, const double* __restrict__ sums,
                                 const double* __restrict__ stats, double* __restrict__ delta, double* __restrict__ resp) {
  const double xx = stats[1], re = stats[4];
  const int n = J0 * SJ;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int64_t lin = (int64_t)J0 * J1 * s0 + e;  // e = j0 + J0 * (j1 + J1 * si)
    const double gv = (double)M.G[lin];
    const double dl = 2.0 * gv * sums[e] + gv * gv * sums[n + e];
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
  int SgStats, SJ;             // stats groups
  int64_t slots;
};

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
  c.SgMax = (int)std::max<int64_t>(1, std::min<int64_t>(c.S, kGramMaxP / c.nYmax));
  c.Pmax = 0;
  for (int q0 = 0; q0 < c.J1; q0 += c.m) {  // the last j_1 chunk may be narrower and take more suffixes
    const int mq = std::min(c.m, c.J1 - q0), nY = mq * (mq + 1) / 2;
    const int sg = (int)std::max<int64_t>(1, std::min<int64_t>(c.S, kGramMaxP / nY));
    c.Pmax = std::max(c.Pmax, sg * nY);
  }
  // stats: 2 * SJ outputs per piece <= 512, 2 * J0 * SJ accumulators <= kStatsEPT * 256
  int sg = (int)std::max<int64_t>(1, std::min<int64_t>(c.S, 256 / c.J1));
  while (sg > 1 && 2 * c.J0 * sg * c.J1 > kStatsEPT * kCoreTask) --sg;
  c.SgStats = sg;
  c.SJ = sg * c.J1;
  c.slots = cap0 + ceil_div(std::max<int64_t>(nnz, 1), kCoreTask) + 1;
  return c;
}

size_t core_scratch_bytes(const vest_model* m, int64_t nnz, int64_t cap0, size_t* y_bytes, size_t* gram_bytes,
                          size_t* part_bytes) {
  const CorePlan c = core_plan(m->ranks, m->order, nnz, cap0);
  const size_t sT = m->dtype == VEST_F64 ? 8 : 4;
  // per-piece gram statistics, later reused for u per non-empty mode-0 row (cap0 x kCoreMaxM)
  *y_bytes = align_up(std::max((size_t)c.slots * c.Pmax, (size_t)(cap0 + 1) * kCoreMaxM) * sT) +
             align_up((size_t)c.slots * 4);
  // the gram region also holds the responsibility sums (2 * J0 * SJ doubles)
  *gram_bytes = align_up(std::max((size_t)c.nblocks * c.nmmax, (size_t)2 * c.J0 * c.SJ) * 8);
  const size_t gemm = (size_t)kGramKSplit * c.nX * c.Pmax * 8;
  const size_t gp = (size_t)kCorePassCtas * kCoreMaxB * 8;
  const size_t st = (size_t)kCorePassCtas * 2 * c.J0 * c.SJ * 8;
  *part_bytes = align_up(std::max({gemm, gp, st}));
  return *y_bytes + *gram_bytes + *part_bytes;
}

template <typename T>
static size_t smem_gram(int nY, int Sg, int P, int kmax) {
  size_t off = (size_t)(kCoreTask + 2) * 8 + (size_t)kCoreTask * nY * sizeof(T) + (size_t)kCoreTask * Sg * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  return off + (size_t)kmax * P * sizeof(T) + (size_t)kMaxLongPieces * P * sizeof(T);
}

template <typename T>
static size_t smem_stats(int J0, int SJ, int P, int kmax) {
  size_t off = (size_t)(kCoreTask + 2) * 8 + (size_t)kCoreTask * J0 * sizeof(T) + (size_t)kCoreTask * SJ * sizeof(T) +
               (size_t)kCoreTask * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  return off + (size_t)kmax * P * sizeof(T) + (size_t)kMaxLongPieces * P * sizeof(T);
}

template <typename T>
static int kmax_for(int P) {
  return (int)std::max<size_t>(1, std::min<size_t>(kCoreKmax, (48 * 1024) / ((size_t)P * sizeof(T))));
}

struct CoreBufs {
  void* Y;
  int32_t* srow;
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
      base + align_up(std::max((size_t)c.slots * c.Pmax, (size_t)(ix->mode[0].cap + 1) * kCoreMaxM) * sT));
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
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntasks, (int64_t)num_sms() * 4));
  for (int qc = 0; qc < c.nq0; ++qc) {
    const int q0 = qc * c.m, mq = std::min(c.m, c.J1 - q0), nY = mq * (mq + 1) / 2;
    const int Sg = (int)std::max<int64_t>(1, std::min<int64_t>(c.S, kGramMaxP / nY));
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
      ga.kmax = kmax_for<T>(ga.P);
      ga.nnz = ix->nnz;
      ga.ntasks = ntasks;
      ga.Y = bf.Y;
      ga.srow = bf.srow;
      VEST_CUDA(cudaMemsetAsync(bf.srow, 0xFF, (size_t)c.slots * 4, s));
      if (ix->nnz > 0) {
        const size_t smem = smem_gram<T>(nY, sg, ga.P, ga.kmax);
        auto kern = core_gram_pass_kernel<T>;
        VEST_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<grid, kCoreTask, smem, s>>>(M, csr, ga);
        VEST_LAUNCH("core_gram_pass_kernel");
      }
      GemmArgs gm{};
      gm.J0 = c.J0;
      gm.nX = c.nX;
      gm.P = ga.P;
      gm.nslots = c.slots;
      gm.Y = bf.Y;
      gm.srow = bf.srow;
      gm.part = bf.part;
      const dim3 gg((unsigned)(((c.nX + 31) / 32) * ((ga.P + 63) / 64)), kGramKSplit);
      core_gram_gemm_kernel<T><<<gg, 256, 0, s>>>(M, csr, gm);
      VEST_LAUNCH("core_gram_gemm_kernel");
      const int b = c.J0 * mq, nm = b * (b + 1) / 2;
      for (int si = 0; si < sg; ++si) {
        const int64_t bi = (s0 + si) * c.nq0 + qc;
        core_gram_merge_kernel<<<(unsigned)ceil_div(nm, 256), 256, 0, s>>>(bf.part, kGramKSplit, c.nX, ga.P, c.J0, mq,
                                                                           nY, si, bf.gram + bi * c.nmmax);
        VEST_LAUNCH("core_gram_merge_kernel");
      }
    }
  }
  return VEST_OK;
}

template <typename T>
vest_status sweep_core_impl(const vest_index* ix, const vest_model* mdl, int reg, double lambda, char* scratch,
                            const ScratchPlan& plan, cudaStream_t s) {
  const DevModel<T> M = dev_model<T>(mdl);
  if (M.N < 2) return fail(VEST_ERR_UNSUPPORTED, "order < 2");
  const CorePlan c = core_plan(M.J, M.N, ix->nnz, ix->mode[0].cap);
  const CoreBufs bf = core_bufs(ix, mdl, scratch, plan);
  T* r0 = reinterpret_cast<T*>(scratch + plan.off_resid);
  double* out = bf.small + 9000 + 3 * kCoreMaxB;
  double* gvec = bf.small + 9000 + 2 * kCoreMaxB;
  double* dbuf[2] = {bf.small + 9000, bf.small + 9000 + kCoreMaxB};
  VEST_TRY(loss_impl<T>(ix, mdl, reg, lambda, out, r0, nullptr, scratch, plan, s));
  VEST_TRY(core_grams<T>(ix, M, c, bf, s));
  const DevMode<T> csr = dev_mode<T>(ix, 0);
  GPassArgs a{};
  a.J0 = c.J0;
  a.J1 = c.J1;
  a.nnz = ix->nnz;
  a.part = bf.part;
  T* U = reinterpret_cast<T*>(bf.Y);  // the per-piece gram region is free again: u per row
  const int nctas_g = kCorePassCtas;
  int64_t iblk = 0;
  for (int64_t sfx = 0; sfx < c.S; ++sfx) {
    for (int qc = 0; qc < c.nq0; ++qc, ++iblk) {
      const int q0 = qc * c.m;
      CoreBlock blk{sfx, q0, std::min(c.m, c.J1 - q0), 0};
      blk.b = c.J0 * blk.m;
      a.cur = blk;
      a.has_prev = iblk > 0;
      if (ix->nnz > 0) {
        if (a.has_prev) {
          core_u_kernel<T><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ix->mode[0].cap, 256), num_sms() * 4)),
                             256, 0, s>>>(M, csr.nzrow, csr.nnzrows, dbuf[(iblk + 1) & 1], c.J0, a.prev.m, U);
          VEST_LAUNCH("core_u_kernel");
        }
        core_g_pass_kernel<T><<<nctas_g, 256, 0, s>>>(M, csr, r0, U, a);
        VEST_LAUNCH("core_g_pass_kernel");
        core_vec_merge_kernel<<<(unsigned)ceil_div(blk.b, 32), 256, 0, s>>>(bf.part, nctas_g, blk.b, gvec);
        VEST_LAUNCH("core_vec_merge_kernel");
      } else {
        VEST_CUDA(cudaMemsetAsync(gvec, 0, (size_t)blk.b * 8, s));
      }
      const size_t ssm = (size_t)(blk.b * (blk.b + 1) / 2) * 8;
      auto sk = core_solve_kernel<T>;
      VEST_CUDA(cudaFuncSetAttribute(sk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm));
      sk<<<1, 256, ssm, s>>>(M, blk, c.J0, c.J1, reg, lambda, bf.gram + iblk * c.nmmax, gvec, dbuf[iblk & 1]);
      VEST_LAUNCH("core_solve_kernel");
      a.prev = blk;
    }
  }
  return VEST_OK;
}

template <typename T>
vest_status core_responsibility(const vest_index* ix, const vest_model* mdl, const T* resid_csr0, const double* stats,
                                double* delta_core, double* resp_core, char* scratch, const ScratchPlan& plan,
                                cudaStream_t s) {
  const DevModel<T> M = dev_model<T>(mdl);
  if (M.N < 2) return fail(VEST_ERR_UNSUPPORTED, "order < 2");
  const CorePlan c = core_plan(M.J, M.N, ix->nnz, ix->mode[0].cap);
  const CoreBufs bf = core_bufs(ix, mdl, scratch, plan);
  const DevMode<T> csr = dev_mode<T>(ix, 0);
  const int64_t ntasks = ceil_div(ix->nnz, kCoreTask);
  const int nctas = (int)std::max<int64_t>(1, std::min<int64_t>(ntasks, kCorePassCtas));
  double* sums = bf.gram;  // reuse the gram region: [2 * J0 * SJ]
  for (int64_t s0 = 0; s0 < c.S; s0 += c.SgStats) {
    StatsArgs a{};
    a.J0 = c.J0;
    a.J1 = c.J1;
    a.s0 = s0;
    a.Sg = (int)std::min<int64_t>(c.SgStats, c.S - s0);
    a.SJ = a.Sg * c.J1;
    a.P = 2 * a.SJ;
    a.kmax = kmax_for<T>(a.P);
    a.nnz = ix->nnz;
    a.ntasks = ntasks;
    a.part = bf.part;
    const int nacc = 2 * c.J0 * a.SJ;
    if (ix->nnz > 0) {
      const size_t smem = smem_stats<T>(c.J0, a.SJ, a.P, a.kmax);
      auto kern = core_stats_kernel<T>;
      VEST_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<nctas, kCoreTask, smem, s>>>(M, csr, resid_csr0, a);
      VEST_LAUNCH("core_stats_kernel");
      core_vec_merge_kernel<<<(unsigned)ceil_div(nacc, 32), 256, 0, s>>>(bf.part, nctas, nacc, sums);
      VEST_LAUNCH("core_vec_merge_kernel");
    } else {
      VEST_CUDA(cudaMemsetAsync(sums, 0, (size_t)nacc * 8, s));
    }
    core_resp_kernel<T><<<(unsigned)ceil_div(c.J0 * a.SJ, 256), 256, 0, s>>>(M, c.J0, c.J1, s0, a.SJ, sums, stats,
                                                                              delta_core, resp_core);
    VEST_LAUNCH("core_resp_kernel");
  }
  return VEST_OK;
}

template vest_status sweep_core_impl<float>(const vest_index*, const vest_model*, int, double, char*,
                                            const ScratchPlan&, cudaStream_t);
template vest_status sweep_core_impl<double>(const vest_index*, const vest_model*, int, double, char*,
                                             const ScratchPlan&, cudaStream_t);
template vest_status core_responsibility<float>(const vest_index*, const vest_model*, const float*, const double*,
                                                double*, double*, char*, const ScratchPlan&, cudaStream_t);
template vest_status core_responsibility<double>(const vest_index*, const vest_model*, const double*, const double*,
                                                 double*, double*, char*, const ScratchPlan&, cudaStream_t);

}  // namespace vest
