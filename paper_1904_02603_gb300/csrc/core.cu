// Core sweep (Lemma 2, Eq. 12; Lemma 4, Eq. 14) and the core part of the
// responsibility (Eq. 5, Algorithm 3).
//
// The core elements are updated one at a time in linear order (j_1 fastest),
// as the paper requires (Section 3.6).  On the GPU this is blocked
// Gauss-Seidel, equal to the one-at-a-time sweep in exact arithmetic:
//   - a block is b = J_0 * m consecutive core elements, (j_0, j_1) in
//     J_0 x [q0, q0 + m) for one fixed suffix (j_2, ..., j_{N-1});
//   - one pass over the mode-0 CSR computes, from the residual r at the block
//     start, g_k = sum_alpha r_alpha P_alpha(k) and the block Gram
//     M_kl = sum_alpha P_alpha(k) P_alpha(l), with P_alpha(j_0, j_1) =
//     a0[i_0, j_0] * a1[i_1, j_1] * c_alpha and c_alpha = prod_{n>=2}
//     a_n[i_n, s_n].  Entries are grouped by their mode-0 row, so per row
//     piece only Q = sum w w^T and h = sum r w with w(q) = a1[i_1, q0+q] c_alpha
//     are formed, and M += (a0 a0^T) (x) Q, g += a0 (x) h;
//   - one thread block then runs the b updates in order exactly:
//     sum_alpha r_alpha P_alpha(k) at step k is g_k - sum_{l<k} Delta_l M_lk;
//   - the next pass first applies this block's Delta to r.
// Per-block sums: per piece in the storage type, across pieces in a
// Kahan-compensated accumulator (FP32) or FP64, across thread blocks in FP64
// in a fixed order.
#include <algorithm>

#include "delta.cuh"

namespace vest {

constexpr int kCoreTask = 256;
constexpr int kCoreMaxB = 128;
constexpr int kCoreMaxM = 10;
constexpr int kCoreEPT = 24;           // accumulator entries per thread (nz <= 5408 for b <= 128, m <= 10)
constexpr int kCorePassCtas = 296;     // fixed: reduction order does not depend on the device

struct CoreBlock {
  int64_t s;      // suffix linear index over modes >= 2
  int q0, m;      // j_1 range
  int b;          // J_0 * m
};

struct CoreArgs {
  int N, J0, J1;
  int64_t nnz;
  int64_t ntasks;
  CoreBlock cur, prev;
  int has_prev;
  int nent;               // b(b+1)/2 + b entries of the packed Gram and g
  int nz;                 // Kronecker-form accumulator entries
  const double* dprev;    // Delta of the previous block [b_prev]
  double* part;           // [ctas][nent]
};

// c_alpha for a suffix s: prod over modes n >= 2 of a_n[i_n, digit_n(s)]
template <typename T>
__device__ __forceinline__ T suffix_weight(const DevModel<T>& M, const int32_t* __restrict__ oidx, int64_t nnz, int64_t p,
                                           int64_t s) {
  T c = T(1);
  for (int n = 2; n < M.N; ++n) {
    const int d = (int)(s % M.J[n]);
    s /= M.J[n];
    const int64_t in = oidx[(int64_t)(n - 1) * nnz + p];  // mode-0 CSR: oidx rows are modes 1..N-1
    c *= M.A[n][in * M.J[n] + d];
  }
  return c;
}

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

// entry e of the packed accumulator -> (k, l): e < b(b+1)/2 packed upper M (k <= l), else g_k
__device__ __forceinline__ void entry_kl(int e, int b, int& k, int& l) {
  const int nm = b * (b + 1) / 2;
  if (e >= nm) {
    k = e - nm;
    l = -1;
    return;
  }
  int kk = 0, u = e;
  while (u >= b - kk) {
    u -= b - kk;
    ++kk;
  }
  k = kk;
  l = kk + u;
}

// Terms of the per-piece sums: packed upper Q = sum w w^T, then h = sum r w.
template <typename T>
struct CoreTerm {
  const T* sW;
  const T* sR;
  int m;
  __device__ TermPtrs<T> prep(int p) const {
    const int nq = m * (m + 1) / 2;
    if (p >= nq) return TermPtrs<T>{sR, sW + (p - nq), 1, m};
    int u = p, q = 0;
    while (u >= m - q) {
      u -= m - q;
      ++q;
    }
    return TermPtrs<T>{sW + q, sW + q + u, m, m};
  }
};

template <typename T>
__global__ void __launch_bounds__(kCoreTask) core_pass_kernel(DevModel<T> M, DevMode<T> csr, const T* r_in,
                                                              T* r_out, CoreArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int J0 = a.J0, m = a.cur.m, b = a.cur.b;
  const int mp = a.has_prev ? a.prev.m : 0;
  const int QP = m * (m + 1) / 2 + m;
  size_t off = 0;
  int64_t* sptr = reinterpret_cast<int64_t*>(smem_raw + off); off += (size_t)(kCoreTask + 2) * 8;
  double* sdp = reinterpret_cast<double*>(smem_raw + off); off += (size_t)kCoreMaxB * 8;
  T* sA0 = reinterpret_cast<T*>(smem_raw + off); off += (size_t)kCoreTask * J0 * sizeof(T);
  T* sU = reinterpret_cast<T*>(smem_raw + off); off += (size_t)kCoreTask * max(mp, 1) * sizeof(T);
  T* sW = reinterpret_cast<T*>(smem_raw + off); off += (size_t)kCoreTask * m * sizeof(T);
  T* sR = reinterpret_cast<T*>(smem_raw + off); off += (size_t)kCoreTask * sizeof(T);
  T* sQ = reinterpret_cast<T*>(smem_raw + off); off += (size_t)kCoreTask * QP * sizeof(T);
  T* sPart = reinterpret_cast<T*>(smem_raw + off); off += (size_t)kMaxLongPieces * QP * sizeof(T);
  T* sSum = reinterpret_cast<T*>(smem_raw + off); off += (size_t)a.nz * sizeof(T);
  T* sComp = reinterpret_cast<T*>(smem_raw + off);
  __shared__ PieceScratch pscr;

  if (a.has_prev)
    for (int i = threadIdx.x; i < a.prev.b; i += blockDim.x) sdp[i] = a.dprev[i];

  // Block Gram in Kronecker form: Z[xi][yi] = sum over row pieces of
  // X[xi] * Y[yi], X = packed upper a0 a0^T (nX = J0(J0+1)/2 values), Y = packed
  // upper Q (nY = m(m+1)/2), followed by the J0*m products a0[j0] * h[q] of g.
  // Each thread owns entries threadIdx.x + i * blockDim.x, coded as
  // a0 index 1 (8 bits) | a0 index 2 (8 bits, 255 = g entry) | offset into Q/h (16 bits).
  T tacc[kCoreEPT];
  uint32_t code[kCoreEPT];
  int nown = 0;
  const int nY = m * (m + 1) / 2, nX = J0 * (J0 + 1) / 2;
#pragma unroll
  for (int i = 0; i < kCoreEPT; ++i) {
    code[i] = 0xFFFFFFFFu;
    const int e = threadIdx.x + i * blockDim.x;
    if (e < a.nz) {
      if (e < nX * nY) {
        int u = e / nY, ja = 0;
        while (u >= J0 - ja) {
          u -= J0 - ja;
          ++ja;
        }
        code[i] = (uint32_t)ja | ((uint32_t)(ja + u) << 8) | ((uint32_t)(e % nY) << 16);
      } else {
        const int g = e - nX * nY;
        code[i] = (uint32_t)(g % J0) | (255u << 8) | ((uint32_t)(nY + g / J0) << 16);
      }
      nown = i + 1;
      sSum[e] = T(0);
      sComp[e] = T(0);
    }
  }
  const int R = *csr.nnzrows;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  __syncthreads();

  for (int64_t task = blockIdx.x; task < a.ntasks; task += gridDim.x) {
    const int64_t t0 = task * kCoreTask, t1 = min(t0 + (int64_t)kCoreTask, a.nnz);
    const int cnt = (int)(t1 - t0);
    int64_t k0;
    const int nrows = load_task_rows(csr.nzptr, csr.gran, R, t0, t1, sptr, &k0);
    // row data: a0 row and u(q) = sum_j0 Delta_prev(j0, q) a0[j0]
    for (int k = warp; k < nrows; k += nwarps) {
      const int64_t row = csr.nzrow[k0 + k];
      for (int j = lane; j < J0; j += 32) sA0[k * J0 + j] = M.A[0][row * J0 + j];
      __syncwarp();
      for (int q = lane; q < mp; q += 32) {
        T u = T(0);
        for (int j = 0; j < J0; ++j) u += (T)sdp[q * J0 + j] * sA0[k * J0 + j];
        sU[k * mp + q] = u;
      }
    }
    __syncthreads();
    // phase 1: per entry, apply the previous block to r, form w
    if ((int)threadIdx.x < cnt) {
      const int64_t p = t0 + threadIdx.x;
      const int lr = local_row(sptr, nrows, p);
      const int64_t i1 = csr.oidx[p];
      const T* a1 = M.A[1] + i1 * a.J1;
      T r = r_in[p];
      if (a.has_prev) {
        const T cp = suffix_weight<T>(M, csr.oidx, a.nnz, p, a.prev.s);
        T acc2 = T(0);
        for (int q = 0; q < mp; ++q) acc2 += sU[lr * mp + q] * a1[a.prev.q0 + q];
        r -= cp * acc2;
        r_out[p] = r;
      }
      const T c = suffix_weight<T>(M, csr.oidx, a.nnz, p, a.cur.s);
      for (int q = 0; q < m; ++q) sW[threadIdx.x * m + q] = a1[a.cur.q0 + q] * c;
      sR[threadIdx.x] = r;
    }
    __syncthreads();
    // phase 2: per row piece Q (packed upper) and h
    {
      CoreTerm<T> f{sW, sR, m};
      piece_sums<T>(sptr, nrows, t0, t1, QP, sQ, sPart, &pscr, f);
    }
    // phase 3: Z += X (x) Y and g += a0 (x) h over the task's pieces (storage type),
    // then into the block's running sums (Kahan for FP32)
#pragma unroll
    for (int i = 0; i < kCoreEPT; ++i) tacc[i] = T(0);
    for (int k = 0; k < nrows; ++k) {
      const T* a0 = sA0 + k * J0;
      const T* Q = sQ + k * QP;
#pragma unroll
      for (int i = 0; i < kCoreEPT; ++i) {
        if (i >= nown) continue;
        const uint32_t c = code[i];
        const int ia = (int)(c & 255u), ib = (int)((c >> 8) & 255u), iq = (int)(c >> 16);
        const T xa = ib == 255 ? a0[ia] : a0[ia] * a0[ib];
        tacc[i] += xa * Q[iq];
      }
    }
#pragma unroll
    for (int i = 0; i < kCoreEPT; ++i)
      if (i < nown) {
        const int e = threadIdx.x + i * blockDim.x;
        CoreAcc<T>::add(sSum[e], sComp[e], tacc[i]);
      }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < kCoreEPT; ++i)
    if (i < nown) {
      const int e = threadIdx.x + i * blockDim.x;
      a.part[(size_t)blockIdx.x * a.nz + e] = CoreAcc<T>::value(sSum[e], sComp[e]);
    }
}

__device__ __forceinline__ int sym_index(int x, int y, int n) {
  const int lo = min(x, y), hi = max(x, y);
  return lo * n - (lo * (lo - 1)) / 2 + (hi - lo);
}

// Fixed-order FP64 sum of the per-block partials, expanded from the Kronecker
// form into the packed block Gram M (k <= l) followed by g.
__global__ void core_merge_kernel(const double* __restrict__ part, int nctas, int nz, int nent, int b, int J0, int m,
                                  double* __restrict__ tot) {
  const int nm = b * (b + 1) / 2, nY = m * (m + 1) / 2, nX = J0 * (J0 + 1) / 2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nent; e += gridDim.x * blockDim.x) {
    int z;
    if (e < nm) {
      int k, l;
      entry_kl(e, b, k, l);
      z = sym_index(k % J0, l % J0, J0) * nY + sym_index(k / J0, l / J0, m);
    } else {
      const int k = e - nm;
      z = nX * nY + (k % J0) + J0 * (k / J0);
    }
    double s = 0.0;
    for (int c = 0; c < nctas; ++c) s += part[(size_t)c * nz + z];
    tot[e] = s;
  }
}


// Exact sequential updates of one block (Eq. 12 / Eq. 14), one thread block.
template <typename T>
__global__ void core_solve_kernel(DevModel<T> M, CoreBlock blk, int J0, int J1, int reg, double lambda,
                                  const double* __restrict__ tot, double* __restrict__ dout) {
  __shared__ double grad[kCoreMaxB];
  __shared__ double dk_s;
  const int b = blk.b;
  const int nm = b * (b + 1) / 2;
  for (int k = threadIdx.x; k < b; k += blockDim.x) grad[k] = tot[nm + k];
  __syncthreads();
  auto Mkl = [&](int k, int l) {
    const int lo = min(k, l), hi = max(k, l);
    return tot[lo * b - (lo * (lo - 1)) / 2 + (hi - lo)];
  };
  for (int k = 0; k < b; ++k) {
    const int j0 = k % J0, q = k / J0;
    const int64_t lin = (int64_t)j0 + (int64_t)J0 * (blk.q0 + q) + (int64_t)J0 * J1 * blk.s;
    if (threadIdx.x == 0) {
      double dk = 0.0;
      if (!M.Gmask[lin]) {
        const double gold = (double)M.G[lin];
        const double mkk = Mkl(k, k);
        const double num = grad[k] + gold * mkk;
        double nv;
        if (reg == VEST_REG_L1) {
          const double gc = -2.0 * num, dc = 2.0 * mkk;
          nv = gc > lambda ? (lambda - gc) / dc : (gc < -lambda ? -(lambda + gc) / dc : 0.0);
        } else {
          nv = num / (lambda + mkk);
        }
        const T st = (T)nv;
        M.G[lin] = st;
        dk = (double)st - gold;
      }
      dk_s = dk;
      dout[k] = dk;
    }
    __syncthreads();
    const double dk = dk_s;
    if (dk != 0.0)
      for (int l = k + 1 + threadIdx.x; l < b; l += blockDim.x) grad[l] -= dk * Mkl(k, l);
    __syncthreads();
  }
}

// Responsibility of the block's core elements from g (sum r P) and diag(M) (sum P^2).
template <typename T>
__global__ void core_resp_kernel(DevModel<T> M, CoreBlock blk, int J0, int J1, const double* __restrict__ tot,
                                 const double* __restrict__ stats, double* __restrict__ delta, double* __restrict__ resp) {
  const int b = blk.b, nm = b * (b + 1) / 2;
  const double xx = stats[1], re = stats[4];
  for (int k = threadIdx.x; k < b; k += blockDim.x) {
    const int j0 = k % J0, q = k / J0;
    const int64_t lin = (int64_t)j0 + (int64_t)J0 * (blk.q0 + q) + (int64_t)J0 * J1 * blk.s;
    const double gv = (double)M.G[lin];
    const double mkk = tot[k * b - (k * (k - 1)) / 2];
    const double dl = 2.0 * gv * tot[nm + k] + gv * gv * mkk;
    delta[lin] = dl;
    if (resp) resp[lin] = re > 0.0 ? (sqrt(fmax(re * re + dl / xx, 0.0)) - re) / re : 0.0;
  }
}

// ------------------------------------------------------------------ host side
// m = j_1 values per block: b = J_0 * m <= 128, and m <= 10 so the per-piece
// Q buffers (m(m+1)/2 + m values per row piece) fit in shared memory.
static void plan_blocks(const int32_t* J, int N, int* m_out, int64_t* nsuffix) {
  const int J0 = J[0], J1 = J[1];
  int m = std::max(1, kCoreMaxB / J0);
  m = std::min(std::min(m, J1), kCoreMaxM);
  *m_out = m;
  int64_t S = 1;
  for (int n = 2; n < N; ++n) S *= J[n];
  *nsuffix = S;
}

size_t core_part_bytes(const vest_model* m) {
  int mm;
  int64_t S;
  plan_blocks(m->ranks, m->order, &mm, &S);
  const int J0 = m->ranks[0];
  return (size_t)kCorePassCtas * (size_t)((J0 * (J0 + 1) / 2) * (mm * (mm + 1) / 2) + J0 * mm) * 8;
}

template <typename T>
static size_t pass_smem(int J0, int m, int mp, int nz) {
  const int QP = m * (m + 1) / 2 + m;
  size_t off = (size_t)(kCoreTask + 2) * 8 + (size_t)kCoreMaxB * 8;
  off += (size_t)kCoreTask * J0 * sizeof(T);
  off += (size_t)kCoreTask * std::max(mp, 1) * sizeof(T);
  off += (size_t)kCoreTask * m * sizeof(T);
  off += (size_t)kCoreTask * sizeof(T);
  off += (size_t)kCoreTask * QP * sizeof(T);
  off += (size_t)kMaxLongPieces * QP * sizeof(T);
  off += 2 * (size_t)nz * sizeof(T);
  return off;
}

// Runs the block passes; with solve = true this is the core sweep, otherwise it
// collects the responsibility statistics of every core element.
template <typename T>
static vest_status core_blocks(const vest_index* ix, const vest_model* mdl, int reg, double lambda, bool solve,
                               T* r0, const double* stats, double* delta_core, double* resp_core, char* scratch,
                               const ScratchPlan& plan, cudaStream_t s) {
  const DevModel<T> M = dev_model<T>(mdl);
  if (M.N < 2) return fail(VEST_ERR_UNSUPPORTED, "order < 2");
  int m;
  int64_t S;
  plan_blocks(M.J, M.N, &m, &S);
  const DevMode<T> csr = dev_mode<T>(ix, 0);
  CoreArgs a{};
  a.N = M.N;
  a.J0 = M.J[0];
  a.J1 = M.J[1];
  a.nnz = ix->nnz;
  a.ntasks = ceil_div(ix->nnz, kCoreTask);
  a.part = reinterpret_cast<double*>(scratch + plan.off_part);
  double* small = reinterpret_cast<double*>(scratch + plan.off_small);
  double* tot = small;                       // [<= 128*129/2 + 128]
  double* dbuf[2] = {small + 9000, small + 9000 + kCoreMaxB};
  const int nctas = (int)std::max<int64_t>(1, std::min<int64_t>(a.ntasks, kCorePassCtas));
  int iblk = 0;
  for (int64_t sfx = 0; sfx < S; ++sfx) {
    for (int q0 = 0; q0 < a.J1; q0 += m) {
      CoreBlock blk{sfx, q0, std::min(m, a.J1 - q0), 0};
      blk.b = a.J0 * blk.m;
      a.cur = blk;
      a.nent = blk.b * (blk.b + 1) / 2 + blk.b;
      a.nz = (a.J0 * (a.J0 + 1) / 2) * (blk.m * (blk.m + 1) / 2) + a.J0 * blk.m;
      if ((size_t)nctas * a.nz * 8 > plan.part_bytes) return fail(VEST_ERR_WORKSPACE, "core partial region too small");
      if (a.nz > kCoreEPT * kCoreTask) return fail(VEST_ERR_UNSUPPORTED, "core block too large");
      a.has_prev = (solve && iblk > 0) ? 1 : 0;
      a.dprev = dbuf[(iblk + 1) & 1];
      if (ix->nnz > 0) {
        const size_t smem = pass_smem<T>(a.J0, blk.m, a.has_prev ? a.prev.m : 0, a.nz);
        auto kern = core_pass_kernel<T>;
        VEST_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<nctas, kCoreTask, smem, s>>>(M, csr, r0, r0, a);
        VEST_LAUNCH("core_pass_kernel");
        core_merge_kernel<<<(unsigned)ceil_div(a.nent, 256), 256, 0, s>>>(a.part, nctas, a.nz, a.nent, blk.b, a.J0,
                                                                          blk.m, tot);
        VEST_LAUNCH("core_merge_kernel");
      } else {
        VEST_CUDA(cudaMemsetAsync(tot, 0, (size_t)a.nent * 8, s));
      }
      if (solve) {
        core_solve_kernel<T><<<1, 128, 0, s>>>(M, blk, a.J0, a.J1, reg, lambda, tot, dbuf[iblk & 1]);
        VEST_LAUNCH("core_solve_kernel");
      } else {
        core_resp_kernel<T><<<1, 128, 0, s>>>(M, blk, a.J0, a.J1, tot, stats, delta_core, resp_core);
        VEST_LAUNCH("core_resp_kernel");
      }
      a.prev = blk;
      ++iblk;
    }
  }
  return VEST_OK;
}

template <typename T>
vest_status sweep_core_impl(const vest_index* ix, const vest_model* m, int reg, double lambda, char* scratch,
                            const ScratchPlan& plan, cudaStream_t s) {
  T* r0 = reinterpret_cast<T*>(scratch + plan.off_resid);
  double* out = reinterpret_cast<double*>(scratch + plan.off_small) + 9000 + 2 * kCoreMaxB;
  VEST_TRY(loss_impl<T>(ix, m, reg, lambda, out, r0, nullptr, scratch, plan, s));
  return core_blocks<T>(ix, m, reg, lambda, true, r0, nullptr, nullptr, nullptr, scratch, plan, s);
}

template <typename T>
vest_status core_responsibility(const vest_index* ix, const vest_model* m, const T* resid_csr0, const double* stats,
                                double* delta_core, double* resp_core, char* scratch, const ScratchPlan& plan,
                                cudaStream_t s) {
  return core_blocks<T>(ix, m, 0, 0.0, false, const_cast<T*>(resid_csr0), stats, delta_core, resp_core, scratch,
                        plan, s);
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
