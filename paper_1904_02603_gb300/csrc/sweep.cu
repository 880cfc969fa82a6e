// Factor sweep (Algorithm 4; Lemma 1, Eq. 9-11; Lemma 3, Eq. 13) and the
// factor part of the responsibility (Eq. 6, Algorithm 3) over the mode-n CSR.
//
// Work is cut into tasks of TASK consecutive CSR positions (nnz-balanced, so
// heavy Zipf rows and one-entry rows cost the same per entry):
//   phase 1  E entries per thread: delta_alpha (Eq. 11) into shared memory,
//            every core fibre read once for the thread's E entries;
//   phase 2  the row sums c_j = sum X delta_j and V_jt = sum delta_j delta_t
//            (Eq. 10) for the update, or sum r delta_j and sum delta_j^2 for the
//            responsibility, per row piece (accumulator: T): short pieces one
//            warp each, long pieces cut into 32-entry chunks over all warps and
//            combined in chunk order; at most KMAX pieces per round;
//   phase 3  one thread per row: a row that ends inside the block's task range
//            stores its sums in the row buffer (a row cut by task edges inside
//            the range is carried from task to task with Kahan compensation);
//            a row cut by the edges of the range writes its piece to a spill
//            slot, and the block where the row starts registers it for the
//            fix-up kernel, which adds the pieces in block order in FP64 and
//            stores the sums likewise.
// A last kernel finishes every non-empty row from the row buffer, one thread
// per row (sequential CD over j in FP64), so the FP64 work runs in full warps
// instead of one lane per row inside the task kernel.  Rows of A^(n) are
// independent (delta does not involve A^(n)), so the order is free.
#include <algorithm>
#include <cstdlib>

#include "tc_delta.cuh"

namespace vest {

enum { kModeUpdate = 0, kModeResp = 1 };

struct SweepArgs {
  ModeRoles r;
  int path;  // vest_delta_path: 0 tensor cores where they apply, 1 FMA kernels, 2 tensor cores required
  int reg;
  double lambda;
  int64_t ntasks;
  int64_t tpc;  // consecutive tasks per thread block
  int task;  // entries per task (blockDim * E)
  int kmax;  // row pieces per phase-2 round
  int P;
  int use_smem_core;
  const uint8_t* onz;
  double* spill;       // [ntasks][2][P]
  int32_t* spanning;   // [ntasks]
  void* rowbuf;        // [non-empty rows][P]: the sums of every row, storage type
  template <typename T>
  __host__ __device__ T* rowbuf_t() const { return static_cast<T*>(rowbuf); }
  // responsibility
  const void* resid_coo;
  const double* stats;  // device {.., x_norm2 at [1], .., RE at [4]}
  double* delta;        // I_n x J_n
  double* resp;         // nullable
};

__host__ __device__ inline int packed_row(int j, int Jn) { return j * Jn - (j * (j - 1)) / 2; }

// Finish a row from its sums (FP64).  kModeUpdate: sequential CD over j (Eq. 9
// or Eq. 13 with g = -2(c_j - sum_{t!=j} V_jt a_t), d = 2 V_jj), each new value
// rounded to the storage type before the next j uses it.  kModeResp: Delta and
// Resp per element (Eq. 3, 6).
template <typename T, typename S, int MODE>
__device__ void finish_row(const DevModel<T>& M, int n, int64_t row, const S* sums, const SweepArgs& a) {
  const int Jn = M.J[n];
  T* arow = M.A[n] + row * Jn;
  if constexpr (MODE == kModeUpdate) {
    const uint8_t* mrow = M.mask[n] + row * Jn;
    double av[kMaxRank];
    for (int t = 0; t < Jn; ++t) av[t] = (double)arow[t];
    for (int j = 0; j < Jn; ++j) {
      if (mrow[j]) continue;
      double num = (double)sums[j];
      for (int t = 0; t < Jn; ++t) {
        if (t == j) continue;
        const int lo = t < j ? t : j, hi = t < j ? j : t;
        num -= (double)sums[Jn + packed_row(lo, Jn) + (hi - lo)] * av[t];
      }
      const double vjj = (double)sums[Jn + packed_row(j, Jn)];
      double nv;
      if (a.reg == VEST_REG_L1) {
        const double g = -2.0 * num, d = 2.0 * vjj;
        nv = g > a.lambda ? (a.lambda - g) / d : (g < -a.lambda ? -(a.lambda + g) / d : 0.0);
      } else {
        nv = num / (vjj + a.lambda);
      }
      const T st = (T)nv;
      arow[j] = st;
      av[j] = (double)st;
    }
  } else {
    const double xx = a.stats[1], re = a.stats[4];
    for (int j = 0; j < Jn; ++j) {
      const double aij = (double)arow[j];
      const double dl = 2.0 * aij * (double)sums[j] + aij * aij * (double)sums[Jn + j];
      a.delta[row * Jn + j] = dl;
      if (a.resp) a.resp[row * Jn + j] = re > 0.0 ? (sqrt(fmax(re * re + dl / xx, 0.0)) - re) / re : 0.0;
    }
  }
}

// Chunks of the long pieces of one task: sum of ceil(len / kPieceChunk) over pieces
// longer than kPieceChunk, at most task / kPieceChunk + task / (kPieceChunk + 1).
__host__ __device__ inline int long_chunks(int task) { return task / kPieceChunk + task / (kPieceChunk + 1); }

// Row-sum tiles over the staged vectors V = (delta_0 .. delta_{JN-1}, X, 0).
// kModeUpdate: outer 2 x 2 tiles (I, J), I <= J over column pairs, the (X, 0) pair
// with itself left out; each product delta_j delta_t (j <= t < Jn) goes to the packed
// Gram output Jn + packed(j, t), X delta_j to output j.  kModeResp: square tiles, one
// per pair of columns: r delta_j to output j, delta_j^2 to output Jn + j.
__host__ __device__ inline int sweep_tiles(int JN, int mode) {
  const int nb = (JN + 2) / 2;
  return mode == kModeUpdate ? nb * (nb + 1) / 2 - 1 : JN / 2;
}

__device__ inline void sweep_tile(int t, int JN, int Jn, int mode, int2& cab, int4& out) {
  int o[4] = {-1, -1, -1, -1};
  if (mode == kModeUpdate) {
    const int nb = (JN + 2) / 2;
    int I = 0, u = t;
    while (u >= nb - I) {
      u -= nb - I;
      ++I;
    }
    const int J = I + u;
    cab = make_int2(2 * I, 2 * J);
    for (int i = 0; i < 4; ++i) {
      const int j = 2 * I + (i >> 1), tt = 2 * J + (i & 1);
      if (I == J && (i >> 1) > (i & 1)) continue;  // the lower copy of a diagonal tile
      if (j >= Jn) continue;
      if (tt < Jn) o[i] = Jn + packed_row(j, Jn) + (tt - j);
      else if (tt == JN) o[i] = j;
    }
  } else {
    cab = make_int2(2 * t, 0);
    const int j0 = 2 * t, j1 = 2 * t + 1;
    if (j0 < Jn) {
      o[0] = j0;
      o[2] = Jn + j0;
    }
    if (j1 < Jn) {
      o[1] = j1;
      o[3] = Jn + j1;
    }
  }
  out = make_int4(o[0], o[1], o[2], o[3]);
}

// Shared memory of a task after the kernel's own leading region (`off` bytes): row starts,
// staged vectors V, per-piece sums, long-piece partials, tile table, carried row sums.
template <typename T>
struct TaskSmem {
  int64_t* sptr;
  T* sV;
  T* sAcc;
  T* sPart;
  int4* sOut;
  int2* sCab;
  T* sCarry;
};

// With v_ext set, V lives there (a region the caller shares with something else) and no
// room is carved for it.
template <typename T>
__device__ __forceinline__ TaskSmem<T> carve_task_smem(unsigned char* base, size_t off, int TASK, int L, int KMAX, int P,
                                                       int NT, T* v_ext = nullptr) {
  TaskSmem<T> t;
  off = (off + 15) & ~(size_t)15;
  t.sptr = reinterpret_cast<int64_t*>(base + off);
  off += (size_t)(TASK + 2) * 8;
  off = (off + 15) & ~(size_t)15;
  if (v_ext) {
    t.sV = v_ext;
  } else {
    t.sV = reinterpret_cast<T*>(base + off);
    off += (size_t)TASK * L * sizeof(T);
  }
  off = (off + 15) & ~(size_t)15;
  t.sAcc = reinterpret_cast<T*>(base + off);
  off += (size_t)KMAX * P * sizeof(T);
  t.sPart = reinterpret_cast<T*>(base + off);
  off += (size_t)long_chunks(TASK) * NT * 4 * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  t.sOut = reinterpret_cast<int4*>(base + off);
  off += (size_t)NT * sizeof(int4);
  t.sCab = reinterpret_cast<int2*>(base + off);
  off += (size_t)NT * sizeof(int2);
  off = (off + 15) & ~(size_t)15;
  t.sCarry = reinterpret_cast<T*>(base + off);
  return t;
}

// Phases 2 and 3 of one task, after its staged vectors V are in shared memory: per-row sums
// over the task's row pieces, then store, carry or spill them (see the top of this file).
template <typename T, int MODE>
__device__ __forceinline__ void task_row_sums(const SweepArgs& a, int JN, int64_t task, int64_t tb, int64_t te,
                                              int64_t t0, int64_t t1, int nrows, int64_t k0, const int64_t* sptr,
                                              int NT, const int2* sCab, const int4* sOut, const T* sV, T* sAcc,
                                              T* sPart, PieceScratch* pscr, T* cin, T* cout) {
  const int KMAX = a.kmax, P = a.P, TASK = a.task;
  const int L = JN + 2;
  const int64_t rt0 = tb * TASK;
  for (int r0 = 0; r0 < nrows; r0 += KMAX) {
    const int nr = min(KMAX, nrows - r0);
    // phase 2: per-row sums over the task's pieces r0 .. r0 + nr - 1
    piece_sums<T, MODE == kModeResp>(sptr + r0, nr, t0, t1, NT, P, sCab, sOut, sV, L, JN, sAcc, sPart, pscr);
    // phase 3: store the sums of rows that end here; carry a row that continues into
    // the block's next task; spill rows cut by the edges of the block's task range.  One
    // thread per (row, output): the P outputs of a row are independent, so a row carried
    // across tasks costs one Kahan step per thread, not P in a row on one thread.
    for (int idx = threadIdx.x; idx < nr * P; idx += blockDim.x) {
      const int kr = idx / P, i = idx - kr * P;
      const int k = r0 + kr;
      const int64_t rs = sptr[k], re = sptr[k + 1];
      const T pv = sAcc[kr * P + i];
      const bool carried_in = (k == 0) && rs < t0 && task > tb;  // earlier pieces are in cin
      const bool continues = re > t1;
      const bool started_here = rs >= rt0;
      if (!continues && !carried_in && rs >= t0) {
        a.rowbuf_t<T>()[(size_t)(k0 + k) * P + i] = pv;
      } else {
        // running sums of a row cut by task edges: (sum, compensation) in T
        T* as = continues ? cout : cin;
        const T sum = carried_in ? cin[i] : T(0), cmp = carried_in ? cin[P + i] : T(0);
        const T y = pv - cmp;
        const T t = sum + y;
        const T c = (t - sum) - y;
        as[P + i] = c;
        as[i] = t;
        if (!continues) {
          if (started_here) a.rowbuf_t<T>()[(size_t)(k0 + k) * P + i] = t - c;
          else a.spill[((size_t)blockIdx.x * 2 + 0) * P + i] = (double)t - (double)c;  // incoming partial
        } else if (task + 1 == te) {  // leaves the block's range
          a.spill[((size_t)blockIdx.x * 2 + (started_here ? 1 : 0)) * P + i] = (double)t - (double)c;
        }
      }
      if (i == 0 && k == nrows - 1 && task + 1 == te)
        a.spanning[blockIdx.x] = (continues && started_here) ? (int32_t)(k0 + k) : -1;
    }
    __syncthreads();
  }
}

template <typename T, int JN, int JF, int NSLOW, int MODE, int E>
__global__ void __launch_bounds__(256 / E, (delta_min_blocks<T, JN, JF, E>(256 / E))) sweep_task_kernel(DevModel<T> M, DevMode<T> csr, const T* __restrict__ gcore,
                                                         SweepArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ModeRoles& r = a.r;
  const int TASK = a.task, KMAX = a.kmax;
  constexpr int L = JN + 2;  // staged vector: delta_0 .. delta_{JN-1}, X, 0
  const int P = a.P;
  const int NT = sweep_tiles(JN, MODE);
  const int64_t core_elems = r.n_outer * r.Jf * JN;
  // shared layout: core | sptr | V | acc | long-piece partials | tile table | carry
  T* sG = reinterpret_cast<T*>(smem_raw);
  const TaskSmem<T> ts = carve_task_smem<T>(smem_raw, a.use_smem_core ? (size_t)core_elems * sizeof(T) : 0, TASK,
                                            L, KMAX, P, NT);
  int64_t* sptr = ts.sptr;
  T* sV = ts.sV;
  int4* sOut = ts.sOut;
  int2* sCab = ts.sCab;
  T* sCarry = ts.sCarry;  // [2][sum, compensation][P]: row sums carried to the next task
  __shared__ PieceScratch pscr;

  const T* g = gcore;
  if (a.use_smem_core) {
    for (int64_t e = threadIdx.x; e < core_elems; e += blockDim.x) sG[e] = gcore[e];
    g = sG;
  }
  for (int t = threadIdx.x; t < NT; t += blockDim.x) sweep_tile(t, JN, r.Jn, MODE, sCab[t], sOut[t]);
  const int R = *csr.nnzrows;
  const int64_t nnz = csr.nnz;
  __syncthreads();

  // this block's consecutive tasks [tb, te)
  const int64_t tb = blockIdx.x * a.tpc, te = min(tb + a.tpc, a.ntasks);
  for (int64_t task = tb; task < te; ++task) {
    const int64_t t0 = task * TASK, t1 = min(t0 + (int64_t)TASK, nnz);
    const int cnt = (int)(t1 - t0);
    int64_t k0;
    const int nrows = load_task_rows(csr.nzptr, csr.gran, R, t0, t1, sptr, &k0);
    T* cin = sCarry + (task & 1) * 2 * P;         // carried in from task - 1 (same block)
    T* cout = sCarry + ((task + 1) & 1) * 2 * P;  // carried out to task + 1

    // phase 1: delta for the thread's E entries (threadIdx.x + e * blockDim.x)
    if ((int)threadIdx.x < cnt) {
      const T* rowf[E];
      SlowRows sr[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int q = threadIdx.x + e * blockDim.x;
        const int64_t p = t0 + (q < cnt ? q : (int)threadIdx.x);
        rowf[e] = gather_rows<T, NSLOW>(M, r, csr.oidx, nnz, p, sr[e]);
      }
      T d[E][JN];
      compute_delta_multi<T, JN, JF, NSLOW, E>(d, g, a.onz, r.n_outer, r.Jf, rowf, sr, r.nslow);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int q = threadIdx.x + e * blockDim.x;
        if (q < cnt) {
          T* dst = sV + q * L;
#pragma unroll
          for (int j = 0; j < JN; ++j) dst[j] = d[e][j];
          if constexpr (MODE == kModeUpdate) dst[JN] = csr.val[t0 + q];
          else dst[JN] = static_cast<const T*>(a.resid_coo)[csr.perm[t0 + q]];
          dst[JN + 1] = T(0);
        }
      }
    }
    __syncthreads();

    task_row_sums<T, MODE>(a, JN, task, tb, te, t0, t1, nrows, k0, sptr, NT, sCab, sOut, sV, ts.sAcc, ts.sPart, &pscr,
                           cin, cout);
  }
}

// ------------------------------------------------------------------ tensor-core delta (FP32)
// The task kernel with phase 1 on the tensor cores (tc_delta.cuh): per task two groups of 128
// entries, each group's A rows written by their own lanes, the MMAs issued by one thread,
// stage 2 read back from the accumulator, then phases 2 and 3 as in sweep_task_kernel.  The
// A region of shared memory takes the staged vectors V once the task's last MMA has completed.
// A wait that runs out marks the device status and ends the CTA's work after its in-flight
// MMAs are given the same bounded wait.
static __device__ unsigned int g_sweep_status;  // bit 0: an MMA completion wait gave up

// One staged vector V of L floats (L even; its start is L * 4 * q bytes into a 16-byte aligned
// array): 16-byte stores when L is a multiple of 4 (at L = 12 the 32 lanes' pieces then fill
// whole wavefronts), 8-byte stores otherwise.
template <int L>
__device__ __forceinline__ void store_row(float* dst, const float (&v)[L]) {
  if constexpr (L % 4 == 0) {
#pragma unroll
    for (int i = 0; i < L; i += 4) *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < L; i += 2) *reinterpret_cast<float2*>(dst + i) = make_float2(v[i], v[i + 1]);
  }
}

template <int JN, int MODE, int NA>
__global__ void __launch_bounds__(128, NA == 1 ? 4 : 2)
    sweep_task_tc_kernel(DevModel<float> M, DevMode<float> csr, const float* __restrict__ gp, SweepArgs a, TcPlan tp) {
  using T = float;
  constexpr int E = 2;  // entries per thread: two groups of 128
  constexpr int L = JN + 2;
  extern __shared__ __align__(128) unsigned char tc_smem_raw[];
  __shared__ uint64_t mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int wait_failed;
  __shared__ PieceScratch pscr;
  const ModeRoles& r = a.r;
  const int TASK = a.task, KMAX = a.kmax, P = a.P;
  const int NT = sweep_tiles(JN, MODE);
  const int tid = threadIdx.x, warp = tid >> 5;
  // shared layout: B hi | B lo | U = (A hi | A lo) or V | sptr | acc | long-piece partials | tiles | carry
  uint32_t* sBhi = reinterpret_cast<uint32_t*>(tc_smem_raw);
  uint32_t* sBlo = reinterpret_cast<uint32_t*>(tc_smem_raw + tp.btile);
  unsigned char* U = tc_smem_raw + 2 * tp.btile;
  uint32_t* sAhi = reinterpret_cast<uint32_t*>(U);
  uint32_t* sAlo = reinterpret_cast<uint32_t*>(U + tp.atile);
  const TaskSmem<T> ts =
      carve_task_smem<T>(tc_smem_raw, 2 * tp.btile + tp.ubytes, TASK, L, KMAX, P, NT, reinterpret_cast<T*>(U));

  tc_fill_b<JN, NA>(sBhi, sBlo, gp, r, tp);
  for (int t = tid; t < NT; t += blockDim.x) sweep_tile(t, JN, r.Jn, MODE, ts.sCab[t], ts.sOut[t]);
  if (tid == 0) {
    tc::mbar_init(&mma_bar, 1);
    wait_failed = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tmem_slot, (uint32_t)tp.ncols);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_slot;
  TcCta<NA> tcc;
  tcc.init(tbase, tp, sBhi, sBlo, sAhi, sAlo);
  uint32_t phase = 0;

  const int64_t nnz = csr.nnz;
  const int64_t tb = blockIdx.x * a.tpc, te = min(tb + a.tpc, a.ntasks);

  // gathers for both entries of the thread in task `tk`: rows of the A modes, the remaining
  // mode's row, X (or r).  The next task's are issued before the current task's row sums, so
  // their latency hides behind that phase.
  // The task's row table comes from the same prefetch: the non-empty-row number of each entry
  // (and of the entry before each warp's first), the first and last row of the task, where the
  // first row starts and the last one ends.
  float a0[E][16], a1[E][NA == 2 ? 16 : 1], wr[E][16], xv[E];
  int rk[E], rkprev[E];
  int kfirst = 0, klast = 0;
  int64_t rs_first = 0, re_last = 0;
  auto gather = [&](int64_t tk) {
    const int64_t g0 = tk * TASK;
    const int gcnt = (int)(min(g0 + (int64_t)TASK, nnz) - g0);
    kfirst = csr.rowk[g0];
    klast = csr.rowk[g0 + gcnt - 1];
    if (tid == 0) {
      rs_first = csr.nzptr[kfirst];
      re_last = csr.nzptr[klast + 1];
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int q = tid + e * 128;
      const bool valid = q < gcnt;
      const int64_t p = g0 + (valid ? q : 0);
      rk[e] = csr.rowk[p];
      rkprev[e] = (valid && q > 0 && (q & 31) == 0) ? csr.rowk[p - 1] : rk[e];
      tc_row(a0[e], tp, M.A[r.f], csr.oidx[p], r.Jf, valid);
      if constexpr (NA == 2) tc_row(a1[e], tp, M.A[r.slow[0]], csr.oidx[nnz + p], tp.JA1, valid);
      if (tp.has_rest) {
        tc_row(wr[e], tp, M.A[r.slow[NA - 1]], csr.oidx[(int64_t)NA * nnz + p], tp.O, valid);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) wr[e][i] = i == 0 ? 1.f : 0.f;
      }
      if constexpr (MODE == kModeUpdate) xv[e] = valid ? csr.val[p] : 0.f;
      else xv[e] = valid ? static_cast<const T*>(a.resid_coo)[csr.perm[p]] : 0.f;
    }
  };
  if (tb < te) gather(tb);

  for (int64_t task = tb; task < te; ++task) {
    const int64_t t0 = task * TASK, t1 = min(t0 + (int64_t)TASK, nnz);
    const int cnt = (int)(t1 - t0);
    const int64_t k0 = kfirst;
    const int nrows = klast - kfirst + 1;
    T* cin = ts.sCarry + (task & 1) * 2 * P;
    T* cout = ts.sCarry + ((task + 1) & 1) * 2 * P;

    float d[E][JN];
#pragma unroll
    for (int g = 0; g < E; ++g) {
      tcc.write_a(tid, a0[g], a1[g]);
      __syncthreads();
      if (tid == 0) tcc.issue(&mma_bar);
      __syncwarp();
      const bool done = tc::mbar_wait_bounded(&mma_bar, phase, kTcWaitPolls);
      phase ^= 1u;
      if (__any_sync(0xffffffffu, !done) && (tid & 31) == 0) wait_failed = 1;  // checked after the task's V barrier
      tc::fence_after_sync();
      tcc.template delta<JN>(tp.Np, tp.O, wr[g], d[g]);
      tc::fence_before_sync();  // this group's accumulator reads before the next group's MMAs
    }
    // every MMA of the task has completed (each thread waited): V may take over the A region
#pragma unroll
    for (int g = 0; g < E; ++g) {
      const int q = tid + g * 128;
      if (q < cnt) {
        float v[L];
#pragma unroll
        for (int j = 0; j < JN; ++j) v[j] = d[g][j];
        v[JN] = xv[g];
        v[JN + 1] = 0.f;
        store_row<L>(ts.sV + q * L, v);
      }
    }
    // row table: sptr[k - k0] = start of every row that starts inside the task, sptr[0] and
    // sptr[nrows] the first row's start and the last row's end (they may lie outside it)
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int q = tid + e * 128;
      const int up = __shfl_up_sync(0xffffffffu, rk[e], 1);
      const int before = (q & 31) == 0 ? rkprev[e] : up;
      if (q > 0 && q < cnt && rk[e] != before) ts.sptr[rk[e] - kfirst] = t0 + q;
    }
    if (tid == 0) {
      ts.sptr[0] = rs_first;
      ts.sptr[nrows] = re_last;
    }
    if (task + 1 < te) gather(task + 1);
    __syncthreads();
    if (wait_failed) break;  // uniform: read after the barrier
    task_row_sums<T, MODE>(a, JN, task, tb, te, t0, t1, nrows, k0, ts.sptr, NT, ts.sCab, ts.sOut, ts.sV, ts.sAcc,
                           ts.sPart, &pscr, cin, cout);
  }
  if (wait_failed) {
    // the MMAs may still be in flight: give them another bounded wait before tensor memory is freed
    if (tid == 0) atomicOr(&g_sweep_status, 1u);
    tc::mbar_wait_bounded(&mma_bar, phase ^ 1u, kTcWaitPolls);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, (uint32_t)tp.ncols);
}

// Rows cut by the edges of the blocks' task ranges: the block where the row starts
// wrote its outgoing partial (slot 1), every later block the row reaches wrote
// its incoming partial (slot 0); add them in block order (FP64) and finish.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) sweep_fixup_kernel(DevModel<T> M, DevMode<T> csr, SweepArgs a, int nblocks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* part = reinterpret_cast<double*>(smem_raw);  // [groups][P]
  const int P = a.P;
  const int groups = max(1, (int)blockDim.x / P);
  for (int64_t c = blockIdx.x; c < nblocks; c += gridDim.x) {
    const int32_t kg = a.spanning[c];
    if (kg < 0) continue;  // uniform across the block
    const int64_t re = csr.nzptr[kg + 1];
    const int64_t clast = ((re - 1) / a.task) / a.tpc;
    // groups > 1: thread (gi, pi) sums output pi over blocks c + gi, c + gi + groups, ...;
    // groups == 1 (P > blockDim): each thread sums outputs threadIdx.x + k * blockDim over all blocks
    const int gi = groups > 1 ? (int)threadIdx.x / P : 0;
    const int pstart = groups > 1 ? (int)threadIdx.x % P : (int)threadIdx.x;
    const int pstep = groups > 1 ? P : (int)blockDim.x;
    if (gi < groups) {
      for (int pp = pstart; pp < P; pp += pstep) {
        double acc = 0.0;
        if (c + gi <= clast) acc = a.spill[((size_t)(c + gi) * 2 + (gi == 0 ? 1 : 0)) * P + pp];
        double c8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int64_t cc = c + gi + groups;
        for (; cc + 7 * groups <= clast; cc += 8 * groups) {
#pragma unroll
          for (int u = 0; u < 8; ++u) c8[u] += a.spill[((size_t)(cc + u * groups) * 2) * P + pp];
        }
        for (int u = 0; cc <= clast; cc += groups, ++u) c8[u & 7] += a.spill[((size_t)cc * 2) * P + pp];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += c8[u];
        part[gi * P + pp] = acc;
      }
    }
    __syncthreads();
    for (int pp = threadIdx.x; pp < P; pp += blockDim.x) {
      double acc = 0.0;
      for (int gg = 0; gg < groups; ++gg) acc += part[gg * P + pp];
      a.rowbuf_t<T>()[(size_t)kg * P + pp] = (T)acc;
    }
    __syncthreads();
  }
}

// Every non-empty row from its sums in the row buffer, one thread per row (FP64 CD).
template <typename T, int MODE>
__global__ void __launch_bounds__(128) finish_rows_kernel(DevModel<T> M, DevMode<T> csr, SweepArgs a) {
  const int64_t R = *csr.nnzrows;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < R; k += (int64_t)gridDim.x * blockDim.x)
    finish_row<T, T, MODE>(M, a.r.n, (int64_t)csr.nzrow[k], a.rowbuf_t<T>() + (size_t)k * a.P, a);
}

// Rows with no observed entry: the update gives 0; their Delta is 0.
template <typename T, int MODE>
__global__ void empty_rows_kernel(DevModel<T> M, int n, const int64_t* __restrict__ row_ptr, double* delta,
                                  double* resp) {
  const int Jn = M.J[n];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M.I[n]; i += (int64_t)gridDim.x * blockDim.x) {
    if (row_ptr[i] != row_ptr[i + 1]) continue;
    for (int j = 0; j < Jn; ++j) {
      if constexpr (MODE == kModeUpdate) {
        M.A[n][i * Jn + j] = T(0);
      } else {
        delta[i * Jn + j] = 0.0;
        if (resp) resp[i * Jn + j] = 0.0;
      }
    }
  }
}

// ------------------------------------------------------------------ host side
static int outputs_per_row(int Jn, int mode_kind) {
  return mode_kind == kModeUpdate ? Jn + Jn * (Jn + 1) / 2 : 2 * Jn;
}

constexpr size_t kSmemBudget = 200 * 1024;
constexpr size_t kSmemMax = 227 * 1024;
constexpr size_t kAccBudget = 32 * 1024;
constexpr int kTask = 256;
constexpr int64_t kSweepBlocks = 3040;  // fixed (sum order device-independent): 4 waves of 5 blocks on 152 SMs

template <typename T>
static int pieces_per_round(int P) {
  return (int)std::max<size_t>(1, std::min<size_t>(64, kAccBudget / ((size_t)P * sizeof(T))));
}

template <typename T>
static size_t task_smem(int task, int kmax, int JN, int P, int mode, size_t core_bytes, bool own_v = true) {
  const int NT = sweep_tiles(JN, mode);
  size_t off = (core_bytes + 15) & ~(size_t)15;
  off += (size_t)(task + 2) * 8;
  off = (off + 15) & ~(size_t)15;
  if (own_v) off += (size_t)task * (JN + 2) * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  off += (size_t)kmax * P * sizeof(T);
  off += (size_t)long_chunks(task) * NT * 4 * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  off += (size_t)NT * (sizeof(int4) + sizeof(int2));
  off = (off + 15) & ~(size_t)15;
  off += 4 * (size_t)P * sizeof(T);
  return off;
}

// Task geometry: 256 entries per task; the core goes to shared memory when it fits.
template <typename T>
int sweep_task_size(int Jn, int P, int64_t core_elems, int* use_smem_core) {
  const int JN = jn_bucket(Jn);
  // the update's tiles outnumber the responsibility's: size for the update
  *use_smem_core =
      task_smem<T>(kTask, pieces_per_round<T>(P), JN, P, kModeUpdate, (size_t)core_elems * sizeof(T)) <= kSmemBudget;
  return kTask;
}

template int sweep_task_size<float>(int, int, int64_t, int*);
template int sweep_task_size<double>(int, int, int64_t, int*);

template <typename T, int JN, int JF, int NSLOW, int MODE, int E>
static vest_status launch_task(const DevModel<T>& M, const DevMode<T>& csr, const T* gp, const SweepArgs& a,
                               size_t smem, cudaStream_t s) {
  auto kern = sweep_task_kernel<T, JN, JF, NSLOW, MODE, E>;
  VEST_TRY(allow_smem(kern, smem));
  kern<<<(unsigned)ceil_div(a.ntasks, a.tpc), a.task / E, smem, s>>>(M, csr, gp, a);
  VEST_LAUNCH("sweep_task_kernel");
  return VEST_OK;
}

// FP32: two entries per thread, the f-mode rank in registers when it equals the
// bucket width; FP64 (the accuracy reference path): one entry per thread.
template <typename T, int JN, int MODE>
static vest_status dispatch_nslow(int nslow, int Jf, const DevModel<T>& M, const DevMode<T>& csr, const T* gp,
                                  const SweepArgs& a, size_t smem, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (nslow == 1 && Jf == JN) return launch_task<T, JN, JN, 1, MODE, 2>(M, csr, gp, a, smem, s);
    if (nslow == 1) return launch_task<T, JN, 0, 1, MODE, 2>(M, csr, gp, a, smem, s);
    if (nslow == 2 && Jf == JN) return launch_task<T, JN, JN, 2, MODE, 2>(M, csr, gp, a, smem, s);
    if (nslow == 2) return launch_task<T, JN, 0, 2, MODE, 2>(M, csr, gp, a, smem, s);
    return launch_task<T, JN, 0, -1, MODE, 1>(M, csr, gp, a, smem, s);
  } else {
    if (nslow == 1) return launch_task<T, JN, 0, 1, MODE, 1>(M, csr, gp, a, smem, s);
    if (nslow == 2) return launch_task<T, JN, 0, 2, MODE, 1>(M, csr, gp, a, smem, s);
    return launch_task<T, JN, 0, -1, MODE, 1>(M, csr, gp, a, smem, s);
  }
}

template <typename T, int MODE>
static vest_status dispatch_jn(int JN, int nslow, int Jf, const DevModel<T>& M, const DevMode<T>& csr, const T* gp,
                               const SweepArgs& a, size_t smem, cudaStream_t s) {
  switch (JN) {
    case 4: return dispatch_nslow<T, 4, MODE>(nslow, Jf, M, csr, gp, a, smem, s);
    case 8: return dispatch_nslow<T, 8, MODE>(nslow, Jf, M, csr, gp, a, smem, s);
    case 10: return dispatch_nslow<T, 10, MODE>(nslow, Jf, M, csr, gp, a, smem, s);
    case 12: return dispatch_nslow<T, 12, MODE>(nslow, Jf, M, csr, gp, a, smem, s);
    case 16: return dispatch_nslow<T, 16, MODE>(nslow, Jf, M, csr, gp, a, smem, s);
    default: return dispatch_nslow<T, 32, MODE>(nslow, Jf, M, csr, gp, a, smem, s);
  }
}

// ------------------------------------------------------------------ tensor-core path selection
template <int JN, int MODE>
static vest_status launch_tc(const DevModel<float>& M, const DevMode<float>& csr, const float* gp, SweepArgs a,
                             const TcPlan& tp, cudaStream_t s) {
  a.kmax = std::min(a.kmax, 32);  // fewer row pieces per round: room for four CTAs per SM
  size_t smem = task_smem<float>(a.task, a.kmax, JN, a.P, MODE, 2 * tp.btile + tp.ubytes, false);
  // no more CTAs on an SM than its 512 TMEM columns hold, so no allocation ever waits
  const size_t sm_bytes = 228 * 1024, reserved = 1024;
  smem = std::max(smem, sm_bytes / (tp.per_sm + 1) - reserved + 16);
  if (smem > kSmemMax) return fail(VEST_ERR_UNSUPPORTED, "tensor-core factor sweep: shared memory exceeds 227 KB");
  TcPlan tpl = tp;
  tpl.base8 = 1;
  for (int k = 0; k < M.N; ++k)
    if (reinterpret_cast<uintptr_t>(M.A[k]) % 8 != 0) tpl.base8 = 0;
  auto kern = tp.na == 2 ? sweep_task_tc_kernel<JN, MODE, 2> : sweep_task_tc_kernel<JN, MODE, 1>;
  VEST_TRY(allow_smem(kern, smem));
  kern<<<(unsigned)ceil_div(a.ntasks, a.tpc), 128, smem, s>>>(M, csr, gp, a, tpl);
  VEST_LAUNCH("sweep_task_tc_kernel");
  return VEST_OK;
}

template <int MODE>
static vest_status dispatch_tc(int JN, const DevModel<float>& M, const DevMode<float>& csr, const float* gp,
                               const SweepArgs& a, const TcPlan& tp, cudaStream_t s) {
  switch (JN) {
    case 4: return launch_tc<4, MODE>(M, csr, gp, a, tp, s);
    case 8: return launch_tc<8, MODE>(M, csr, gp, a, tp, s);
    case 10: return launch_tc<10, MODE>(M, csr, gp, a, tp, s);
    case 12: return launch_tc<12, MODE>(M, csr, gp, a, tp, s);
    case 16: return launch_tc<16, MODE>(M, csr, gp, a, tp, s);
    default: return launch_tc<32, MODE>(M, csr, gp, a, tp, s);
  }
}

template <typename T, int MODE>
static vest_status run_mode(const vest_index* ix, const DevModel<T>& M, int n, SweepArgs a, char* scratch,
                            const ScratchPlan& plan, cudaStream_t s) {
  const ModeRoles r = mode_roles(M.J, M.N, n);
  a.r = r;
  const int JN = jn_bucket(r.Jn);
  T* gp = reinterpret_cast<T*>(scratch + plan.off_gperm);
  const int64_t core_elems = r.n_outer * r.Jf * JN;
  uint8_t* onz = reinterpret_cast<uint8_t*>(scratch + plan.off_gperm + align_up((size_t)core_elems * sizeof(T)));
  if (align_up((size_t)core_elems * sizeof(T)) + align_up((size_t)r.n_outer) > plan.gperm_bytes)
    return fail(VEST_ERR_WORKSPACE, "scratch region for the permuted core too small");
  prep_core_kernel<T><<<(unsigned)std::min<int64_t>(r.n_outer, 4096), 128, 0, s>>>(M.G, r, JN, gp, onz);
  VEST_LAUNCH("prep_core_kernel");
  a.onz = onz;
  a.P = outputs_per_row(r.Jn, MODE);
  int use_smem = 0;
  a.task = sweep_task_size<T>(r.Jn, a.P, core_elems, &use_smem);
  a.kmax = pieces_per_round<T>(a.P);
  a.use_smem_core = use_smem;
  a.ntasks = ceil_div(ix->nnz, a.task);
  // a fixed number of thread blocks, each over consecutive tasks: the order of every
  // sum is the same on any device
  a.tpc = std::max<int64_t>(1, ceil_div(a.ntasks, kSweepBlocks));
  const int64_t nblocks = std::max<int64_t>(1, ceil_div(a.ntasks, a.tpc));
  if ((size_t)nblocks * 2 * a.P * 8 > plan.spill_bytes || nblocks > plan.ntasks)
    return fail(VEST_ERR_WORKSPACE, "scratch spill region too small");
  a.spill = reinterpret_cast<double*>(scratch + plan.off_spill);
  if ((size_t)ix->mode[n].cap * a.P * 8 > plan.rowbuf_bytes) return fail(VEST_ERR_WORKSPACE, "scratch row buffer too small");
  a.rowbuf = scratch + plan.off_rowbuf;
  a.spanning = reinterpret_cast<int32_t*>(scratch + plan.off_spanning);
  const DevMode<T> csr = dev_mode<T>(ix, n);
  const int eg = std::max(1, std::min<int>((int)ceil_div(M.I[n], 256), num_sms() * 8));
  empty_rows_kernel<T, MODE><<<eg, 256, 0, s>>>(M, n, ix->mode[n].row_ptr, a.delta, a.resp);
  VEST_LAUNCH("empty_rows_kernel");
  if (ix->nnz == 0) return VEST_OK;
  size_t smem = task_smem<T>(a.task, a.kmax, JN, a.P, MODE, use_smem ? (size_t)core_elems * sizeof(T) : 0);
  while (smem > kSmemMax && a.kmax > 1) {  // large ranks in FP64: fewer pieces per round
    a.kmax = std::max(1, a.kmax / 2);
    smem = task_smem<T>(a.task, a.kmax, JN, a.P, MODE, use_smem ? (size_t)core_elems * sizeof(T) : 0);
  }
  if (smem > kSmemMax) return fail(VEST_ERR_UNSUPPORTED, "factor sweep: shared memory of one task exceeds 227 KB");
  TcPlan tp{};
  const bool use_tc = sizeof(T) == 4 && a.task == 256 &&
                      (a.path == VEST_DELTA_TENSOR || (a.path == VEST_DELTA_AUTO && tensor_cores_enabled())) &&
                      tc_plan(r, M.N, JN, (size_t)kTask * (JN + 2) * 4, &tp);
  if constexpr (sizeof(T) == 4) {
    if (use_tc) VEST_TRY(dispatch_tc<MODE>(JN, M, csr, gp, a, tp, s));
    else VEST_TRY(dispatch_jn<T, MODE>(JN, r.nslow, r.Jf, M, csr, gp, a, smem, s));
  } else {
    VEST_TRY(dispatch_jn<T, MODE>(JN, r.nslow, r.Jf, M, csr, gp, a, smem, s));
  }
  const size_t fsmem = (size_t)std::max(1, 256 / a.P) * a.P * 8 + 8 * a.P;
  auto fk = sweep_fixup_kernel<T, MODE>;
  VEST_TRY(allow_smem(fk, fsmem));
  const int64_t fgrid = std::min<int64_t>(nblocks, (int64_t)num_sms() * 8);
  fk<<<(unsigned)fgrid, 256, fsmem, s>>>(M, csr, a, (int)nblocks);
  VEST_LAUNCH("sweep_fixup_kernel");
  const int64_t rgrid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(ix->mode[n].cap, 128), (int64_t)num_sms() * 8));
  finish_rows_kernel<T, MODE><<<(unsigned)rgrid, 128, 0, s>>>(M, csr, a);
  VEST_LAUNCH("finish_rows_kernel");
  return VEST_OK;
}

template <typename T>
vest_status sweep_factors_mode(const vest_index* ix, const vest_model* m, int reg, double lambda, int mode,
                               char* scratch, const ScratchPlan& plan, cudaStream_t s, int path) {
  const DevModel<T> M = dev_model<T>(m);
  SweepArgs a{};
  a.path = path;
  a.reg = reg;
  a.lambda = lambda;
  return run_mode<T, kModeUpdate>(ix, M, mode, a, scratch, plan, s);
}

template <typename T>
vest_status responsibility_factors(const vest_index* ix, const vest_model* m, const double* stats,
                                   double* const* delta_factor, double* const* resp_factor, char* scratch,
                                   const ScratchPlan& plan, cudaStream_t s) {
  const DevModel<T> M = dev_model<T>(m);
  for (int n = 0; n < M.N; ++n) {
    SweepArgs a{};
    a.resid_coo = scratch + plan.off_resid_coo;
    a.stats = stats;
    a.delta = delta_factor[n];
    a.resp = resp_factor ? resp_factor[n] : nullptr;
    VEST_TRY((run_mode<T, kModeResp>(ix, M, n, a, scratch, plan, s)));
  }
  return VEST_OK;
}

// Whether the tensor-core delta serves mode n of this FP32 model.
bool sweep_tc_applies(const vest_model* m, int n) {
  if (m->dtype != VEST_F32) return false;
  const ModeRoles r = mode_roles(m->ranks, m->order, n);
  TcPlan tp{};
  return tc_plan(r, m->order, jn_bucket(r.Jn), (size_t)kTask * (jn_bucket(r.Jn) + 2) * 4, &tp);
}

// Bits set by the factor-sweep kernels since the last clear (bit 0: a bounded wait on the
// tensor cores gave up); synchronises the device to read them.
vest_status sweep_device_status(uint32_t* flags, bool clear) {
  VEST_CUDA(cudaDeviceSynchronize());
  unsigned int v = 0;
  VEST_CUDA(cudaMemcpyFromSymbol(&v, g_sweep_status, sizeof(v)));
  if (clear && v) {
    const unsigned int z = 0;
    VEST_CUDA(cudaMemcpyToSymbol(g_sweep_status, &z, sizeof(z)));
  }
  *flags = v;
  return VEST_OK;
}

template vest_status sweep_factors_mode<float>(const vest_index*, const vest_model*, int, double, int, char*,
                                               const ScratchPlan&, cudaStream_t, int);
template vest_status sweep_factors_mode<double>(const vest_index*, const vest_model*, int, double, int, char*,
                                                const ScratchPlan&, cudaStream_t, int);
template vest_status responsibility_factors<float>(const vest_index*, const vest_model*, const double*,
                                                   double* const*, double* const*, char*, const ScratchPlan&,
                                                   cudaStream_t);
template vest_status responsibility_factors<double>(const vest_index*, const vest_model*, const double*,
                                                    double* const*, double* const*, char*, const ScratchPlan&,
                                                    cudaStream_t);

}  // namespace vest
