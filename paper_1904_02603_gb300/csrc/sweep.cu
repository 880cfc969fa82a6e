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

#include "delta.cuh"
#include "tcgen05.cuh"

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
// Eq. 11 in two stages for each group of 128 entries (one entry per accumulator row):
//   stage 1, tcgen05 MMA in split TF32 (hi*hi + hi*lo + lo*hi, about FP32 accuracy):
//     T[e][(o, j)] = sum_k A[e][k] B[k][(o, j)], with A[e] the row of the other mode f
//     (NA = 1) or the Khatri-Rao product of the rows of f and of the first slow mode
//     (NA = 2), and B the core permuted to (k, (o, j_n)), o over the one remaining other
//     mode (or a single o when none remains);
//   stage 2, FP32 FMAs: delta_e(j) = sum_o w_e(o) T[e][(o, j)], w_e the row of the
//     remaining mode (1 when none remains).
// With the dense 10 x 10 x 10 core of the Zipf workload this moves 1000 of the 1100 FMAs
// per entry of the staged contraction onto the tensor cores.  B sits in shared memory
// (K-major, no swizzle) and the accumulator in tensor memory, column o * JN + j.  With one
// A mode, A is written to shared memory by the lane of its entry (the MMA reads both
// operands there; the region is reused for the staged vectors V once the task's last MMA
// has completed), so the allocation is the accumulator alone: 128 columns for the Zipf
// workload, four CTAs per SM.  With two A modes the wider A goes to tensor memory.  One
// thread issues the MMAs and commits them to an mbarrier that every thread waits on with a
// bounded number of polls; a wait that runs out marks the device status and ends the CTA's
// work after its in-flight MMAs are given the same bounded wait.
struct TcPlan {
  int na;        // other modes folded into A: 1 (A in shared memory) or 2 (A in tensor memory)
  int jf8;       // rank of mode f rounded up to 8: A columns per row of the second A mode
  int JA1;       // rank of the second A mode (1 when na = 1)
  int Kp;        // A width: jf8 * JA1, a multiple of 8 (the MMA's K step)
  int O;         // rank of the remaining mode (1 when none)
  int has_rest;  // a remaining mode exists
  int Np;        // MMA N: O * JN rounded up to 16
  int colD;      // first accumulator column: 0 (na = 1) or 2 Kp after A hi and lo (na = 2)
  int ncols;     // TMEM columns allocated: power of two >= colD + Np
  int per_sm;    // CTAs per SM that the allocation allows: 512 / ncols
  size_t btile;  // bytes of one B tile (hi or lo): Np * Kp * 4
  size_t atile;  // bytes of one A tile (hi or lo) in shared memory: 128 * Kp * 4 (0 when na = 2)
  size_t ubytes; // shared region of A hi, A lo and, later, V: max(2 atile, V bytes), 128-aligned
};

constexpr uint32_t kTcWaitPolls = 1u << 22;  // bounded mbarrier wait (seconds at worst, never in practice)
constexpr int kTcMaxChunks = 14;             // accumulator columns read in 16-column chunks: Np <= 224
static __device__ unsigned int g_sweep_status;  // bit 0: an MMA completion wait gave up

// stage 2 for one lane: delta(j) += w(o) T[o * JN + j] over the accumulator's Np columns
template <int JN>
__device__ __forceinline__ void contract_rest(uint32_t taddr, int Np, int O, const float (&w)[16], float (&d)[JN]) {
#pragma unroll
  for (int c = 0; c < kTcMaxChunks * 16; c += 16) {
    if (c < Np) {
      uint32_t u[16];
      tc::ld16(taddr + (uint32_t)c, u);
      tc::wait_ld();
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int col = c + i, o = col / JN, j = col - o * JN;
        if (o < 16 && o < O) d[j] = fmaf(w[o], __uint_as_float(u[i]), d[j]);
      }
    }
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

  // B tiles from the permuted core gp[((o_full * Jf + cf) * JN + j]: element (n, k) with
  // n = o * JN + j, k = s0 * jf8 + cf (s0 = 0 when na = 1), o_full = o (na = 1) or s0 + JA1 o
  for (int e = tid; e < tp.Np * tp.Kp; e += blockDim.x) {
    const int n = e / tp.Kp, k = e - n * tp.Kp;
    const int o = n / JN, j = n - o * JN;
    const int s0 = NA == 2 ? k / tp.jf8 : 0, cf = NA == 2 ? k - s0 * tp.jf8 : k;
    float v = 0.f;
    if (j < r.Jn && cf < r.Jf && o < tp.O && s0 < tp.JA1) {
      const int64_t of = NA == 2 ? (int64_t)s0 + (int64_t)tp.JA1 * o : (int64_t)o;
      v = gp[(of * r.Jf + cf) * JN + j];
    }
    uint32_t hi, lo;
    tc::split_tf32(v, hi, lo);
    const uint32_t wi = tc::kmajor_offset(n, k, tp.Kp) >> 2;
    sBhi[wi] = hi;
    sBlo[wi] = lo;
  }
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
  const uint32_t lane = (uint32_t)(32 * (warp & 3)) << 16;
  const uint32_t colAlo = (uint32_t)tp.Kp, colD = (uint32_t)tp.colD;
  const uint32_t idesc = tc::idesc_tf32(128, tp.Np);
  const uint32_t sbo = (uint32_t)tp.Kp * 32u;
  const uint32_t bhi_addr = tc::smem_u32(sBhi), blo_addr = tc::smem_u32(sBlo);
  const uint32_t ahi_addr = tc::smem_u32(sAhi), alo_addr = tc::smem_u32(sAlo);
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
      const float* ra0 = M.A[r.f] + (int64_t)csr.oidx[p] * r.Jf;
#pragma unroll
      for (int i = 0; i < 16; ++i) a0[e][i] = (valid && i < r.Jf) ? __ldg(ra0 + i) : 0.f;
      if constexpr (NA == 2) {
        const float* ra1 = M.A[r.slow[0]] + (int64_t)csr.oidx[nnz + p] * tp.JA1;
#pragma unroll
        for (int i = 0; i < 16; ++i) a1[e][i] = (valid && i < tp.JA1) ? __ldg(ra1 + i) : 0.f;
      }
      if (tp.has_rest) {
        const float* rr = M.A[r.slow[NA - 1]] + (int64_t)csr.oidx[(int64_t)NA * nnz + p] * tp.O;
#pragma unroll
        for (int i = 0; i < 16; ++i) wr[e][i] = (valid && i < tp.O) ? __ldg(rr + i) : 0.f;
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
      // A operand of this group's entry tid: hi and lo, in shared memory (na = 1, the row is
      // the entry, 16-byte pieces of four k) or in this lane's tensor-memory row (na = 2)
      if constexpr (NA == 1) {
#pragma unroll
        for (int c = 0; c < 16; c += 4) {
          if (c < tp.Kp) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) tc::split_tf32(a0[g][c + i], h[i], l[i]);
            const uint32_t wi = tc::kmajor_offset(tid, c, tp.Kp) >> 2;
            *reinterpret_cast<uint4*>(sAhi + wi) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4*>(sAlo + wi) = make_uint4(l[0], l[1], l[2], l[3]);
          }
        }
        tc::fence_async_smem();
      } else {
#pragma unroll
        for (int s0 = 0; s0 < 16; ++s0) {
          if (s0 < tp.JA1) {
            const float w0 = a1[g][s0];
#pragma unroll
            for (int c = 0; c < 16; c += 8) {
              if (c < tp.jf8) {
                uint32_t h[8], l[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) tc::split_tf32(a0[g][c + i] * w0, h[i], l[i]);
                const uint32_t col = (uint32_t)(s0 * tp.jf8 + c);
                tc::st8(tbase + lane + col, h);
                tc::st8(tbase + lane + colAlo + col, l);
              }
            }
          }
        }
        tc::wait_st();
      }
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
        for (int ks = 0; ks < tp.Kp / 8; ++ks) {
          const uint64_t bh = tc::smem_desc(bhi_addr + (uint32_t)ks * 256u, 128u, sbo);
          const uint64_t bl = tc::smem_desc(blo_addr + (uint32_t)ks * 256u, 128u, sbo);
          if constexpr (NA == 1) {
            const uint64_t ah = tc::smem_desc(ahi_addr + (uint32_t)ks * 256u, 128u, sbo);
            const uint64_t al = tc::smem_desc(alo_addr + (uint32_t)ks * 256u, 128u, sbo);
            tc::mma_tf32_ss(tbase + colD, ah, bh, idesc, ks > 0 ? 1u : 0u);
            tc::mma_tf32_ss(tbase + colD, ah, bl, idesc, 1u);
            tc::mma_tf32_ss(tbase + colD, al, bh, idesc, 1u);
          } else {
            tc::mma_tf32_ts(tbase + colD, tbase + ks * 8, bh, idesc, ks > 0 ? 1u : 0u);
            tc::mma_tf32_ts(tbase + colD, tbase + ks * 8, bl, idesc, 1u);
            tc::mma_tf32_ts(tbase + colD, tbase + colAlo + ks * 8, bh, idesc, 1u);
          }
        }
        tc::mma_commit(&mma_bar);
      }
      __syncwarp();
      const bool done = tc::mbar_wait_bounded(&mma_bar, phase, kTcWaitPolls);
      phase ^= 1u;
      if (__any_sync(0xffffffffu, !done) && (tid & 31) == 0) wait_failed = 1;  // checked after the task's V barrier
      tc::fence_after_sync();
      // stage 2: delta(j) = sum_o w(o) T[o * JN + j]
#pragma unroll
      for (int j = 0; j < JN; ++j) d[g][j] = 0.f;
      contract_rest<JN>(tbase + lane + colD, tp.Np, tp.O, wr[g], d[g]);
      tc::fence_before_sync();  // this group's accumulator reads before the next group's MMAs
    }
    // every MMA of the task has completed (each thread waited): V may take over the A region
#pragma unroll
    for (int g = 0; g < E; ++g) {
      const int q = tid + g * 128;
      if (q < cnt) {
        T* dst = ts.sV + q * L;
#pragma unroll
        for (int j = 0; j < JN; ++j) dst[j] = d[g][j];
        dst[JN] = xv[g];
        dst[JN + 1] = T(0);
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
// The tensor-core delta serves FP32 models whose other modes split into one or two A modes
// (ranks <= 16) and at most one remaining mode (rank <= 16), with 2 Kp + Np <= 256 TMEM
// columns.  Among the feasible splits the one with the least CUDA-core work per entry is
// taken: stage 2's O * JN FMAs plus the A split (and, with two A modes, their products).
// VEST_TENSOR_CORES=0 in the environment selects the FMA kernels everywhere.
static bool tensor_cores_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("VEST_TENSOR_CORES");
    return !(v && v[0] == '0');
  }();
  return on;
}

static bool tc_plan(const ModeRoles& r, int order, int JN, TcPlan* out) {
  int best = 1 << 30;
  bool found = false;
  for (int na = 1; na <= 2; ++na) {
    const int nother = order - 1;
    if (na > nother) break;
    const int nrest = nother - na;
    if (nrest > 1) continue;
    const int ja1 = na == 2 ? r.Js[0] : 1;
    const int jr = nrest ? r.Js[na - 1] : 1;
    if (r.Jf > 16 || ja1 > 16 || jr > 16) continue;
    TcPlan p{};
    p.na = na;
    p.jf8 = (r.Jf + 7) / 8 * 8;
    p.JA1 = ja1;
    p.Kp = p.jf8 * ja1;
    p.O = jr;
    p.has_rest = nrest;
    p.Np = (jr * JN + 15) / 16 * 16;
    if (p.Np > kTcMaxChunks * 16) continue;
    p.colD = na == 1 ? 0 : 2 * p.Kp;
    if (p.colD + p.Np > 256) continue;
    p.ncols = 32;
    while (p.ncols < p.colD + p.Np) p.ncols *= 2;
    p.per_sm = 512 / p.ncols;
    p.btile = (size_t)p.Np * p.Kp * 4;
    p.atile = na == 1 ? (size_t)128 * p.Kp * 4 : 0;
    p.ubytes = align_up(std::max(2 * p.atile, (size_t)kTask * (JN + 2) * 4), 128);
    const int cost = jr * JN + (na == 2 ? 3 : 2) * p.Kp;
    if (cost < best) {
      best = cost;
      *out = p;
      found = true;
    }
  }
  return found;
}

template <int JN, int MODE>
static vest_status launch_tc(const DevModel<float>& M, const DevMode<float>& csr, const float* gp, SweepArgs a,
                             const TcPlan& tp, cudaStream_t s) {
  a.kmax = std::min(a.kmax, 32);  // fewer row pieces per round: room for four CTAs per SM
  size_t smem = task_smem<float>(a.task, a.kmax, JN, a.P, MODE, 2 * tp.btile + tp.ubytes, false);
  // no more CTAs on an SM than its 512 TMEM columns hold, so no allocation ever waits
  const size_t sm_bytes = 228 * 1024, reserved = 1024;
  smem = std::max(smem, sm_bytes / (tp.per_sm + 1) - reserved + 16);
  if (smem > kSmemMax) return fail(VEST_ERR_UNSUPPORTED, "tensor-core factor sweep: shared memory exceeds 227 KB");
  auto kern = tp.na == 2 ? sweep_task_tc_kernel<JN, MODE, 2> : sweep_task_tc_kernel<JN, MODE, 1>;
  VEST_TRY(allow_smem(kern, smem));
  kern<<<(unsigned)ceil_div(a.ntasks, a.tpc), 128, smem, s>>>(M, csr, gp, a, tp);
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
                      tc_plan(r, M.N, JN, &tp);
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
  return tc_plan(r, m->order, jn_bucket(r.Jn), &tp);
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
