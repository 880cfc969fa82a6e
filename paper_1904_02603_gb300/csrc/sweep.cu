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

#include "delta.cuh"

namespace vest {

enum { kModeUpdate = 0, kModeResp = 1 };

struct SweepArgs {
  ModeRoles r;
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
  // shared layout: core | sptr | V | acc | long-piece partials | tile table
  T* sG = reinterpret_cast<T*>(smem_raw);
  size_t off = a.use_smem_core ? (size_t)core_elems * sizeof(T) : 0;
  off = (off + 15) & ~(size_t)15;
  int64_t* sptr = reinterpret_cast<int64_t*>(smem_raw + off);
  off += (size_t)(TASK + 2) * 8;
  off = (off + 15) & ~(size_t)15;
  T* sV = reinterpret_cast<T*>(smem_raw + off);
  off += (size_t)TASK * L * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  T* sAcc = reinterpret_cast<T*>(smem_raw + off);
  off += (size_t)KMAX * P * sizeof(T);
  T* sPart = reinterpret_cast<T*>(smem_raw + off);
  off += (size_t)long_chunks(TASK) * NT * 4 * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  int4* sOut = reinterpret_cast<int4*>(smem_raw + off);
  off += (size_t)NT * sizeof(int4);
  int2* sCab = reinterpret_cast<int2*>(smem_raw + off);
  off += (size_t)NT * sizeof(int2);
  off = (off + 15) & ~(size_t)15;
  T* sCarry = reinterpret_cast<T*>(smem_raw + off);  // [2][sum, compensation][P]: row sums carried to the next task
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

  // this block's consecutive tasks [tb, te) and the positions [rt0, rt1) they cover
  const int64_t tb = blockIdx.x * a.tpc, te = min(tb + a.tpc, a.ntasks);
  const int64_t rt0 = tb * TASK;
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

    for (int r0 = 0; r0 < nrows; r0 += KMAX) {
      const int nr = min(KMAX, nrows - r0);
      // phase 2: per-row sums over the task's pieces r0 .. r0 + nr - 1
      piece_sums<T, MODE == kModeResp>(sptr + r0, nr, t0, t1, NT, P, sCab, sOut, sV, L, JN, sAcc, sPart, &pscr);
      // phase 3: store the sums of rows that end here; carry a row that continues into
      // the block's next task; spill rows cut by the edges of the block's task range
      for (int kr = threadIdx.x; kr < nr; kr += blockDim.x) {
        const int k = r0 + kr;
        const int64_t rs = sptr[k], re = sptr[k + 1];
        const T* piece = sAcc + kr * P;
        const bool carried_in = (k == 0) && rs < t0 && task > tb;  // earlier pieces are in cin
        const bool continues = re > t1;
        const bool started_here = rs >= rt0;
        if (!continues && !carried_in && rs >= t0) {
          T* dst = a.rowbuf_t<T>() + (size_t)(k0 + k) * P;
          for (int i = 0; i < P; ++i) dst[i] = piece[i];
        } else {
          // running sums of a row cut by task edges: (sum, compensation) in T
          T* as = continues ? cout : cin;
          T* ac = as + P;
          for (int i = 0; i < P; ++i) {
            T sum = carried_in ? cin[i] : T(0), cmp = carried_in ? cin[P + i] : T(0);
            const T y = piece[i] - cmp;
            const T t = sum + y;
            ac[i] = (t - sum) - y;
            as[i] = t;
          }
          if (!continues) {
            if (started_here) {
              T* dst = a.rowbuf_t<T>() + (size_t)(k0 + k) * P;
              for (int i = 0; i < P; ++i) dst[i] = as[i] - ac[i];
            } else {  // the row entered the block's range from an earlier block: incoming partial
              double* sp = a.spill + ((size_t)blockIdx.x * 2 + 0) * P;
              for (int i = 0; i < P; ++i) sp[i] = (double)as[i] - (double)ac[i];
            }
          } else if (task + 1 == te) {  // leaves the block's range
            double* sp = a.spill + ((size_t)blockIdx.x * 2 + (started_here ? 1 : 0)) * P;
            for (int i = 0; i < P; ++i) sp[i] = (double)as[i] - (double)ac[i];
            a.spanning[blockIdx.x] = started_here ? (int32_t)(k0 + k) : -1;
          }
        }
        if (k == nrows - 1 && task + 1 == te && !(continues && started_here)) a.spanning[blockIdx.x] = -1;
      }
      __syncthreads();
    }
  }
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
static size_t task_smem(int task, int kmax, int JN, int P, int mode, size_t core_bytes) {
  const int NT = sweep_tiles(JN, mode);
  size_t off = (core_bytes + 15) & ~(size_t)15;
  off += (size_t)(task + 2) * 8;
  off = (off + 15) & ~(size_t)15;
  off += (size_t)task * (JN + 2) * sizeof(T);
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
  VEST_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
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
  VEST_TRY(dispatch_jn<T, MODE>(JN, r.nslow, r.Jf, M, csr, gp, a, smem, s));
  const size_t fsmem = (size_t)std::max(1, 256 / a.P) * a.P * 8 + 8 * a.P;
  auto fk = sweep_fixup_kernel<T, MODE>;
  VEST_CUDA(cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
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
                               char* scratch, const ScratchPlan& plan, cudaStream_t s) {
  const DevModel<T> M = dev_model<T>(m);
  SweepArgs a{};
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

template vest_status sweep_factors_mode<float>(const vest_index*, const vest_model*, int, double, int, char*,
                                               const ScratchPlan&, cudaStream_t);
template vest_status sweep_factors_mode<double>(const vest_index*, const vest_model*, int, double, int, char*,
                                                const ScratchPlan&, cudaStream_t);
template vest_status responsibility_factors<float>(const vest_index*, const vest_model*, const double*,
                                                   double* const*, double* const*, char*, const ScratchPlan&,
                                                   cudaStream_t);
template vest_status responsibility_factors<double>(const vest_index*, const vest_model*, const double*,
                                                    double* const*, double* const*, char*, const ScratchPlan&,
                                                    cudaStream_t);

}  // namespace vest
