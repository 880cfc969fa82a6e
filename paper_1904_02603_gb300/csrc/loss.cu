// Loss / RE (Eq. 1, Eq. 2, Eq. 4), entry-wise reconstruction (Eq. 7),
// column normalisation (the final step of Algorithm 2) and zero counts.
//
// B(alpha) = sum_j a0[i_0, j] delta^(0)_alpha(j): the mode-0 delta of Eq. 11
// dotted with the entry's mode-0 factor row, over the mode-0 CSR.  Products and
// delta run in the storage type; r^2 and X^2 are summed in FP64 per thread, then
// per thread block in a fixed shuffle tree, then across a fixed number of thread
// blocks in a fixed order, so the loss is bitwise reproducible.
#include <algorithm>

#include "tc_delta.cuh"

namespace vest {

constexpr int kLossTask = 256;
constexpr int kLossCtas = 760;  // fixed (sum order device-independent): one wave of 5 CTAs on 152 SMs
constexpr int kLossTcCtas = 608;  // the tensor-core loss: one wave of 4 CTAs on 152 SMs, fixed likewise
constexpr int kRegCtas = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// deterministic block sum; all threads must call; result valid in thread 0
__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) t += sh[w];
  __syncthreads();
  return t;
}

struct LossArgs {
  ModeRoles r;
  int64_t ntasks;
  const uint8_t* onz;
  int use_smem_core;
  double* part;  // [ctas][2]
};

// E entries per thread (threadIdx.x + e * blockDim.x of each 256-entry task).
template <typename T, int JN, int JF, int NSLOW, int E>
__global__ void __launch_bounds__(kLossTask / E, (delta_min_blocks<T, JN, JF, E>(kLossTask / E, JF > 0 ? 0 : 24))) loss_kernel(DevModel<T> M, DevMode<T> csr, const T* __restrict__ gcore,
                                                         LossArgs a, T* __restrict__ resid_csr0,
                                                         T* __restrict__ resid_coo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const ModeRoles& r = a.r;
  const int64_t core_elems = r.n_outer * r.Jf * JN;
  T* sG = reinterpret_cast<T*>(smem_raw);
  const T* g = gcore;
  if (a.use_smem_core) {
    for (int64_t e = threadIdx.x; e < core_elems; e += blockDim.x) sG[e] = gcore[e];
    g = sG;
  }
  const int64_t nnz = csr.nnz;
  const int J0 = M.J[0];
  // per-thread sums in the storage type with Kahan compensation, FP64 across threads
  T sq = T(0), sqc = T(0), xx = T(0), xxc = T(0);
  auto kadd = [](T& s, T& c, T v) {
    const T y = v - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  };
  __syncthreads();
  for (int64_t task = blockIdx.x; task < a.ntasks; task += gridDim.x) {
    const int64_t t0 = task * kLossTask, t1 = min(t0 + (int64_t)kLossTask, nnz);
    const int cnt = (int)(t1 - t0);
    if ((int)threadIdx.x < cnt) {
      const T* rowf[E];
      SlowRows sr[E];
      int64_t i0[E];  // mode-0 row of each entry, resolved before the contraction
      T xv[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int q = threadIdx.x + e * blockDim.x;
        const int64_t pe = t0 + (q < cnt ? q : (int)threadIdx.x);
        rowf[e] = gather_rows<T, NSLOW>(M, r, csr.oidx, nnz, pe, sr[e]);
        i0[e] = csr.nzrow[csr.rowk[pe]];
        xv[e] = csr.val[pe];
      }
      T d[E][JN];
      compute_delta_multi<T, JN, JF, NSLOW, E>(d, g, a.onz, r.n_outer, r.Jf, rowf, sr, r.nslow);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int q = threadIdx.x + e * blockDim.x;
        if (q >= cnt) continue;
        const int64_t p = t0 + q;
        const T* a0 = M.A[0] + i0[e] * J0;
        T b = T(0);
#pragma unroll
        for (int j = 0; j < JN; ++j)
          if (j < J0) b += __ldg(a0 + j) * d[e][j];
        const T x = xv[e];
        const T res = x - b;
        if (resid_csr0) resid_csr0[p] = res;
        if (resid_coo) resid_coo[csr.perm[p]] = res;
        kadd(sq, sqc, res * res);
        kadd(xx, xxc, x * x);
      }
    }
  }
  const double s1 = block_sum((double)sq - (double)sqc, red);
  const double s2 = block_sum((double)xx - (double)xxc, red);
  if (threadIdx.x == 0) {
    a.part[blockIdx.x * 2 + 0] = s1;
    a.part[blockIdx.x * 2 + 1] = s2;
  }
}

// The same loss with delta^(0) on the tensor cores (FP32 models the plan of tc_delta.cuh
// serves, mode-0 rank <= 16): per task of 256 mode-0 CSR positions two groups of 128 entries,
// each group's A rows written by their own lanes, the MMAs issued by one thread, delta read
// back from the accumulator and dotted with the entry's mode-0 row.  Sums as in loss_kernel.
// A wait that runs out marks the device status, abandons the CTA's entries and, after the
// in-flight MMAs get the same bounded wait, frees tensor memory.
static __device__ unsigned int g_loss_status;  // bit 1: an MMA completion wait gave up

template <int JN, int NA>
__global__ void __launch_bounds__(128, NA == 1 ? 4 : 2)
    loss_tc_kernel(DevModel<float> M, DevMode<float> csr, const float* __restrict__ gp, LossArgs a, TcPlan tp,
                   float* __restrict__ resid_csr0, float* __restrict__ resid_coo) {
  constexpr int E = 2;
  extern __shared__ __align__(128) unsigned char ltc_smem[];
  __shared__ uint64_t mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int wait_failed;
  __shared__ double red[32];
  const ModeRoles& r = a.r;
  const int tid = threadIdx.x, warp = tid >> 5;
  uint32_t* sBhi = reinterpret_cast<uint32_t*>(ltc_smem);
  uint32_t* sBlo = reinterpret_cast<uint32_t*>(ltc_smem + tp.btile);
  uint32_t* sAhi = reinterpret_cast<uint32_t*>(ltc_smem + 2 * tp.btile);
  uint32_t* sAlo = reinterpret_cast<uint32_t*>(ltc_smem + 2 * tp.btile + tp.atile);
  tc_fill_b<JN, NA>(sBhi, sBlo, gp, r, tp);
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
  const int J0 = M.J[0];
  float sq = 0.f, sqc = 0.f, xx = 0.f, xxc = 0.f;
  auto kadd = [](float& s, float& c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  };
  // gathers of both entries of the thread in task tk; the next task's are issued once the
  // current one's rows are used, so their latency overlaps the current task's MMAs and sums
  float a0[E][16], a1[E][NA == 2 ? 16 : 1], wr[E][16], am[E][16], xv[E];
  auto gather = [&](int64_t tk) {
    const int64_t g0 = tk * kLossTask;
    const int gcnt = (int)(min(g0 + (int64_t)kLossTask, nnz) - g0);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int q = tid + e * 128;
      const bool valid = q < gcnt;
      const int64_t p = g0 + (valid ? q : 0);
      tc_row(a0[e], tp, M.A[r.f], csr.oidx[p], r.Jf, valid);
      if constexpr (NA == 2) tc_row(a1[e], tp, M.A[r.slow[0]], csr.oidx[nnz + p], tp.JA1, valid);
      if (tp.has_rest) {
        tc_row(wr[e], tp, M.A[r.slow[NA - 1]], csr.oidx[(int64_t)NA * nnz + p], tp.O, valid);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) wr[e][i] = i == 0 ? 1.f : 0.f;
      }
      tc_row(am[e], tp, M.A[0], csr.nzrow[csr.rowk[p]], J0, valid);
      xv[e] = valid ? csr.val[p] : 0.f;
    }
  };
  if ((int64_t)blockIdx.x < a.ntasks) gather(blockIdx.x);
  for (int64_t task = blockIdx.x; task < a.ntasks && !wait_failed; task += gridDim.x) {
    const int64_t t0 = task * kLossTask;
    const int cnt = (int)(min(t0 + (int64_t)kLossTask, nnz) - t0);
    float res[E];
#pragma unroll
    for (int g = 0; g < E; ++g) {
      tcc.write_a(tid, a0[g], a1[g]);
      __syncthreads();
      if (tid == 0) tcc.issue(&mma_bar);
      __syncwarp();
      const bool done = tc::mbar_wait_bounded(&mma_bar, phase, kTcWaitPolls);
      phase ^= 1u;
      if (__any_sync(0xffffffffu, !done) && (tid & 31) == 0) wait_failed = 1;
      tc::fence_after_sync();
      float d[JN];
      tcc.template delta<JN>(tp.Np, tp.O, wr[g], d);
      tc::fence_before_sync();  // this group's accumulator reads before the next group's MMAs
      float b = 0.f;
#pragma unroll
      for (int j = 0; j < JN; ++j)
        if (j < 16) b += am[g][j] * d[j];
      res[g] = xv[g] - b;
    }
#pragma unroll
    for (int g = 0; g < E; ++g) {
      const int q = tid + g * 128;
      if (q < cnt) {
        const int64_t p = t0 + q;
        if (resid_csr0) resid_csr0[p] = res[g];
        if (resid_coo) resid_coo[csr.perm[p]] = res[g];
        kadd(sq, sqc, res[g] * res[g]);
        kadd(xx, xxc, xv[g] * xv[g]);
      }
    }
    if (task + gridDim.x < a.ntasks) gather(task + gridDim.x);
    __syncthreads();  // wait_failed is read uniformly by the loop condition
  }
  if (wait_failed) {
    if (tid == 0) atomicOr(&g_loss_status, 2u);
    tc::mbar_wait_bounded(&mma_bar, phase ^ 1u, kTcWaitPolls);
  }
  const double s1 = block_sum((double)sq - (double)sqc, red);
  const double s2 = block_sum((double)xx - (double)xxc, red);
  if (tid == 0) {
    a.part[blockIdx.x * 2 + 0] = s1;
    a.part[blockIdx.x * 2 + 1] = s2;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, (uint32_t)tp.ncols);
}

// regulariser partial sums over every factor and core element
template <typename T>
__global__ void reg_kernel(DevModel<T> M, int reg, double* __restrict__ part) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int seg = 0; seg <= M.N; ++seg) {
    const T* v = seg < M.N ? M.A[seg] : M.G;
    const int64_t size = seg < M.N ? M.I[seg] * M.J[seg] : M.gsize;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < size; e += (int64_t)gridDim.x * blockDim.x) {
      const double x = (double)v[e];
      acc += reg == VEST_REG_L1 ? fabs(x) : x * x;
    }
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void loss_final_kernel(const double* __restrict__ lpart, int nl, const double* __restrict__ rpart, int nr,
                                  double lambda, double* __restrict__ out) {
  __shared__ double red[32];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nl; i += blockDim.x) {
    a += lpart[2 * i];
    b += lpart[2 * i + 1];
  }
  for (int i = threadIdx.x; i < nr; i += blockDim.x) c += rpart[i];
  const double sq = block_sum(a, red);
  const double xx = block_sum(b, red);
  const double rg = block_sum(c, red);
  if (threadIdx.x == 0) {
    out[0] = sq;
    out[1] = xx;
    out[2] = lambda * rg;
    out[3] = sq + lambda * rg;
    out[4] = xx > 0.0 ? sqrt(sq) / sqrt(xx) : 0.0;
  }
}

constexpr size_t kLossSmemBudget = 160 * 1024;

template <typename T, int JN, int JF, int NSLOW, int E>
static vest_status launch_loss(const DevModel<T>& M, const DevMode<T>& csr, const T* gp, const LossArgs& a,
                               size_t smem, int grid, T* r0, T* rc, cudaStream_t s) {
  auto kern = loss_kernel<T, JN, JF, NSLOW, E>;
  VEST_TRY(allow_smem(kern, smem));
  kern<<<grid, kLossTask / E, smem, s>>>(M, csr, gp, a, r0, rc);
  VEST_LAUNCH("loss_kernel");
  return VEST_OK;
}

// FP32: two entries per thread, f-mode rows in registers when the rank equals the bucket width.
template <typename T, int JN>
static vest_status loss_nslow(int nslow, int Jf, const DevModel<T>& M, const DevMode<T>& csr, const T* gp,
                              const LossArgs& a, size_t smem, int grid, T* r0, T* rc, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (nslow == 1 && Jf == JN) return launch_loss<T, JN, JN, 1, 2>(M, csr, gp, a, smem, grid, r0, rc, s);
    if (nslow == 1) return launch_loss<T, JN, 0, 1, 2>(M, csr, gp, a, smem, grid, r0, rc, s);
    if (nslow == 2 && Jf == JN) return launch_loss<T, JN, JN, 2, 2>(M, csr, gp, a, smem, grid, r0, rc, s);
    if (nslow == 2) return launch_loss<T, JN, 0, 2, 2>(M, csr, gp, a, smem, grid, r0, rc, s);
  } else {
    if (nslow == 1) return launch_loss<T, JN, 0, 1, 1>(M, csr, gp, a, smem, grid, r0, rc, s);
    if (nslow == 2) return launch_loss<T, JN, 0, 2, 1>(M, csr, gp, a, smem, grid, r0, rc, s);
  }
  return launch_loss<T, JN, 0, -1, 1>(M, csr, gp, a, smem, grid, r0, rc, s);
}

template <int JN, int NA>
static vest_status launch_loss_tc_jn(const DevModel<float>& M, const DevMode<float>& csr, const float* gp,
                                     const LossArgs& a, const TcPlan& tp, int grid, float* r0, float* rc,
                                     cudaStream_t s) {
  TcPlan tpl = tp;
  tpl.base8 = 1;
  for (int k = 0; k < M.N; ++k)
    if (reinterpret_cast<uintptr_t>(M.A[k]) % 8 != 0) tpl.base8 = 0;
  size_t smem = 2 * tp.btile + tp.ubytes;
  // no more CTAs on an SM than its 512 TMEM columns hold, so no allocation ever waits
  smem = std::max(smem, (size_t)(228 * 1024) / (tp.per_sm + 1) - 1024 + 16);
  auto kern = loss_tc_kernel<JN, NA>;
  VEST_TRY(allow_smem(kern, smem));
  kern<<<grid, 128, smem, s>>>(M, csr, gp, a, tpl, r0, rc);
  VEST_LAUNCH("loss_tc_kernel");
  return VEST_OK;
}

template <typename T>
static vest_status launch_loss_tc(int JN, const DevModel<T>& M, const DevMode<T>& csr, const T* gp, const LossArgs& a,
                                  const TcPlan& tp, int grid, T* r0, T* rc, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    const bool two = tp.na == 2;
    switch (JN) {
      case 4: return two ? launch_loss_tc_jn<4, 2>(M, csr, gp, a, tp, grid, r0, rc, s)
                         : launch_loss_tc_jn<4, 1>(M, csr, gp, a, tp, grid, r0, rc, s);
      case 8: return two ? launch_loss_tc_jn<8, 2>(M, csr, gp, a, tp, grid, r0, rc, s)
                         : launch_loss_tc_jn<8, 1>(M, csr, gp, a, tp, grid, r0, rc, s);
      case 10: return two ? launch_loss_tc_jn<10, 2>(M, csr, gp, a, tp, grid, r0, rc, s)
                          : launch_loss_tc_jn<10, 1>(M, csr, gp, a, tp, grid, r0, rc, s);
      case 12: return two ? launch_loss_tc_jn<12, 2>(M, csr, gp, a, tp, grid, r0, rc, s)
                          : launch_loss_tc_jn<12, 1>(M, csr, gp, a, tp, grid, r0, rc, s);
      default: return two ? launch_loss_tc_jn<16, 2>(M, csr, gp, a, tp, grid, r0, rc, s)
                          : launch_loss_tc_jn<16, 1>(M, csr, gp, a, tp, grid, r0, rc, s);
    }
  }
  return fail(VEST_ERR_UNSUPPORTED, "tensor-core loss needs an FP32 model");
}

template <typename T>
vest_status loss_impl(const vest_index* ix, const vest_model* m, int reg, double lambda, double* out, T* resid_csr0,
                      T* resid_coo, char* scratch, const ScratchPlan& plan, cudaStream_t s) {
  const DevModel<T> M = dev_model<T>(m);
  const ModeRoles r = mode_roles(M.J, M.N, 0);
  const int JN = jn_bucket(r.Jn);
  const int64_t core_elems = r.n_outer * r.Jf * JN;
  T* gp = reinterpret_cast<T*>(scratch + plan.off_gperm);
  uint8_t* onz = reinterpret_cast<uint8_t*>(scratch + plan.off_gperm + align_up((size_t)core_elems * sizeof(T)));
  if (align_up((size_t)core_elems * sizeof(T)) + align_up((size_t)r.n_outer) > plan.gperm_bytes)
    return fail(VEST_ERR_WORKSPACE, "scratch region for the permuted core too small");
  prep_core_kernel<T><<<(unsigned)std::min<int64_t>(r.n_outer, 4096), 128, 0, s>>>(M.G, r, JN, gp, onz);
  VEST_LAUNCH("prep_core_kernel");
  LossArgs a{};
  a.r = r;
  a.onz = onz;
  a.ntasks = ceil_div(ix->nnz, kLossTask);
  const size_t core_bytes = align_up((size_t)core_elems * sizeof(T), 16);
  a.use_smem_core = core_bytes <= kLossSmemBudget;
  const size_t smem = a.use_smem_core ? core_bytes : 0;
  double* lpart = reinterpret_cast<double*>(scratch + plan.off_part);
  double* rpart = lpart + 2 * kLossCtas;
  a.part = lpart;
  int grid = (int)std::max<int64_t>(1, std::min<int64_t>(a.ntasks, kLossCtas));
  TcPlan tp{};
  if constexpr (sizeof(T) == 4) {
    if (ix->nnz > 0 && JN <= 16 && tensor_cores_enabled() && tc_plan(r, M.N, JN, 0, &tp)) {
      grid = (int)std::max<int64_t>(1, std::min<int64_t>(a.ntasks, kLossTcCtas));
      VEST_TRY(launch_loss_tc(JN, M, dev_mode<T>(ix, 0), gp, a, tp, grid, resid_csr0, resid_coo, s));
      reg_kernel<T><<<kRegCtas, 256, 0, s>>>(M, reg, rpart);
      VEST_LAUNCH("reg_kernel");
      loss_final_kernel<<<1, 256, 0, s>>>(lpart, grid, rpart, kRegCtas, lambda, out);
      VEST_LAUNCH("loss_final_kernel");
      return VEST_OK;
    }
  }
  if (ix->nnz > 0) {
    const DevMode<T> csr = dev_mode<T>(ix, 0);
    switch (JN) {
      case 4: VEST_TRY((loss_nslow<T, 4>(r.nslow, r.Jf, M, csr, gp, a, smem, grid, resid_csr0, resid_coo, s))); break;
      case 8: VEST_TRY((loss_nslow<T, 8>(r.nslow, r.Jf, M, csr, gp, a, smem, grid, resid_csr0, resid_coo, s))); break;
      case 10: VEST_TRY((loss_nslow<T, 10>(r.nslow, r.Jf, M, csr, gp, a, smem, grid, resid_csr0, resid_coo, s))); break;
      case 12: VEST_TRY((loss_nslow<T, 12>(r.nslow, r.Jf, M, csr, gp, a, smem, grid, resid_csr0, resid_coo, s))); break;
      case 16: VEST_TRY((loss_nslow<T, 16>(r.nslow, r.Jf, M, csr, gp, a, smem, grid, resid_csr0, resid_coo, s))); break;
      default: VEST_TRY((loss_nslow<T, 32>(r.nslow, r.Jf, M, csr, gp, a, smem, grid, resid_csr0, resid_coo, s))); break;
    }
  }
  reg_kernel<T><<<kRegCtas, 256, 0, s>>>(M, reg, rpart);
  VEST_LAUNCH("reg_kernel");
  loss_final_kernel<<<1, 256, 0, s>>>(lpart, ix->nnz > 0 ? grid : 0, rpart, kRegCtas, lambda, out);
  VEST_LAUNCH("loss_final_kernel");
  return VEST_OK;
}

size_t loss_part_bytes() { return (size_t)(2 * kLossCtas + kRegCtas) * 8; }

// Bits set by the tensor-core loss kernel since the last clear (bit 1: a bounded wait gave up).
vest_status loss_device_status(uint32_t* flags, bool clear) {
  unsigned int v = 0;
  VEST_CUDA(cudaMemcpyFromSymbol(&v, g_loss_status, sizeof(v)));
  if (clear && v) {
    const unsigned int z = 0;
    VEST_CUDA(cudaMemcpyToSymbol(g_loss_status, &z, sizeof(z)));
  }
  *flags = v;
  return VEST_OK;
}

// Loss from per-CTA (sum r^2, sum x^2) partials already in the loss region (nl of them,
// at most kLossCtas): adds the regulariser and writes the five loss values.
template <typename T>
vest_status loss_finish(const vest_model* m, int reg, double lambda, int nl, double* out, char* scratch,
                        const ScratchPlan& plan, cudaStream_t s) {
  const DevModel<T> M = dev_model<T>(m);
  double* lpart = reinterpret_cast<double*>(scratch + plan.off_part);
  double* rpart = lpart + 2 * kLossCtas;
  reg_kernel<T><<<kRegCtas, 256, 0, s>>>(M, reg, rpart);
  VEST_LAUNCH("reg_kernel");
  loss_final_kernel<<<1, 256, 0, s>>>(lpart, nl, rpart, kRegCtas, lambda, out);
  VEST_LAUNCH("loss_final_kernel");
  return VEST_OK;
}

int loss_ctas() { return kLossCtas; }

template vest_status loss_finish<float>(const vest_model*, int, double, int, double*, char*, const ScratchPlan&,
                                        cudaStream_t);
template vest_status loss_finish<double>(const vest_model*, int, double, int, double*, char*, const ScratchPlan&,
                                         cudaStream_t);

template vest_status loss_impl<float>(const vest_index*, const vest_model*, int, double, double*, float*, float*, char*,
                                      const ScratchPlan&, cudaStream_t);
template vest_status loss_impl<double>(const vest_index*, const vest_model*, int, double, double*, double*, double*,
                                       char*, const ScratchPlan&, cudaStream_t);

// ------------------------------------------------------------------ completion queries (Eq. 7)
template <typename T>
__global__ void reconstruct_kernel(DevModel<T> M, const int32_t* __restrict__ q, int64_t count, T* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    bool in_range = true;  // a tuple outside the tensor reads nothing and gives NaN
    for (int n = 0; n < M.N; ++n) {
      const int32_t v = q[(int64_t)n * count + i];
      in_range = in_range && v >= 0 && (int64_t)v < M.I[n];
    }
    if (!in_range) {
      out[i] = T(NAN);
      continue;
    }
    // B = sum over core elements, staged: fold the slowest mode first
    T acc = T(0);
    int64_t lin = 0;
    const int64_t gs = M.gsize;
    int dig[kMaxOrder];
    for (int n = 0; n < M.N; ++n) dig[n] = 0;
    for (lin = 0; lin < gs; ++lin) {
      T p = M.G[lin];
      if (p != T(0)) {
        for (int n = 0; n < M.N; ++n) p *= M.A[n][(int64_t)q[(int64_t)n * count + i] * M.J[n] + dig[n]];
        acc += p;
      }
      for (int n = 0; n < M.N; ++n) {
        if (++dig[n] < M.J[n]) break;
        dig[n] = 0;
      }
    }
    out[i] = acc;
  }
}

template <typename T>
vest_status reconstruct_impl(const vest_model* m, const int32_t* q_idx, int64_t count, T* out, cudaStream_t s) {
  if (count <= 0) return VEST_OK;
  const DevModel<T> M = dev_model<T>(m);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(count, 256), (int64_t)num_sms() * 8));
  reconstruct_kernel<T><<<grid, 256, 0, s>>>(M, q_idx, count, out);
  VEST_LAUNCH("reconstruct_kernel");
  return VEST_OK;
}
template vest_status reconstruct_impl<float>(const vest_model*, const int32_t*, int64_t, float*, cudaStream_t);
template vest_status reconstruct_impl<double>(const vest_model*, const int32_t*, int64_t, double*, cudaStream_t);

// ------------------------------------------------------------------ normalisation
constexpr int kNormCtas = 128;

template <typename T>
__global__ void colnorm_partial_kernel(const T* __restrict__ A, int64_t I, int J, double* __restrict__ part) {
  __shared__ double sh[256];
  const int per = blockDim.x / J;  // threads per column group
  const int j = threadIdx.x % J, rl = threadIdx.x / J;
  double acc = 0.0;
  if (rl < per) {
    const int64_t rows_per_cta = ceil_div(I, (int64_t)gridDim.x);
    const int64_t r0 = blockIdx.x * rows_per_cta, r1 = min(I, r0 + rows_per_cta);
    for (int64_t i = r0 + rl; i < r1; i += per) {
      const double x = (double)A[i * J + j];
      acc += x * x;
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < J) {
    double t = 0.0;
    for (int q = 0; q < per; ++q) t += sh[q * J + threadIdx.x];
    part[blockIdx.x * J + threadIdx.x] = t;
  }
}

__global__ void colnorm_final_kernel(const double* __restrict__ part, int nctas, int J, double* __restrict__ b) {
  const int j = threadIdx.x;
  if (j < J) {
    double t = 0.0;
    for (int c = 0; c < nctas; ++c) t += part[c * J + j];
    b[j] = sqrt(t);
  }
}

template <typename T>
__global__ void scale_columns_kernel(T* __restrict__ A, int64_t I, int J, const double* __restrict__ b) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < I * J; e += (int64_t)gridDim.x * blockDim.x) {
    const double bj = b[e % J];
    if (bj > 0.0) A[e] = (T)((double)A[e] / bj);
  }
}

template <typename T>
__global__ void scale_core_kernel(DevModel<T> M, const double* __restrict__ b /* [N][32] */) {
  for (int64_t lin = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; lin < M.gsize; lin += (int64_t)gridDim.x * blockDim.x) {
    double g = (double)M.G[lin];
    int64_t rem = lin;
    for (int n = 0; n < M.N; ++n) {
      const int jn = (int)(rem % M.J[n]);
      rem /= M.J[n];
      g = (double)(T)(g * b[n * kMaxRank + jn]);
    }
    M.G[lin] = (T)g;
  }
}

template <typename T>
vest_status normalize_impl(const vest_model* m, char* scratch, cudaStream_t s) {
  const DevModel<T> M = dev_model<T>(m);
  double* part = reinterpret_cast<double*>(scratch);
  double* b = part + (size_t)kNormCtas * kMaxRank;
  for (int n = 0; n < M.N; ++n) {
    const int J = M.J[n];
    const int threads = std::max(J, 256 / J * J);
    colnorm_partial_kernel<T><<<kNormCtas, threads, 0, s>>>(M.A[n], M.I[n], J, part);
    VEST_LAUNCH("colnorm_partial");
    colnorm_final_kernel<<<1, 32, 0, s>>>(part, kNormCtas, J, b + n * kMaxRank);
    VEST_LAUNCH("colnorm_final");
    const int grid = std::max(1, std::min<int>((int)ceil_div(M.I[n] * J, 256), num_sms() * 8));
    scale_columns_kernel<T><<<grid, 256, 0, s>>>(M.A[n], M.I[n], J, b + n * kMaxRank);
    VEST_LAUNCH("scale_columns");
  }
  const int grid = std::max(1, std::min<int>((int)ceil_div(M.gsize, 256), num_sms() * 8));
  scale_core_kernel<T><<<grid, 256, 0, s>>>(M, b);
  VEST_LAUNCH("scale_core");
  return VEST_OK;
}
template vest_status normalize_impl<float>(const vest_model*, char*, cudaStream_t);
template vest_status normalize_impl<double>(const vest_model*, char*, cudaStream_t);

size_t normalize_scratch_bytes() { return (size_t)(kNormCtas + kMaxOrder) * kMaxRank * 8; }

// ------------------------------------------------------------------ zero counts
template <typename T>
__global__ void count_zeros_kernel(DevModel<T> M, unsigned long long* __restrict__ out) {
  for (int seg = 0; seg <= M.N; ++seg) {
    const T* v = seg < M.N ? M.A[seg] : M.G;
    const int64_t size = seg < M.N ? M.I[seg] * M.J[seg] : M.gsize;
    unsigned long long c = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < size; e += (int64_t)gridDim.x * blockDim.x)
      c += (v[e] == T(0));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out + seg, c);
  }
}

template <typename T>
vest_status count_zeros_impl(const vest_model* m, int64_t* out, char* scratch, cudaStream_t s) {
  (void)scratch;
  const DevModel<T> M = dev_model<T>(m);
  VEST_CUDA(cudaMemsetAsync(out, 0, (size_t)(M.N + 1) * 8, s));
  count_zeros_kernel<T><<<num_sms() * 2, 256, 0, s>>>(M, reinterpret_cast<unsigned long long*>(out));
  VEST_LAUNCH("count_zeros");
  return VEST_OK;
}
template vest_status count_zeros_impl<float>(const vest_model*, int64_t*, char*, cudaStream_t);
template vest_status count_zeros_impl<double>(const vest_model*, int64_t*, char*, cudaStream_t);

}  // namespace vest
