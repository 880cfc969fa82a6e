// Peak-rate probes of the GB300 units the hot path leans on, timed with CUDA events on the
// caller's stream: FP32 FMA and FP64 FMA issue rates (independent FMA chains in every lane
// of every SM), the tcgen05 TF32 MMA rate with A in tensor memory (M = 128, N = 256, K = 8,
// the operand placement of the factor sweep) and the L2 random-gather rate of 16-byte
// reads from a table that fits in L2.  The results are the denominators of the roofline
// fractions the benchmark reports.  Nothing here allocates: the gather table lives in the
// caller's buffer.
#include <cstdio>

#include "tcgen05.cuh"
#include "vest_internal.cuh"

namespace vest {

namespace {

constexpr int kChains = 8;

__device__ double g_probe_sink[4];

template <typename F>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, F seed) {
  F a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + (F)(threadIdx.x + c);
  const F b = (F)0.999999, d = (F)1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], b, d);
  }
  F s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == (F)-1.2345) g_probe_sink[0] = (double)s;  // never true; keeps the chains live
}

// One CTA per SM (its dynamic shared memory keeps a second one off) allocates all 512 TMEM
// columns, keeps A (128 x 8 TF32) in TMEM and B (256 x 8 TF32) in shared memory, and issues
// `count` MMAs of 128 x 256 x 8 into one accumulator, committed every 64 and waited on with a
// bounded number of polls.
__global__ void __launch_bounds__(128) mma_tf32_probe_kernel(int count, unsigned int* status) {
  __shared__ __align__(128) uint32_t sB[256 * 8];
  __shared__ uint64_t bar;
  __shared__ uint32_t slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < 256 * 8; i += blockDim.x) sB[i] = tc::to_tf32(1.0f / (float)(1 + (i & 7)));
  if (tid == 0) tc::mbar_init(&bar, 1);
  if (warp == 0) tc::tmem_alloc(&slot, 512);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = slot, lane = (uint32_t)(32 * (warp & 3)) << 16;
  uint32_t av[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) av[i] = tc::to_tf32(0.5f);
  tc::st8(tbase + lane, av);
  tc::wait_st();
  tc::fence_before_sync();
  __syncthreads();
  bool ok = true;
  if (tid == 0) {
    tc::fence_after_sync();
    const uint64_t bd = tc::smem_desc(tc::smem_u32(sB), 128u, 8u * 32u);
    const uint32_t idesc = tc::idesc_tf32(128, 256);
    uint32_t phase = 0;
    for (int i = 0; i < count && ok; ++i) {
      tc::mma_tf32_ts(tbase + 8, tbase, bd, idesc, i > 0 ? 1u : 0u);
      if ((i & 63) == 63 || i + 1 == count) {
        tc::mma_commit(&bar);
        ok = tc::mbar_wait_bounded(&bar, phase, 1u << 22);
        phase ^= 1u;
      }
    }
    if (!ok) atomicOr(status, 2u);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

__global__ void __launch_bounds__(256) gather_probe_kernel(const float4* __restrict__ table, uint32_t mask, int iters) {
  uint32_t h = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = 0; i < iters; ++i) {
    uint32_t idx[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      h ^= h << 13;
      h ^= h >> 17;
      h ^= h << 5;
      idx[u] = h & mask;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float4 v = __ldg(table + idx[u]);
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
  }
  if (acc.x + acc.y + acc.z + acc.w == -1.2345f) g_probe_sink[1] = acc.x;
}

}  // namespace

static __device__ unsigned int g_probe_status;

}  // namespace vest

using namespace vest;

extern "C" vest_status vest_probe_peak(int32_t kind, double* rate, void* buffer, size_t buffer_bytes, void* stream) {
  if (!rate) return fail(VEST_ERR_INVALID, "rate is NULL");
  const cudaStream_t s = as_stream(stream);
  const int sms = num_sms();
  cudaEvent_t e0, e1;
  VEST_CUDA(cudaEventCreate(&e0));
  VEST_CUDA(cudaEventCreate(&e1));
  double work = 0.0;
  unsigned int* status = nullptr;
  VEST_CUDA(cudaGetSymbolAddress((void**)&status, g_probe_status));
  for (int rep = 0; rep < 2; ++rep) {  // the first run warms clocks and caches up; the second is timed
    VEST_CUDA(cudaEventRecord(e0, s));
    if (kind == 0 || kind == 1) {
      const int blocks = sms * 8, threads = 256, iters = kind == 0 ? 4096 : 256;
      if (kind == 0) fma_probe_kernel<float><<<blocks, threads, 0, s>>>(iters, 1.0f);
      else fma_probe_kernel<double><<<blocks, threads, 0, s>>>(iters, 1.0);
      VEST_LAUNCH("fma_probe_kernel");
      work = 2.0 * kChains * 16.0 * iters * (double)blocks * threads;  // flops
    } else if (kind == 2) {
      const int count = 8192, blocks = sms;
      const int pad = 120 * 1024;  // more than half of an SM's shared memory: one CTA per SM
      VEST_TRY(allow_smem(mma_tf32_probe_kernel, pad));
      mma_tf32_probe_kernel<<<blocks, 128, pad, s>>>(count, status);
      VEST_LAUNCH("mma_tf32_probe_kernel");
      work = 2.0 * 128 * 256 * 8 * (double)count * blocks;  // flops
    } else if (kind == 3) {
      if (!buffer || buffer_bytes < (size_t(1) << 22))
        return fail(VEST_ERR_WORKSPACE, "gather probe needs a buffer of at least 4 MiB");
      size_t n = 1;
      while (n * 2 * sizeof(float4) <= buffer_bytes && n * 2 * sizeof(float4) <= (size_t(32) << 20)) n *= 2;
      const int blocks = sms * 8, threads = 256, iters = 1024;
      if (rep == 0) VEST_CUDA(cudaMemsetAsync(buffer, 0, n * sizeof(float4), s));
      gather_probe_kernel<<<blocks, threads, 0, s>>>(static_cast<const float4*>(buffer), (uint32_t)(n - 1), iters);
      VEST_LAUNCH("gather_probe_kernel");
      work = 16.0 * 8.0 * iters * (double)blocks * threads;  // bytes
    } else {
      return fail(VEST_ERR_INVALID, "probe kind must be 0 (FP32 FMA), 1 (FP64 FMA), 2 (TF32 MMA) or 3 (L2 gather)");
    }
    VEST_CUDA(cudaEventRecord(e1, s));
  }
  VEST_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  VEST_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  unsigned int st = 0;
  VEST_CUDA(cudaMemcpy(&st, status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st) return fail(VEST_ERR_TIMEOUT, "the TF32 MMA probe's bounded wait gave up");
  *rate = work / (ms * 1e-3) / 1e12;  // TFLOP/s or TB/s
  return VEST_OK;
}
