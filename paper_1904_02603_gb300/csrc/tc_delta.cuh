// delta_alpha (Eq. 11) on the tensor cores for FP32 models, shared by the factor sweep
// (sweep.cu) and the loss (loss.cu).
//
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
// A mode, A is written to shared memory by the lane of its entry and the MMA reads both
// operands there, so the allocation is the accumulator alone: 128 columns for the Zipf
// workload, four CTAs per SM.  With two A modes the wider A goes to tensor memory.  One
// thread issues the MMAs and commits them to an mbarrier that every thread waits on with a
// bounded number of polls.
#pragma once

#include <algorithm>
#include <cstdlib>

#include "delta.cuh"
#include "tcgen05.cuh"

namespace vest {

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
  size_t ubytes; // shared region of A hi and lo, shared with whatever the caller stages after the
                 // MMAs: max(2 atile, the caller's bytes), 128-aligned
  int base8;     // every factor array starts 8-byte aligned (rows of even length are read 8 bytes at a time)
};

// A factor row of `len` <= 16 elements into registers, zero beyond it.  With an 8-byte aligned
// factor base (base8) and an even length every row is 8-byte aligned and is read in 8-byte
// pieces: half the load instructions and L1 wavefronts of a gather across 32 rows.
__device__ __forceinline__ void load_row16(float (&v)[16], const float* __restrict__ row, int len, bool base8) {
  if (base8 && (len & 1) == 0) {
    const float2* r2 = reinterpret_cast<const float2*>(row);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 x = 2 * i < len ? __ldg(r2 + i) : make_float2(0.f, 0.f);
      v[2 * i] = x.x;
      v[2 * i + 1] = x.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = i < len ? __ldg(row + i) : 0.f;
  }
}

// Row `idx` of a factor with rank J for the tensor-core kernels (zero when the entry is not valid).
__device__ __forceinline__ void tc_row(float (&v)[16], const TcPlan& tp, const float* A, int64_t idx, int J,
                                       bool valid) {
  load_row16(v, A + idx * J, valid ? J : 0, tp.base8);
}

constexpr uint32_t kTcWaitPolls = 1u << 22;  // bounded mbarrier wait (seconds at worst, never in practice)
constexpr int kTcMaxChunks = 14;             // accumulator columns read in 16-column chunks: Np <= 224

// VEST_TENSOR_CORES=0 in the environment turns the automatic choice to the FMA kernels.
inline bool tensor_cores_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("VEST_TENSOR_CORES");
    return !(v && v[0] == '0');
  }();
  return on;
}

// The tensor-core delta serves FP32 models whose other modes split into one or two A modes
// (ranks <= 16) and at most one remaining mode (rank <= 16), within the 256 TMEM columns of
// one CTA.  Among the feasible splits the one with the least CUDA-core work per entry is
// taken: stage 2's O * JN FMAs plus the A split (and, with two A modes, their products).
// `after_bytes`: what the caller keeps in the A region once the MMAs are done.
inline bool tc_plan(const ModeRoles& r, int order, int JN, size_t after_bytes, TcPlan* out) {
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
    p.ubytes = align_up(std::max(2 * p.atile, after_bytes), 128);
    const int cost = jr * JN + (na == 2 ? 3 : 2) * p.Kp;
    if (cost < best) {
      best = cost;
      *out = p;
      found = true;
    }
  }
  return found;
}

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

// B tiles (hi and lo) from the permuted core gp[((o_full * Jf + cf) * JN + j]: element (n, k)
// with n = o * JN + j, k = s0 * jf8 + cf (s0 = 0 when na = 1), o_full = o (na = 1) or
// s0 + JA1 o; zero outside the model's ranks.  All threads of the CTA take part.
template <int JN, int NA>
__device__ __forceinline__ void tc_fill_b(uint32_t* sBhi, uint32_t* sBlo, const float* __restrict__ gp,
                                          const ModeRoles& r, const TcPlan& tp) {
  for (int e = threadIdx.x; e < tp.Np * tp.Kp; e += blockDim.x) {
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
}

// Per-CTA state of the tensor-core delta and its two steps on a group of 128 entries: each
// thread writes its entry's A row (write_a), then one thread issues the MMAs (issue).
template <int NA>
struct TcCta {
  uint32_t tbase;   // TMEM allocation
  uint32_t lane;    // this warp's TMEM lane quadrant, << 16
  uint32_t colAlo;  // A lo columns (na = 2)
  uint32_t colD;    // accumulator columns
  uint32_t idesc, sbo;
  uint32_t bhi, blo, ahi, alo;  // shared addresses of the operand tiles
  uint32_t* sAhi;
  uint32_t* sAlo;
  int Kp, jf8, JA1;

  __device__ void init(uint32_t tmem, const TcPlan& tp, uint32_t* Bhi, uint32_t* Blo, uint32_t* Ahi, uint32_t* Alo) {
    tbase = tmem;
    lane = (uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16;
    colAlo = (uint32_t)tp.Kp;
    colD = (uint32_t)tp.colD;
    idesc = tc::idesc_tf32(128, tp.Np);
    sbo = (uint32_t)tp.Kp * 32u;
    bhi = tc::smem_u32(Bhi);
    blo = tc::smem_u32(Blo);
    ahi = tc::smem_u32(Ahi);
    alo = tc::smem_u32(Alo);
    sAhi = Ahi;
    sAlo = Alo;
    Kp = tp.Kp;
    jf8 = tp.jf8;
    JA1 = tp.JA1;
  }

  // A operand of accumulator row `row` (the calling thread's entry): hi and lo, in shared
  // memory (na = 1, 16-byte pieces of four k) or in this lane's tensor-memory row (na = 2).
  // Ends with the fence the MMA's reads need; the caller then synchronises the CTA.
  __device__ void write_a(int row, const float (&a0)[16], const float (&a1)[NA == 2 ? 16 : 1]) const {
    if constexpr (NA == 1) {
#pragma unroll
      for (int c = 0; c < 16; c += 4) {
        if (c < Kp) {
          uint32_t h[4], l[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) tc::split_tf32(a0[c + i], h[i], l[i]);
          const uint32_t wi = tc::kmajor_offset(row, c, Kp) >> 2;
          *reinterpret_cast<uint4*>(sAhi + wi) = make_uint4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<uint4*>(sAlo + wi) = make_uint4(l[0], l[1], l[2], l[3]);
        }
      }
      tc::fence_async_smem();
    } else {
#pragma unroll
      for (int s0 = 0; s0 < 16; ++s0) {
        if (s0 < JA1) {
          const float w0 = a1[s0];
#pragma unroll
          for (int c = 0; c < 16; c += 8) {
            if (c < jf8) {
              uint32_t h[8], l[8];
#pragma unroll
              for (int i = 0; i < 8; ++i) tc::split_tf32(a0[c + i] * w0, h[i], l[i]);
              const uint32_t col = (uint32_t)(s0 * jf8 + c);
              tc::st8(tbase + lane + col, h);
              tc::st8(tbase + lane + colAlo + col, l);
            }
          }
        }
      }
      tc::wait_st();
    }
    tc::fence_before_sync();
  }

  // One thread, after the CTA barrier that follows write_a: the split-TF32 products over the
  // K steps into the accumulator, committed to `bar`.
  __device__ void issue(uint64_t* bar) const {
    tc::fence_after_sync();
    for (int ks = 0; ks < Kp / 8; ++ks) {
      const uint64_t bh = tc::smem_desc(bhi + (uint32_t)ks * 256u, 128u, sbo);
      const uint64_t bl = tc::smem_desc(blo + (uint32_t)ks * 256u, 128u, sbo);
      if constexpr (NA == 1) {
        const uint64_t ah = tc::smem_desc(ahi + (uint32_t)ks * 256u, 128u, sbo);
        const uint64_t al = tc::smem_desc(alo + (uint32_t)ks * 256u, 128u, sbo);
        tc::mma_tf32_ss(tbase + colD, ah, bh, idesc, ks > 0 ? 1u : 0u);
        tc::mma_tf32_ss(tbase + colD, ah, bl, idesc, 1u);
        tc::mma_tf32_ss(tbase + colD, al, bh, idesc, 1u);
      } else {
        tc::mma_tf32_ts(tbase + colD, tbase + ks * 8, bh, idesc, ks > 0 ? 1u : 0u);
        tc::mma_tf32_ts(tbase + colD, tbase + ks * 8, bl, idesc, 1u);
        tc::mma_tf32_ts(tbase + colD, tbase + colAlo + ks * 8, bh, idesc, 1u);
      }
    }
    tc::mma_commit(bar);
  }

  // The accumulator row of this lane's entry: delta(j) = sum_o w(o) T[o * JN + j].
  template <int JN>
  __device__ void delta(int Np, int O, const float (&w)[16], float (&d)[JN]) const {
#pragma unroll
    for (int j = 0; j < JN; ++j) d[j] = 0.f;
    contract_rest<JN>(tbase + lane + colD, Np, O, w, d);
  }
};

}  // namespace vest
