// delta_alpha^(n) (Eq. 11) on the GPU: the core permuted for mode n into a
// [outer][j_f][JN] layout (j_n contiguous, padded to the bucket width JN with
// zeros), then one staged contraction per observed entry with the other
// modes' factor rows.  "f" is the lowest-numbered mode other than n; the
// remaining other modes ("slow" modes) are folded into one weight per outer
// index.  Outer slices whose core fibres are all zero are skipped uniformly.
#pragma once

#include "vest_internal.cuh"

namespace vest {

// Mode roles for a sweep of mode n.
struct ModeRoles {
  int n, f;                  // updated mode, fastest other mode (-1 if order 1)
  int nslow;                 // number of slow modes
  int slow[kMaxOrder];       // slow modes, fastest first
  int Jn, Jf;
  int Js[kMaxOrder];         // ranks of the slow modes
  int64_t n_outer;           // prod of slow ranks
  int64_t stride[kMaxOrder]; // core linear strides of every mode
};

inline ModeRoles mode_roles(const int32_t* J, int N, int n) {
  ModeRoles r{};
  r.n = n;
  r.Jn = J[n];
  int64_t s = 1;
  for (int k = 0; k < N; ++k) {
    r.stride[k] = s;
    s *= J[k];
  }
  int q = 0;
  r.f = -1;
  for (int k = 0; k < N; ++k) {
    if (k == n) continue;
    if (r.f < 0) {
      r.f = k;
      r.Jf = J[k];
    } else {
      r.slow[q] = k;
      r.Js[q] = J[k];
      ++q;
    }
  }
  r.nslow = q;
  r.n_outer = 1;
  for (int i = 0; i < q; ++i) r.n_outer *= r.Js[i];
  return r;
}

// JN bucket widths instantiated by the kernels.
inline int jn_bucket(int J) {
  if (J <= 4) return 4;
  if (J <= 8) return 8;
  if (J <= 10) return 10;
  if (J <= 12) return 12;
  if (J <= 16) return 16;
  return 32;
}

// Permuted, padded core for mode n: gp[(o * Jf + cf) * JN + j] = G[lin(j_n=j, j_f=cf, slow digits of o)],
// zero for j >= Jn; onz[o] = 1 iff the outer slice o holds a nonzero.
template <typename T>
__global__ void prep_core_kernel(const T* __restrict__ G, ModeRoles r, int JN, T* __restrict__ gp,
                                 uint8_t* __restrict__ onz) {
  const int64_t slice = (int64_t)r.Jf * JN;
  for (int64_t o = blockIdx.x; o < r.n_outer; o += gridDim.x) {
    int64_t base = 0, rem = o;
    for (int i = 0; i < r.nslow; ++i) {
      base += (rem % r.Js[i]) * r.stride[r.slow[i]];
      rem /= r.Js[i];
    }
    int any = 0;
    for (int64_t e = threadIdx.x; e < slice; e += blockDim.x) {
      const int cf = (int)(e / JN), j = (int)(e % JN);
      T v = T(0);
      if (j < r.Jn) v = G[base + (int64_t)cf * r.stride[r.f] + (int64_t)j * r.stride[r.n]];
      gp[o * slice + e] = v;
      any |= (v != T(0));
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) onz[o] = (uint8_t)any;
  }
}

// Slow-mode row pointers and ranks for one entry.
struct SlowRows {
  const void* row[kMaxOrder];
  int J[kMaxOrder];
};

// ---------------------------------------------------------------- delta for E entries at once
// The core fibre of each (o, j_f) is read from shared memory once and feeds all
// E entries of the thread.  JF > 0: the rank of mode f is JF at compile time and
// the E rows of mode f sit in registers.
template <typename T, int JN>
__device__ __forceinline__ void load_fibre(T (&v)[JN], const T* __restrict__ g) {
  if constexpr (sizeof(T) == 4 && JN % 4 == 0) {
#pragma unroll
    for (int j = 0; j < JN; j += 4) {
      const float4 x = *reinterpret_cast<const float4*>(g + j);
      v[j] = x.x;
      v[j + 1] = x.y;
      v[j + 2] = x.z;
      v[j + 3] = x.w;
    }
  } else if constexpr (sizeof(T) == 4 && JN % 2 == 0) {
#pragma unroll
    for (int j = 0; j < JN; j += 2) {
      const float2 x = *reinterpret_cast<const float2*>(g + j);
      v[j] = x.x;
      v[j + 1] = x.y;
    }
  } else if constexpr (sizeof(T) == 8 && JN % 2 == 0) {
#pragma unroll
    for (int j = 0; j < JN; j += 2) {
      const double2 x = *reinterpret_cast<const double2*>(g + j);
      v[j] = x.x;
      v[j + 1] = x.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < JN; ++j) v[j] = g[j];
  }
}

// Minimum resident blocks per SM for the __launch_bounds__ of kernels that run the
// contraction below with `threads` threads per block.  Without it ptxas keeps these kernels
// at 64 registers and spills the per-entry fibre weights inside the contraction loop.  The
// estimate counts the live registers of the loop (accumulators, fibre weights, one core
// fibre, ~48 for addressing and loop state, `extra` for the caller's own live values) and asks for as many blocks as that allows.
template <typename T, int JN, int JF, int E>
constexpr int delta_min_blocks(int threads, int extra = 0) {
  const int w = (int)sizeof(T) / 4;
  const int need = E * JN * w + E * JF * w + JN * w + 48 + extra;
  const int b = 65536 / (threads * need);
  return b < 1 ? 1 : (b > 8 ? 8 : b);
}

template <typename T, int JN, int JF, int E>
__device__ __forceinline__ void delta_slice(T (&d)[E][JN], const T (&w)[E], const T* __restrict__ go, int Jf,
                                            const T* const (&rowf)[E], const T (&rf)[E][JF > 0 ? JF : 1]) {
  if constexpr (JF > 0) {
#pragma unroll
    for (int cf = 0; cf < JF; ++cf) {
      T gv[JN];
      load_fibre<T, JN>(gv, go + cf * JN);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const T wf = w[e] * rf[e][cf];
#pragma unroll
        for (int j = 0; j < JN; ++j) d[e][j] = fma(wf, gv[j], d[e][j]);
      }
    }
  } else {
    for (int cf = 0; cf < Jf; ++cf) {
      T gv[JN];
      load_fibre<T, JN>(gv, go + cf * JN);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const T wf = w[e] * __ldg(rowf[e] + cf);
#pragma unroll
        for (int j = 0; j < JN; ++j) d[e][j] = fma(wf, gv[j], d[e][j]);
      }
    }
  }
}

template <typename T, int JN, int JF, int NSLOW, int E>
__device__ __forceinline__ void compute_delta_multi(T (&d)[E][JN], const T* __restrict__ g,
                                                    const uint8_t* __restrict__ onz, int64_t n_outer, int Jf,
                                                    const T* const (&rowf)[E], const SlowRows (&sr)[E], int nslow) {
#pragma unroll
  for (int e = 0; e < E; ++e)
#pragma unroll
    for (int j = 0; j < JN; ++j) d[e][j] = T(0);
  T rf[E][JF > 0 ? JF : 1];
  if constexpr (JF > 0) {
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int cf = 0; cf < JF; ++cf) rf[e][cf] = __ldg(rowf[e] + cf);
  }
  const int64_t slice = (int64_t)Jf * JN;
  T w[E];
  if constexpr (NSLOW == 0) {
#pragma unroll
    for (int e = 0; e < E; ++e) w[e] = T(1);
    delta_slice<T, JN, JF, E>(d, w, g, Jf, rowf, rf);
  } else if constexpr (NSLOW == 1) {
    for (int o = 0; o < (int)n_outer; ++o) {
      if (!onz[o]) continue;
      bool any = false;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        w[e] = __ldg(static_cast<const T*>(sr[e].row[0]) + o);
        any |= (w[e] != T(0));
      }
      if (!any) continue;
      delta_slice<T, JN, JF, E>(d, w, g + o * slice, Jf, rowf, rf);
    }
  } else if constexpr (NSLOW == 2) {
    const int J0 = sr[0].J[0], J1 = sr[0].J[1];
    for (int d1 = 0; d1 < J1; ++d1) {
      T w1[E];
      bool any1 = false;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        w1[e] = __ldg(static_cast<const T*>(sr[e].row[1]) + d1);
        any1 |= (w1[e] != T(0));
      }
      if (!any1) continue;
      for (int d0 = 0; d0 < J0; ++d0) {
        const int o = d0 + J0 * d1;
        if (!onz[o]) continue;
        bool any = false;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          w[e] = w1[e] * __ldg(static_cast<const T*>(sr[e].row[0]) + d0);
          any |= (w[e] != T(0));
        }
        if (!any) continue;
        delta_slice<T, JN, JF, E>(d, w, g + o * slice, Jf, rowf, rf);
      }
    }
  } else {
    int dig[kMaxOrder];
    for (int i = 0; i < nslow; ++i) dig[i] = 0;
    for (int64_t o = 0; o < n_outer; ++o) {
      if (onz[o]) {
        bool any = false;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          T x = T(1);
          for (int i = 0; i < nslow; ++i) x *= __ldg(static_cast<const T*>(sr[e].row[i]) + dig[i]);
          w[e] = x;
          any |= (x != T(0));
        }
        if (any) delta_slice<T, JN, JF, E>(d, w, g + o * slice, Jf, rowf, rf);
      }
      for (int i = 0; i < nslow; ++i) {  // odometer, slow[0] fastest
        if (++dig[i] < sr[0].J[i]) break;
        dig[i] = 0;
      }
    }
  }
}

// Row pointers of the other modes for the entry at CSR position p of mode n.
// oidx rows are the other modes in ascending order: f first, then the slow ones.
// NSLOW >= 0: the number of slow modes is a compile-time constant (keeps SlowRows in registers).
template <typename T, int NSLOW = -1>
__device__ __forceinline__ const T* gather_rows(const DevModel<T>& M, const ModeRoles& r, const int32_t* __restrict__ oidx,
                                                int64_t nnz, int64_t p, SlowRows& sr) {
  const int64_t i_f = oidx[p];
  const int ns = NSLOW >= 0 ? NSLOW : r.nslow;
#pragma unroll
  for (int i = 0; i < (NSLOW >= 0 ? NSLOW : kMaxOrder); ++i) {
    if (i >= ns) break;
    const int k = r.slow[i];
    const int64_t ik = oidx[(int64_t)(i + 1) * nnz + p];
    sr.row[i] = M.A[k] + ik * M.J[k];
    sr.J[i] = M.J[k];
  }
  return M.A[r.f] + i_f * M.J[r.f];
}

// ---------------------------------------------------------------- task -> rows
// A task is a contiguous range [t0, t1) of positions in a mode's CSR order,
// t0 a multiple of 32.  Loads nzptr[k0 .. k1+1] into sptr and returns the number
// of rows overlapping the task: k0 from the granule table, k1 from the granule of
// t1 - 1 plus one warp-wide probe of the (at most 31) row starts after it.
__device__ __forceinline__ int load_task_rows(const int64_t* __restrict__ nzptr, const int32_t* __restrict__ gran,
                                              int R, int64_t t0, int64_t t1, int64_t* sptr, int64_t* sk0) {
  __shared__ int64_t k_range[2];
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const int64_t kb = gran[(t1 - 1) >> 5];
    const int64_t kk = kb + 1 + lane;
    const bool starts = kk <= R && nzptr[kk] <= t1 - 1;
    const unsigned bal = __ballot_sync(0xffffffffu, starts);
    if (lane == 0) {
      k_range[0] = gran[t0 >> 5];
      k_range[1] = kb + __popc(bal);
    }
  }
  __syncthreads();
  const int64_t k0 = k_range[0];
  const int nrows = (int)(k_range[1] - k0 + 1);
  for (int i = threadIdx.x; i <= nrows; i += blockDim.x) sptr[i] = nzptr[k0 + i];
  *sk0 = k0;
  __syncthreads();
  return nrows;
}

// ---------------------------------------------------------------- per-piece sums
// The task's staged vectors V[q][0..L), L even: delta_0 .. delta_{JN-1}, X, 0 for the
// task-local entries q.  A tile sums four products over the entries of a row piece
// (task-local positions [max(sptr[k], t0), min(sptr[k+1], t1)) - t0):
//   outer tile (ca, cb):  A = V[q][ca, ca+1], B = V[q][cb, cb+1]:  A0 B0, A0 B1, A1 B0, A1 B1
//   square tile (ca):     A = V[q][ca, ca+1], x = V[q][xcol]:      x A0, x A1, A0^2, A1^2
// into the outputs out.x, .y, .z, .w of the piece (-1: none).  Every output of a piece
// belongs to exactly one tile.  Pieces of at most kPieceChunk entries: one warp per
// piece, lanes over tiles.  Longer pieces (at most TASK / kPieceChunk + 1 of them): cut
// into kPieceChunk-entry chunks spread over every thread, partials combined in chunk
// order.  Each chain keeps two accumulator sets (even / odd entries).  Fixed order
// throughout.
constexpr int kPieceChunk = 32;
constexpr int kMaxLongPieces = 16;

struct PieceScratch {
  int nlong;
  int total;                       // items of long pieces
  int k[kMaxLongPieces];           // long piece ids
  int q[kMaxLongPieces];           // chunks per long piece
  int item0[kMaxLongPieces + 1];   // first item of each long piece
};

template <typename S>
__device__ __forceinline__ void load2(const S* p, S& a, S& b) {
  if constexpr (sizeof(S) == 4) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    a = v.x;
    b = v.y;
  } else {
    const double2 v = *reinterpret_cast<const double2*>(p);
    a = v.x;
    b = v.y;
  }
}

template <typename S, bool SQUARE>
__device__ __forceinline__ void tile_chain(const S* V, int L, int xcol, int2 cab, int s, int e, S (&r)[4]) {
  S a[4] = {S(0), S(0), S(0), S(0)}, b[4] = {S(0), S(0), S(0), S(0)};
  const S* p = V + s * L;
  int q = s;
  for (; q + 1 < e; q += 2, p += 2 * L) {
    S x0, x1, y0, y1;
    load2<S>(p + cab.x, x0, x1);
    load2<S>(p + L + cab.x, y0, y1);
    if constexpr (SQUARE) {
      const S u = p[xcol], v = p[L + xcol];
      a[0] += u * x0; a[1] += u * x1; a[2] += x0 * x0; a[3] += x1 * x1;
      b[0] += v * y0; b[1] += v * y1; b[2] += y0 * y0; b[3] += y1 * y1;
    } else {
      S u0, u1, v0, v1;
      load2<S>(p + cab.y, u0, u1);
      load2<S>(p + L + cab.y, v0, v1);
      a[0] += x0 * u0; a[1] += x0 * u1; a[2] += x1 * u0; a[3] += x1 * u1;
      b[0] += y0 * v0; b[1] += y0 * v1; b[2] += y1 * v0; b[3] += y1 * v1;
    }
  }
  if (q < e) {
    S x0, x1;
    load2<S>(p + cab.x, x0, x1);
    if constexpr (SQUARE) {
      const S u = p[xcol];
      a[0] += u * x0; a[1] += u * x1; a[2] += x0 * x0; a[3] += x1 * x1;
    } else {
      S u0, u1;
      load2<S>(p + cab.y, u0, u1);
      a[0] += x0 * u0; a[1] += x0 * u1; a[2] += x1 * u0; a[3] += x1 * u1;
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) r[i] = a[i] + b[i];
}

__device__ __forceinline__ int out_at(const int4& o, int i) { return i == 0 ? o.x : i == 1 ? o.y : i == 2 ? o.z : o.w; }

template <typename S, bool SQUARE>
__device__ void piece_sums(const int64_t* sptr, int nrows, int64_t t0, int64_t t1, int NT, int P, const int2* cab,
                           const int4* outs, const S* V, int L, int xcol, S* sums, S* part, PieceScratch* ps) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // short pieces
  for (int k = warp; k < nrows; k += nwarps) {
    const int s = (int)(max(sptr[k], t0) - t0), e = (int)(min(sptr[k + 1], t1) - t0);
    if (e - s > kPieceChunk) continue;
    for (int t = lane; t < NT; t += 32) {
      S r[4];
      tile_chain<S, SQUARE>(V, L, xcol, cab[t], s, e, r);
      const int4 o = outs[t];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int pi = out_at(o, i);
        if (pi >= 0) sums[k * P + pi] = r[i];
      }
    }
  }
  // collect long pieces (warp 0)
  if (warp == 0) {
    int n = 0;
    for (int k0 = 0; k0 < nrows; k0 += 32) {
      const int k = k0 + lane;
      bool lg = false;
      if (k < nrows) lg = (min(sptr[k + 1], t1) - max(sptr[k], t0)) > kPieceChunk;
      const unsigned b = __ballot_sync(0xffffffffu, lg);
      if (lg) {
        const int slot = n + __popc(b & ((1u << lane) - 1u));
        if (slot < kMaxLongPieces) ps->k[slot] = k;
      }
      n += __popc(b);
    }
    __syncwarp();
    if (lane == 0) {
      ps->nlong = min(n, kMaxLongPieces);
      int it = 0;
      for (int i = 0; i < ps->nlong; ++i) {
        const int k = ps->k[i];
        const int len = (int)(min(sptr[k + 1], t1) - max(sptr[k], t0));
        ps->q[i] = (len + kPieceChunk - 1) / kPieceChunk;
        ps->item0[i] = it;
        it += ps->q[i] * NT;
      }
      ps->item0[ps->nlong] = it;
      ps->total = it;
    }
  }
  __syncthreads();
  const int nlong = ps->nlong, total = ps->total;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    int j = 0;
    while (i >= ps->item0[j + 1]) ++j;
    const int k = ps->k[j], r = i - ps->item0[j];
    const int q = r / NT, t = r % NT;
    const int s0 = (int)(max(sptr[k], t0) - t0), e0 = (int)(min(sptr[k + 1], t1) - t0);
    const int s = s0 + q * kPieceChunk, e = min(e0, s + kPieceChunk);
    S rr[4];
    tile_chain<S, SQUARE>(V, L, xcol, cab[t], s, e, rr);
#pragma unroll
    for (int u = 0; u < 4; ++u) part[i * 4 + u] = rr[u];
  }
  __syncthreads();
  for (int j = 0; j < nlong; ++j) {
    const int k = ps->k[j], nq = ps->q[j], base = ps->item0[j];
    for (int tu = threadIdx.x; tu < NT * 4; tu += blockDim.x) {
      const int t = tu >> 2, u = tu & 3;
      const int pi = out_at(outs[t], u);
      if (pi < 0) continue;
      S a = S(0);
      for (int q = 0; q < nq; ++q) a += part[(base + q * NT + t) * 4 + u];
      sums[k * P + pi] = a;
    }
  }
  __syncthreads();
}

}  // namespace vest
