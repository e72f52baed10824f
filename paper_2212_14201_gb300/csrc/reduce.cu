// Read-only reductions of the state: marginal probabilities (prob_run_list /
// prob_run_dict), <Z_i> for every qubit, and Pauli-sum expectations (the paper's
// probability / expectation tools, Section "A variety of convenient tools"; qop,
// Section "Variational quantum circuit").
//
// Every reduction is deterministic: per-thread partials are combined by a fixed
// warp-shuffle tree, CTA partials go to the workspace in CTA order and one
// final CTA adds them in that order.  Results do not depend on timing.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include "fixed.h"
#include "internal.h"
#include "pauli_plan.h"

namespace qs {

__device__ __forceinline__ double prob(double2 a) { return __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y)); }
__device__ __forceinline__ double acc_prob(double2 a, double s) { return fma(a.y, a.y, fma(a.x, a.x, s)); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of one value per thread (blockDim.x == 256); result valid in all threads.
__device__ double block_sum256(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) r += sh[i];
  return r;
}

// ---- full probability vector -------------------------------------------------------
// per-CTA partial sums of |a_x|^2 (four interleaved accumulators per thread)
template <class T>
__global__ void __launch_bounds__(256) k_norm2(const T* __restrict__ a, uint64_t N, double* __restrict__ part) {
  __shared__ double sh[8];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  // |a|^2 accumulated as two fused multiply-adds (two FP64 instructions per
  // amplitude: the FP64 pipe, not HBM, bounds this kernel on GB300)
  for (; i + 3 * stride < N; i += 4 * stride) {
    s0 = acc_prob(ld_amp(a, i), s0);
    s1 = acc_prob(ld_amp(a, i + stride), s1);
    s2 = acc_prob(ld_amp(a, i + 2 * stride), s2);
    s3 = acc_prob(ld_amp(a, i + 3 * stride), s3);
  }
  for (; i < N; i += stride) s0 = acc_prob(ld_amp(a, i), s0);
  const double t = block_sum256((s0 + s1) + (s2 + s3), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

template <class T>
__global__ void k_probs_full(const T* __restrict__ a, double* __restrict__ p, uint64_t N) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += stride) p[i] = prob(ld_amp(a, i));
}

// ---- marginal over nq <= 12 qubits: per-CTA shared histogram ---------------------
struct MargArgs {
  uint64_t N;
  int nq;
  int q[12];
};

__device__ __forceinline__ uint32_t extract_bits(uint64_t x, const MargArgs& g) {
  uint32_t k = 0;
  for (int j = 0; j < g.nq; ++j) k |= (uint32_t)((x >> g.q[j]) & 1) << j;
  return k;
}

// Each CTA owns a contiguous range of the state; a thread accumulates its own
// elements into a shared histogram with shared-memory atomics would make the sum
// order timing-dependent, so instead each warp owns a private histogram slice
// and adds its lanes' values in lane order.
template <class T>
__global__ void __launch_bounds__(256) k_marginal_small(const T* __restrict__ a, double* __restrict__ part,
                                                         const MargArgs g, uint64_t per_cta) {
  extern __shared__ double hist[];  // [8 warps][2^nq]
  const int H = 1 << g.nq;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int i = threadIdx.x; i < 8 * H; i += blockDim.x) hist[i] = 0.0;
  __syncthreads();
  uint64_t begin = blockIdx.x * per_cta, end = min(g.N, begin + per_cta);
  double* mine = hist + w * H;
  for (uint64_t base = begin + (uint64_t)w * 32; base < end; base += 256) {
    uint64_t x = base + l;
    double p = x < end ? prob(ld_amp(a, x)) : 0.0;
    uint32_t k = extract_bits(x, g);
    // lanes add in lane order (deterministic)
    for (int src = 0; src < 32; ++src) {
      double ps = __shfl_sync(0xffffffffu, p, src);
      uint32_t ks = __shfl_sync(0xffffffffu, k, src);
      if (l == 0 && base + src < end) mine[ks] += ps;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    double s = 0.0;
    for (int ww = 0; ww < 8; ++ww) s += hist[ww * H + i];
    part[(size_t)blockIdx.x * H + i] = s;
  }
}

// Marginal over nq <= 3 qubits (a measured qubit, a few bits): every thread keeps
// one partial per outcome over its grid-stride elements, the CTA adds them with
// the fixed shuffle tree, CTA partials go to part[cta][outcome] (then
// k_marginal_finish in CTA order).
template <class T, int NQ>
__global__ void __launch_bounds__(256) k_marginal_tiny(const T* __restrict__ a, double* __restrict__ part,
                                                        const MargArgs g) {
  __shared__ double sh[8];
  constexpr int H = 1 << NQ;
  double acc[H];
#pragma unroll
  for (int k = 0; k < H; ++k) acc[k] = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < g.N; x += stride) {
    const double2 v = ld_amp(a, x);
    uint32_t kb = 0;
#pragma unroll
    for (int j = 0; j < NQ; ++j) kb |= (uint32_t)((x >> g.q[j]) & 1) << j;
#pragma unroll
    for (int k = 0; k < H; ++k)
      if (k == (int)kb) acc[k] = acc_prob(v, acc[k]);
  }
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const double t = block_sum256(acc[k], sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * H + k] = t;
  }
}

// ---- exact integer marginals over at most three qubits (and the squared norm) ------
// For states whose components are known to lie within the Q60 bound (norm <= 1.25,
// e.g. |0> after unitary gates): each component is rounded once to Q60 (2^-60
// resolution, |error| <= 2^-61) and its square is summed exactly as a 128-bit
// integer in units of 2^-120, so the only errors are those roundings (a total below
// 2^-60 sum |a_x| <= 2^-45 for n <= 30) and one final conversion to double.  Integer
// arithmetic runs on pipes that GB300 issues at full rate; the FP64 form above is
// bound by the FP64 pipe (1/74 of the FP32 rate) rather than by HBM.
// The sum of all squares is at most 1.5625 * 2^120 < 2^128.
using u128 = unsigned __int128;

__device__ __forceinline__ u128 sq120(double2 v) {
  const int64_t r = q60_from_double(v.x), i = q60_from_double(v.y);
  const uint64_t ur = (uint64_t)(r < 0 ? -r : r), ui = (uint64_t)(i < 0 ? -i : i);
  return (u128)ur * ur + (u128)ui * ui;
}

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int o) {
  const uint64_t lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)(uint64_t)v, o);
  const uint64_t hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(uint64_t)(v >> 64), o);
  return ((u128)hi << 64) | lo;
}

// per-CTA exact partials: part[(block * H + k) * 2 + {0, 1}] = low and high words
template <class T, int NQ>
__global__ void __launch_bounds__(256) k_marginal_exact(const T* __restrict__ a, uint64_t* __restrict__ part,
                                                         const MargArgs g) {
  constexpr int H = 1 << NQ;
  __shared__ uint64_t sh[8][H][2];
  u128 acc[H];
#pragma unroll
  for (int k = 0; k < H; ++k) acc[k] = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  auto add = [&](uint64_t x, u128 p) {
    uint32_t kb = 0;
#pragma unroll
    for (int j = 0; j < NQ; ++j) kb |= (uint32_t)((x >> g.q[j]) & 1) << j;
#pragma unroll
    for (int k = 0; k < H; ++k)
      if (k == (int)kb) acc[k] += p;
  };
  uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  // four independent loads in flight per thread (the loop is otherwise bound by
  // the latency of one 16-byte load per iteration)
  for (; x + 3 * stride < g.N; x += 4 * stride) {
    const double2 v0 = ld_amp(a, x), v1 = ld_amp(a, x + stride), v2 = ld_amp(a, x + 2 * stride),
                  v3 = ld_amp(a, x + 3 * stride);
    add(x, sq120(v0));
    add(x + stride, sq120(v1));
    add(x + 2 * stride, sq120(v2));
    add(x + 3 * stride, sq120(v3));
  }
  for (; x < g.N; x += stride) add(x, sq120(ld_amp(a, x)));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    u128 v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor_u128(v, o);
    if (l == 0) {
      sh[w][k][0] = (uint64_t)v;
      sh[w][k][1] = (uint64_t)(v >> 64);
    }
  }
  __syncthreads();
  if (threadIdx.x < H) {
    u128 t = 0;
    for (int i = 0; i < 8; ++i) t += ((u128)sh[i][threadIdx.x][1] << 64) | sh[i][threadIdx.x][0];
    part[((size_t)blockIdx.x * H + threadIdx.x) * 2] = (uint64_t)t;
    part[((size_t)blockIdx.x * H + threadIdx.x) * 2 + 1] = (uint64_t)(t >> 64);
  }
}

__global__ void k_exact_finish(const uint64_t* __restrict__ part, int nblocks, int H, double* __restrict__ out) {
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    u128 t = 0;
    for (int b = 0; b < nblocks; ++b)
      t += ((u128)part[((size_t)b * H + i) * 2 + 1] << 64) | part[((size_t)b * H + i) * 2];
    const double v = (double)(uint64_t)(t >> 64) * 18446744073709551616.0 + (double)(uint64_t)t;
    out[i] = v * 0x1p-120;
  }
}

__global__ void k_marginal_finish(const double* __restrict__ part, int nblocks, int H, double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < H; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * H + i];
    out[i] = s;
  }
}

// ---- marginal over many qubits: one thread per output entry -----------------------
struct MargBigArgs {
  uint64_t H;         // 2^nq outputs
  uint64_t R;         // 2^(n-nq) terms per output
  int nq, nr;
  int q[QS_MAX_QUBITS];   // listed qubits
  int r[QS_MAX_QUBITS];   // remaining qubits, ascending
};

template <class T>
__global__ void k_marginal_big(const T* __restrict__ a, double* __restrict__ out, const MargBigArgs g) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < g.H; k += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t xb = 0;
    for (int j = 0; j < g.nq; ++j) xb |= ((k >> j) & 1ull) << g.q[j];
    double s = 0.0;
    for (uint64_t r = 0; r < g.R; ++r) {
      uint64_t x = xb;
      for (int j = 0; j < g.nr; ++j) x |= ((r >> j) & 1ull) << g.r[j];
      s += prob(ld_amp(a, x));
    }
    out[k] = s;
  }
}

// ---- <Z_i> for all i -----------------------------------------------------------------
// CTA c owns the contiguous range [c*2^r, (c+1)*2^r).  Thread t handles elements
// t + 256*j: bits 0..7 of the index are t, bits 8..r-1 are j, bits >= r are the CTA.
// Each thread keeps its total and, for every bit of j, the sum over its elements
// with that bit set; the CTA combines them into S_i = sum_{x_i = 1} p_x.
constexpr int ZMAXJ = 26;
template <class A>
__global__ void __launch_bounds__(256) k_expect_z(const A* __restrict__ a, int r, double* __restrict__ part) {
  __shared__ double sh[8];
  const int jbits = r - 8;
  const uint64_t base = (uint64_t)blockIdx.x << r;
  double tot = 0.0;
  double bs[ZMAXJ];
#pragma unroll
  for (int b = 0; b < ZMAXJ; ++b) bs[b] = 0.0;
  const uint64_t J = 1ull << jbits;
  for (uint64_t j = 0; j < J; ++j) {
    double p = prob(ld_amp(a, base + threadIdx.x + (j << 8)));
    tot += p;
#pragma unroll
    for (int b = 0; b < ZMAXJ; ++b)
      if (b < jbits && ((j >> b) & 1)) bs[b] += p;
  }
  // outputs: [0] total, [1 + i] = S_i for i < r  (bits >= r are handled by the finisher)
  double* o = part + (size_t)blockIdx.x * (r + 1);
  double T = block_sum256(tot, sh);
  if (threadIdx.x == 0) o[0] = T;
  for (int i = 0; i < 8; ++i) {
    double v = block_sum256(((threadIdx.x >> i) & 1) ? tot : 0.0, sh);
    if (threadIdx.x == 0) o[1 + i] = v;
  }
  for (int b = 0; b < jbits; ++b) {
    double v = 0.0;
#pragma unroll
    for (int bb = 0; bb < ZMAXJ; ++bb)
      if (bb == b) v = bs[bb];
    v = block_sum256(v, sh);
    if (threadIdx.x == 0) o[1 + 8 + b] = v;
  }
}

// The same sums exactly, for a state within the Q60 bound and 4 <= r - 8 <= ZEXJ
// loop bits: squares of the Q60-rounded components as 128-bit integers (units
// 2^-120).  A thread takes its amplitudes sixteen at a time (loop bits 0..3, whose
// sums stay in registers); the sixteen-amplitude total is then added, in shared
// memory, to the sum of every higher loop bit set in that step, the same for all
// lanes.  Outputs per CTA as in k_expect_z, each value as two words (low, high).
constexpr int ZEXJ = 12;
template <class A>
__global__ void __launch_bounds__(256, 3) k_expect_z_exact(const A* __restrict__ a, int r, uint64_t* __restrict__ part) {
  __shared__ uint64_t sh[8][2];
  __shared__ uint4 hs[ZEXJ - 4][256];  // per-thread sums of loop bits 4.. (low, high words)
  const int jbits = r - 8;
  const uint64_t base = ((uint64_t)blockIdx.x << r) + threadIdx.x;
  for (int b = 0; b < jbits - 4; ++b) hs[b][threadIdx.x] = make_uint4(0, 0, 0, 0);
  u128 tot = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
  const uint64_t J = 1ull << jbits;
  for (uint64_t j = 0; j < J; j += 16) {
    u128 t16 = 0;
#pragma unroll
    for (int h = 0; h < 16; h += 8) {
      double2 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = ld_amp(a, base + ((j + h + q) << 8));
      u128 t8 = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const u128 p = sq120(v[q]);
        t8 += p;
        if (q & 1) b0 += p;
        if (q & 2) b1 += p;
        if (q & 4) b2 += p;
      }
      if (h) b3 += t8;
      t16 += t8;
    }
    tot += t16;
    const uint32_t jh = (uint32_t)(j >> 4);
    if (jh) {
      for (int b = 0; b < jbits - 4; ++b) {
        if ((jh >> b) & 1) {
          uint4 c = hs[b][threadIdx.x];
          u128 v = (((u128)(((uint64_t)c.w << 32) | c.z)) << 64) | (((uint64_t)c.y << 32) | c.x);
          v += t16;
          const uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
          hs[b][threadIdx.x] = make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32));
        }
      }
    }
  }
  auto block_sum = [&](u128 v) {  // fixed shuffle tree, then warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor_u128(v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
      sh[w][0] = (uint64_t)v;
      sh[w][1] = (uint64_t)(v >> 64);
    }
    __syncthreads();
    u128 t = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) t += ((u128)sh[i][1] << 64) | sh[i][0];
    return t;
  };
  uint64_t* o = part + (size_t)blockIdx.x * (r + 1) * 2;
  auto put = [&](int k, u128 v) {
    if (threadIdx.x == 0) {
      o[2 * k] = (uint64_t)v;
      o[2 * k + 1] = (uint64_t)(v >> 64);
    }
  };
  put(0, block_sum(tot));
  for (int i = 0; i < 8; ++i) put(1 + i, block_sum(((threadIdx.x >> i) & 1) ? tot : (u128)0));
  put(9, block_sum(b0));
  put(10, block_sum(b1));
  put(11, block_sum(b2));
  put(12, block_sum(b3));
  for (int b = 0; b < jbits - 4; ++b) {
    const uint4 c = hs[b][threadIdx.x];
    put(13 + b, block_sum((((u128)(((uint64_t)c.w << 32) | c.z)) << 64) | (((uint64_t)c.y << 32) | c.x)));
  }
}

// out[i] = T - 2 S_i from the exact CTA partials (bits >= r: CTA index bits).
__global__ void k_expect_z_exact_finish(const uint64_t* __restrict__ part, int nblocks, int r, int n,
                                        double* __restrict__ out) {
  const int i = threadIdx.x;
  if (i >= n) return;
  u128 T = 0, S = 0;
  for (int c = 0; c < nblocks; ++c) {
    const uint64_t* o = part + (size_t)c * (r + 1) * 2;
    const u128 t = ((u128)o[1] << 64) | o[0];
    T += t;
    if (i < r) S += ((u128)o[2 * (1 + i) + 1] << 64) | o[2 * (1 + i)];
    else if ((c >> (i - r)) & 1) S += t;
  }
  const bool neg = T < 2 * S;  // T - 2S may be negative
  const u128 m = neg ? 2 * S - T : T - 2 * S;
  const double d = (double)(uint64_t)(m >> 64) * 18446744073709551616.0 + (double)(uint64_t)m;
  out[i] = (neg ? -d : d) * 0x1p-120;
}

__global__ void k_expect_z_finish(const double* __restrict__ part, int nblocks, int r, int n, double* __restrict__ out) {
  // out[i] = T - 2 S_i; thread i handles qubit i; CTA partials added in CTA order.
  int i = threadIdx.x;
  if (i >= n) return;
  double T = 0.0, S = 0.0;
  for (int c = 0; c < nblocks; ++c) {
    const double* o = part + (size_t)c * (r + 1);
    T += o[0];
    if (i < r) S += o[1 + i];
    else if ((c >> (i - r)) & 1) S += o[0];
  }
  out[i] = T - 2.0 * S;
}

// ---- Pauli terms ------------------------------------------------------------------------
// For a term (xm, zm, ny = popcount(xm & zm)):
//   <P> = sum_x Re( i^ny (-1)^{popcount(x & zm)} conj(a_{x^xm}) a_x ).
// Up to 8 terms per launch; per-CTA partials, then a fixed-order finish.
struct PauliArgs {
  uint64_t N;
  int nt;
  uint64_t xm[8], zm[8];
  int ny[8];
};

template <class T>
__global__ void __launch_bounds__(256) k_pauli(const T* __restrict__ a, const PauliArgs g, double* __restrict__ part) {
  __shared__ double sh[8];
  double acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < g.N; x += stride) {
    double2 v = ld_amp(a, x);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (k >= g.nt) break;
      double2 u = ld_amp(a, x ^ g.xm[k]);
      // w = conj(u) * v ; term = Re(i^ny * w) with sign (-1)^{popcount(x & zm)}
      double w;
      if (g.ny[k] & 1) w = fma(u.y, v.x, -u.x * v.y);   // Re(i*w) = -Im(w) = u.y v.x - u.x v.y
      else w = fma(u.x, v.x, u.y * v.y);                // Re(w)
      int neg = (__popcll(x & g.zm[k]) + (g.ny[k] >> 1)) & 1;
      acc[k] += neg ? -w : w;
    }
  }
  for (int k = 0; k < g.nt; ++k) {
    double s = block_sum256(acc[k], sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * 8 + k] = s;
  }
}

__global__ void k_pauli_finish(const double* __restrict__ part, int nblocks, int nt, double* __restrict__ out) {
  int k = threadIdx.x;
  if (k >= nt) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * 8 + k];
  out[k] = s;
}

// ---- Pauli sums, exact integer form ---------------------------------------------------
// For a state within the Q60 bound (norm <= 1.25) every term is computed from the
// Q60-rounded amplitudes with exact 128-bit integer sums (units 2^-120).  A term
// P = (xm, zm) with ny = popcount(xm & zm) pairs x0 with x1 = x0 ^ xm; with
// w = conj(a_x1) a_x0 and s0 = (-1)^popcount(x0 & zm) the pair contributes
//   ny = 0: 2 s0 Re w,  1: -2 s0 Im w,  2: -2 s0 Re w,  3: 2 s0 Im w,
// and a term with xm = 0 contributes s0 |a_x0|^2 per index.
//
// One pass reads the state once, as tiles {base ^ span(bm_0 .. bm_{T-1})} of
// 2^T <= 4096 amplitudes: the basis holds qubits 0..3 (so a tile is made of runs
// of 16 consecutive amplitudes) and X masks reduced to distinct leading bits, which
// every tile base has clear.  A CTA stages a tile in shared memory with cp.async,
// decodes it to split Q60 once, serves the |a|^2 slots from the decoded values,
// then every pair slot whose X mask lies in the span from shared memory.  A slot
// (xm, zm, part) accumulates pos = the sum of its values v (Re w, Im w or |a|^2)
// over pairs with s0 = +1; the term is mult * (2 pos - tot), tot = the same sum
// with zm = 0 (its own slot).  The passes are planned on the host (pauli_plan.h).
struct PTile {
  uint64_t ntiles;          // 2^(n - T)
  int T;                    // tile coordinates, ordered by leading bit
  int lead[PT_TMAX];        // leading bit of each basis vector (ascending)
  uint64_t bm[PT_TMAX];     // basis vector of each coordinate
  int nt, nz;               // slots in this pass; the first nz are |a|^2 slots
  uint64_t zm[PS_MAX];
  uint32_t zc[PS_MAX];      // bit i = parity(bm[i] & zm)
  uint32_t xc[PS_MAX];      // pair slots: X mask = XOR of bm[i] over the bits i of xc
  int top[PS_MAX];          // pair slots: highest bit of xc
  uint8_t im[PS_MAX];       // pair slots: 0 = Re w, 1 = Im w
};

__device__ __forceinline__ uint64_t insert0(uint64_t c, int b) {
  return ((c >> b) << (b + 1)) | (c & ((1ull << b) - 1));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ Sp sp_h(int4 u) { return {u.x, u.y}; }
// acc += v when bit 0 of c is clear: a predicated 128-bit add (carry chain)
__device__ __forceinline__ void add128_if_even(u128& acc, u128 v, uint32_t c) {
  uint64_t lo = (uint64_t)acc, hi = (uint64_t)(acc >> 64);
  asm("{\n\t.reg .pred p;\n\t.reg .b32 t;\n\tand.b32 t, %4, 1;\n\tsetp.eq.u32 p, t, 0;\n\t"
      "@p add.cc.u64 %0, %0, %2;\n\t@p addc.u64 %1, %1, %3;\n\t}"
      : "+l"(lo), "+l"(hi)
      : "l"((uint64_t)v), "l"((uint64_t)(v >> 64)), "r"(c));
  acc = ((u128)hi << 64) | lo;
}
__device__ __forceinline__ Sp sp_i(int4 u) { return {u.z, u.w}; }

template <class A>
__global__ void __launch_bounds__(256, 3) k_pauli_tile(const A* __restrict__ a, const PTile g,
                                                       uint64_t* __restrict__ part) {
  extern __shared__ int4 tile[];  // 2^T entries: the raw amplitude, then (r.h, r.l, i.h, i.l)
  __shared__ uint64_t sh[8][PS_MAX][2];
  const int E = 1 << g.T;
  u128 pos[PS_MAX];
#pragma unroll
  for (int k = 0; k < PS_MAX; ++k) pos[k] = 0;
  __shared__ uint64_t span_hi[1 << (PT_TMAX - 8)];  // span of coordinates 8.. for e >> 8
  uint64_t span_t = 0;                              // span of this thread's coordinates 0..7
  for (int i = 0; i < g.T && i < 8; ++i)
    if ((threadIdx.x >> i) & 1) span_t ^= g.bm[i];
  if (threadIdx.x < (1 << (PT_TMAX - 8))) {
    uint64_t v = 0;
    for (int i = 8; i < g.T; ++i)
      if ((threadIdx.x >> (i - 8)) & 1) v ^= g.bm[i];
    span_hi[threadIdx.x] = v;
  }
  // |a|^2 slots: the sign of entry e is bit k of (pbm ^ tpar ^ zub[e >> 8]), with
  // tpar the parities of this thread's coordinates 0..7 and zub those of 8..
  __shared__ uint32_t zub[1 << (PT_TMAX - 8)];
  uint32_t tpar = 0;
#pragma unroll
  for (int k = 0; k < PS_MAX; ++k)
    if (k < g.nz) tpar |= (uint32_t)(__popc(threadIdx.x & g.zc[k] & 0xffu) & 1) << k;
  if (threadIdx.x < (1 << (PT_TMAX - 8))) {
    uint32_t u = 0;
    for (int k = 0; k < g.nz; ++k) u |= (uint32_t)(__popc(threadIdx.x & (g.zc[k] >> 8)) & 1) << k;
    zub[threadIdx.x] = u;
  }
  __syncthreads();
  for (uint64_t c = blockIdx.x; c < g.ntiles; c += gridDim.x) {
    uint64_t base = c;
    for (int i = 0; i < g.T; ++i) base = insert0(base, g.lead[i]);
    const uint64_t bt = base ^ span_t;
    for (int e = threadIdx.x; e < E; e += 256) {
      const uint64_t x = bt ^ span_hi[e >> 8];
      if (sizeof(A) == 16) cp_async16(&tile[e], a + x);
      else cp_async8(&tile[e], a + x);
    }
    cp_async_wait_all();  // each thread decodes the entries it copied
    uint32_t pbm = 0;     // bit k: parity(base & zm_k)
#pragma unroll
    for (int k = 0; k < PS_MAX; ++k)
      if (k < g.nt) pbm |= (uint32_t)(__popcll(base & g.zm[k]) & 1) << k;
    for (int e = threadIdx.x; e < E; e += 256) {
      double re, im;
      if (sizeof(A) == 16) {
        const double2 v = *reinterpret_cast<const double2*>(&tile[e]);
        re = v.x;
        im = v.y;
      } else {
        const float2 v = *reinterpret_cast<const float2*>(&tile[e]);
        re = v.x;
        im = v.y;
      }
      const Sp r = split31(q60_from_double(re)), i = split31(q60_from_double(im));
      tile[e] = make_int4(r.h, r.l, i.h, i.l);
      if (g.nz > 0) {
        const u128 p = dot2_exact(r, r, i, i);
        const uint32_t m = pbm ^ tpar ^ zub[e >> 8];
#pragma unroll
        for (int k = 0; k < PS_MAX; ++k)
          if (k < g.nz) add128_if_even(pos[k], p, m >> k);
      }
    }
    __syncthreads();
    // pair slots: pairs outer, slots inner (one product live, recomputed when the
    // slot's (X mask, part) changes)
    for (int t = threadIdx.x; t < E / 2; t += 256) {
      int key = -1;
      u128 wv = 0;
      uint32_t s0 = 0;
#pragma unroll
      for (int k = 0; k < PS_MAX; ++k) {
        if (k >= g.nz && k < g.nt) {
          const uint32_t xc = g.xc[k];
          const int kk = (int)xc * 2 + g.im[k];
          if (kk != key) {
            key = kk;
            const int top = g.top[k];
            s0 = (((uint32_t)t >> top) << (top + 1)) | ((uint32_t)t & ((1u << top) - 1u));
            const int4 u0 = tile[s0], u1 = tile[s0 ^ xc];
            wv = g.im[k] ? dot2_exact(sp_h(u1), sp_i(u0), sp_neg(sp_i(u1)), sp_h(u0))
                         : dot2_exact(sp_h(u1), sp_h(u0), sp_i(u1), sp_i(u0));
          }
          if (g.zc[k] == 0) {  // sign the same over the tile
            if (((pbm >> k) & 1u) == 0) pos[k] += wv;
          } else {
            add128_if_even(pos[k], wv, (pbm >> k) ^ (uint32_t)__popc(s0 & g.zc[k]));
          }
        }
      }
    }
    __syncthreads();  // the next tile's copies overwrite this one
  }
  const int wp = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < PS_MAX; ++k) {
    if (k < g.nt) {
      u128 t = pos[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += shfl_xor_u128(t, o);
      if (l == 0) {
        sh[wp][k][0] = (uint64_t)t;
        sh[wp][k][1] = (uint64_t)(t >> 64);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < g.nt) {
    u128 t = 0;
    for (int q = 0; q < 8; ++q) t += ((u128)sh[q][threadIdx.x][1] << 64) | sh[q][threadIdx.x][0];
    part[((size_t)blockIdx.x * PS_MAX + threadIdx.x) * 2] = (uint64_t)t;
    part[((size_t)blockIdx.x * PS_MAX + threadIdx.x) * 2 + 1] = (uint64_t)(t >> 64);
  }
}

// sums[slot0 + k] = the CTA partials of slot k added (modulo 2^128)
__global__ void k_pauli_exact_finish(const uint64_t* __restrict__ part, int nblocks, int nt, uint64_t* __restrict__ sums) {
  const int k = threadIdx.x;
  if (k >= nt) return;
  u128 t = 0;
  for (int b = 0; b < nblocks; ++b)
    t += ((u128)part[((size_t)b * PS_MAX + k) * 2 + 1] << 64) | part[((size_t)b * PS_MAX + k) * 2];
  sums[2 * k] = (uint64_t)t;
  sums[2 * k + 1] = (uint64_t)(t >> 64);
}

}  // namespace qs

using namespace qs;

static int read_back(qs_state* s, const double* dev, size_t count, double* host) {
  QS_TRY(ensure_pinned(s, count * sizeof(double)));
  QS_CUDA(cudaMemcpyAsync(s->pinned, dev, count * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  memcpy(host, s->pinned, count * sizeof(double));
  return QS_OK;
}

static int marginal_device(qs_state* s, const int* qubits, int nq, double* dout, bool allow_exact = true) {
  const int n = s->n;
  const uint64_t N = 1ull << n;
  bool identity = nq == n;
  for (int j = 0; j < nq && identity; ++j) identity = qubits[j] == j;
  KTimer kt(s, QS_K_REDUCE, nq, 1, 0, 0, (double)N, 3.0 * (double)N);
  if (identity) {
    with_amps(s, [&](auto* a) {
      k_probs_full<<<(int)std::min<uint64_t>((N + 255) / 256, 152 * 32), 256, 0, s->stream>>>(a, dout, N);
      return QS_OK;
    });
    return launch_check("probs_full");
  }
  if (nq <= 3 && s->bound == 1 && allow_exact) {  // exact integer sums (see k_marginal_exact)
    MargArgs g;
    g.N = N;
    g.nq = nq;
    for (int j = 0; j < nq; ++j) g.q[j] = qubits[j];
    const int nblocks = (int)std::min<uint64_t>(1216, std::max<uint64_t>(1, N / 1024));
    uint64_t* part = (uint64_t*)s->ws;
    note_launch(1);
    with_amps(s, [&](auto* a) {
      using T = std::remove_cv_t<std::remove_pointer_t<decltype(a)>>;
      const T* ca = a;
      switch (nq) {
        case 0: k_marginal_exact<T, 0><<<nblocks, 256, 0, s->stream>>>(ca, part, g); break;
        case 1: k_marginal_exact<T, 1><<<nblocks, 256, 0, s->stream>>>(ca, part, g); break;
        case 2: k_marginal_exact<T, 2><<<nblocks, 256, 0, s->stream>>>(ca, part, g); break;
        default: k_marginal_exact<T, 3><<<nblocks, 256, 0, s->stream>>>(ca, part, g); break;
      }
      return QS_OK;
    });
    QS_TRY(launch_check("marginal_exact"));
    k_exact_finish<<<1, 32, 0, s->stream>>>(part, nblocks, 1 << nq, dout);
    return launch_check("marginal_exact finish");
  }
  if (nq == 0) {  // squared norm: per-thread sums, a fixed shuffle tree, CTA partials in order
    const int nblocks = (int)std::min<uint64_t>(608, std::max<uint64_t>(1, N / 1024));
    double* part = (double*)s->ws;
    with_amps(s, [&](auto* a) {
      k_norm2<<<nblocks, 256, 0, s->stream>>>(a, N, part);
      return QS_OK;
    });
    QS_TRY(launch_check("norm2"));
    k_marginal_finish<<<1, 32, 0, s->stream>>>(part, nblocks, 1, dout);
    return launch_check("norm2 finish");
  }
  if (nq <= 3) {
    MargArgs g;
    g.N = N;
    g.nq = nq;
    for (int j = 0; j < nq; ++j) g.q[j] = qubits[j];
    const int nblocks = (int)std::min<uint64_t>(608, std::max<uint64_t>(1, N / 1024));
    double* part = (double*)s->ws;
    with_amps(s, [&](auto* a) {
      using T = std::remove_cv_t<std::remove_pointer_t<decltype(a)>>;
      const T* ca = a;
      switch (nq) {
        case 1: k_marginal_tiny<T, 1><<<nblocks, 256, 0, s->stream>>>(ca, part, g); break;
        case 2: k_marginal_tiny<T, 2><<<nblocks, 256, 0, s->stream>>>(ca, part, g); break;
        default: k_marginal_tiny<T, 3><<<nblocks, 256, 0, s->stream>>>(ca, part, g); break;
      }
      return QS_OK;
    });
    QS_TRY(launch_check("marginal_tiny"));
    const int H = 1 << nq;
    k_marginal_finish<<<1, 32, 0, s->stream>>>(part, nblocks, H, dout);
    return launch_check("marginal_finish");
  }
  if (nq <= 10) {  // 8 warp-private histograms of 2^nq doubles fit in shared memory
    MargArgs g;
    g.N = N;
    g.nq = nq;
    for (int j = 0; j < nq; ++j) g.q[j] = qubits[j];
    int nblocks = (int)std::min<uint64_t>(304, std::max<uint64_t>(1, N / 256));
    uint64_t per = (N + nblocks - 1) / nblocks;
    per = (per + 255) / 256 * 256;
    nblocks = (int)((N + per - 1) / per);
    size_t smem = (size_t)8 * (1 << nq) * sizeof(double);
    double* part = (double*)s->ws;
    QS_TRY(with_amps(s, [&](auto* a) {
      using T = std::remove_cv_t<std::remove_pointer_t<decltype(a)>>;
      if (smem > 48 * 1024)
        QS_CUDA(cudaFuncSetAttribute(k_marginal_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_marginal_small<<<nblocks, 256, smem, s->stream>>>((const T*)a, part, g, per);
      return QS_OK;
    }));
    QS_TRY(launch_check("marginal_small"));
    int H = 1 << nq;
    k_marginal_finish<<<(H + 255) / 256, 256, 0, s->stream>>>(part, nblocks, H, dout);
    return launch_check("marginal_finish");
  }
  MargBigArgs g;
  g.nq = nq;
  g.H = 1ull << nq;
  g.R = 1ull << (n - nq);
  uint64_t used = 0;
  for (int j = 0; j < nq; ++j) {
    g.q[j] = qubits[j];
    used |= 1ull << qubits[j];
  }
  g.nr = 0;
  for (int b = 0; b < n; ++b)
    if (!((used >> b) & 1)) g.r[g.nr++] = b;
  with_amps(s, [&](auto* a) {
    k_marginal_big<<<(int)std::min<uint64_t>((g.H + 255) / 256, 152 * 32), 256, 0, s->stream>>>(a, dout, g);
    return QS_OK;
  });
  return launch_check("marginal_big");
}

static int check_qubit_list(const qs_state* s, const int* qubits, int nq) {
  if (nq < 0 || nq > s->n) return fail(QS_ERR_INVALID_ARG, "nq=%d outside 0..n", nq);
  if (nq && !qubits) return fail(QS_ERR_INVALID_ARG, "qubits is NULL");
  uint64_t seen = 0;
  for (int j = 0; j < nq; ++j) {
    if (qubits[j] < 0 || qubits[j] >= s->n || ((seen >> qubits[j]) & 1))
      return fail(QS_ERR_INVALID_ARG, "bad or repeated qubit %d", qubits[j]);
    seen |= 1ull << qubits[j];
  }
  return QS_OK;
}

namespace qs {
// Marginal probabilities into host memory; allow_exact = false forces the FP64
// kernels (relative accuracy for tiny probabilities, where the exact integer form
// is only accurate to 2^-45 absolute).
int marginal_host(qs_state* s, const int* qubits, int nq, double* out, bool allow_exact) {
  size_t H = (size_t)1 << nq;
  double* tmp = nullptr;
  QS_CUDA(dmalloc_async(&tmp, H * sizeof(double), s->stream));
  int rc = marginal_device(s, qubits, nq, tmp, allow_exact);
  if (rc == QS_OK) {
    cudaError_t e = cudaMemcpyAsync(out, tmp, H * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "probs readback");
  }
  cudaFreeAsync(tmp, s->stream);
  return rc;
}
}  // namespace qs

extern "C" int qs_probs(const qs_state* cs, const int* qubits, int nq, double* out, int on_device) {
  clear_error();
  qs_state* s = const_cast<qs_state*>(cs);
  QS_TRY(check_state(s));
  QS_TRY(check_qubit_list(s, qubits, nq));
  if (!out) return fail(QS_ERR_INVALID_ARG, "out is NULL");
  size_t H = (size_t)1 << nq;
  if (on_device) return marginal_device(s, qubits, nq, out);
  double* tmp = nullptr;
  QS_CUDA(dmalloc_async(&tmp, H * sizeof(double), s->stream));
  int rc = marginal_device(s, qubits, nq, tmp);
  if (rc == QS_OK) {
    cudaError_t e = cudaMemcpyAsync(out, tmp, H * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "probs readback");
  }
  cudaFreeAsync(tmp, s->stream);
  return rc;
}

extern "C" int qs_probs_dict(const qs_state* cs, const int* qubits, int nq, double threshold, uint64_t* idx,
                             double* p, size_t cap, size_t* count) {
  clear_error();
  qs_state* s = const_cast<qs_state*>(cs);
  QS_TRY(check_state(s));
  QS_TRY(check_qubit_list(s, qubits, nq));
  if (!count || (cap && (!idx || !p))) return fail(QS_ERR_INVALID_ARG, "NULL output");
  if (nq > 28) return fail(QS_ERR_UNSUPPORTED, "probs_dict over more than 28 qubits");
  size_t H = (size_t)1 << nq;
  std::vector<double> host(H);
  QS_TRY(qs_probs(s, qubits, nq, host.data(), 0));
  size_t c = 0;
  for (size_t k = 0; k < H; ++k) {
    if (host[k] > threshold) {
      if (c < cap) {
        idx[c] = k;
        p[c] = host[k];
      }
      ++c;
    }
  }
  *count = c;
  return QS_OK;
}

// Whether the state is within the Q60 bound (norm <= 1.25), measuring the norm
// once when that is unknown (after qs_set_state or a non-unitary matrix).
static int ensure_bound(qs_state* s) {
  if (s->bound != 0) return QS_OK;
  double norm2 = 0.0;
  QS_TRY(qs_probs(s, nullptr, 0, &norm2, 0));
  s->bound = (norm2 <= Q60_MAX_ABS * Q60_MAX_ABS) ? 1 : 2;
  return QS_OK;
}

extern "C" int qs_expect_z_all(const qs_state* cs, double* out) {
  clear_error();
  qs_state* s = const_cast<qs_state*>(cs);
  QS_TRY(check_state(s));
  if (!out) return fail(QS_ERR_INVALID_ARG, "out is NULL");
  const int n = s->n;
  double* part = (double*)s->ws;
  double* dres = part + (size_t)1024 * 72 - 64;
  if (n < 8) {
    // tiny states: marginal per qubit
    for (int i = 0; i < n; ++i) {
      double m2[2];
      int q = i;
      QS_TRY(qs_probs(s, &q, 1, m2, 0));
      out[i] = m2[0] - m2[1];
    }
    return QS_OK;
  }
  QS_TRY(ensure_bound(s));
  KTimer kt(s, QS_K_REDUCE, n, 1, 0, 0, (double)(1ull << n), 5.0 * (double)(1ull << n));
  if (s->bound == 1 && n >= 12 && n <= 20 + ZEXJ - 2) {  // exact integer sums (k_expect_z_exact)
    // r bits per CTA: 4 <= r - 8 <= ZEXJ loop bits, at most 1024 CTAs
    const int r = std::max(12, n - 10);
    const int nblocks = 1 << (n - r);
    uint64_t* ipart = (uint64_t*)s->ws;
    note_launch(1);
    with_amps(s, [&](auto* a) {
      k_expect_z_exact<<<nblocks, 256, 0, s->stream>>>(a, r, ipart);
      return QS_OK;
    });
    QS_TRY(launch_check("expect_z"));
    k_expect_z_exact_finish<<<1, 64, 0, s->stream>>>(ipart, nblocks, r, n, dres);
    QS_TRY(launch_check("expect_z_finish"));
    return read_back(s, dres, n, out);
  }
  // r = bits per CTA: at least 8 (one element per thread), at most 8 + ZMAXJ; CTAs <= 1024
  int r = std::max(8, n - 10);
  r = std::min(r, std::min(n, 8 + ZMAXJ));
  int nblocks = 1 << (n - r);
  with_amps(s, [&](auto* a) {
    k_expect_z<<<nblocks, 256, 0, s->stream>>>(a, r, part);
    return QS_OK;
  });
  QS_TRY(launch_check("expect_z"));
  k_expect_z_finish<<<1, 64, 0, s->stream>>>(part, nblocks, r, n, dres);
  QS_TRY(launch_check("expect_z_finish"));
  return read_back(s, dres, n, out);
}

// <sum_k coef_k P_k> with the exact passes of k_pauli_exact.  Slots are keyed by
// (xm, zm, part); X masks are taken two at a time as a cell basis, every other
// X mask in their span joins that pass, and |a|^2 slots fill the free places
// (then passes of their own over cells of bits 0 and 1).
static int pauli_exact(qs_state* s, const qs_pauli* terms, size_t nterms, double* out) {
  const int n = s->n;
  const size_t kChunk = 16384;  // terms per plan: at most 2 slots each
  double e = 0.0;
  std::vector<double> vals;
  for (size_t t0 = 0; t0 < nterms; t0 += kChunk) {
    const size_t nt = std::min(kChunk, nterms - t0);
    std::vector<uint64_t> xmv(nt), zmv(nt);
    for (size_t k = 0; k < nt; ++k) {
      xmv[k] = terms[t0 + k].xmask;
      zmv[k] = terms[t0 + k].zmask;
    }
    const PauliPlan plan = plan_pauli(n, xmv.data(), zmv.data(), nt);
    const auto& slots = plan.slots;
    const auto& passes = plan.passes;
    const auto& tslot = plan.tslot;
    const auto& ttot = plan.ttot;
    const auto& tmult = plan.tmult;
    // launch
    const size_t nslots = slots.size();
    std::vector<int> gidx(nslots, -1);
    uint64_t* part = (uint64_t*)s->ws;
    const size_t part_words = (size_t)1216 * PS_MAX * 2;
    uint64_t* sums = part + part_words;
    if ((part_words + 2 * nslots) * sizeof(uint64_t) > s->ws_bytes)
      return fail(QS_ERR_UNSUPPORTED, "Pauli slot sums exceed the workspace");
    static std::once_flag smem_once;
    std::call_once(smem_once, [] {
      cudaFuncSetAttribute(k_pauli_tile<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 16 << PT_TMAX);
      cudaFuncSetAttribute(k_pauli_tile<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 16 << PT_TMAX);
    });
    int next = 0;
    for (const auto& P : passes) {
      PTile g{};
      g.T = (int)P.bm.size();
      g.ntiles = 1ull << (n - g.T);
      for (int q = 0; q < g.T; ++q) {
        g.bm[q] = P.bm[q];
        g.lead[q] = pp_lead(P.bm[q]);
      }
      g.nt = (int)P.sl.size();
      g.nz = 0;
      for (int q = 0; q < g.nt; ++q) {
        const PauliSlot& sl = slots[P.sl[q]];
        gidx[P.sl[q]] = next + q;
        g.zm[q] = sl.zm;
        g.im[q] = (uint8_t)sl.im;
        uint32_t zc = 0;
        for (int t = 0; t < g.T; ++t) zc |= (uint32_t)(__builtin_popcountll(P.bm[t] & sl.zm) & 1) << t;
        g.zc[q] = zc;
        if (!sl.xm) {
          ++g.nz;
          g.xc[q] = 0;
          g.top[q] = 0;
        } else {
          uint32_t xc = 0;
          pp_reduce(P.bm, sl.xm, &xc);
          g.xc[q] = xc;
          g.top[q] = 31 - __builtin_clz(xc);
        }
      }
      const int nblocks = (int)std::min<uint64_t>(3 * 152, g.ntiles);  // three CTAs per SM
      KTimer kt(s, QS_K_REDUCE, n, g.nt, 0, 0, (double)(1ull << n), 8.0 * g.nt * (double)(1ull << n));
      note_launch(2);
      with_amps(s, [&](auto* a) {
        using T = std::remove_cv_t<std::remove_pointer_t<decltype(a)>>;
        k_pauli_tile<T><<<nblocks, 256, (size_t)16 << g.T, s->stream>>>(a, g, part);
        return QS_OK;
      });
      QS_TRY(launch_check("pauli_tile"));
      k_pauli_exact_finish<<<1, 32, 0, s->stream>>>(part, nblocks, g.nt, sums + 2 * (size_t)next);
      QS_TRY(launch_check("pauli_exact_finish"));
      next += g.nt;
    }
    std::vector<uint64_t> hs(2 * nslots);
    if (nslots) QS_TRY(read_back(s, (const double*)sums, 2 * nslots, (double*)hs.data()));
    auto sum_of = [&](int k) {
      const int g2 = gidx[k];
      return ((unsigned __int128)hs[2 * g2 + 1] << 64) | hs[2 * g2];
    };
    for (size_t k = 0; k < nt; ++k) {
      const __int128 d = (__int128)(2 * sum_of(tslot[k]) - sum_of(ttot[k]));
      const double v = (double)tmult[k] * ((double)d * 0x1p-120);
      e += terms[t0 + k].coef * v;
    }
  }
  *out = e;
  return QS_OK;
}

extern "C" int qs_expect_pauli(const qs_state* cs, const qs_pauli* terms, size_t nterms, double* out) {
  clear_error();
  qs_state* s = const_cast<qs_state*>(cs);
  QS_TRY(check_state(s));
  if (!out || (nterms && !terms)) return fail(QS_ERR_INVALID_ARG, "NULL argument");
  const uint64_t full = s->n >= 64 ? ~0ull : ((1ull << s->n) - 1);
  for (size_t k = 0; k < nterms; ++k)
    if ((terms[k].xmask | terms[k].zmask) & ~full) return fail(QS_ERR_INVALID_ARG, "term %zu exceeds n", k);
  QS_TRY(ensure_bound(s));
  if (s->bound == 1) return pauli_exact(s, terms, nterms, out);
  const uint64_t N = 1ull << s->n;
  const int nblocks = (int)std::min<uint64_t>(608, std::max<uint64_t>(1, N / 256));
  double* part = (double*)s->ws;
  double* dres = part + (size_t)nblocks * 8;
  std::vector<double> vals(nterms);
  for (size_t k0 = 0; k0 < nterms; k0 += 8) {
    PauliArgs g;
    g.N = N;
    g.nt = (int)std::min<size_t>(8, nterms - k0);
    for (int k = 0; k < g.nt; ++k) {
      g.xm[k] = terms[k0 + k].xmask;
      g.zm[k] = terms[k0 + k].zmask;
      g.ny[k] = __builtin_popcountll(terms[k0 + k].xmask & terms[k0 + k].zmask) & 3;
    }
    KTimer kt(s, QS_K_REDUCE, s->n, g.nt, 0, 0, (double)N, 4.0 * g.nt * (double)N);
    with_amps(s, [&](auto* a) {
      k_pauli<<<nblocks, 256, 0, s->stream>>>(a, g, part);
      return QS_OK;
    });
    QS_TRY(launch_check("pauli"));
    k_pauli_finish<<<1, 32, 0, s->stream>>>(part, nblocks, g.nt, dres);
    QS_TRY(launch_check("pauli_finish"));
    QS_TRY(read_back(s, dres, g.nt, vals.data() + k0));
  }
  double e = 0.0;
  for (size_t k = 0; k < nterms; ++k) e += terms[k].coef * vals[k];
  *out = e;
  return QS_OK;
}

// ---- <Z_i> without any allocation ------------------------------------------------------
// For callers that cannot allocate device memory (see the declaration in qsim.h):
// the per-CTA partial sums live in this file-scope device array instead of a
// state's workspace.  Its size covers the largest launch of k_expect_z:
// at most 1024 CTAs, each writing r + 1 <= 25 values for n <= 34.
#define QS_NOALLOC_EZ_MIN_QUBITS 8
#define QS_NOALLOC_EZ_MAX_QUBITS 34
#define QS_NOALLOC_EZ_SLOTS (1024 * 25)
static __device__ __align__(256) double g_noalloc_ez_partials[QS_NOALLOC_EZ_SLOTS];

// Register bits r of k_expect_z for n qubits (as the entry point chooses them) and
// the partials a launch writes: 2^(n - r) CTAs, r + 1 values each.
constexpr int noalloc_ez_r(int n) {
  return std::min(std::max(8, n - 10), std::min(n, 8 + ZMAXJ));
}
constexpr bool noalloc_ez_fits() {
  for (int n = QS_NOALLOC_EZ_MIN_QUBITS; n <= QS_NOALLOC_EZ_MAX_QUBITS; ++n)
    if ((1ll << (n - noalloc_ez_r(n))) * (noalloc_ez_r(n) + 1) > QS_NOALLOC_EZ_SLOTS) return false;
  return true;
}
static_assert(noalloc_ez_fits(), "the static partials array must hold the largest launch of its qubit range");

// Device address of g_noalloc_ez_partials (the name itself is only a host-side
// stand-in and must not be passed to a kernel).  Outside stream capture it is
// looked up on every call (cudaGetSymbolAddress allocates nothing), so a context
// that was torn down and created again cannot leave a stale address; during
// capture, when runtime calls may not be allowed, the address of the last call
// on the device is used.
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[64] = {nullptr};

static int noalloc_scratch(cudaStream_t st, double** out) {
  int dev = 0;
  QS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(QS_ERR_UNSUPPORTED, "device ordinal %d", dev);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  QS_CUDA(cudaStreamIsCapturing(st, &cs));
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_ez_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_ez_partials)");
    g_noalloc_ptr[dev] = (double*)p;
  } else if (!g_noalloc_ptr[dev]) {
    return fail(QS_ERR_UNSUPPORTED, "make the first qs_expect_z_all_noalloc call on a device before stream capture");
  }
  *out = g_noalloc_ptr[dev];
  return QS_OK;
}

extern "C" int qs_expect_z_all_noalloc(const double* device_amps, int n, double* device_out, void* stream) {
  clear_error();
  if (!device_amps || !device_out) return fail(QS_ERR_INVALID_ARG, "NULL device pointer");
  if (n < QS_NOALLOC_EZ_MIN_QUBITS || n > QS_NOALLOC_EZ_MAX_QUBITS)
    return fail(QS_ERR_INVALID_ARG, "qs_expect_z_all_noalloc supports %d <= n <= %d qubits (got n=%d)",
                QS_NOALLOC_EZ_MIN_QUBITS, QS_NOALLOC_EZ_MAX_QUBITS, n);
  if ((uintptr_t)device_amps & 15) return fail(QS_ERR_INVALID_ARG, "amplitudes not 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  double* part = nullptr;
  QS_TRY(noalloc_scratch(st, &part));
  const int r = noalloc_ez_r(n);
  const int nblocks = 1 << (n - r);
  note_launch(2);
  // every partial that k_expect_z_finish reads is written first by k_expect_z, so
  // nothing left over from an earlier call is read
  k_expect_z<<<nblocks, 256, 0, st>>>((const double2*)device_amps, r, part);
  QS_TRY(launch_check("expect_z (no-alloc)"));
  k_expect_z_finish<<<1, 64, 0, st>>>(part, nblocks, r, n, device_out);
  return launch_check("expect_z_finish (no-alloc)");
}
