// Computational-basis sampling (measure_all / run_with_configuration in the
// paper's API) with a bit-reproducible definition:
//   u_s  = (SplitMix64 output s of the stream seeded `seed` >> 11) * 2^-53
//          (Steele, Lea & Flood 2014; counter form: state = seed + (s+1)*gamma);
//   p_x  = re*re + im*im, each product and the sum rounded separately;
//   L    = min(1024, 2^n); T_b = p_{bL} + ... + p_{bL+L-1} summed left to right;
//   G    = min(1024, number of blocks); superblock c holds blocks [cG, cG + G);
//   F_c(i) = T_{cG} + ... + T_{cG+i} left to right; P_0 = 0, P_{c+1} = P_c + F_c(G-1);
//   E_0 = 0, E_{cG+i+1} = P_c + F_c(i)  (for n <= 20: E_{b+1} = E_b + T_b);
//   shot s -> smallest x in the first block b with E_{b+1} > u_s such that
//             E_b + (left-to-right partial sum of block b up to x) > u_s;
//             if no block qualifies, the largest x with p_x > 0.
// Kernels: block totals (one thread per block, sequential; the running sum is
// also kept after every K = min(32, L) amplitudes), the superblock prefixes (one
// CTA per superblock, its sequential sum staged through shared memory), the
// prefix of the superblock totals (one CTA), the offset of every superblock's
// prefixes, and one thread per shot (binary search over E, then over the block's
// running-sum checkpoints, then a sequential scan of at most K amplitudes that
// continues the block's left-to-right sum from the checkpoint before them: the
// same additions in the same order as a scan from the block's start).
#include <algorithm>

#include "ieee_sq.h"
#include "internal.h"

namespace qs {

__device__ __forceinline__ double p_exact(double2 a) { return __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y)); }

// T[b] = left-to-right block total; lastnz[b] = largest x in block b with p_x > 0,
// or -1; cp[b * (L / K) + m] = the running sum after amplitude (m + 1) K - 1 of the
// block (K = min(32, L); the last checkpoint is T[b]).
template <class A>
__global__ void k_block_totals(const A* __restrict__ a, int64_t nb, int64_t L, int64_t K, double* __restrict__ T,
                               long long* __restrict__ lastnz, double* __restrict__ cp) {
  const int64_t M = L / K;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    const A* p = a + b * L;
    double S = 0.0;
    long long last = -1;
    for (int64_t j = 0; j < L; j += 4) {
      const double2 v[4] = {ld_amp(p, j), ld_amp(p, j + 1 < L ? j + 1 : j), ld_amp(p, j + 2 < L ? j + 2 : j),
                            ld_amp(p, j + 3 < L ? j + 3 : j)};
      // p = fl(fl(re^2) + fl(im^2)) on the integer pipes (bit-identical to the FP64
      // operations) when every component of the four is in range; else, for the
      // whole warp, on the FP64 pipe (one vote, so the fallback is a real branch)
      double pq[4];
      bool ok = true;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        bool o1, o2, o3 = true;
        const double sr = sq_rn_int(v[k].x, &o1), si = sq_rn_int(v[k].y, &o2);
        // the sum on the integer pipes for half of the amplitudes, on the FP64 pipe
        // for the other half: the two pipes then finish together
        pq[k] = (k & 1) ? __dadd_rn(sr, si) : add_rn_pos_int(sr, si, &o3);
        ok = ok && o1 && o2 && o3;
      }
      if (!__all_sync(__activemask(), ok)) {
#pragma unroll
        for (int k = 0; k < 4; ++k) pq[k] = p_exact(v[k]);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (k == 0 || j + k < L) {
          const double q = pq[k];
          S = __dadd_rn(S, q);
          if (q_bits(q) != 0) last = b * L + j + k;  // q >= +0: a nonzero bit pattern is q > 0
        }
      }
      if (K >= 4 && ((j + 4) & (K - 1)) == 0 && j + 4 < L) cp[b * M + (j + 4) / K - 1] = S;
    }
    T[b] = S;
    cp[b * M + M - 1] = S;
    lastnz[b] = last;
  }
}

// One CTA per segment c of G entries of T (a superblock of blocks, or the
// superblock totals): out[c*G + i + 1] = T[c*G] + ... + T[c*G + i], left to right;
// tot[c] = the segment's total; lmax[c] = max of lastnz over the segment.  CTA 0
// also writes out[0] = 0.  The operands are staged through shared memory in
// chunks so the one thread that adds waits only on its own additions.
constexpr int kSegMax = 1024;
__global__ void k_seg_prefix(const double* __restrict__ T, int64_t G, double* __restrict__ out,
                             double* __restrict__ tot, const long long* __restrict__ lastnz,
                             long long* __restrict__ lmax) {
  __shared__ double buf[kSegMax];
  __shared__ long long wmax[32];
  __shared__ double carry;
  const int64_t c0 = (int64_t)blockIdx.x * G;
  long long lm = -1;
  if (threadIdx.x == 0) carry = 0.0;
  for (int64_t k0 = 0; k0 < G; k0 += kSegMax) {
    const int cnt = (int)min((int64_t)kSegMax, G - k0);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      buf[i] = T[c0 + k0 + i];
      lm = max(lm, lastnz[c0 + k0 + i]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double e = carry;
      int i = 0;
      for (; i + 8 <= cnt; i += 8) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = buf[i + k];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          e = __dadd_rn(e, v[k]);
          v[k] = e;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) buf[i + k] = v[k];
      }
      for (; i < cnt; ++i) {
        e = __dadd_rn(e, buf[i]);
        buf[i] = e;
      }
      carry = e;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) out[c0 + k0 + i + 1] = buf[i];
    __syncthreads();
  }
  // the largest nonzero index: a max (any order gives the same)
  for (int o = 16; o > 0; o >>= 1) lm = max(lm, __shfl_xor_sync(0xffffffffu, lm, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = lm;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long l = -1;
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) l = max(l, wmax[wv]);
    lmax[blockIdx.x] = l;
    tot[blockIdx.x] = carry;
    if (blockIdx.x == 0) out[0] = 0.0;
  }
}

// E[b + 1] = P[b / G] + E[b + 1] for the blocks of superblocks 1, 2, ... (superblock
// 0 has P = 0); lastnz[nb] = the last nonzero index (0 for the zero vector).
__global__ void k_seg_offset(double* __restrict__ E, int64_t nb, int G, const double* __restrict__ P,
                             const long long* __restrict__ lall, long long* __restrict__ lastnz) {
  for (int64_t b = G + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x)
    E[b + 1] = __dadd_rn(P[b / G], E[b + 1]);
  if (blockIdx.x == 0 && threadIdx.x == 0) lastnz[nb] = lall[0] < 0 ? 0 : lall[0];
}

template <class A>
__global__ void k_sample(const A* __restrict__ a, const double* __restrict__ E, const long long* __restrict__ lastnz,
                         const double* __restrict__ cp, int64_t nb, int64_t L, int64_t K, uint64_t seed,
                         uint64_t shots, uint64_t* __restrict__ out) {
  const int64_t M = L / K;
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < shots; s += (uint64_t)gridDim.x * blockDim.x) {
    double u = u01_of(splitmix64(seed, s));
    int64_t lo = 0, hi = nb;
    while (lo < hi) {
      int64_t mid = lo + ((hi - lo) >> 1);
      if (E[mid + 1] > u) hi = mid;
      else lo = mid + 1;
    }
    if (lo == nb) {
      out[s] = (uint64_t)lastnz[nb];
      continue;
    }
    const int64_t b = lo;
    const double eb = E[b];
    const double* c = cp + b * M;
    // first K-run whose end passes u (E_b + running sum is nondecreasing in x)
    int64_t lo2 = 0, hi2 = M;
    while (lo2 < hi2) {
      const int64_t mid = lo2 + ((hi2 - lo2) >> 1);
      if (__dadd_rn(eb, c[mid]) > u) hi2 = mid;
      else lo2 = mid + 1;
    }
    int64_t pick = b * L + L - 1;
    if (lo2 < M) {
      const A* p = a + b * L;
      double S = lo2 ? c[lo2 - 1] : 0.0;
      for (int64_t j = lo2 * K; j < lo2 * K + K; ++j) {
        S = __dadd_rn(S, p_exact(ld_amp(p, j)));
        if (__dadd_rn(eb, S) > u) {
          pick = b * L + j;
          break;
        }
      }
    }
    out[s] = (uint64_t)pick;
  }
}

}  // namespace qs

using namespace qs;

extern "C" int qs_sample(const qs_state* cs, uint64_t seed, uint64_t shots, uint64_t* out, int on_device) {
  clear_error();
  qs_state* s = const_cast<qs_state*>(cs);
  QS_TRY(check_state(s));
  if (shots == 0) return QS_OK;
  if (!out) return fail(QS_ERR_INVALID_ARG, "out is NULL");
  const int64_t N = (int64_t)1 << s->n;
  const int64_t L = N < 1024 ? N : 1024;
  const int64_t nb = N / L;
  const int64_t G = nb < kSegMax ? nb : kSegMax;  // blocks per superblock
  const int64_t nsb = nb / G;                      // superblocks (nb, G powers of two)
  double* T = (double*)s->ws;
  double* E = T + (nb + 1);
  long long* lastnz = (long long*)(E + (nb + 1));
  double* Ssb = (double*)(lastnz + (nb + 1));  // superblock totals
  double* P = Ssb + (nsb + 1);                 // superblock prefixes
  long long* lsb = (long long*)(P + (nsb + 1));
  long long* lall = lsb + (nsb + 1);
  const int64_t K = L < 32 ? L : 32;  // amplitudes per running-sum checkpoint
  struct StreamBuf {                   // freed on the stream when the call returns
    void* p = nullptr;
    cudaStream_t st;
    ~StreamBuf() {
      if (p) cudaFreeAsync(p, st);
    }
  } cpb{nullptr, s->stream};
  QS_CUDA(dmalloc_async(&cpb.p, (size_t)(N / K) * sizeof(double), s->stream));  // 1/64 of the state's bytes
  double* cp = (double*)cpb.p;
  int g1 = (int)std::min<int64_t>((nb + 127) / 128, 152 * 16);
  KTimer kt(s, QS_K_REDUCE, s->n, 3, 0, 0, (double)N, 4.0 * (double)N);
  note_launch(4);
  with_amps(s, [&](auto* a) {
    k_block_totals<<<g1, 128, 0, s->stream>>>(a, nb, L, K, T, lastnz, cp);
    return QS_OK;
  });
  QS_TRY(launch_check("block_totals"));
  k_seg_prefix<<<(unsigned)nsb, 128, 0, s->stream>>>(T, G, E, Ssb, lastnz, lsb);
  QS_TRY(launch_check("superblock prefix"));
  k_seg_prefix<<<1, 128, 0, s->stream>>>(Ssb, nsb, P, Ssb + nsb, lsb, lall);
  QS_TRY(launch_check("superblock totals prefix"));
  const int g2 = (int)std::max<int64_t>(1, std::min<int64_t>((nb + 255) / 256, 152 * 8));
  k_seg_offset<<<g2, 256, 0, s->stream>>>(E, nb, (int)G, P, lall, lastnz);
  QS_TRY(launch_check("superblock offset"));
  uint64_t* dout = out;
  if (!on_device) {
    const cudaError_t e = dmalloc_async((void**)&dout, shots * sizeof(uint64_t), s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(samples)");
  }
  int g3 = (int)std::min<uint64_t>((shots + 127) / 128, 152 * 16);
  with_amps(s, [&](auto* a) {
    k_sample<<<g3, 128, 0, s->stream>>>(a, E, lastnz, cp, nb, L, K, seed, shots, dout);
    return QS_OK;
  });
  int rc = launch_check("sample");
  if (!on_device) {
    if (rc == QS_OK) {
      cudaError_t e = cudaMemcpyAsync(out, dout, shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, s->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
      if (e != cudaSuccess) rc = cuda_fail(e, "sample readback");
    }
    cudaFreeAsync(dout, s->stream);
  }
  return rc;
}
