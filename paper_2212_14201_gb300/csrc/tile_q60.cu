// Register-phase tile pass on the Q60 engine (the paper's circuit fusion,
// Section "Quantum circuit fusion", with gate data in fast on-chip memory,
// Section "GPU optimization").
//
// For each tile (2^m amplitudes x = deposit(r, outside bits) | deposit(j, tile
// bits)) the CTA reads the amplitudes once from HBM, converts them to Q60 (two
// int64 per amplitude) and keeps them in shared memory at the swizzled index
// j ^ sw(j).  Each register phase then has every thread load the 16 amplitudes
// of its group (tile index gb | dep(k), k = 0..15 over the phase's four register
// bits), apply the phase's ops to them in registers and store them back; one
// barrier separates phases.  The tile is converted back and written once.
//
// Arithmetic per op (limb products, 3 wide multiply-adds each, fixed.h):
//   PAIR  two real rotations on register bits r0 < r1 as one real 4x4 on quads:
//         16 products per quad and component (the same as the two apart), half the
//         limb splits and roundings;
//   REAL  real 2x2: 4 products per pair and component;
//   GEN   general 2x2, Gauss form: 6 products per output;
//   TABLE a full-tile diagonal, one Gauss-form complex product per amplitude,
//         entries read from L2 in the order the phase's threads use them.
#include <algorithm>

#include "regtile.h"

namespace qs {

__constant__ uint8_t c_rt_swz[16] = {1, 2, 4, 3, 5, 6, 7, 1, 2, 4, 3, 5, 6, 7, 1, 2};  // RP_SWZ

// Physical shared-memory index of a single tile bit b.
__device__ __forceinline__ uint32_t rt_bit_phys(int b) { return (1u << b) ^ (b < 3 ? 0u : (uint32_t)c_rt_swz[b]); }

// Nearest double to V * 2^-60 (round half to even) without branches, integer
// operations only (the FP64 pipe runs at 1/64 of the integer rate).
__device__ __forceinline__ double rt_to_double(int64_t V) {
  const uint64_t s = (uint64_t)(V >> 63);
  const uint64_t a = ((uint64_t)V ^ s) - s;  // |V|; |V| < 2^62 here
  const int lz = __clzll((long long)a);       // 64 for a == 0
  const uint64_t x = a << (lz & 63);          // leading one at bit 63
  uint64_t mant = x >> 11;                    // 53 bits with the leading one
  const uint32_t rem = (uint32_t)x & 0x7FFu;
  mant += (uint64_t)((rem > 0x400u) | ((rem == 0x400u) & (uint32_t)mant & 1u));
  // leading bit 63 - lz of V: biased exponent 1026 - lz; the leading one of mant
  // adds 1 to the exponent field, and a carry to 2^53 adds one more
  const uint64_t bits = ((uint64_t)(1025 - lz) << 52) + mant;
  return a ? __longlong_as_double((long long)((s << 63) | bits)) : 0.0;
}

__device__ __forceinline__ longlong2 rt_load(const double2& x) {
  return make_longlong2(q60_from_double_nb(x.x), q60_from_double_nb(x.y));
}
__device__ __forceinline__ double2 rt_store(const longlong2& v) {
  return make_double2(rt_to_double(v.x), rt_to_double(v.y));
}

// c + i d (table entry as Q60 limbs c.h c.l d.h d.l) times a, Gauss form:
// K1 = c (a_r + a_i), K2 = a_r (d - c), K3 = a_i (c + d); re = K1 - K3, im = K1 + K2.
// The sums of limbs are redundant limb pairs (low limbs in (-2^30, 2^31)); the
// accumulators stay below 8 * 2^60 for |amplitude| <= 1.25.
__device__ __forceinline__ longlong2 rt_tab_mul(const int4 e, const longlong2 a) {
  const QL r = q60_split(a.x), i = q60_split(a.y);
  const QL s{r.h + i.h, r.l + i.l};
  const QL c{e.x, e.y};
  const QL dmc{e.z - e.x, e.w - e.y};
  const QL cpd{e.x + e.z, e.y + e.w};
  QAcc k1 = qacc_new(), k2{0, 0}, k3{0, 0};
  qacc_add(k1, c, s);
  qacc_add(k2, dmc, r);
  qacc_add(k3, cpd, i);
  return make_longlong2(qacc_round(QAcc{k1.hi - k3.hi, k1.mid - k3.mid}),
                        qacc_round(QAcc{k1.hi + k2.hi, k1.mid + k2.mid}));
}

// a times a unit code or a general entry u (re, im, -im limbs, qc_make form)
__device__ __forceinline__ longlong2 rt_mul(const longlong2 a, int code, const QL* u) {
  switch (code) {
    case U_ONE: return a;
    case U_I: return make_longlong2(-a.y, a.x);
    case U_MINUS_ONE: return make_longlong2(-a.x, -a.y);
    case U_MINUS_I: return make_longlong2(a.y, -a.x);
    default: {
      const QL ar = q60_split(a.x), ai = q60_split(a.y);
      const QL ur = u[0], ui = u[1], un = u[2];
      QAcc re = qacc_new(), im = qacc_new();
      qacc_add(re, ur, ar);
      qacc_add(re, un, ai);
      qacc_add(im, ur, ai);
      qacc_add(im, ui, ar);
      return make_longlong2(qacc_round(re), qacc_round(im));
    }
  }
}

// Two real rotations on register bits R0 < R1 as a real 4x4 on the four quads of
// the 16 registers (quad index bit(R0) + 2 bit(R1)); with TAB the table entries
// of the quad multiply first.
template <int R0, int R1, bool TAB>
__device__ __forceinline__ void rt_pair(longlong2 (&v)[16], const QL* __restrict__ c, const int4* __restrict__ tab) {
  constexpr int S0 = 1 << R0, S1 = 1 << R1;
#pragma unroll
  for (int k0 = 0; k0 < 16; ++k0) {
    if (k0 & (S0 | S1)) continue;
    const int kk[4] = {k0, k0 | S0, k0 | S1, k0 | S0 | S1};
    QL r[4], im[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      longlong2 x = v[kk[q]];
      if (TAB) x = rt_tab_mul(__ldg(tab + kk[q]), x);
      r[q] = q60_split(x.x);
      im[q] = q60_split(x.y);
    }
#pragma unroll
    for (int row = 0; row < 4; ++row) {
      QAcc xr = qacc_new(), xi = qacc_new();
#pragma unroll
      for (int col = 0; col < 4; ++col) {
        const QL u = c[4 * row + col];
        qacc_add(xr, u, r[col]);
        qacc_add(xi, u, im[col]);
      }
      v[kk[row]] = make_longlong2(qacc_round(xr), qacc_round(xi));
    }
  }
}

template <int R>
__device__ __forceinline__ void rt_real(longlong2 (&v)[16], const QL* __restrict__ c, uint32_t cr) {
  constexpr int S = 1 << R;
  const QL m00 = c[0], m01 = c[1], m10 = c[2], m11 = c[3];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (k & S) continue;
    if (((uint32_t)k & cr) != cr) continue;
    const longlong2 a0 = v[k], a1 = v[k | S];
    const QL r0 = q60_split(a0.x), i0 = q60_split(a0.y), r1 = q60_split(a1.x), i1 = q60_split(a1.y);
    QAcc x = qacc_new(), y = qacc_new(), z = qacc_new(), w = qacc_new();
    qacc_add(x, m00, r0);
    qacc_add(x, m01, r1);
    qacc_add(y, m00, i0);
    qacc_add(y, m01, i1);
    qacc_add(z, m10, r0);
    qacc_add(z, m11, r1);
    qacc_add(w, m10, i0);
    qacc_add(w, m11, i1);
    v[k] = make_longlong2(qacc_round(x), qacc_round(y));
    v[k | S] = make_longlong2(qacc_round(z), qacc_round(w));
  }
}

template <int R>
__device__ __forceinline__ void rt_gen(longlong2 (&v)[16], const QL* __restrict__ c, uint32_t cr) {
  constexpr int S = 1 << R;
  const QC u0{c[0], c[1], c[2]}, u1{c[3], c[4], c[5]}, u2{c[6], c[7], c[8]}, u3{c[9], c[10], c[11]};
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (k & S) continue;
    if (((uint32_t)k & cr) != cr) continue;
    const longlong2 a0 = v[k], a1 = v[k | S];
    const QL r0 = q60_split(a0.x), i0 = q60_split(a0.y), r1 = q60_split(a1.x), i1 = q60_split(a1.y);
    const QL s0 = q60_split(a0.x + a0.y), s1 = q60_split(a1.x + a1.y);
    int64_t re, im;
    q60_gauss_row(u0, u1, r0, i0, s0, r1, i1, s1, &re, &im);
    v[k] = make_longlong2(re, im);
    q60_gauss_row(u2, u3, r0, i0, s0, r1, i1, s1, &re, &im);
    v[k | S] = make_longlong2(re, im);
  }
}

// Antidiagonal (kind 0), diagonal (1) or |1>-phase (2) op on register bit R.
template <int R>
__device__ __forceinline__ void rt_unit(longlong2 (&v)[16], const RtOp& op, const QL* __restrict__ c, int form) {
  constexpr int S = 1 << R;
  const uint32_t cr = op.cr;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (k & S) continue;
    if (((uint32_t)k & cr) != cr) continue;
    if (form == 0) {
      const longlong2 a0 = v[k], a1 = v[k | S];
      v[k] = rt_mul(a1, op.code0, c + 3);
      v[k | S] = rt_mul(a0, op.code1, c + 6);
    } else {
      if (form == 1) v[k] = rt_mul(v[k], op.code0, c);
      v[k | S] = rt_mul(v[k | S], op.code1, c + 9);
    }
  }
}

template <int R>
__device__ __forceinline__ void rt_single(longlong2 (&v)[16], const RtOp& op, const QL* __restrict__ c) {
  switch (op.kind) {
    case RK_REAL: rt_real<R>(v, c, op.cr); break;
    case RK_GEN: rt_gen<R>(v, c, op.cr); break;
    case RK_ANTI: rt_unit<R>(v, op, c, 0); break;
    case RK_DIAG: rt_unit<R>(v, op, c, 1); break;
    default: rt_unit<R>(v, op, c, 2); break;
  }
}

template <bool TAB>
__device__ __forceinline__ void rt_pair_any(longlong2 (&v)[16], int r0, int r1, const QL* __restrict__ c,
                                            const int4* __restrict__ tab) {
  switch (r0 * 4 + r1) {
    case 1: rt_pair<0, 1, TAB>(v, c, tab); break;
    case 2: rt_pair<0, 2, TAB>(v, c, tab); break;
    case 3: rt_pair<0, 3, TAB>(v, c, tab); break;
    case 6: rt_pair<1, 2, TAB>(v, c, tab); break;
    case 7: rt_pair<1, 3, TAB>(v, c, tab); break;
    default: rt_pair<2, 3, TAB>(v, c, tab); break;
  }
}

#ifndef QS_RT_MINB
#define QS_RT_MINB 1
#endif

template <int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS >= 256 ? QS_RT_MINB : 1)
    k_tile_q60(double2* __restrict__ a, const __grid_constant__ RtArgs g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = g.m;
  const uint32_t TS = 1u << m;
  const uint32_t H = 1u << g.nhigh;
  const int L = m - g.nhigh;
  const uint32_t lowmask = (1u << L) - 1;
  const uint32_t tid = threadIdx.x;
  const uint32_t G = TS >> 4;  // groups of 16 amplitudes: one per thread
  uint64_t* offs = reinterpret_cast<uint64_t*>(smem_raw);                 // [H] offsets of the high tile bits
  uint8_t* swt = reinterpret_cast<uint8_t*>(smem_raw + (size_t)H * 8);    // [TS / 8] swizzle of j >> 3
  longlong2* tile = reinterpret_cast<longlong2*>(smem_raw + (((size_t)H * 8 + (TS >> 3) + 15) & ~(size_t)15));
  for (uint32_t h = tid; h < H; h += THREADS) {
    uint64_t o = 0;
    for (int b = 0; b < g.nhigh; ++b) o |= (uint64_t)((h >> b) & 1u) << g.qhigh[b];
    offs[h] = o;
  }
  for (uint32_t h = tid; h < (TS >> 3); h += THREADS) {
    uint32_t sw = 0;
    for (int b = 0; b + 3 < m; ++b)
      if ((h >> b) & 1u) sw ^= c_rt_swz[b + 3];
    swt[h] = (uint8_t)sw;
  }
  const int ngb = m - 4;
  for (uint64_t r = blockIdx.x; r < g.ntiles; r += gridDim.x) {
    uint64_t base = 0;
    for (int b = 0; b < g.nout; ++b) base |= ((r >> b) & 1ull) << g.outpos[b];
    __syncthreads();  // offs / swt ready; the previous tile's store has read the tile
    for (uint32_t j = tid; j < TS; j += THREADS)
      tile[j ^ swt[j >> 3]] = rt_load(a[base + offs[j >> L] + (j & lowmask)]);
    __syncthreads();
    for (int p = 0; p < g.nphases; ++p) {
      if (tid < G) {
        const RtPhase& ph = g.phases[p];
        uint32_t gb = 0;
        for (int i = 0; i < ngb; ++i) gb |= ((tid >> i) & 1u) << ph.gl[i];
        const uint32_t sb = gb ^ swt[gb >> 3];
        const uint32_t d0 = rt_bit_phys(ph.rb[0]), d1 = rt_bit_phys(ph.rb[1]), d2 = rt_bit_phys(ph.rb[2]),
                       d3 = rt_bit_phys(ph.rb[3]);
        longlong2 v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const uint32_t dk = ((k & 1) ? d0 : 0u) ^ ((k & 2) ? d1 : 0u) ^ ((k & 4) ? d2 : 0u) ^ ((k & 8) ? d3 : 0u);
          v[k] = tile[sb ^ dk];
        }
        for (int o = ph.op_begin; o < ph.op_end; ++o) {
          const RtOp& op = g.ops[o];
          if ((base & op.ext) != op.ext) continue;  // uniform across the CTA
          if ((gb & op.gmask) != op.gmask) continue;
          const QL* c = g.coef + op.coef;
          const int kind = op.kind;
          if (kind == RK_PAIR) {
            if (op.table >= 0)
              rt_pair_any<true>(v, op.r0, op.r1, c, g.tables + ((size_t)op.table << m) + (size_t)tid * 16);
            else
              rt_pair_any<false>(v, op.r0, op.r1, c, nullptr);
          } else if (kind == RK_TABLE) {
            const int4* tab = g.tables + ((size_t)op.table << m) + (size_t)tid * 16;
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = rt_tab_mul(__ldg(tab + k), v[k]);
          } else if (kind == RK_SCAL) {
            const uint32_t bit = op.sout ? (uint32_t)((base >> op.sbit) & 1ull) : ((gb >> op.sbit) & 1u);
            const int code = bit ? op.code1 : op.code0;
            if (code == U_ONE) continue;
            const QL* u = c + (bit ? 9 : 0);
            const uint32_t cr = op.cr;
#pragma unroll
            for (int k = 0; k < 16; ++k)
              if (((uint32_t)k & cr) == cr) v[k] = rt_mul(v[k], code, u);
          } else {
            switch (op.r0) {
              case 0: rt_single<0>(v, op, c); break;
              case 1: rt_single<1>(v, op, c); break;
              case 2: rt_single<2>(v, op, c); break;
              default: rt_single<3>(v, op, c); break;
            }
          }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const uint32_t dk = ((k & 1) ? d0 : 0u) ^ ((k & 2) ? d1 : 0u) ^ ((k & 4) ? d2 : 0u) ^ ((k & 8) ? d3 : 0u);
          tile[sb ^ dk] = v[k];
        }
      }
      __syncthreads();
    }
    for (uint32_t j = tid; j < TS; j += THREADS)
      a[base + offs[j >> L] + (j & lowmask)] = rt_store(tile[j ^ swt[j >> 3]]);
  }
}

template <int THREADS>
static int launch_rt(qs_state* s, const RtArgs& g, size_t smem) {
  static int sms = 0;
  static bool attr = false;
  if (!attr) {
    QS_CUDA(cudaFuncSetAttribute(k_tile_q60<THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
    attr = true;
  }
  int per_sm = 0;
  QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_q60<THREADS>, THREADS, smem));
  const uint64_t grid = std::min<uint64_t>(g.ntiles, (uint64_t)std::max(1, sms) * std::max(1, per_sm));
  k_tile_q60<THREADS><<<(unsigned)grid, THREADS, smem, s->stream>>>(s->amps, g);
  return launch_check("register tile kernel");
}

int launch_tile_q60(qs_state* s, const RtArgs& g, double int_ops, int ngates, uint64_t qmask) {
  if (g.m < RT_MIN_M || g.m > RT_MAX_M) return fail(QS_ERR_INVALID_ARG, "internal: register tile width %d", g.m);
  const size_t TS = (size_t)1 << g.m, H = (size_t)1 << g.nhigh;
  const size_t smem = ((H * 8 + (TS >> 3) + 15) & ~(size_t)15) + TS * 16;
  KTimer kt(s, QS_K_TILE, g.m, ngates, qmask, 0, (double)(1ull << g.n), 0.0, int_ops);
  const size_t groups = TS >> 4;
  if (groups > 128) return launch_rt<256>(s, g, smem);
  if (groups > 64) return launch_rt<128>(s, g, smem);
  if (groups > 32) return launch_rt<64>(s, g, smem);
  return launch_rt<32>(s, g, smem);
}

}  // namespace qs
