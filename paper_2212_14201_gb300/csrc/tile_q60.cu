// Register-phase tile pass on the Q60 engine (the paper's circuit fusion,
// Section "Quantum circuit fusion", with gate data in fast on-chip memory,
// Section "GPU optimization").
//
// For each tile (2^m amplitudes x = deposit(r, outside bits) | deposit(j, tile
// bits)) the CTA reads the amplitudes once from HBM, converts them to Q60 (two
// int64 per amplitude) and keeps them in shared memory at the swizzled index
// j ^ sw(j).  In a register phase every thread owns the 16 amplitudes of its
// group (tile index gb | dep(k), k = 0..15 over the phase's four register bits);
// the phase's runs stream the group's four quads through registers, each quad
// loaded once per run and taken through every op of the run.  One barrier
// separates phases; the tile is converted back and written once.
//
// Arithmetic per op (limb products, 3 wide multiply-adds each, fixed.h):
//   PAIR  two real rotations on the run's bits as two complex products on the
//         quad (q60pair.cuh): 8 products per quad and component, half of what
//         the two rotations cost apart;
//   REAL  real 2x2: 4 products per pair and component;
//   GEN   general 2x2, Gauss form: 6 products per output;
//   TABLE a full-tile diagonal, one Gauss-form complex product per amplitude,
//         entries read from L2 in the order the phase's threads use them.
#include <algorithm>

#include "q60pair.cuh"
#include "regtile.h"

namespace qs {

__constant__ uint8_t c_rt_swz[16] = {1, 2, 4, 3, 5, 6, 7, 1, 2, 4, 3, 5, 6, 7, 1, 2};  // RP_SWZ

// Physical shared-memory index of a single tile bit b.
__device__ __forceinline__ uint32_t rt_bit_phys(int b) { return (1u << b) ^ (b < 3 ? 0u : (uint32_t)c_rt_swz[b]); }

__device__ __forceinline__ longlong2 rt_load(const double2& x) {
  return make_longlong2(q60_from_double_nb(x.x), q60_from_double_nb(x.y));
}
__device__ __forceinline__ double2 rt_store(const longlong2& v) {
  return make_double2(q60_to_double_nb(v.x), q60_to_double_nb(v.y));
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

// A quad in registers: a[i] is register index kk[i] of the group, quad index
// i = bit(run r0) + 2 bit(run r1).
struct RtQuad {
  longlong2 a[4];
  uint32_t kk[4];
};

__device__ __forceinline__ void rt_q_pair(RtQuad& q, const QL* __restrict__ c, int flags, const int4* __restrict__ tab) {
  if (tab) {
#pragma unroll
    for (int i = 0; i < 4; ++i) q.a[i] = rt_tab_mul(__ldg(tab + q.kk[i]), q.a[i]);
  }
  q60_pair_quad(q.a[0], q.a[1], q.a[2], q.a[3], c, flags);
}

// A one-qubit op on the amplitude pair (a0, a1) = (bit 0, bit 1 of its target).
__device__ __forceinline__ void rt_2x2(longlong2& a0, longlong2& a1, const RtOp& op, const QL* __restrict__ c) {
  switch (op.kind) {
    case RK_REAL: {
      const QL r0 = q60_split(a0.x), i0 = q60_split(a0.y), r1 = q60_split(a1.x), i1 = q60_split(a1.y);
      QAcc x = qacc_new(), y = qacc_new(), z = qacc_new(), w = qacc_new();
      qacc_add(x, c[0], r0);
      qacc_add(x, c[1], r1);
      qacc_add(y, c[0], i0);
      qacc_add(y, c[1], i1);
      qacc_add(z, c[2], r0);
      qacc_add(z, c[3], r1);
      qacc_add(w, c[2], i0);
      qacc_add(w, c[3], i1);
      a0 = make_longlong2(qacc_round(x), qacc_round(y));
      a1 = make_longlong2(qacc_round(z), qacc_round(w));
      break;
    }
    case RK_GEN: {
      const QL r0 = q60_split(a0.x), i0 = q60_split(a0.y), r1 = q60_split(a1.x), i1 = q60_split(a1.y);
      const QL s0 = q60_split(a0.x + a0.y), s1 = q60_split(a1.x + a1.y);
      const QC u0{c[0], c[1], c[2]}, u1{c[3], c[4], c[5]}, u2{c[6], c[7], c[8]}, u3{c[9], c[10], c[11]};
      int64_t re, im;
      q60_gauss_row(u0, u1, r0, i0, s0, r1, i1, s1, &re, &im);
      const longlong2 b0 = make_longlong2(re, im);
      q60_gauss_row(u2, u3, r0, i0, s0, r1, i1, s1, &re, &im);
      a0 = b0;
      a1 = make_longlong2(re, im);
      break;
    }
    case RK_ANTI: {
      const longlong2 x0 = a0;
      a0 = rt_mul(a1, op.code0, c + 3);
      a1 = rt_mul(x0, op.code1, c + 6);
      break;
    }
    case RK_DIAG:
      a0 = rt_mul(a0, op.code0, c);
      a1 = rt_mul(a1, op.code1, c + 9);
      break;
    default:  // RK_PH1
      a1 = rt_mul(a1, op.code1, c + 9);
      break;
  }
}

__device__ __forceinline__ void rt_q_op(RtQuad& q, const RtOp& op, const QL* __restrict__ c, const int4* tab0,
                                        uint64_t base, uint32_t gb) {
  const uint32_t cr = op.cr;
  switch (op.kind) {
    case RK_PAIR:
      rt_q_pair(q, c, op.role, op.table >= 0 ? tab0 : nullptr);
      break;
    case RK_TABLE: {
#pragma unroll
      for (int i = 0; i < 4; ++i) q.a[i] = rt_tab_mul(__ldg(tab0 + q.kk[i]), q.a[i]);
      break;
    }
    case RK_SCAL: {
      const uint32_t bit = op.sout ? (uint32_t)((base >> op.sbit) & 1ull) : ((gb >> op.sbit) & 1u);
      const int code = bit ? op.code1 : op.code0;
      const QL* u = c + (bit ? 9 : 0);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if ((q.kk[i] & cr) == cr) q.a[i] = rt_mul(q.a[i], code, u);
      break;
    }
    default:
      if (op.role == 0) {
        if ((q.kk[0] & cr) == cr) rt_2x2(q.a[0], q.a[1], op, c);
        if ((q.kk[2] & cr) == cr) rt_2x2(q.a[2], q.a[3], op, c);
      } else {
        if ((q.kk[0] & cr) == cr) rt_2x2(q.a[0], q.a[2], op, c);
        if ((q.kk[1] & cr) == cr) rt_2x2(q.a[1], q.a[3], op, c);
      }
      break;
  }
}

#ifndef QS_RT_MINB
#define QS_RT_MINB 3
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
  // this thread's slice of every table (entry k at + k)
  const int4* tab_t = g.tables + (size_t)tid * 16;
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
        const uint32_t p0 = rt_bit_phys(ph.rb[0]), p1 = rt_bit_phys(ph.rb[1]), p2 = rt_bit_phys(ph.rb[2]),
                       p3 = rt_bit_phys(ph.rb[3]);
        auto dsel = [&](int i) { return i == 0 ? p0 : (i == 1 ? p1 : (i == 2 ? p2 : p3)); };
        for (int u = ph.run_begin; u < ph.run_end; ++u) {
          const RtRun run = g.runs[u];
          const int r0 = run.r0, r1 = run.r1;
          const int o0 = (r0 != 0 && r1 != 0) ? 0 : ((r0 != 1 && r1 != 1) ? 1 : 2);
          const int o1 = 6 - r0 - r1 - o0;
          const uint32_t d0 = dsel(r0), d1 = dsel(r1), e0 = dsel(o0), e1 = dsel(o1);
          const uint32_t k0 = 1u << r0, k1 = 1u << r1, f0 = 1u << o0, f1 = 1u << o1;
#pragma unroll 1
          for (int qi = 0; qi < 4; ++qi) {
            const uint32_t ob = sb ^ ((qi & 1) ? e0 : 0u) ^ ((qi & 2) ? e1 : 0u);
            const uint32_t kq = ((qi & 1) ? f0 : 0u) | ((qi & 2) ? f1 : 0u);
            RtQuad q;
            const uint32_t ad[4] = {ob, ob ^ d0, ob ^ d1, ob ^ d0 ^ d1};
            q.kk[0] = kq;
            q.kk[1] = kq | k0;
            q.kk[2] = kq | k1;
            q.kk[3] = kq | k0 | k1;
#pragma unroll
            for (int i = 0; i < 4; ++i) q.a[i] = tile[ad[i]];
            for (int o = run.op_begin; o < run.op_end; ++o) {
              const RtOp& op = g.ops[o];
              if ((base & op.ext) != op.ext) continue;  // uniform across the CTA
              if ((gb & op.gmask) != op.gmask) continue;
              rt_q_op(q, op, g.coef + op.coef, tab_t + ((size_t)(op.table < 0 ? 0 : op.table) << m), base, gb);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) tile[ad[i]] = q.a[i];
          }
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
