// Shared Q60 tile machinery of the batched and the single-state adjoint passes:
// op descriptors in global memory, tile ops on int64 (Q60) amplitude pairs, and the
// generator inner product Im <lambda| G |psi> over a tile.
#pragma once

#include <string.h>

#include <vector>

#include "fixed.h"
#include "internal.h"

namespace qs {

constexpr int BT_THREADS = 256;
constexpr int BT_M = 11;          // tile qubits: psi and lambda tiles of 2^11 x 16 B
constexpr int BT_MAX_OPS = 128;   // ops (and gradient slots) per pass: keeps 3 CTAs per SM
constexpr int BT_MAX_N = 24;
constexpr int BT_OFFS = 1 << (BT_M - 3);  // high-bit offset table: tiles hold qubits 0..2 (or all of n < 3)

// BK_DGROUP: a group of up to four uncontrolled diagonal gates on distinct tile
// qubits, run as one op: amplitude j gets E[idx], idx = the member target bits
// of j (member m at bit m), E = the product of the members' diagonals (16 entries
// per group, Gauss form).  The members follow the head as BK_MEMBER records
// (nothing to run on their own) and keep their generator slots.
// BK_RPAIR: two uncontrolled real ops on distinct tile qubits a (first member)
// and b, run as one real 4x4 M = R_b (x) R_a on the quads (j, j|a, j|b, j|a|b)
// (entries row-major, quad index 2*bit(b) + bit(a); 16 limb pairs per pair,
// gate = pair index); in the backward sweep the op also takes both members'
// generator terms from the quads it has loaded.
enum : int8_t { BK_SCALAR = 9, BK_DGROUP = 10, BK_MEMBER = 11, BK_RPAIR = 12 };
constexpr int BT_DG_MAX = 4;  // members per group
enum : int8_t { BG_NONE = 0, BG_X = 1, BG_Y = 2, BG_Z = 3, BG_P = 4 };

struct BPass {
  int m, nhigh, nout, op_begin, op_end, nslots;
  int qhigh[16];
  int outpos[32];
};

struct BOp {
  uint64_t ext;     // controls outside the tile
  uint32_t lcm;     // controls inside the tile (local bits)
  int gate;         // global gate index (matrix tables)
  int param;        // global parameter index, or -1
  double gsign;     // generator sign (-1 for a dagger record)
  int16_t slot;     // gradient slot within the pass, or -1
  int8_t kf, kb;    // op class forward / adjoint
  int8_t tb;        // local target bit (global target bit for SCALAR)
  int8_t gen;
  int8_t c0f, c1f, c0b, c1b;
  int8_t nmem;      // BK_DGROUP head: members following it (gate = group index)
};

// Diagonal group (see BK_DGROUP): a_j *= E[idx(j)].
static __device__ void bt_apply_dgroup(longlong2* tile, uint32_t TS, const BOp* mem, int nm, const QC* E) {
  int tbs[BT_DG_MAX];
#pragma unroll
  for (int m = 0; m < BT_DG_MAX; ++m) tbs[m] = m < nm ? mem[m].tb : 0;
  for (uint32_t j = threadIdx.x; j < TS; j += BT_THREADS) {
    uint32_t idx = 0;
#pragma unroll
    for (int m = 0; m < BT_DG_MAX; ++m)
      if (m < nm) idx |= ((j >> tbs[m]) & 1u) << m;
    const QC u = E[idx];
    const longlong2 a = tile[j];
    int64_t re, im;
    q60_gauss_mul(u, q60_split(a.x), q60_split(a.y), q60_split(a.x + a.y), &re, &im);
    tile[j] = make_longlong2(re, im);
  }
}

// One output component of the 4x4 real M (row k) on four split inputs.
__device__ __forceinline__ int64_t bt_row4(const QL* M, int k, const QL* x) {
  QAcc acc = qacc_new();
#pragma unroll
  for (int c = 0; c < 4; ++c) qacc_add(acc, M[4 * k + c], x[c]);
  return qacc_round(acc);
}

// Generator term of one pair (amplitudes 0 and 1 of the pair) for generator `gen`,
// as the signed products of bt_gen_partial, exactly in Q60 units.
__device__ __forceinline__ int64_t bt_pair_gen(int gen, QL l0x, QL l0y, QL l1x, QL l1y, QL p0x, QL p0y, QL p1x,
                                               QL p1y) {
  QAccF pos{0, 0, 0}, neg{0, 0, 0};
  switch (gen) {
    case BG_X:  // l0x p1y - l0y p1x + l1x p0y - l1y p0x
      qaccf_add(pos, l0x, p1y); qaccf_add(neg, l0y, p1x); qaccf_add(pos, l1x, p0y); qaccf_add(neg, l1y, p0x);
      break;
    case BG_Y:  // -l0x p1x - l0y p1y + l1x p0x + l1y p0y
      qaccf_add(neg, l0x, p1x); qaccf_add(neg, l0y, p1y); qaccf_add(pos, l1x, p0x); qaccf_add(pos, l1y, p0y);
      break;
    case BG_Z:  // l0x p0y - l0y p0x - l1x p1y + l1y p1x
      qaccf_add(pos, l0x, p0y); qaccf_add(neg, l0y, p0x); qaccf_add(neg, l1x, p1y); qaccf_add(pos, l1y, p1x);
      break;
    case BG_P:  // -2 (l1x p1y - l1y p1x)
      qaccf_add(neg, l1x, p1y); qaccf_add(pos, l1y, p1x);
      return 2 * (qaccf_result(pos) - qaccf_result(neg));
    default:
      return 0;
  }
  return qaccf_result(pos) - qaccf_result(neg);
}

// Real pair forward: the quads of the tile through M.
static __device__ __noinline__ void bt_rpair(longlong2* tile, uint32_t TS, uint32_t ta, uint32_t tbb,
                                             const QL* __restrict__ M) {
  const uint32_t lo = min(ta, tbb), hi = max(ta, tbb);
  for (uint32_t i = threadIdx.x; i < (TS >> 2); i += BT_THREADS) {
    uint32_t j = i + (i & ~(lo - 1));
    j = j + (j & ~(hi - 1));
    const uint32_t jj[4] = {j, j | ta, j | tbb, j | ta | tbb};
    QL r[4], im[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const longlong2 v = tile[jj[c]];
      r[c] = q60_split(v.x);
      im[c] = q60_split(v.y);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) tile[jj[k]] = make_longlong2(bt_row4(M, k, r), bt_row4(M, k, im));
  }
}

// Real pair backward: both members' generator terms (member a on the pairs
// (0,1), (2,3) of the quad, member b on (0,2), (1,3)), then M on both tiles.
static __device__ __noinline__ void bt_rpair_back(longlong2* P, longlong2* Lt, uint32_t TS, uint32_t ta,
                                                  uint32_t tbb, int gen_a, int gen_b, const QL* __restrict__ M,
                                                  int64_t* out_a, int64_t* out_b) {
  int64_t sa = 0, sb = 0;
  const uint32_t lo = min(ta, tbb), hi = max(ta, tbb);
  for (uint32_t i = threadIdx.x; i < (TS >> 2); i += BT_THREADS) {
    uint32_t j = i + (i & ~(lo - 1));
    j = j + (j & ~(hi - 1));
    const uint32_t jj[4] = {j, j | ta, j | tbb, j | ta | tbb};
    QL pr[4], pi[4], lr[4], li[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const longlong2 v = P[jj[c]], w = Lt[jj[c]];
      pr[c] = q60_split(v.x);
      pi[c] = q60_split(v.y);
      lr[c] = q60_split(w.x);
      li[c] = q60_split(w.y);
    }
    if (gen_a != BG_NONE) {
      sa += bt_pair_gen(gen_a, lr[0], li[0], lr[1], li[1], pr[0], pi[0], pr[1], pi[1]);
      sa += bt_pair_gen(gen_a, lr[2], li[2], lr[3], li[3], pr[2], pi[2], pr[3], pi[3]);
    }
    if (gen_b != BG_NONE) {
      sb += bt_pair_gen(gen_b, lr[0], li[0], lr[2], li[2], pr[0], pi[0], pr[2], pi[2]);
      sb += bt_pair_gen(gen_b, lr[1], li[1], lr[3], li[3], pr[1], pi[1], pr[3], pi[3]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      P[jj[k]] = make_longlong2(bt_row4(M, k, pr), bt_row4(M, k, pi));
      Lt[jj[k]] = make_longlong2(bt_row4(M, k, lr), bt_row4(M, k, li));
    }
  }
  *out_a = sa;
  *out_b = sb;
}

// Backward step of a diagonal group in one sweep: per amplitude the members'
// generator terms (as bt_gen_dgroup) and then E on psi and on lambda.
static __device__ void bt_back_dgroup(longlong2* P, longlong2* Lt, uint32_t TS, const BOp* mem, int nm,
                                      const QC* __restrict__ E, int64_t* out) {
  int tbs[BT_DG_MAX], gens[BT_DG_MAX];
#pragma unroll
  for (int m = 0; m < BT_DG_MAX; ++m) {
    out[m] = 0;
    tbs[m] = m < nm ? mem[m].tb : 0;
    gens[m] = m < nm ? mem[m].gen : BG_NONE;
  }
  for (uint32_t j = threadIdx.x; j < TS; j += BT_THREADS) {
    const longlong2 p = P[j], l = Lt[j];
    const QL px = q60_split(p.x), py = q60_split(p.y), lx = q60_split(l.x), ly = q60_split(l.y);
    QAccF pos{0, 0, 0}, neg{0, 0, 0};
    qaccf_add(pos, lx, py);
    qaccf_add(neg, ly, px);
    const int64_t w = qaccf_result(pos) - qaccf_result(neg);
    uint32_t idx = 0;
#pragma unroll
    for (int m = 0; m < BT_DG_MAX; ++m) {
      const bool one = (j >> tbs[m]) & 1u;
      if (m < nm) idx |= (uint32_t)one << m;
      if (gens[m] == BG_Z) out[m] += one ? -w : w;
      else if (gens[m] == BG_P && one) out[m] -= 2 * w;
    }
    const QC u = E[idx];
    int64_t re, im;
    q60_gauss_mul(u, px, py, q60_split(p.x + p.y), &re, &im);
    P[j] = make_longlong2(re, im);
    q60_gauss_mul(u, lx, ly, q60_split(l.x + l.y), &re, &im);
    Lt[j] = make_longlong2(re, im);
  }
}

// Generator partials of every member of a diagonal group on the same tiles, in
// Q60 units: w_j = Im(conj(l_j) p_j) once per amplitude, then per member Z:
// (-1)^bit w_j, P: -2 [bit] w_j (the members commute with each other and with
// each other's generators, so every term may be taken before the group runs).
// Bounds as in bt_gen_partial.
static __device__ void bt_gen_dgroup(const longlong2* P, const longlong2* Lt, uint32_t TS, const BOp* mem, int nm,
                                     int64_t* out) {
  int tbs[BT_DG_MAX], gens[BT_DG_MAX];
#pragma unroll
  for (int m = 0; m < BT_DG_MAX; ++m) {
    out[m] = 0;
    tbs[m] = m < nm ? mem[m].tb : 0;
    gens[m] = m < nm ? mem[m].gen : BG_NONE;
  }
  for (uint32_t j = threadIdx.x; j < TS; j += BT_THREADS) {
    const longlong2 p = P[j], l = Lt[j];
    QAccF acc{0, 0, 0};
    qaccf_add(acc, q60_split(l.x), q60_split(p.y));
    qaccf_add(acc, q60_split(-l.y), q60_split(p.x));
    const int64_t w = qaccf_result(acc);
#pragma unroll
    for (int m = 0; m < BT_DG_MAX; ++m) {
      const bool one = (j >> tbs[m]) & 1u;
      if (gens[m] == BG_Z) out[m] += one ? -w : w;
      else if (gens[m] == BG_P && one) out[m] -= 2 * w;
    }
  }
}


__device__ __forceinline__ longlong2 bt_unit(longlong2 a, int code) {
  switch (code) {
    case U_ONE: return a;
    case U_I: return make_longlong2(-a.y, a.x);
    case U_MINUS_ONE: return make_longlong2(-a.x, -a.y);
    default: return make_longlong2(a.y, -a.x);
  }
}

// Matrices of these passes are in Gauss form (qc_make_gauss): u * a with three
// limb products; a real entry keeps its value in u.re.
__device__ __forceinline__ longlong2 bt_mul(longlong2 a, int code, const QC& u) {
  if (code != U_GENERAL) return bt_unit(a, code);
  int64_t re, im;
  q60_gauss_mul(u, q60_split(a.x), q60_split(a.y), q60_split(a.x + a.y), &re, &im);
  return make_longlong2(re, im);
}

__device__ __forceinline__ uint32_t bt_expand(uint32_t i, uint32_t fixed, uint32_t set) {
  while (fixed) {
    int f = __ffs(fixed) - 1;
    fixed &= fixed - 1;
    i = ((i >> f) << (f + 1)) | (i & ((1u << f) - 1));
  }
  return i | set;
}

static __device__ void bt_apply(longlong2* tile, uint32_t TS, const BOp& op, int kind, int c0, int c1, const QC* U,
                         uint64_t base) {
  const uint32_t lcm = op.lcm;
  if (kind == BK_SCALAR) {
    const bool one = (base >> op.tb) & 1ull;
    const int code = one ? c1 : c0;
    if (code == U_ONE) return;
    const QC& u = U[one ? 3 : 0];
    const uint32_t cnt = TS >> __popc(lcm);
    for (uint32_t i = threadIdx.x; i < cnt; i += BT_THREADS) {
      uint32_t j = bt_expand(i, lcm, lcm);
      tile[j] = bt_mul(tile[j], code, u);
    }
    return;
  }
  const uint32_t tb = 1u << op.tb;
  const uint32_t fixed = lcm | tb;
  const uint32_t cnt = TS >> __popc(fixed);
  for (uint32_t i = threadIdx.x; i < cnt; i += BT_THREADS) {
    // without in-tile controls the insertion of one zero bit is a mask and an add
    const uint32_t j0 = lcm ? bt_expand(i, fixed, lcm) : i + (i & ~(tb - 1)), j1 = j0 | tb;
    if (kind == OP_PHASE1) {
      tile[j1] = bt_mul(tile[j1], c1, U[3]);
      continue;
    }
    longlong2 a0 = tile[j0], a1 = tile[j1], b0, b1;
    if (kind == OP_DIAG) {
      b0 = bt_mul(a0, c0, U[0]);
      b1 = bt_mul(a1, c1, U[3]);
    } else if (kind == OP_ANTI) {
      b0 = bt_mul(a1, c0, U[1]);
      b1 = bt_mul(a0, c1, U[2]);
    } else if (kind == OP_GENERAL) {
      const QL r0 = q60_split(a0.x), i0 = q60_split(a0.y), r1 = q60_split(a1.x), i1 = q60_split(a1.y);
      const QL s0 = q60_split(a0.x + a0.y), s1 = q60_split(a1.x + a1.y);
      int64_t re, im;
      q60_gauss_row(U[0], U[1], r0, i0, s0, r1, i1, s1, &re, &im);
      b0 = make_longlong2(re, im);
      q60_gauss_row(U[2], U[3], r0, i0, s0, r1, i1, s1, &re, &im);
      b1 = make_longlong2(re, im);
    } else {  // real entries: u.re of the Gauss form
      const QL r0 = q60_split(a0.x), i0 = q60_split(a0.y), r1 = q60_split(a1.x), i1 = q60_split(a1.y);
      int64_t out[4];
#pragma unroll
      for (int row = 0; row < 2; ++row) {
        const QC& u0 = U[2 * row];
        const QC& u1 = U[2 * row + 1];
        QAcc re = qacc_new(), im = qacc_new();
        qacc_add(re, u0.re, r0);
        qacc_add(re, u1.re, r1);
        qacc_add(im, u0.re, i0);
        qacc_add(im, u1.re, i1);
        out[2 * row] = qacc_round(re);
        out[2 * row + 1] = qacc_round(im);
      }
      b0 = make_longlong2(out[0], out[1]);
      b1 = make_longlong2(out[2], out[3]);
    }
    tile[j0] = b0;
    tile[j1] = b1;
  }
}

// sum_k s_k * l_k * p_k for four signed products of Q60 values, in Q60 units
// (all four limb products kept, one rounding: these terms are summed over the
// whole state).
__device__ __forceinline__ int64_t bt_dot4(const int64_t* l, const int64_t* p, const int* sg) {
  QAccF acc{0, 0, 0};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (sg[k] == 0) continue;
    qaccf_add(acc, q60_split(sg[k] > 0 ? l[k] : -l[k]), q60_split(p[k]));
  }
  return qaccf_result(acc);
}

// This thread's share of Im <lambda| G |psi> over the op's pairs in the tile, in
// Q60 units, summed exactly in an int64: every partial sum is bounded by
// sum |l_x| |p_y| over distinct pairs (x, y) times the generator's largest
// weight (2), i.e. by 2 ||lambda|| ||psi|| <= 2 * 1.25^2 < 4 (Cauchy-Schwarz),
// so it stays below 2^62.  No FP64 arithmetic per pair (GB300 issues FP64 at
// 1/74 of its FP32 rate).
static __device__ int64_t bt_gen_partial(const longlong2* P, const longlong2* Lt, uint32_t TS, const BOp& op,
                                         uint64_t base) {
  if (op.kf == BK_SCALAR) {
    // diagonal generator on a qubit outside the tile: per amplitude,
    // Z -> (-1)^bit Im(conj(l) p), P -> -2 [bit] Im(conj(l) p)
    const bool one = (base >> op.tb) & 1ull;
    if (op.gen == BG_P && !one) return 0;
    const int64_t w = op.gen == BG_P ? -2 : (one ? -1 : 1);
    const uint32_t cnt = TS >> __popc(op.lcm);
    int64_t acc = 0;
    for (uint32_t i = threadIdx.x; i < cnt; i += BT_THREADS) {
      const uint32_t j = bt_expand(i, op.lcm, op.lcm);
      const int64_t l[4] = {Lt[j].x, Lt[j].y, 0, 0}, p[4] = {P[j].y, P[j].x, 0, 0};
      const int sg[4] = {1, -1, 0, 0};
      acc += w * bt_dot4(l, p, sg);
    }
    return acc;
  }
  const uint32_t tb = 1u << op.tb;
  const uint32_t fixed = op.lcm | tb;
  const uint32_t cnt = TS >> __popc(fixed);
  int64_t acc = 0;
  for (uint32_t i = threadIdx.x; i < cnt; i += BT_THREADS) {
    const uint32_t j0 = op.lcm ? bt_expand(i, fixed, op.lcm) : i + (i & ~(tb - 1)), j1 = j0 | tb;
    const longlong2 p0 = P[j0], p1 = P[j1], l0 = Lt[j0], l1 = Lt[j1];
    int64_t l[4], p[4];
    int sg[4];
    switch (op.gen) {
      case BG_X:  // l0x p1y - l0y p1x + l1x p0y - l1y p0x
        l[0] = l0.x; p[0] = p1.y; sg[0] = 1; l[1] = l0.y; p[1] = p1.x; sg[1] = -1;
        l[2] = l1.x; p[2] = p0.y; sg[2] = 1; l[3] = l1.y; p[3] = p0.x; sg[3] = -1;
        break;
      case BG_Y:  // -l0x p1x - l0y p1y + l1x p0x + l1y p0y
        l[0] = l0.x; p[0] = p1.x; sg[0] = -1; l[1] = l0.y; p[1] = p1.y; sg[1] = -1;
        l[2] = l1.x; p[2] = p0.x; sg[2] = 1; l[3] = l1.y; p[3] = p0.y; sg[3] = 1;
        break;
      case BG_Z:  // l0x p0y - l0y p0x - l1x p1y + l1y p1x
        l[0] = l0.x; p[0] = p0.y; sg[0] = 1; l[1] = l0.y; p[1] = p0.x; sg[1] = -1;
        l[2] = l1.x; p[2] = p1.y; sg[2] = -1; l[3] = l1.y; p[3] = p1.x; sg[3] = 1;
        break;
      default:    // P: -2 (l1x p1y - l1y p1x)
        l[0] = l1.x; p[0] = p1.y; sg[0] = -1; l[1] = l1.y; p[1] = p1.x; sg[1] = 1;
        l[2] = 0; p[2] = 0; sg[2] = 0; l[3] = 0; p[3] = 0; sg[3] = 0;
        break;
    }
    const int64_t v = bt_dot4(l, p, sg);
    acc += op.gen == BG_P ? 2 * v : v;
  }
  return acc;
}

// Backward step of a pair op of class REAL with a generator (RY, H-type rows):
// for each of this thread's pairs, the generator term and then U on the psi pair
// and on the lambda pair, from one load and one limb split of each (real entries
// in u.re of the Gauss form).  Returns the thread's partial.
static __device__ int64_t bt_back_real(longlong2* P, longlong2* Lt, uint32_t TS, const BOp& op,
                                       const QC* __restrict__ U) {
  const uint32_t tb = 1u << op.tb;
  const uint32_t fixed = op.lcm | tb;
  const uint32_t cnt = TS >> __popc(fixed);
  int64_t acc = 0;
  for (uint32_t i = threadIdx.x; i < cnt; i += BT_THREADS) {
    const uint32_t j0 = op.lcm ? bt_expand(i, fixed, op.lcm) : i + (i & ~(tb - 1)), j1 = j0 | tb;
    const longlong2 p0 = P[j0], p1 = P[j1], l0 = Lt[j0], l1 = Lt[j1];
    const QL p0x = q60_split(p0.x), p0y = q60_split(p0.y), p1x = q60_split(p1.x), p1y = q60_split(p1.y);
    const QL l0x = q60_split(l0.x), l0y = q60_split(l0.y), l1x = q60_split(l1.x), l1y = q60_split(l1.y);
    acc += bt_pair_gen(op.gen, l0x, l0y, l1x, l1y, p0x, p0y, p1x, p1y);
#pragma unroll
    for (int row = 0; row < 2; ++row) {
      const QL u0 = U[2 * row].re, u1 = U[2 * row + 1].re;
      QAcc pr = qacc_new(), pi = qacc_new(), lr = qacc_new(), li = qacc_new();
      qacc_add(pr, u0, p0x);
      qacc_add(pr, u1, p1x);
      qacc_add(pi, u0, p0y);
      qacc_add(pi, u1, p1y);
      qacc_add(lr, u0, l0x);
      qacc_add(lr, u1, l1x);
      qacc_add(li, u0, l0y);
      qacc_add(li, u1, l1y);
      const uint32_t jr = row ? j1 : j0;
      P[jr] = make_longlong2(qacc_round(pr), qacc_round(pi));
      Lt[jr] = make_longlong2(qacc_round(lr), qacc_round(li));
    }
  }
  return acc;
}

// An antidiagonal op with unit factors (X, CNOT, Y, Toffoli) on psi and lambda in
// one sweep over the pairs: swaps with sign or i factors, no arithmetic.
static __device__ void bt_anti_both(longlong2* P, longlong2* Lt, uint32_t TS, const BOp& op, int c0, int c1) {
  const uint32_t tb = 1u << op.tb;
  const uint32_t fixed = op.lcm | tb;
  const uint32_t cnt = TS >> __popc(fixed);
  for (uint32_t i = threadIdx.x; i < cnt; i += BT_THREADS) {
    const uint32_t j0 = op.lcm ? bt_expand(i, fixed, op.lcm) : i + (i & ~(tb - 1)), j1 = j0 | tb;
    const longlong2 p0 = P[j0], p1 = P[j1], l0 = Lt[j0], l1 = Lt[j1];
    P[j0] = bt_unit(p1, c0);
    P[j1] = bt_unit(p0, c1);
    Lt[j0] = bt_unit(l1, c0);
    Lt[j1] = bt_unit(l0, c1);
  }
}

// Adds this thread's partial (Q60 units) to its warp's accumulator of `slot`
// without a CTA barrier: the warp sums exactly by integer shuffles (the bound of
// bt_gen_partial holds for the warp's total too), lane 0 converts once and owns
// the warp's row, so the order of the FP64 additions is fixed.  wacc holds
// (BT_THREADS / 32) rows of nslots.
__device__ __forceinline__ void bt_warp_accumulate(int64_t v, double* wacc, int nslots, int slot) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += (int64_t)__shfl_xor_sync(0xffffffffu, (long long)v, o);
  if ((threadIdx.x & 31) == 0) wacc[(threadIdx.x >> 5) * nslots + slot] += q60_to_double(v);
}

// After a barrier: the CTA's total of `slot`, warps added in warp order.
__device__ __forceinline__ double bt_warp_total(const double* wacc, int nslots, int slot) {
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < BT_THREADS / 32; ++w) t += wacc[w * nslots + slot];
  return t;
}

static __device__ double bt_block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
#pragma unroll
  for (int i = 0; i < BT_THREADS / 32; ++i) r += red[i];
  return r;
}

// Runs of up to BT_DG_MAX consecutive uncontrolled diagonal ops (forward and
// adjoint class) on distinct tile qubits, with a Z, P or no generator, of the
// ops [begin, end) become diagonal groups: a BK_DGROUP head (gate = group index,
// nmem members) is inserted before the members, which turn into BK_MEMBER
// records.  Heads are appended to `heads` (their index in the new op list);
// src[i - begin] receives the old index of new op i (-1 for a head).
// Consecutive uncontrolled real ops on distinct tile qubits become real pairs
// the same way (a BK_RPAIR head, gate = index into `pairs`, two BK_MEMBER records).
static inline void group_diagonals(std::vector<BOp>& ops, size_t begin, std::vector<int>* heads,
                                   std::vector<int>* src, std::vector<int>* pairs = nullptr) {
  auto eligible = [](const BOp& o) {
    const bool df = o.kf == OP_DIAG || o.kf == OP_PHASE1, db = o.kb == OP_DIAG || o.kb == OP_PHASE1;
    return df && db && o.lcm == 0 && o.ext == 0 && (o.gen == BG_NONE || o.gen == BG_Z || o.gen == BG_P);
  };
  auto real = [](const BOp& o) { return o.kf == OP_REAL && o.kb == OP_REAL && o.lcm == 0 && o.ext == 0; };
  std::vector<BOp> out(ops.begin(), ops.begin() + begin);
  src->clear();
  size_t i = begin;
  while (i < ops.size()) {
    if (pairs && i + 1 < ops.size() && real(ops[i]) && real(ops[i + 1]) && ops[i].tb != ops[i + 1].tb) {
      BOp h;
      memset(&h, 0, sizeof h);
      h.kf = h.kb = BK_RPAIR;
      h.nmem = 2;
      h.gate = (int)pairs->size();
      h.slot = -1;
      h.param = -1;
      h.gen = BG_NONE;
      pairs->push_back((int)out.size());
      out.push_back(h);
      src->push_back(-1);
      for (size_t k = i; k < i + 2; ++k) {
        BOp mo = ops[k];
        mo.kf = mo.kb = BK_MEMBER;
        out.push_back(mo);
        src->push_back((int)k);
      }
      i += 2;
      continue;
    }
    size_t j = i;
    uint32_t bits = 0;
    while (j < ops.size() && j - i < (size_t)BT_DG_MAX && eligible(ops[j]) && !((bits >> ops[j].tb) & 1)) {
      bits |= 1u << ops[j].tb;
      ++j;
    }
    if (j - i >= 2) {
      BOp h;
      memset(&h, 0, sizeof h);
      h.kf = h.kb = BK_DGROUP;
      h.nmem = (int8_t)(j - i);
      h.gate = (int)heads->size();
      h.slot = -1;
      h.param = -1;
      h.gen = BG_NONE;
      heads->push_back((int)out.size());
      out.push_back(h);
      src->push_back(-1);
      for (size_t k = i; k < j; ++k) {
        BOp mo = ops[k];
        mo.kf = mo.kb = BK_MEMBER;
        out.push_back(mo);
        src->push_back((int)k);
      }
      i = j;
    } else {
      out.push_back(ops[i]);
      src->push_back((int)i);
      ++i;
    }
  }
  ops.swap(out);
}

}  // namespace qs
