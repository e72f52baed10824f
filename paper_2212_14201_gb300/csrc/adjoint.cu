// Adjoint differentiation of <psi(theta)| H |psi(theta)> for parametrised
// circuits (the paper's variational circuits, Section "Variational quantum
// circuit", with qop expectations; it does not say how gradients are taken --
// this is the adjoint recursion of Jones & Gacon, arXiv:2009.02823):
//   psi = U_G ... U_1 |0>,  lambda = H psi,  E = Re <psi|lambda>,
//   for k = G..1:  dE/dtheta_k += Im <lambda| G_k |psi>   (if U_k = exp(-i theta G_k / 2))
//                  psi <- U_k^dag psi,  lambda <- U_k^dag lambda.
// One fused kernel per backward gate reads both vectors once, forms the
// generator inner product (FP64, deterministic per-CTA partials) and applies
// U_k^dag to both.  lambda is kept scaled by 1/S, S a power of two >= sum|coef|,
// so that its components stay inside the Q60 range of the gate engine.
#include <math.h>

#include <algorithm>
#include <vector>

#include "fixed.h"
#include "internal.h"
#include "q60tile.cuh"

namespace qs {

enum GenKind : int { GEN_NONE = 0, GEN_X = 1, GEN_Y = 2, GEN_Z = 3, GEN_P = 4 };

struct AdjArgs {
  double2 m[4];     // U^dag (FP64 engine)
  QC q[4];          // U^dag (Q60 engine)
  uint64_t cmask;
  int64_t items;
  int t, nfix;
  int fix[16];
  int cls, code0, code1;
  int gen;          // GenKind
  double gsign;     // -1 for a dagger record
  int slot;         // partial-sum slot of this gate
};

__device__ __forceinline__ double adj_neg(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

__device__ __forceinline__ double2 adj_unit(double2 a, int code) {
  switch (code) {
    case U_ONE: return a;
    case U_I: return make_double2(adj_neg(a.y), a.x);
    case U_MINUS_ONE: return make_double2(adj_neg(a.x), adj_neg(a.y));
    default: return make_double2(a.y, adj_neg(a.x));
  }
}

// Apply the op to the pair (a0, a1) in place.
template <bool FX>
__device__ __forceinline__ void adj_pair(const AdjArgs& g, double2& a0, double2& a1) {
  const int cls = g.cls;
  if (!FX) {
    auto mulc = [](double2 a, int code, double2 u) {
      if (code != U_GENERAL) return adj_unit(a, code);
      return make_double2(fma(u.x, a.x, -u.y * a.y), fma(u.x, a.y, u.y * a.x));
    };
    if (cls == OP_PHASE1) {
      a1 = mulc(a1, g.code1, g.m[3]);
    } else if (cls == OP_DIAG) {
      a0 = mulc(a0, g.code0, g.m[0]);
      a1 = mulc(a1, g.code1, g.m[3]);
    } else if (cls == OP_ANTI) {
      double2 b0 = mulc(a1, g.code0, g.m[1]), b1 = mulc(a0, g.code1, g.m[2]);
      a0 = b0;
      a1 = b1;
    } else if (cls == OP_REAL) {
      double2 b0 = make_double2(fma(g.m[0].x, a0.x, g.m[1].x * a1.x), fma(g.m[0].x, a0.y, g.m[1].x * a1.y));
      double2 b1 = make_double2(fma(g.m[2].x, a0.x, g.m[3].x * a1.x), fma(g.m[2].x, a0.y, g.m[3].x * a1.y));
      a0 = b0;
      a1 = b1;
    } else if (cls == OP_GENERAL) {
      const double2 u0 = g.m[0], u1 = g.m[1], u2 = g.m[2], u3 = g.m[3];
      double2 b0, b1;
      b0.x = fma(u0.x, a0.x, fma(-u0.y, a0.y, fma(u1.x, a1.x, -u1.y * a1.y)));
      b0.y = fma(u0.x, a0.y, fma(u0.y, a0.x, fma(u1.x, a1.y, u1.y * a1.x)));
      b1.x = fma(u2.x, a0.x, fma(-u2.y, a0.y, fma(u3.x, a1.x, -u3.y * a1.y)));
      b1.y = fma(u2.x, a0.y, fma(u2.y, a0.x, fma(u3.x, a1.y, u3.y * a1.x)));
      a0 = b0;
      a1 = b1;
    }
    return;
  }
  auto qmul = [](double2 a, int code, const QC& u) {
    if (code != U_GENERAL) return adj_unit(a, code);
    const QL ar = q60_split(q60_from_double(a.x)), ai = q60_split(q60_from_double(a.y));
    QAcc re = qacc_new(), im = qacc_new();
    qacc_add(re, u.re, ar);
    qacc_add(re, u.nim, ai);
    qacc_add(im, u.re, ai);
    qacc_add(im, u.im, ar);
    return make_double2(q60_to_double(qacc_round(re)), q60_to_double(qacc_round(im)));
  };
  if (cls == OP_PHASE1) {
    a1 = qmul(a1, g.code1, g.q[3]);
  } else if (cls == OP_DIAG) {
    a0 = qmul(a0, g.code0, g.q[0]);
    a1 = qmul(a1, g.code1, g.q[3]);
  } else if (cls == OP_ANTI) {
    double2 b0 = qmul(a1, g.code0, g.q[1]), b1 = qmul(a0, g.code1, g.q[2]);
    a0 = b0;
    a1 = b1;
  } else if (cls == OP_REAL || cls == OP_GENERAL) {
    const QL r0 = q60_split(q60_from_double(a0.x)), i0 = q60_split(q60_from_double(a0.y));
    const QL r1 = q60_split(q60_from_double(a1.x)), i1 = q60_split(q60_from_double(a1.y));
    int64_t out[4];
#pragma unroll
    for (int row = 0; row < 2; ++row) {
      const QC& u0 = g.q[2 * row];
      const QC& u1 = g.q[2 * row + 1];
      QAcc re = qacc_new(), im = qacc_new();
      qacc_add(re, u0.re, r0);
      qacc_add(re, u1.re, r1);
      qacc_add(im, u0.re, i0);
      qacc_add(im, u1.re, i1);
      if (cls == OP_GENERAL) {
        qacc_add(re, u0.nim, i0);
        qacc_add(re, u1.nim, i1);
        qacc_add(im, u0.im, r0);
        qacc_add(im, u1.im, r1);
      }
      out[2 * row] = qacc_round(re);
      out[2 * row + 1] = qacc_round(im);
    }
    a0 = make_double2(q60_to_double(out[0]), q60_to_double(out[1]));
    a1 = make_double2(q60_to_double(out[2]), q60_to_double(out[3]));
  }
}

// Im <lambda| G |psi> over one pair.
__device__ __forceinline__ double gen_im(int gen, double2 l0, double2 l1, double2 p0, double2 p1) {
  switch (gen) {
    case GEN_X: return fma(l0.x, p1.y, -l0.y * p1.x) + fma(l1.x, p0.y, -l1.y * p0.x);
    case GEN_Y: return -fma(l0.x, p1.x, l0.y * p1.y) + fma(l1.x, p0.x, l1.y * p0.y);
    case GEN_Z: return fma(l0.x, p0.y, -l0.y * p0.x) - fma(l1.x, p1.y, -l1.y * p1.x);
    case GEN_P: return -2.0 * fma(l1.x, p1.y, -l1.y * p1.x);
    default: return 0.0;
  }
}

__device__ __forceinline__ double adj_block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  return r;
}

template <bool FX>
__global__ void __launch_bounds__(256) k_adj_step(double2* __restrict__ psi, double2* __restrict__ lam,
                                                  const AdjArgs g, double* __restrict__ part) {
  __shared__ double sh[8];
  const uint64_t tb = 1ull << g.t;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (uint64_t)g.items; i += stride) {
    uint64_t x0 = i;
    for (int k = 0; k < g.nfix; ++k) {
      int f = g.fix[k];
      x0 = ((x0 >> f) << (f + 1)) | (x0 & ((1ull << f) - 1));
    }
    x0 |= g.cmask;
    const uint64_t x1 = x0 | tb;
    double2 p0 = psi[x0], p1 = psi[x1], l0 = lam[x0], l1 = lam[x1];
    if (g.gen != GEN_NONE) acc += gen_im(g.gen, l0, l1, p0, p1);
    adj_pair<FX>(g, p0, p1);
    adj_pair<FX>(g, l0, l1);
    psi[x0] = p0;
    psi[x1] = p1;
    lam[x0] = l0;
    lam[x1] = l1;
  }
  if (g.gen != GEN_NONE) {
    double s = adj_block_sum(acc, sh);
    if (threadIdx.x == 0) part[(size_t)g.slot * gridDim.x + blockIdx.x] = s * g.gsign;
  }
}

// lambda = (H / S) psi, as a gather over groups of terms sharing an X mask:
//   lambda[y] = sum_g D_g(y) psi[y ^ xm_g],
//   D_g(y) = sum_{k in g} c_k i^{ny_k} (-1)^{popcount((y ^ xm_g) & zm_k)}.
constexpr int HMAX = 48;
struct HArgs {
  uint64_t N;
  int nterms, ngroups, accumulate;
  uint64_t gxm[HMAX];
  int gstart[HMAX + 1];
  uint64_t zm[HMAX];
  double c[HMAX];   // coef / S times the real unit of i^ny (+-1) ...
  int64_t cq[HMAX]; // (the same in Q60)
  int imag[HMAX];   // ... placed in the imaginary part when ny is odd
};

__global__ void __launch_bounds__(256) k_apply_h(const double2* __restrict__ psi, double2* __restrict__ lam,
                                                 const __grid_constant__ HArgs h) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  // Q60 integers (the FP64 pipe would bound this loop on GB300): the signed
  // coefficient sums of a group are exact in int64 (sum |c_k| <= 1), each group's
  // product with psi is rounded once, and the launch's total (|.| <= |psi|_inf)
  // is converted once.
  for (uint64_t y = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; y < h.N; y += stride) {
    int64_t ore = 0, oim = 0;
    for (int gi = 0; gi < h.ngroups; ++gi) {
      const uint64_t x = y ^ h.gxm[gi];
      int64_t dre = 0, dim = 0;
      for (int k = h.gstart[gi]; k < h.gstart[gi + 1]; ++k) {
        const int64_t v = (__popcll(x & h.zm[k]) & 1) ? -h.cq[k] : h.cq[k];
        if (h.imag[k]) dim += v;
        else dre += v;
      }
      const double2 p = psi[x];
      const QL px = q60_split(q60_from_double(p.x)), py = q60_split(q60_from_double(p.y));
      const QL qr = q60_split(dre), qi = q60_split(dim), nqi = q60_split(-dim);
      QAcc r = qacc_new(), i = qacc_new();
      qacc_add(r, qr, px);  // re: dre px - dim py
      qacc_add(r, nqi, py);
      qacc_add(i, qr, py);  // im: dre py + dim px
      qacc_add(i, qi, px);
      ore += qacc_round(r);
      oim += qacc_round(i);
    }
    double2 out = make_double2(q60_to_double(ore), q60_to_double(oim));
    if (h.accumulate) {
      const double2 prev = lam[y];
      out.x += prev.x;
      out.y += prev.y;
    }
    lam[y] = out;
  }
}

// per-CTA partials of Re <psi|lambda>
__global__ void __launch_bounds__(256) k_dot_re(const double2* __restrict__ a, const double2* __restrict__ b, uint64_t N,
                                                double* __restrict__ part) {
  __shared__ double sh[8];
  double acc = 0.0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    const double2 u = a[i], v = b[i];
    acc += fma(u.x, v.x, u.y * v.y);
  }
  double s = adj_block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out[j] = sum over the CTA partials of slot j, in CTA order.
__global__ void k_slot_sums(const double* __restrict__ part, int nslots, int nblocks, double* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nslots; j += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)j * nblocks + b];
    out[j] = s;
  }
}

// ---- fused backward sweep (Q60): tile passes over psi and lambda at once --------------
// The backward sweep applies U_G^dag .. U_1^dag, so it is the forward sweep of the
// reversed, daggered program; greedy tile passes over that list only reorder ops
// that commute, and an op that commutes with U_k also commutes with U_k's
// generator (same qubits, same diagonal structure), so every generator inner
// product is taken on the same (psi, lambda) as in the gate-by-gate sweep.
constexpr int ADJ_GRID_STRIDE = 608;  // partial-sum slots per gradient (>= CTAs of any pass)

struct AdjPassArgs {
  BPass ps;
  const BOp* ops;   // ops of this pass (device), in execution order
  const QC* mats;   // 4 entries per op (device)
  const QC* dgm;    // 16 entries per diagonal group (device)
  const QL* rpm;    // 16 entries per real pair (device)
  double* part;     // [slot][ADJ_GRID_STRIDE]
  int slot_base;
};

__global__ void __launch_bounds__(BT_THREADS, 3) k_adj_pass(double2* __restrict__ psi, double2* __restrict__ lam,
                                                         const AdjPassArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const BPass& ps = a.ps;
  const int m = ps.m;
  const int L = m - ps.nhigh;
  const uint32_t TS = 1u << m;
  const uint32_t H = 1u << ps.nhigh;
  longlong2* tP = reinterpret_cast<longlong2*>(smem);
  longlong2* tL = tP + TS;
  uint64_t* offs = reinterpret_cast<uint64_t*>(tL + TS);
  double* wacc = reinterpret_cast<double*>(offs + H);  // [warps][nslots]
  for (uint32_t h = threadIdx.x; h < H; h += BT_THREADS) {
    uint64_t o = 0;
    for (int b = 0; b < ps.nhigh; ++b) o |= (uint64_t)((h >> b) & 1u) << ps.qhigh[b];
    offs[h] = o;
  }
  for (int s = threadIdx.x; s < ps.nslots * (BT_THREADS / 32); s += BT_THREADS) wacc[s] = 0.0;
  const uint32_t lowmask = (1u << L) - 1;
  const uint64_t ntiles = 1ull << ps.nout;
  for (uint64_t r = blockIdx.x; r < ntiles; r += gridDim.x) {
    uint64_t base = 0;
    for (int b = 0; b < ps.nout; ++b) base |= ((r >> b) & 1ull) << ps.outpos[b];
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < TS; j += BT_THREADS) {
      const uint64_t x = base + offs[j >> L] + (j & lowmask);
      const double2 u = psi[x], v = lam[x];
      tP[j] = make_longlong2(q60_from_double(u.x), q60_from_double(u.y));
      tL[j] = make_longlong2(q60_from_double(v.x), q60_from_double(v.y));
    }
    __syncthreads();
    for (int k = ps.op_begin; k < ps.op_end; ++k) {
      const BOp op = a.ops[k];
      if (op.kb == BK_MEMBER || (base & op.ext) != op.ext) continue;
      // each thread reads and then rewrites only its own pairs (amplitudes) of this
      // op, so the generator partial and the update need no barrier between them
      if (op.kb == BK_DGROUP) {
        int64_t gp[BT_DG_MAX];
        const BOp* mem = a.ops + k + 1;
        bt_back_dgroup(tP, tL, TS, mem, op.nmem, a.dgm + 16 * op.gate, gp);
        for (int mm = 0; mm < op.nmem; ++mm)
          if (mem[mm].slot >= 0) bt_warp_accumulate(gp[mm], wacc, ps.nslots, mem[mm].slot);
        __syncthreads();
        continue;
      }
      if (op.kb == BK_RPAIR) {
        const BOp* mem = a.ops + k + 1;
        int64_t ga, gb;
        bt_rpair_back(tP, tL, TS, 1u << mem[0].tb, 1u << mem[1].tb, mem[0].gen, mem[1].gen, a.rpm + 16 * op.gate,
                      &ga, &gb);
        if (mem[0].slot >= 0) bt_warp_accumulate(ga, wacc, ps.nslots, mem[0].slot);
        if (mem[1].slot >= 0) bt_warp_accumulate(gb, wacc, ps.nslots, mem[1].slot);
        __syncthreads();
        continue;
      }
      if (op.slot < 0 && op.kb == OP_ANTI && op.c0b != U_GENERAL && op.c1b != U_GENERAL) {
        bt_anti_both(tP, tL, TS, op, op.c0b, op.c1b);  // psi and lambda in one sweep
        __syncthreads();
        continue;
      }
      if (op.slot >= 0 && op.kb == OP_REAL) {  // one pass over the pairs
        bt_warp_accumulate(bt_back_real(tP, tL, TS, op, a.mats + 4 * k), wacc, ps.nslots, op.slot);
        __syncthreads();
        continue;
      }
      if (op.slot >= 0) bt_warp_accumulate(bt_gen_partial(tP, tL, TS, op, base), wacc, ps.nslots, op.slot);
      bt_apply(tP, TS, op, op.kb, op.c0b, op.c1b, a.mats + 4 * k, base);
      bt_apply(tL, TS, op, op.kb, op.c0b, op.c1b, a.mats + 4 * k, base);
      __syncthreads();
    }
    for (uint32_t j = threadIdx.x; j < TS; j += BT_THREADS) {
      const uint64_t x = base + offs[j >> L] + (j & lowmask);
      psi[x] = make_double2(q60_to_double(tP[j].x), q60_to_double(tP[j].y));
      lam[x] = make_double2(q60_to_double(tL[j].x), q60_to_double(tL[j].y));
    }
  }
  __syncthreads();
  for (int k = ps.op_begin + threadIdx.x; k < ps.op_end; k += BT_THREADS) {
    const BOp& op = a.ops[k];
    if (op.slot >= 0)
      a.part[(size_t)(a.slot_base + op.slot) * ADJ_GRID_STRIDE + blockIdx.x] =
          bt_warp_total(wacc, ps.nslots, op.slot) * op.gsign;
  }
}

static int gen_of(const qs_gate& g);

// Backward sweep as tile passes; slot_param receives, per gradient slot in
// execution order, the parameter it belongs to.
static int backward_fused(qs_state* s, double2* lam, const qs_gate* gates, size_t ng, const double* params,
                          double* part, std::vector<int>& slot_param) {
  const int n = s->n;
  std::vector<qs_gate> R(ng);
  std::vector<int> tgt(ng);
  std::vector<uint64_t> cms(ng);
  for (size_t i = 0; i < ng; ++i) {
    R[i] = gates[ng - 1 - i];
    R[i].dagger = !R[i].dagger;
    QS_TRY(gate_qubits(R[i], n, &tgt[i], &cms[i]));
  }
  const int m = std::min(n, BT_M);
  const uint64_t low = (1ull << std::min(n, 3)) - 1;
  std::vector<uint32_t> remaining(ng), pass, rest;
  for (size_t i = 0; i < ng; ++i) remaining[i] = (uint32_t)i;
  std::vector<BOp> ops;
  std::vector<Mat2> opm;  // each op's matrix (double), parallel to ops
  std::vector<QC> mats;
  std::vector<QC> dgm;    // 16 Gauss-form entries per diagonal group
  std::vector<int> dgheads, dgsrc, rpheads;
  std::vector<QL> rpm;    // 16 limb pairs per real pair
  std::vector<BPass> passes;
  int slot_base = 0;
  std::vector<int> slot_bases;
  while (!remaining.empty()) {
    const uint64_t Q = greedy_pass(R.data(), tgt, cms, remaining, m, low, BT_MAX_OPS, pass, rest);
    BPass bp;
    memset(&bp, 0, sizeof bp);
    int local[64];
    int mm = 0;
    for (int b = 0; b < n; ++b) local[b] = ((Q >> b) & 1) ? mm++ : -1;
    int L = 0;
    while (L < n && ((Q >> L) & 1)) ++L;
    bp.m = mm;
    for (int b = L; b < n; ++b)
      if ((Q >> b) & 1) bp.qhigh[bp.nhigh++] = b;
    for (int b = 0; b < n; ++b)
      if (!((Q >> b) & 1)) bp.outpos[bp.nout++] = b;
    bp.op_begin = (int)ops.size();
    int slot = 0;
    for (uint32_t i : pass) {
      const qs_gate& orig = gates[ng - 1 - i];
      Mat2 mt;
      QS_TRY(gate_matrix(R[i], params, &mt));
      Op1 o1 = classify(tgt[i], cms[i], mt);
      BOp op;
      memset(&op, 0, sizeof op);
      op.gen = orig.param_idx >= 0 ? (int8_t)gen_of(orig) : (int8_t)BG_NONE;
      if (o1.cls == OP_IDENTITY && op.gen == BG_NONE) continue;
      op.kb = op.kf = (int8_t)o1.cls;
      op.c0b = (int8_t)o1.code0;
      op.c1b = (int8_t)o1.code1;
      uint32_t lcm = 0;
      uint64_t ext = 0;
      for (int b = 0; b < n; ++b)
        if ((cms[i] >> b) & 1) {
          if (local[b] >= 0) lcm |= 1u << local[b];
          else ext |= 1ull << b;
        }
      op.lcm = lcm;
      op.ext = ext;
      if (local[tgt[i]] >= 0) {
        op.tb = (int8_t)local[tgt[i]];
        if (o1.cls == OP_IDENTITY) op.kb = op.kf = OP_PHASE1;  // identity matrix, kept for its gradient slot
      } else {
        op.tb = (int8_t)tgt[i];
        op.kb = op.kf = BK_SCALAR;
      }
      op.gsign = orig.dagger ? -1.0 : 1.0;
      op.slot = -1;
      op.param = orig.param_idx;
      if (op.gen != BG_NONE) {
        op.slot = (int16_t)slot++;
        slot_param.push_back(orig.param_idx);
      }
      ops.push_back(op);
      opm.push_back(mt);
    }
    // runs of diagonal ops -> diagonal groups; then the matrix tables in op order
    const size_t ng0 = dgheads.size(), np0 = rpheads.size();
    group_diagonals(ops, bp.op_begin, &dgheads, &dgsrc, &rpheads);
    std::vector<Mat2> pm(dgsrc.size());
    for (size_t k = 0; k < dgsrc.size(); ++k) {
      if (dgsrc[k] >= 0) pm[k] = opm[dgsrc[k]];
      else pm[k] = Mat2{};
    }
    opm.resize(bp.op_begin);
    opm.insert(opm.end(), pm.begin(), pm.end());
    for (size_t k = bp.op_begin; k < ops.size(); ++k)
      for (int e = 0; e < 4; ++e) mats.push_back(qc_make_gauss(opm[k].m[e].re, opm[k].m[e].im));  // bt_apply's form
    for (size_t gi = ng0; gi < dgheads.size(); ++gi) {
      const int head = dgheads[gi];
      const int nm = ops[head].nmem;
      for (int idx = 0; idx < 16; ++idx) {
        double re = 1.0, im = 0.0;
        for (int mm = 0; mm < nm && idx < (1 << nm); ++mm) {
          const C2 u = opm[head + 1 + mm].m[((idx >> mm) & 1) ? 3 : 0];
          const double r2 = re * u.re - im * u.im, i2 = re * u.im + im * u.re;
          re = r2;
          im = i2;
        }
        dgm.push_back(qc_make_gauss(re, im));
      }
    }
    for (size_t pi = np0; pi < rpheads.size(); ++pi) {  // M = R_b (x) R_a, a = first member
      const Mat2& ra = opm[rpheads[pi] + 1];
      const Mat2& rb = opm[rpheads[pi] + 2];
      for (int k = 0; k < 4; ++k)
        for (int c = 0; c < 4; ++c)
          rpm.push_back(q60_split(q60_from_double(rb.m[2 * (k >> 1) + (c >> 1)].re * ra.m[2 * (k & 1) + (c & 1)].re)));
    }
    bp.op_end = (int)ops.size();
    bp.nslots = slot;
    passes.push_back(bp);
    slot_bases.push_back(slot_base);
    slot_base += slot;
    remaining.swap(rest);
  }
  BOp* d_ops = nullptr;
  QC* d_mats = nullptr;
  QC* d_dgm = nullptr;
  QL* d_rpm = nullptr;
  QS_CUDA(dmalloc_async((void**)&d_ops, sizeof(BOp) * std::max<size_t>(1, ops.size()), s->stream));
  cudaError_t e = dmalloc_async((void**)&d_mats, sizeof(QC) * std::max<size_t>(4, mats.size()), s->stream);
  if (e == cudaSuccess) e = dmalloc_async((void**)&d_dgm, sizeof(QC) * std::max<size_t>(16, dgm.size()), s->stream);
  if (e == cudaSuccess) e = dmalloc_async((void**)&d_rpm, sizeof(QL) * std::max<size_t>(16, rpm.size()), s->stream);
  if (e == cudaSuccess && !rpm.empty())
    e = cudaMemcpyAsync(d_rpm, rpm.data(), sizeof(QL) * rpm.size(), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess && !ops.empty())
    e = cudaMemcpyAsync(d_ops, ops.data(), sizeof(BOp) * ops.size(), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess && !mats.empty())
    e = cudaMemcpyAsync(d_mats, mats.data(), sizeof(QC) * mats.size(), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess && !dgm.empty())
    e = cudaMemcpyAsync(d_dgm, dgm.data(), sizeof(QC) * dgm.size(), cudaMemcpyHostToDevice, s->stream);
  int rc = e == cudaSuccess ? QS_OK : cuda_fail(e, "adjoint op tables");
  static bool attr = false;
  if (rc == QS_OK && !attr) {
    e = cudaFuncSetAttribute(k_adj_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    if (e != cudaSuccess) rc = cuda_fail(e, "adjoint pass attribute");
    attr = true;
  }
  for (size_t p = 0; rc == QS_OK && p < passes.size(); ++p) {
    AdjPassArgs a;
    a.ps = passes[p];
    a.ops = d_ops;
    a.mats = d_mats;
    a.dgm = d_dgm;
    a.rpm = d_rpm;
    a.part = part;
    a.slot_base = slot_bases[p];
    const uint32_t TS = 1u << a.ps.m;
    const size_t smem = 2 * sizeof(longlong2) * TS + sizeof(uint64_t) * ((size_t)1 << a.ps.nhigh) +
                        sizeof(double) * ((size_t)a.ps.nslots * (BT_THREADS / 32) + 8);
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(3, (220 * 1024) / (smem + 1024)));
    const uint64_t grid = std::min<uint64_t>(1ull << a.ps.nout, (uint64_t)std::min(ADJ_GRID_STRIDE, 152 * per_sm));
    {
      KTimer kt(s, QS_K_ADJOINT, a.ps.m, a.ps.op_end - a.ps.op_begin, 0, 0, 2.0 * (double)(1ull << n), 0.0);
      k_adj_pass<<<(unsigned)grid, BT_THREADS, smem, s->stream>>>(s->amps, lam, a);
    }
    rc = launch_check("adjoint pass");
  }
  cudaFreeAsync(d_ops, s->stream);
  cudaFreeAsync(d_mats, s->stream);
  cudaFreeAsync(d_dgm, s->stream);
  cudaFreeAsync(d_rpm, s->stream);
  return rc;
}

static bool g_adj_fused = true;

extern "C" int qs_set_adjoint_fused(int on) {
  g_adj_fused = on != 0;
  return QS_OK;
}

static int gen_of(const qs_gate& g) {
  switch (g.type) {
    case QS_RX: return GEN_X;
    case QS_RY: return GEN_Y;
    case QS_RZ: return GEN_Z;
    case QS_P: case QS_CR: return GEN_P;
    default: return GEN_NONE;
  }
}

// Launch lambda = (H/S) psi for the whole Pauli sum (several launches if it is long).
static int apply_hamiltonian(qs_state* s, const double2* psi, double2* lam, const qs_pauli* terms, size_t nterms,
                             double S) {
  // group by X mask, preserving first-appearance order
  std::vector<uint64_t> xms;
  std::vector<std::vector<size_t>> members;
  for (size_t k = 0; k < nterms; ++k) {
    size_t gidx = 0;
    while (gidx < xms.size() && xms[gidx] != terms[k].xmask) ++gidx;
    if (gidx == xms.size()) {
      xms.push_back(terms[k].xmask);
      members.emplace_back();
    }
    members[gidx].push_back(k);
  }
  HArgs* h = new (std::nothrow) HArgs;
  if (!h) return fail(QS_ERR_OOM, "host allocation failed");
  h->N = 1ull << s->n;
  h->accumulate = 0;
  int rc = QS_OK;
  size_t gi = 0;
  const int grid = (int)std::min<uint64_t>((h->N + 255) / 256, 152 * 16);
  while (gi < xms.size() || (xms.empty() && !h->accumulate)) {
    h->nterms = 0;
    h->ngroups = 0;
    while (gi < xms.size() && h->ngroups < HMAX && h->nterms + (int)members[gi].size() <= HMAX) {
      h->gxm[h->ngroups] = xms[gi];
      h->gstart[h->ngroups] = h->nterms;
      for (size_t k : members[gi]) {
        const qs_pauli& t = terms[k];
        int ny = __builtin_popcountll(t.xmask & t.zmask) & 3;
        double c = t.coef / S;
        h->zm[h->nterms] = t.zmask;
        h->c[h->nterms] = (ny >= 2) ? -c : c;
        h->cq[h->nterms] = q60_from_double(h->c[h->nterms]);
        h->imag[h->nterms] = ny & 1;
        ++h->nterms;
      }
      ++h->ngroups;
      ++gi;
    }
    if (h->ngroups == 0 && gi < xms.size()) {
      rc = fail(QS_ERR_UNSUPPORTED, "more than %d terms share one X mask", HMAX);
      break;
    }
    h->gstart[h->ngroups] = h->nterms;
    {
      KTimer kt(s, QS_K_ADJOINT, 0, h->nterms, 0, 0, (double)h->N * (1 + h->ngroups), 0.0);
      k_apply_h<<<grid, 256, 0, s->stream>>>(psi, lam, *h);
    }
    if ((rc = launch_check("apply_h")) != QS_OK) break;
    h->accumulate = 1;
    if (xms.empty()) break;
  }
  delete h;
  return rc;
}

}  // namespace qs

using namespace qs;

extern "C" int qs_adjoint_grad(qs_state* s, const qs_gate* gates, size_t ng, const double* params, size_t np,
                               const qs_pauli* terms, size_t nterms, double* energy, double* grad) {
  clear_error();
  QS_TRY(check_state(s));
  if (s->prec == 64) return fail(QS_ERR_UNSUPPORTED, "adjoint gradients need a complex128 state");
  if (!energy || (np && !grad) || (nterms && !terms)) return fail(QS_ERR_INVALID_ARG, "NULL argument");
  QS_TRY(validate_gates(gates, ng, s->n, params));
  const uint64_t full = s->n >= 64 ? ~0ull : ((1ull << s->n) - 1);
  double csum = 0.0;
  for (size_t k = 0; k < nterms; ++k) {
    if ((terms[k].xmask | terms[k].zmask) & ~full) return fail(QS_ERR_INVALID_ARG, "term %zu exceeds n", k);
    csum += fabs(terms[k].coef);
  }
  size_t nslots = 0;
  for (size_t k = 0; k < ng; ++k) {
    if (gates[k].param_idx < 0) continue;
    if ((size_t)gates[k].param_idx >= np) return fail(QS_ERR_INVALID_ARG, "gate %zu reads params[%d] >= np", k,
                                                      gates[k].param_idx);
    if (gen_of(gates[k]) == GEN_NONE)
      return fail(QS_ERR_UNSUPPORTED, "gate %zu: gradients are defined for RX, RY, RZ, P and CR parameters", k);
    ++nslots;
  }
  const int n = s->n;
  const uint64_t N = 1ull << n;
  const size_t bytes = N * sizeof(double2);
  // lambda lives next to the state for the duration of the call
  double2* lam = nullptr;
  QS_CUDA(dmalloc_async((void**)&lam, bytes, s->stream));
  const int nblocks = 608;
  double* part = nullptr;
  double* sums = nullptr;
  int rc = QS_OK;
  auto cleanup = [&]() {
    if (lam) cudaFreeAsync(lam, s->stream);
    if (part) cudaFreeAsync(part, s->stream);
    if (sums) cudaFreeAsync(sums, s->stream);
  };
  cudaError_t e = dmalloc_async((void**)&part, sizeof(double) * nblocks * (nslots + 1), s->stream);
  if (e == cudaSuccess) e = dmalloc_async((void**)&sums, sizeof(double) * (nslots + 1), s->stream);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "adjoint workspace");
  }
  // forward: psi = U_G ... U_1 |0>, fused
  const double S = csum > 0 ? exp2(ceil(log2(csum))) : 1.0;
  qs_plan* plan = nullptr;
  if ((rc = qs_set_zero(s)) == QS_OK && (rc = qs_plan_create(n, gates, ng, QS_PLAN_GREEDY, 5, &plan)) == QS_OK)
    rc = qs_apply(s, gates, ng, params, plan);
  if (plan) qs_plan_free(plan);
  bool fixed = false;
  if (rc == QS_OK) rc = choose_fixed(s, &fixed);
  if (rc == QS_OK) rc = apply_hamiltonian(s, s->amps, lam, terms, nterms, S);
  if (rc == QS_OK) {
    KTimer kt(s, QS_K_ADJOINT, 0, 0, 0, 0, 2.0 * N, 2.0 * N);
    k_dot_re<<<nblocks, 256, 0, s->stream>>>(s->amps, lam, N, part + (size_t)nslots * nblocks);
    rc = launch_check("dot");
  }
  // backward
  std::vector<int> slot_param;
  size_t slot = 0;
  const bool fused = fixed && g_adj_fused;
  if (rc == QS_OK && fused) {
    e = cudaMemsetAsync(part, 0, sizeof(double) * nblocks * nslots, s->stream);
    rc = e == cudaSuccess ? backward_fused(s, lam, gates, ng, params, part, slot_param) : cuda_fail(e, "memset");
  }
  for (size_t kk = fused ? 0 : ng; rc == QS_OK && kk-- > 0;) {
    const qs_gate& g = gates[kk];
    qs_gate inv = g;
    inv.dagger = !g.dagger;
    int t;
    uint64_t cm;
    Mat2 m;
    if ((rc = gate_qubits(inv, n, &t, &cm)) != QS_OK) break;
    if ((rc = gate_matrix(inv, params, &m)) != QS_OK) break;
    Op1 op = classify(t, cm, m);
    AdjArgs a;
    for (int i = 0; i < 4; ++i) {
      a.m[i] = make_double2(m.m[i].re, m.m[i].im);
      a.q[i] = qc_make(m.m[i].re, m.m[i].im);
    }
    a.cmask = cm;
    a.t = t;
    a.cls = op.cls;
    a.code0 = op.code0;
    a.code1 = op.code1;
    a.gen = g.param_idx >= 0 ? gen_of(g) : GEN_NONE;
    a.gsign = g.dagger ? -1.0 : 1.0;
    a.slot = (int)slot;
    if (a.gen == GEN_NONE && op.cls == OP_IDENTITY) continue;
    uint64_t fx = cm | (1ull << t);
    a.nfix = 0;
    for (int b = 0; b < 64; ++b)
      if ((fx >> b) & 1) a.fix[a.nfix++] = b;
    a.items = (int64_t)1 << (n - a.nfix);
    {
      KTimer kt(s, QS_K_ADJOINT, 1, 1, 1ull << t, cm, 4.0 * a.items, a.gen != GEN_NONE ? 8.0 * a.items : 0.0);
      if (fixed) k_adj_step<true><<<nblocks, 256, 0, s->stream>>>(s->amps, lam, a, part);
      else k_adj_step<false><<<nblocks, 256, 0, s->stream>>>(s->amps, lam, a, part);
    }
    rc = launch_check("adjoint step");
    if (a.gen != GEN_NONE) {
      slot_param.push_back(g.param_idx);
      ++slot;
    }
  }
  std::vector<double> host(nslots + 1);
  if (rc == QS_OK) {
    k_slot_sums<<<(int)((nslots + 1 + 127) / 128), 128, 0, s->stream>>>(part, (int)nslots + 1, nblocks, sums);
    rc = launch_check("slot sums");
  }
  if (rc == QS_OK) {
    e = cudaMemcpyAsync(host.data(), sums, sizeof(double) * (nslots + 1), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "adjoint readback");
  }
  cleanup();
  if (rc != QS_OK) return rc;
  *energy = host[nslots] * S;
  for (size_t j = 0; j < np; ++j) grad[j] = 0.0;
  for (size_t j = 0; j < nslots; ++j) grad[slot_param[j]] += host[j] * S;
  // the state now holds U_1^dag ... U_G^dag psi_G = |0> up to rounding
  return QS_OK;
}
