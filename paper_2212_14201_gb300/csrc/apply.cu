// Per-gate (plain mode) application kernels and the dense k-qubit matrix gate.
//
// Section "High-performance simulation" of the paper: a circuit is an iteration of
// gates and each gate sweeps the amplitude vector; "Performance of basic gates":
// X / CNOT / Toffoli are pure data movement.  Here every one-qubit op with any
// control mask is one launch that touches only the amplitudes it changes:
//   PHASE1  diag(1, d)     : amplitudes with target = 1 and controls = 1
//   DIAG    diag(d0, d1)   : the control-satisfied subspace
//   ANTI    [[0,b],[c,0]]  : swap (X, Y, CNOT, Toffoli) -- unit factors by sign flips
//   REAL / GENERAL 2x2     : pairs (x, x | 2^t) in the control-satisfied subspace
// Work items enumerate only the control-satisfied subspace by inserting zero bits
// at the sorted target/control positions, so a CNOT reads and writes half the
// vector and a Toffoli a quarter.
#include <algorithm>

#include "fixed.h"
#include "internal.h"

namespace qs {

struct OpArgs {
  double2 m[4];
  uint64_t cmask;   // all control bits (they are set in every touched index)
  int64_t items;    // work items (pairs, or single amplitudes for PHASE1)
  int t;            // target bit
  int nfix;         // sorted fixed positions (target + controls) to insert
  int fix[16];
  int code0, code1;
};

__device__ __forceinline__ double dneg(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

// Multiply by a unit phase given by code (1, i, -1, -i) without FP instructions.
__device__ __forceinline__ double2 mul_unit(double2 a, int code) {
  switch (code) {
    case U_ONE: return a;
    case U_I: return make_double2(dneg(a.y), a.x);
    case U_MINUS_ONE: return make_double2(dneg(a.x), dneg(a.y));
    default: return make_double2(a.y, dneg(a.x));  // U_MINUS_I
  }
}

__device__ __forceinline__ double2 cmul(double2 u, double2 a) {
  return make_double2(fma(u.x, a.x, -u.y * a.y), fma(u.x, a.y, u.y * a.x));
}

__device__ __forceinline__ double2 mul_code(double2 a, int code, double2 u) {
  return code == U_GENERAL ? cmul(u, a) : mul_unit(a, code);
}

__device__ __forceinline__ uint64_t expand(uint64_t i, const OpArgs& g) {
  for (int k = 0; k < g.nfix; ++k) {
    int f = g.fix[k];
    uint64_t lo = i & ((1ull << f) - 1);
    i = ((i >> f) << (f + 1)) | lo;
  }
  return i | g.cmask;
}

template <int CLS>
__global__ void __launch_bounds__(256) k_op1(double2* __restrict__ a, const OpArgs g) {
  const uint64_t tb = 1ull << g.t;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (uint64_t)g.items; i += stride) {
    uint64_t x0 = expand(i, g);
    if (CLS == OP_PHASE1) {
      uint64_t x1 = x0 | tb;
      a[x1] = mul_code(a[x1], g.code1, g.m[3]);
    } else {
      uint64_t x1 = x0 | tb;
      double2 a0 = a[x0], a1 = a[x1];
      double2 b0, b1;
      if (CLS == OP_DIAG) {
        b0 = mul_code(a0, g.code0, g.m[0]);
        b1 = mul_code(a1, g.code1, g.m[3]);
      } else if (CLS == OP_ANTI) {
        b0 = mul_code(a1, g.code0, g.m[1]);
        b1 = mul_code(a0, g.code1, g.m[2]);
      } else if (CLS == OP_REAL) {
        b0 = make_double2(fma(g.m[0].x, a0.x, g.m[1].x * a1.x), fma(g.m[0].x, a0.y, g.m[1].x * a1.y));
        b1 = make_double2(fma(g.m[2].x, a0.x, g.m[3].x * a1.x), fma(g.m[2].x, a0.y, g.m[3].x * a1.y));
      } else {
        b0.x = fma(g.m[0].x, a0.x, fma(-g.m[0].y, a0.y, fma(g.m[1].x, a1.x, -g.m[1].y * a1.y)));
        b0.y = fma(g.m[0].x, a0.y, fma(g.m[0].y, a0.x, fma(g.m[1].x, a1.y, g.m[1].y * a1.x)));
        b1.x = fma(g.m[2].x, a0.x, fma(-g.m[2].y, a0.y, fma(g.m[3].x, a1.x, -g.m[3].y * a1.y)));
        b1.y = fma(g.m[2].x, a0.y, fma(g.m[2].y, a0.x, fma(g.m[3].x, a1.y, g.m[3].y * a1.x)));
      }
      a[x0] = b0;
      a[x1] = b1;
    }
  }
}

// ---- complex64 states: the same ops in FP32 ----------------------------------------
struct OpArgs32 {
  float2 m[4];
  uint64_t cmask;
  int64_t items;
  int t;
  int nfix;
  int fix[16];
  int code0, code1;
};

__device__ __forceinline__ float2 mul_unit32(float2 a, int code) {
  switch (code) {
    case U_ONE: return a;
    case U_I: return make_float2(-a.y, a.x);
    case U_MINUS_ONE: return make_float2(-a.x, -a.y);
    default: return make_float2(a.y, -a.x);
  }
}

__device__ __forceinline__ float2 mul_code32(float2 a, int code, float2 u) {
  return code == U_GENERAL ? make_float2(fmaf(u.x, a.x, -u.y * a.y), fmaf(u.x, a.y, u.y * a.x)) : mul_unit32(a, code);
}

template <int CLS>
__global__ void __launch_bounds__(256) k_op1_c64(float2* __restrict__ a, const OpArgs32 g) {
  const uint64_t tb = 1ull << g.t;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (uint64_t)g.items; i += stride) {
    uint64_t x0 = i;
    for (int k = 0; k < g.nfix; ++k) {
      const int f = g.fix[k];
      x0 = ((x0 >> f) << (f + 1)) | (x0 & ((1ull << f) - 1));
    }
    x0 |= g.cmask;
    const uint64_t x1 = x0 | tb;
    if (CLS == OP_PHASE1) {
      a[x1] = mul_code32(a[x1], g.code1, g.m[3]);
      continue;
    }
    const float2 a0 = a[x0], a1 = a[x1];
    float2 b0, b1;
    if (CLS == OP_DIAG) {
      b0 = mul_code32(a0, g.code0, g.m[0]);
      b1 = mul_code32(a1, g.code1, g.m[3]);
    } else if (CLS == OP_ANTI) {
      b0 = mul_code32(a1, g.code0, g.m[1]);
      b1 = mul_code32(a0, g.code1, g.m[2]);
    } else if (CLS == OP_REAL) {
      b0 = make_float2(fmaf(g.m[0].x, a0.x, g.m[1].x * a1.x), fmaf(g.m[0].x, a0.y, g.m[1].x * a1.y));
      b1 = make_float2(fmaf(g.m[2].x, a0.x, g.m[3].x * a1.x), fmaf(g.m[2].x, a0.y, g.m[3].x * a1.y));
    } else {
      b0.x = fmaf(g.m[0].x, a0.x, fmaf(-g.m[0].y, a0.y, fmaf(g.m[1].x, a1.x, -g.m[1].y * a1.y)));
      b0.y = fmaf(g.m[0].x, a0.y, fmaf(g.m[0].y, a0.x, fmaf(g.m[1].x, a1.y, g.m[1].y * a1.x)));
      b1.x = fmaf(g.m[2].x, a0.x, fmaf(-g.m[2].y, a0.y, fmaf(g.m[3].x, a1.x, -g.m[3].y * a1.y)));
      b1.y = fmaf(g.m[2].x, a0.y, fmaf(g.m[2].y, a0.x, fmaf(g.m[3].x, a1.y, g.m[3].y * a1.x)));
    }
    a[x0] = b0;
    a[x1] = b1;
  }
}

// ---- Q60 fixed-point variant (arithmetic on the integer pipe; see fixed.h) --------
struct OpArgsFx {
  QC u[4];
  uint64_t cmask;
  int64_t items;
  int t, nfix;
  int fix[16];
  int code0, code1;
};

struct QV {
  int64_t re, im;
};

__device__ __forceinline__ QV q_load(const double2& a) { return {q60_from_double(a.x), q60_from_double(a.y)}; }
__device__ __forceinline__ double2 q_store(QV v) { return make_double2(q60_to_double(v.re), q60_to_double(v.im)); }

// real 2x2: u0.re*a0 + u1.re*a1
__device__ __forceinline__ QV q_real2(const QC& u0, QL a0r, QL a0i, const QC& u1, QL a1r, QL a1i) {
  QAcc re = qacc_new(), im = qacc_new();
  qacc_add(re, u0.re, a0r);
  qacc_add(re, u1.re, a1r);
  qacc_add(im, u0.re, a0i);
  qacc_add(im, u1.re, a1i);
  return {qacc_round(re), qacc_round(im)};
}

// u * a with u in Gauss form (three limb products)
__device__ __forceinline__ double2 fx_mul(double2 a, int code, const QC& u) {
  if (code != U_GENERAL) return mul_unit(a, code);
  const QV v = q_load(a);
  int64_t re, im;
  q60_gauss_mul(u, q60_split(v.re), q60_split(v.im), q60_split(v.re + v.im), &re, &im);
  return q_store(QV{re, im});
}

// One pair (x0, x0 | tb) of the op: matrices in Gauss form (real entries in u.re).
template <int CLS>
__device__ __forceinline__ void fx_pair(const OpArgsFx& g, double2 a0, double2 a1, double2& b0, double2& b1) {
  if (CLS == OP_DIAG) {
    b0 = fx_mul(a0, g.code0, g.u[0]);
    b1 = fx_mul(a1, g.code1, g.u[3]);
  } else if (CLS == OP_ANTI) {
    b0 = fx_mul(a1, g.code0, g.u[1]);
    b1 = fx_mul(a0, g.code1, g.u[2]);
  } else {
    const QV v0 = q_load(a0), v1 = q_load(a1);
    const QL r0 = q60_split(v0.re), i0 = q60_split(v0.im), r1 = q60_split(v1.re), i1 = q60_split(v1.im);
    if (CLS == OP_REAL) {
      b0 = q_store(q_real2(g.u[0], r0, i0, g.u[1], r1, i1));
      b1 = q_store(q_real2(g.u[2], r0, i0, g.u[3], r1, i1));
    } else {
      const QL s0 = q60_split(v0.re + v0.im), s1 = q60_split(v1.re + v1.im);
      int64_t re, im;
      q60_gauss_row(g.u[0], g.u[1], r0, i0, s0, r1, i1, s1, &re, &im);
      b0 = q_store(QV{re, im});
      q60_gauss_row(g.u[2], g.u[3], r0, i0, s0, r1, i1, s1, &re, &im);
      b1 = q_store(QV{re, im});
    }
  }
}

__device__ __forceinline__ uint64_t fx_index(const OpArgsFx& g, uint64_t i, uint64_t tb) {
  if (g.nfix == 1) return i + (i & ~(tb - 1));  // no controls: one zero bit at the target
  uint64_t x0 = i;
  for (int k = 0; k < g.nfix; ++k) {
    const int f = g.fix[k];
    x0 = ((x0 >> f) << (f + 1)) | (x0 & ((1ull << f) - 1));
  }
  return x0 | g.cmask;
}

// Two pairs per iteration, both loaded before either is computed (four 16-byte
// loads in flight per thread: the kernel moves the whole state through HBM).
template <int CLS>
__global__ void __launch_bounds__(256) k_op1_fx(double2* __restrict__ a, const OpArgsFx g) {
  const uint64_t tb = 1ull << g.t;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t items = (uint64_t)g.items;
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (CLS == OP_PHASE1) {
    for (; i < items; i += stride) {
      const uint64_t x1 = fx_index(g, i, tb) | tb;
      a[x1] = fx_mul(a[x1], g.code1, g.u[3]);
    }
    return;
  }
  for (; i + stride < items; i += 2 * stride) {
    const uint64_t p0 = fx_index(g, i, tb), q0 = fx_index(g, i + stride, tb);
    const double2 a0 = a[p0], a1 = a[p0 | tb], c0 = a[q0], c1 = a[q0 | tb];
    double2 b0, b1, d0, d1;
    fx_pair<CLS>(g, a0, a1, b0, b1);
    fx_pair<CLS>(g, c0, c1, d0, d1);
    a[p0] = b0;
    a[p0 | tb] = b1;
    a[q0] = d0;
    a[q0 | tb] = d1;
  }
  if (i < items) {
    const uint64_t p0 = fx_index(g, i, tb);
    double2 b0, b1;
    fx_pair<CLS>(g, a[p0], a[p0 | tb], b0, b1);
    a[p0] = b0;
    a[p0 | tb] = b1;
  }
}

static int grid_for(int64_t items, int threads) {
  int64_t b = (items + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

static bool needs_arith(const Op1& op) {
  if (op.cls == OP_REAL || op.cls == OP_GENERAL) return true;
  if (op.cls == OP_PHASE1) return op.code1 == U_GENERAL;
  return op.code0 == U_GENERAL || op.code1 == U_GENERAL;
}

static int launch_op1_c64(qs_state* s, const Op1& op) {
  OpArgs32 g;
  for (int i = 0; i < 4; ++i) g.m[i] = make_float2((float)op.m.m[i].re, (float)op.m.m[i].im);
  g.cmask = op.cmask;
  g.t = op.target;
  g.code0 = op.code0;
  g.code1 = op.code1;
  const uint64_t fixbits = op.cmask | (1ull << op.target);
  const int nf = __builtin_popcountll(fixbits);
  if (nf > 16) return fail(QS_ERR_UNSUPPORTED, "more than 15 controls");
  g.nfix = 0;
  for (int b = 0; b < 64; ++b)
    if ((fixbits >> b) & 1) g.fix[g.nfix++] = b;
  g.items = (int64_t)1 << (s->n - nf);
  const int T = 256;
  const int grid = grid_for(g.items, T);
  const double amps = op.cls == OP_PHASE1 ? (double)g.items : 2.0 * (double)g.items;
  double fpa = 0.0;
  if (op.cls == OP_GENERAL) fpa = 14.0;
  else if (op.cls == OP_REAL) fpa = 6.0;
  else if (op.cls == OP_PHASE1) fpa = op.code1 == U_GENERAL ? 6.0 : 0.0;
  else fpa = 0.5 * ((op.code0 == U_GENERAL ? 6.0 : 0.0) + (op.code1 == U_GENERAL ? 6.0 : 0.0));
  KTimer kt(s, op.cls, 1, 1, 1ull << op.target, op.cmask, amps, fpa * amps);
  float2* a = reinterpret_cast<float2*>(s->amps);
  switch (op.cls) {
    case OP_PHASE1: k_op1_c64<OP_PHASE1><<<grid, T, 0, s->stream>>>(a, g); break;
    case OP_DIAG: k_op1_c64<OP_DIAG><<<grid, T, 0, s->stream>>>(a, g); break;
    case OP_ANTI: k_op1_c64<OP_ANTI><<<grid, T, 0, s->stream>>>(a, g); break;
    case OP_REAL: k_op1_c64<OP_REAL><<<grid, T, 0, s->stream>>>(a, g); break;
    default: k_op1_c64<OP_GENERAL><<<grid, T, 0, s->stream>>>(a, g); break;
  }
  return launch_check("op1 kernel (complex64)");
}

int launch_op1(qs_state* s, const Op1& op, bool fixed) {
  if (op.cls == OP_IDENTITY) return QS_OK;
  if (s->prec == 64) return launch_op1_c64(s, op);
  if (fixed && needs_arith(op)) {
    OpArgsFx g;
    for (int i = 0; i < 4; ++i) g.u[i] = qc_make_gauss(op.m.m[i].re, op.m.m[i].im);  // Gauss form
    g.cmask = op.cmask;
    g.t = op.target;
    g.code0 = op.code0;
    g.code1 = op.code1;
    uint64_t fx = op.cmask | (1ull << op.target);
    int nf = __builtin_popcountll(fx);
    if (nf > 16) return fail(QS_ERR_UNSUPPORTED, "more than 15 controls");
    g.nfix = 0;
    for (int b = 0; b < 64; ++b)
      if ((fx >> b) & 1) g.fix[g.nfix++] = b;
    g.items = (int64_t)1 << (s->n - nf);
    const int T = 256;
    int grid = grid_for(g.items, T);
    double amps = op.cls == OP_PHASE1 ? (double)g.items : 2.0 * (double)g.items;
    // algorithmic limb products: 3 per real product; a general 2x2 needs 8 real
    // products per amplitude, a real 2x2 4, a general phase 4
    double ipa = op.cls == OP_GENERAL ? 24.0 : op.cls == OP_REAL ? 12.0 : 0.0;
    if (op.cls == OP_PHASE1) ipa = 12.0;
    if (op.cls == OP_DIAG || op.cls == OP_ANTI)
      ipa = 6.0 * ((op.code0 == U_GENERAL ? 1.0 : 0.0) + (op.code1 == U_GENERAL ? 1.0 : 0.0));
    KTimer kt(s, op.cls, 1, 1, 1ull << op.target, op.cmask, amps, 0.0, ipa * amps);
    switch (op.cls) {
      case OP_PHASE1: k_op1_fx<OP_PHASE1><<<grid, T, 0, s->stream>>>(s->amps, g); break;
      case OP_DIAG: k_op1_fx<OP_DIAG><<<grid, T, 0, s->stream>>>(s->amps, g); break;
      case OP_ANTI: k_op1_fx<OP_ANTI><<<grid, T, 0, s->stream>>>(s->amps, g); break;
      case OP_REAL: k_op1_fx<OP_REAL><<<grid, T, 0, s->stream>>>(s->amps, g); break;
      default: k_op1_fx<OP_GENERAL><<<grid, T, 0, s->stream>>>(s->amps, g); break;
    }
    return launch_check("op1 fixed-point kernel");
  }
  OpArgs g;
  for (int i = 0; i < 4; ++i) g.m[i] = make_double2(op.m.m[i].re, op.m.m[i].im);
  g.cmask = op.cmask;
  g.t = op.target;
  g.code0 = op.code0;
  g.code1 = op.code1;
  uint64_t fixbits = op.cmask | (1ull << op.target);
  int nf = __builtin_popcountll(fixbits);
  if (nf > 16) return fail(QS_ERR_UNSUPPORTED, "more than 15 controls");
  g.nfix = 0;
  for (int b = 0; b < 64; ++b)
    if ((fixbits >> b) & 1) g.fix[g.nfix++] = b;
  g.items = (int64_t)1 << (s->n - nf);
  const int T = 256;
  int grid = grid_for(g.items, T);
  // amplitudes touched and the floating-point operations the op needs per amplitude
  double amps = op.cls == OP_PHASE1 ? (double)g.items : 2.0 * (double)g.items;
  double fpa = 0.0;
  if (op.cls == OP_GENERAL) fpa = 14.0;
  else if (op.cls == OP_REAL) fpa = 6.0;
  else if (op.cls == OP_PHASE1) fpa = op.code1 == U_GENERAL ? 6.0 : 0.0;
  else if (op.cls == OP_DIAG) fpa = 0.5 * ((op.code0 == U_GENERAL ? 6.0 : 0.0) + (op.code1 == U_GENERAL ? 6.0 : 0.0));
  else if (op.cls == OP_ANTI) fpa = 0.5 * ((op.code0 == U_GENERAL ? 6.0 : 0.0) + (op.code1 == U_GENERAL ? 6.0 : 0.0));
  KTimer kt(s, op.cls, 1, 1, 1ull << op.target, op.cmask, amps, fpa * amps);
  switch (op.cls) {
    case OP_PHASE1: k_op1<OP_PHASE1><<<grid, T, 0, s->stream>>>(s->amps, g); break;
    case OP_DIAG: k_op1<OP_DIAG><<<grid, T, 0, s->stream>>>(s->amps, g); break;
    case OP_ANTI: k_op1<OP_ANTI><<<grid, T, 0, s->stream>>>(s->amps, g); break;
    case OP_REAL: k_op1<OP_REAL><<<grid, T, 0, s->stream>>>(s->amps, g); break;
    default: k_op1<OP_GENERAL><<<grid, T, 0, s->stream>>>(s->amps, g); break;
  }
  return launch_check("op1 kernel");
}

// ---- dense k-qubit matrix (1 <= k <= 5), matrix passed by value ------------------
template <int K>
struct DenseArgs {
  double2 m[(1 << K) * (1 << K)];
  uint64_t cmask;
  int64_t items;
  int tgt[K];
  int nfix;
  int fix[24];
};

template <int K>
__global__ void __launch_bounds__(128) k_dense(double2* __restrict__ a, const __grid_constant__ DenseArgs<K> g) {
  constexpr int D = 1 << K;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (uint64_t)g.items; i += stride) {
    uint64_t x = i;
    for (int k = 0; k < g.nfix; ++k) {
      int f = g.fix[k];
      x = ((x >> f) << (f + 1)) | (x & ((1ull << f) - 1));
    }
    x |= g.cmask;
    uint64_t idx[D];
    double2 v[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      uint64_t y = x;
#pragma unroll
      for (int b = 0; b < K; ++b)
        if ((j >> b) & 1) y |= 1ull << g.tgt[b];
      idx[j] = y;
      v[j] = a[y];
    }
#pragma unroll
    for (int r = 0; r < D; ++r) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        double2 u = g.m[r * D + c];
        re = fma(u.x, v[c].x, fma(-u.y, v[c].y, re));
        im = fma(u.x, v[c].y, fma(u.y, v[c].x, im));
      }
      a[idx[r]] = make_double2(re, im);
    }
  }
}

template <int K>
static int launch_dense_k(qs_state* s, const int* targets, uint64_t cmask, const C2* mat) {
  DenseArgs<K> g;
  constexpr int D = 1 << K;
  for (int i = 0; i < D * D; ++i) g.m[i] = make_double2(mat[i].re, mat[i].im);
  g.cmask = cmask;
  uint64_t fixed = cmask;
  for (int j = 0; j < K; ++j) {
    g.tgt[j] = targets[j];
    fixed |= 1ull << targets[j];
  }
  int nf = __builtin_popcountll(fixed);
  if (nf > 24) return fail(QS_ERR_UNSUPPORTED, "too many controls for a dense block");
  g.nfix = 0;
  for (int b = 0; b < 64; ++b)
    if ((fixed >> b) & 1) g.fix[g.nfix++] = b;
  g.items = (int64_t)1 << (s->n - nf);
  const int T = 128;
  double amps = (double)g.items * D;
  KTimer kt(s, QS_K_DENSE, K, 1, fixed & ~cmask, cmask, amps, (8.0 * D - 2.0) * amps);
  k_dense<K><<<grid_for(g.items, T), T, 0, s->stream>>>(s->amps, g);
  return launch_check("dense kernel");
}

int launch_dense(qs_state* s, const int* targets, int k, uint64_t cmask, const C2* mat) {
  switch (k) {
    case 1: return launch_dense_k<1>(s, targets, cmask, mat);
    case 2: return launch_dense_k<2>(s, targets, cmask, mat);
    case 3: return launch_dense_k<3>(s, targets, cmask, mat);
    case 4: return launch_dense_k<4>(s, targets, cmask, mat);
    case 5: return launch_dense_k<5>(s, targets, cmask, mat);
    default: return fail(QS_ERR_INVALID_ARG, "dense block width %d outside 1..5", k);
  }
}

}  // namespace qs

using namespace qs;

int qs_apply_plan(qs_state* s, const qs_gate* gates, size_t ng, const double* params, const qs_plan* plan,
                  bool fixed);

extern "C" int qs_apply(qs_state* s, const qs_gate* gates, size_t ng, const double* params, const qs_plan* plan) {
  clear_error();
  QS_TRY(check_state(s));
  QS_TRY(validate_gates(gates, ng, s->n, params));
  bool fixed = false;
  QS_TRY(choose_fixed(s, &fixed));
  if (plan) return qs_apply_plan(s, gates, ng, params, plan, fixed);
  for (size_t k = 0; k < ng; ++k) {
    int t;
    uint64_t cm;
    Mat2 m;
    QS_TRY(gate_qubits(gates[k], s->n, &t, &cm));
    QS_TRY(gate_matrix(gates[k], params, &m));
    QS_TRY(launch_op1(s, classify(t, cm, m), fixed));
  }
  return QS_OK;
}

extern "C" int qs_apply_matrix(qs_state* s, const int* targets, int k, uint64_t ctrl_mask, const double* mat) {
  clear_error();
  QS_TRY(check_state(s));
  if (!targets || !mat) return fail(QS_ERR_INVALID_ARG, "NULL targets or matrix");
  if (s->prec == 64) return fail(QS_ERR_UNSUPPORTED, "dense k-qubit matrices need a complex128 state");
  if (k < 1 || k > 5 || k > s->n) return fail(QS_ERR_INVALID_ARG, "k=%d outside 1..min(5, n)", k);
  uint64_t full = s->n >= 64 ? ~0ull : ((1ull << s->n) - 1);
  uint64_t tm = 0;
  for (int j = 0; j < k; ++j) {
    if (targets[j] < 0 || targets[j] >= s->n || ((tm >> targets[j]) & 1))
      return fail(QS_ERR_INVALID_ARG, "bad or repeated target %d", targets[j]);
    tm |= 1ull << targets[j];
  }
  if ((ctrl_mask & ~full) || (ctrl_mask & tm)) return fail(QS_ERR_INVALID_ARG, "bad control mask");
  s->bound = 0;  // the matrix need not be unitary
  return launch_dense(s, targets, k, ctrl_mask, (const C2*)mat);
}
