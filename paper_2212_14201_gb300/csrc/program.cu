// Mid-circuit measurement with collapse, and programs with classical control:
// the paper's QMeasure, QIf, QWhile and ClassicalProg nodes (Section "Core" and
// its QIf / QWhile listings; classical operators per Section "Qif and QWhile").
//
// Measurement of qubit q with a draw u in [0, 1):
//   p0, p1 = squared norms of the parts with bit q = 0 / 1 (one reduction pass);
//   outcome = 0 if u (p0 + p1) < p0, else 1;
//   collapse (one pass): the other part is zeroed (written, not read), the kept
//   part scaled by 1 / sqrt(p_outcome).
// Inside a program, measurement k (0-based, in execution order) draws
// u_k = u01(SplitMix64 output k of the stream seeded `seed`), the sampler's
// generator.  The interpreter runs on the host; every gate run is a qs_apply
// (plain per-gate kernels, or one cached greedy fusion plan per gate run).
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace qs {

// a_x *= scale where (x & mask) == want; a_x = 0 elsewhere (complex128, or
// complex64 scaled in double and rounded once).
__device__ __forceinline__ double2 scaled(double2 v, double c) { return make_double2(v.x * c, v.y * c); }
__device__ __forceinline__ float2 scaled(float2 v, double c) {
  return make_float2((float)((double)v.x * c), (float)((double)v.y * c));
}

template <class A>
__global__ void k_collapse(A* __restrict__ a, uint64_t N, uint64_t mask, uint64_t want, double scale) {
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x) {
    if ((x & mask) == want) a[x] = scaled(a[x], scale);
    else a[x] = A{};
  }
}

static int collapse(qs_state* s, uint64_t mask, uint64_t want, double scale) {
  const uint64_t N = 1ull << s->n;
  constexpr int T = 256;
  int sms = 0;
  QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
  const uint64_t grid = std::min<uint64_t>((N + T - 1) / T, (uint64_t)std::max(1, sms) * 16);
  KTimer kt(s, QS_K_OTHER, 0, 1, mask, 0, (double)N, 2.0 * (double)(N >> __builtin_popcountll(mask)));
  with_amps(s, [&](auto* a) {
    k_collapse<<<(unsigned)grid, T, 0, s->stream>>>(a, N, mask, want, scale);
    return QS_OK;
  });
  return launch_check("collapse kernel");
}

static int measure_one(qs_state* s, int qubit, double u, int* outcome, double* p1_out) {
  double p[2] = {0.0, 0.0};
  QS_TRY(marginal_host(s, &qubit, 1, p, true));
  // the exact integer marginal is accurate to 2^-45 absolute: for a small branch
  // (whose probability scales the collapse) take the FP64 sums instead
  if (std::min(p[0], p[1]) < 0x1p-20) QS_TRY(marginal_host(s, &qubit, 1, p, false));
  const double tot = p[0] + p[1];
  if (!(tot > 0.0)) return fail(QS_ERR_INVALID_ARG, "measurement of a zero state");
  const int o = (u * tot < p[0]) ? 0 : 1;
  const double scale = 1.0 / sqrt(o ? p[1] : p[0]);
  QS_TRY(collapse(s, 1ull << qubit, (uint64_t)o << qubit, scale));
  // the state now has norm 1 up to rounding: it stays within the Q60 bound
  if (s->bound == 2) s->bound = 0;
  *outcome = o;
  if (p1_out) *p1_out = p[1] / tot;
  return QS_OK;
}

// ---- the interpreter -------------------------------------------------------------
struct Runner {
  qs_state* s;
  const qs_pinstr* prog;
  const qs_gate* gates;
  size_t ngates;
  const double* params;
  bool fuse;
  uint64_t seed, max_iters, nmeas = 0;
  int64_t* cbits;
  size_t ncbits;
  double* record;
  size_t record_cap;
  std::vector<qs_plan*> plans;  // per instruction, built on first use

  ~Runner() {
    for (qs_plan* p : plans)
      if (p) qs_plan_free(p);
  }

  int value(int32_t idx, int64_t imm, int64_t* v) const {
    if (idx < 0) {
      *v = imm;
      return QS_OK;
    }
    if ((size_t)idx >= ncbits) return fail(QS_ERR_INVALID_ARG, "classical register %d out of range", idx);
    *v = cbits[idx];
    return QS_OK;
  }

  int write(int32_t idx, int64_t v) {
    if (idx < 0 || (size_t)idx >= ncbits) return fail(QS_ERR_INVALID_ARG, "classical register %d out of range", idx);
    cbits[idx] = v;
    return QS_OK;
  }

  static int alu(int op, int64_t a, int64_t b, int64_t* out) {
    const uint64_t ua = (uint64_t)a, ub = (uint64_t)b;
    switch (op) {
      case QS_CA_MOV: *out = a; break;
      case QS_CA_ADD: *out = (int64_t)(ua + ub); break;
      case QS_CA_SUB: *out = (int64_t)(ua - ub); break;
      case QS_CA_MUL: *out = (int64_t)(ua * ub); break;
      case QS_CA_DIV:
        if (b == 0) return fail(QS_ERR_INVALID_ARG, "classical division by zero");
        if (a == INT64_MIN && b == -1) return fail(QS_ERR_INVALID_ARG, "classical division overflow");
        *out = a / b;
        break;
      case QS_CA_AND: *out = (a != 0 && b != 0) ? 1 : 0; break;
      case QS_CA_OR: *out = (a != 0 || b != 0) ? 1 : 0; break;
      case QS_CA_XOR: *out = a ^ b; break;
      case QS_CA_LT: *out = a < b; break;
      case QS_CA_LE: *out = a <= b; break;
      case QS_CA_GT: *out = a > b; break;
      case QS_CA_GE: *out = a >= b; break;
      case QS_CA_EQ: *out = a == b; break;
      case QS_CA_NE: *out = a != b; break;
      case QS_CA_NOT: *out = a == 0; break;
      default: return fail(QS_ERR_INVALID_ARG, "unknown classical operator %d", op);
    }
    return QS_OK;
  }

  int gates_run(size_t at) {
    const qs_pinstr& in = prog[at];
    if (in.gate_begin > in.gate_end || in.gate_end > ngates)
      return fail(QS_ERR_INVALID_ARG, "instruction %zu: gate range outside the gate array", at);
    const size_t ng = (size_t)(in.gate_end - in.gate_begin);
    if (ng == 0) return QS_OK;
    const qs_gate* g = gates + in.gate_begin;
    if (!fuse) return qs_apply(s, g, ng, params, nullptr);
    if (!plans[at]) QS_TRY(qs_plan_create(s->n, g, ng, QS_PLAN_GREEDY, 5, &plans[at]));
    return qs_apply(s, g, ng, params, plans[at]);
  }

  int block(size_t begin, size_t end) {
    size_t i = begin;
    while (i < end) {
      const qs_pinstr& in = prog[i];
      switch (in.op) {
        case QS_PI_GATES:
          QS_TRY(gates_run(i));
          ++i;
          break;
        case QS_PI_MEASURE: {
          if (in.dst < 0 || (size_t)in.dst >= ncbits)
            return fail(QS_ERR_INVALID_ARG, "instruction %zu: classical register out of range", i);
          if (in.qubit < 0 || in.qubit >= s->n)
            return fail(QS_ERR_INVALID_ARG, "instruction %zu: qubit %d out of range", i, in.qubit);
          int o = 0;
          double p1 = 0.0;
          QS_TRY(measure_one(s, in.qubit, u01_of(splitmix64(seed, nmeas)), &o, &p1));
          if (record && nmeas < record_cap) record[nmeas] = p1;
          ++nmeas;
          cbits[in.dst] = o;
          ++i;
          break;
        }
        case QS_PI_ASSIGN: {
          int64_t a = 0, b = 0, v = 0;
          QS_TRY(value(in.lhs, in.imm, &a));
          QS_TRY(value(in.rhs, in.imm, &b));
          QS_TRY(alu(in.alu, a, b, &v));
          QS_TRY(write(in.dst, v));
          ++i;
          break;
        }
        case QS_PI_IF: {
          const size_t t0 = i + 1, t1 = t0 + in.n_then, e1 = t1 + in.n_else;
          if (e1 > end) return fail(QS_ERR_INVALID_ARG, "instruction %zu: if-blocks run past their parent", i);
          int64_t c = 0;
          QS_TRY(value(in.lhs, in.imm, &c));
          QS_TRY(c != 0 ? block(t0, t1) : block(t1, e1));
          i = e1;
          break;
        }
        case QS_PI_WHILE: {
          const size_t b0 = i + 1, b1 = b0 + in.n_then;
          if (b1 > end || in.n_else != 0)
            return fail(QS_ERR_INVALID_ARG, "instruction %zu: malformed while-block", i);
          for (uint64_t iters = 0;; ++iters) {
            int64_t c = 0;
            QS_TRY(value(in.lhs, in.imm, &c));
            if (c == 0) break;
            if (iters >= max_iters) return fail(QS_ERR_TIMEOUT, "instruction %zu: loop bound reached", i);
            QS_TRY(block(b0, b1));
          }
          i = b1;
          break;
        }
        default:
          return fail(QS_ERR_INVALID_ARG, "instruction %zu: unknown op %d", i, in.op);
      }
    }
    return QS_OK;
  }
};

}  // namespace qs

using namespace qs;

extern "C" int qs_measure(qs_state* s, int qubit, double u, int* outcome, double* p1) {
  clear_error();
  QS_TRY(check_state(s));
  if (!outcome) return fail(QS_ERR_INVALID_ARG, "outcome is NULL");
  if (qubit < 0 || qubit >= s->n) return fail(QS_ERR_INVALID_ARG, "qubit %d out of range", qubit);
  if (!(u >= 0.0 && u < 1.0)) return fail(QS_ERR_INVALID_ARG, "u must lie in [0, 1)");
  return measure_one(s, qubit, u, outcome, p1);
}

extern "C" int qs_run_program(qs_state* s, const qs_pinstr* prog, size_t nprog, const qs_gate* gates, size_t ngates,
                              const double* params, int fuse, uint64_t seed, uint64_t max_iters, int64_t* cbits,
                              size_t ncbits, double* record, size_t record_cap, uint64_t* nmeasured) {
  clear_error();
  QS_TRY(check_state(s));
  if (nprog && !prog) return fail(QS_ERR_INVALID_ARG, "prog is NULL");
  if (ngates && !gates) return fail(QS_ERR_INVALID_ARG, "gates is NULL");
  if (ncbits && !cbits) return fail(QS_ERR_INVALID_ARG, "cbits is NULL");
  if (record_cap && !record) return fail(QS_ERR_INVALID_ARG, "record is NULL");
  Runner r;
  r.s = s;
  r.prog = prog;
  r.gates = gates;
  r.ngates = ngates;
  r.params = params;
  r.fuse = fuse != 0;
  r.seed = seed;
  r.max_iters = max_iters;
  r.cbits = cbits;
  r.ncbits = ncbits;
  r.record = record;
  r.record_cap = record_cap;
  r.plans.assign(nprog, nullptr);
  const int rc = r.block(0, nprog);
  if (nmeasured) *nmeasured = r.nmeas;
  if (rc != QS_OK) return rc;
  QS_CUDA(cudaStreamSynchronize(s->stream));
  return QS_OK;
}
