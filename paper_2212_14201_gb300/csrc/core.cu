// State lifecycle, error reporting and host-side gate resolution of libqsim.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "fixed.h"
#include "internal.h"

namespace qs {

static thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

// ---- host-side fault injection ----------------------------------------------------
// One armed fault for the process: events of kind g_fault_kind (allocations through
// dmalloc / dmalloc_async / hmalloc_pinned, or launch checks) pass g_fault_after
// times, then the next g_fault_count fail (-1: all of them).  QS_FAULT in the
// environment arms it when the library loads.
static std::atomic<int> g_fault_kind{QS_FAULT_NONE};
static std::atomic<long long> g_fault_after{0};
static std::atomic<long long> g_fault_left{0};
static std::atomic<long long> g_fault_fired{0};
static thread_local bool t_injected = false;

static int fault_arm(int kind, long long after, long long count) {
  if (kind != QS_FAULT_NONE && kind != QS_FAULT_ALLOC && kind != QS_FAULT_LAUNCH)
    return fail(QS_ERR_INVALID_ARG, "fault kind %d", kind);
  if (after < 0 || count < -1 || count == 0) return fail(QS_ERR_INVALID_ARG, "fault after=%lld count=%lld", after, count);
  g_fault_kind.store(QS_FAULT_NONE);
  g_fault_after.store(after);
  g_fault_left.store(count);
  g_fault_fired.store(0);
  g_fault_kind.store(kind);
  return QS_OK;
}

bool fault_fire(int kind) {
  if (g_fault_kind.load(std::memory_order_relaxed) != kind) return false;
  if (g_fault_after.fetch_sub(1) > 0) return false;
  g_fault_after.store(0);
  long long left = g_fault_left.load();
  while (true) {
    if (left == 0) return false;
    if (left < 0) break;  // every event fails
    if (g_fault_left.compare_exchange_weak(left, left - 1)) break;
  }
  g_fault_fired.fetch_add(1);
  t_injected = true;
  return true;
}

// QS_FAULT = "alloc" | "launch", optionally ":after" and ":count" (count -1: every
// event after the first `after`); anything else leaves the library unarmed.
static int parse_fault_spec(const char* spec) {
  if (!spec || !*spec) return QS_OK;
  char kind[16] = {0};
  long long after = 0, count = 1;
  int got = sscanf(spec, "%15[a-z]:%lld:%lld", kind, &after, &count);
  if (got < 1) return fail(QS_ERR_INVALID_ARG, "QS_FAULT=%s", spec);
  int k = strcmp(kind, "alloc") == 0 ? QS_FAULT_ALLOC : strcmp(kind, "launch") == 0 ? QS_FAULT_LAUNCH : -1;
  if (k < 0) return fail(QS_ERR_INVALID_ARG, "QS_FAULT=%s: kind is alloc or launch", spec);
  return fault_arm(k, after, count);
}

static const int g_fault_from_env = parse_fault_spec(getenv("QS_FAULT"));

int cuda_fail(cudaError_t e, const char* what) {
  const bool inj = t_injected;
  t_injected = false;
  return fail(e == cudaErrorMemoryAllocation ? QS_ERR_OOM : QS_ERR_CUDA, "%s: %s%s", what,
              cudaGetErrorString(e), inj ? " (injected by the armed fault)" : "");
}

void clear_error() { g_err.clear(); }

int launch_check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  if (fault_fire(QS_FAULT_LAUNCH)) return cuda_fail(cudaErrorLaunchFailure, what);
  return QS_OK;
}

int check_state(const qs_state* s) {
  if (!s || !s->amps || s->n < 1 || s->n > QS_MAX_QUBITS) return fail(QS_ERR_INVALID_ARG, "invalid state handle");
  return QS_OK;
}

// Workspace: per-1024-amplitude block sums and prefixes for the sampler (and per
// superblock of 1024 blocks), plus per-CTA partial results of the reductions.
size_t workspace_bytes(int n) {
  size_t N = (size_t)1 << n;
  size_t L = N < 1024 ? N : 1024;
  size_t nb = N / L;
  size_t nsb = nb < 1024 ? 1 : nb / 1024;
  size_t sampler = (2 * (nb + 1) + 2 * (nsb + 1)) * sizeof(double) + (nb + 1 + 2 * (nsb + 1)) * sizeof(long long) + 256;
  size_t reduce = (size_t)1024 * 72 * sizeof(double) + 256;  // up to 1024 CTAs x (n + 2) values
  size_t hist = (size_t)304 * 4096 * sizeof(double);          // marginal histograms
  return std::max(sampler, std::max(reduce, hist)) + 4096;
}

int ensure_pinned(qs_state* s, size_t bytes) {
  if (s->pinned_bytes >= bytes) return QS_OK;
  if (s->pinned) cudaFreeHost(s->pinned);
  s->pinned = nullptr;
  s->pinned_bytes = 0;
  QS_CUDA(hmalloc_pinned(&s->pinned, bytes));
  s->pinned_bytes = bytes;
  return QS_OK;
}

// ---- instrumentation ------------------------------------------------------------
static unsigned long long g_launches = 0;

void note_launch(int count) { __atomic_fetch_add(&g_launches, (unsigned long long)count, __ATOMIC_RELAXED); }

static cudaEvent_t take_event(qs_state* s) {
  if (!s->event_pool.empty()) {
    cudaEvent_t e = s->event_pool.back();
    s->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

KTimer::KTimer(qs_state* st, int kind, int k, int n_ops, uint64_t qmask, uint64_t cmask, double items, double flops,
               double int_ops)
    : s(st), on(st->timing) {
  note_launch(1);
  if (!on) return;
  pt.rec.kind = kind;
  pt.rec.n = st->n;
  pt.rec.k = k;
  pt.rec.n_ops = n_ops;
  pt.rec.qubit_mask = qmask;
  pt.rec.ctrl_mask = cmask;
  pt.rec.items = items;
  pt.rec.flops = flops;
  pt.rec.int_ops = int_ops;
  pt.rec.ms = 0.0;
  pt.e0 = take_event(st);
  pt.e1 = take_event(st);
  if (!pt.e0 || !pt.e1) {
    on = false;
    return;
  }
  cudaEventRecord(pt.e0, st->stream);
}

KTimer::~KTimer() {
  if (!on) return;
  cudaEventRecord(pt.e1, s->stream);
  s->pending.push_back(pt);
}

// ---- gates --------------------------------------------------------------------

static bool two_qubit(int t) { return t == QS_CNOT || t == QS_CZ || t == QS_CR; }

int gate_qubits(const qs_gate& g, int n, int* target, uint64_t* cmask) {
  if (g.type < QS_I || g.type > QS_CR) return fail(QS_ERR_INVALID_ARG, "unknown gate code %d", g.type);
  if (g.q0 < 0 || g.q0 >= n) return fail(QS_ERR_INVALID_ARG, "qubit %d out of range for n=%d", g.q0, n);
  uint64_t full = n >= 64 ? ~0ull : ((1ull << n) - 1);
  if (g.ctrl_mask & ~full) return fail(QS_ERR_INVALID_ARG, "control mask 0x%llx exceeds n=%d",
                                       (unsigned long long)g.ctrl_mask, n);
  uint64_t cm = g.ctrl_mask;
  int t = g.q0;
  if (two_qubit(g.type)) {
    if (g.q1 < 0 || g.q1 >= n || g.q1 == g.q0)
      return fail(QS_ERR_INVALID_ARG, "two-qubit gate needs distinct qubits in range (got %d, %d)", g.q0, g.q1);
    t = g.q1;
    cm |= 1ull << g.q0;
  }
  if ((cm >> t) & 1) return fail(QS_ERR_INVALID_ARG, "target %d is also a control", t);
  *target = t;
  *cmask = cm;
  return QS_OK;
}

static C2 cexpi(double t) {
  double s, c;
  sincos(t, &s, &c);
  return {c, s};
}

int gate_matrix(const qs_gate& g, const double* params, Mat2* out) {
  double th = g.p[0];
  if (g.param_idx >= 0) {
    if (!params) return fail(QS_ERR_INVALID_ARG, "gate reads params[%d] but params is NULL", g.param_idx);
    th = params[g.param_idx];
  }
  const double r = M_SQRT1_2;
  C2* m = out->m;
  const C2 z{0, 0}, one{1, 0};
  double s, c;
  sincos(0.5 * th, &s, &c);
  switch (g.type) {
    case QS_I: m[0] = one; m[1] = z; m[2] = z; m[3] = one; break;
    case QS_H: m[0] = {r, 0}; m[1] = {r, 0}; m[2] = {r, 0}; m[3] = {-r, 0}; break;
    case QS_X: case QS_CNOT: m[0] = z; m[1] = one; m[2] = one; m[3] = z; break;
    case QS_Y: m[0] = z; m[1] = {0, -1}; m[2] = {0, 1}; m[3] = z; break;
    case QS_Z: case QS_CZ: m[0] = one; m[1] = z; m[2] = z; m[3] = {-1, 0}; break;
    case QS_S: m[0] = one; m[1] = z; m[2] = z; m[3] = {0, 1}; break;
    case QS_T: m[0] = one; m[1] = z; m[2] = z; m[3] = {r, r}; break;
    case QS_RX: m[0] = {c, 0}; m[1] = {0, -s}; m[2] = {0, -s}; m[3] = {c, 0}; break;
    case QS_RY: m[0] = {c, 0}; m[1] = {-s, 0}; m[2] = {s, 0}; m[3] = {c, 0}; break;
    case QS_RZ: m[0] = cexpi(-0.5 * th); m[1] = z; m[2] = z; m[3] = cexpi(0.5 * th); break;
    case QS_U3: {
      C2 el = cexpi(g.p[2]), ep = cexpi(g.p[1]), epl = cexpi(g.p[1] + g.p[2]);
      m[0] = {c, 0};
      m[1] = {-el.re * s, -el.im * s};
      m[2] = {ep.re * s, ep.im * s};
      m[3] = {epl.re * c, epl.im * c};
      break;
    }
    case QS_P: case QS_CR: m[0] = one; m[1] = z; m[2] = z; m[3] = cexpi(th); break;
    default: return fail(QS_ERR_INVALID_ARG, "unknown gate code %d", g.type);
  }
  if (g.dagger) {
    C2 a = m[0], b = m[1], cc = m[2], d = m[3];
    m[0] = {a.re, -a.im};
    m[1] = {cc.re, -cc.im};
    m[2] = {b.re, -b.im};
    m[3] = {d.re, -d.im};
  }
  return QS_OK;
}

int validate_gates(const qs_gate* gates, size_t ng, int n, const double* params) {
  if (ng && !gates) return fail(QS_ERR_INVALID_ARG, "gates is NULL");
  for (size_t k = 0; k < ng; ++k) {
    int t;
    uint64_t cm;
    int rc = gate_qubits(gates[k], n, &t, &cm);
    if (rc) return fail(rc, "gate %zu: %s", k, qs_last_error());
    if (gates[k].param_idx >= 0 && !params)
      return fail(QS_ERR_INVALID_ARG, "gate %zu reads params[%d] but params is NULL", k, gates[k].param_idx);
  }
  return QS_OK;
}

int unit_code(const C2& z) {
  if (z.im == 0.0 && z.re == 1.0) return U_ONE;
  if (z.re == 0.0 && z.im == 1.0) return U_I;
  if (z.im == 0.0 && z.re == -1.0) return U_MINUS_ONE;
  if (z.re == 0.0 && z.im == -1.0) return U_MINUS_I;
  return U_GENERAL;
}

Op1 classify(int target, uint64_t cmask, const Mat2& m) {
  Op1 op;
  op.target = target;
  op.cmask = cmask;
  op.m = m;
  op.code0 = op.code1 = U_GENERAL;
  auto zero = [](const C2& z) { return z.re == 0.0 && z.im == 0.0; };
  const C2* u = m.m;
  if (zero(u[1]) && zero(u[2])) {
    op.code0 = unit_code(u[0]);
    op.code1 = unit_code(u[3]);
    if (op.code0 == U_ONE && op.code1 == U_ONE) op.cls = OP_IDENTITY;
    else if (op.code0 == U_ONE) op.cls = OP_PHASE1;
    else op.cls = OP_DIAG;
  } else if (zero(u[0]) && zero(u[3])) {
    op.cls = OP_ANTI;
    op.code0 = unit_code(u[1]);
    op.code1 = unit_code(u[2]);
  } else if (u[0].im == 0.0 && u[1].im == 0.0 && u[2].im == 0.0 && u[3].im == 0.0) {
    op.cls = OP_REAL;
  } else {
    op.cls = OP_GENERAL;
  }
  return op;
}

}  // namespace qs

using namespace qs;

// ---- C ABI: library + states ----------------------------------------------------

extern "C" const char* qs_last_error(void) { return g_err.c_str(); }

extern "C" int qs_max_qubits(void) { return QS_MAX_QUBITS; }

extern "C" int qs_fault_set(int kind, long long after, long long count) {
  clear_error();
  return fault_arm(kind, after, count);
}

extern "C" int qs_fault_get(int* kind, long long* after, long long* left, long long* fired, int* env_status) {
  if (kind) *kind = g_fault_kind.load();
  if (after) *after = std::max(0ll, g_fault_after.load());
  if (left) *left = g_fault_left.load();
  if (fired) *fired = g_fault_fired.load();
  if (env_status) *env_status = g_fault_from_env;
  return QS_OK;
}

__global__ void k_set_zero(double2* __restrict__ a, size_t N) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < N; i += stride) a[i] = make_double2(i == 0 ? 1.0 : 0.0, 0.0);
}

__global__ void k_set_zero(float2* __restrict__ a, size_t N) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < N; i += stride) a[i] = make_float2(i == 0 ? 1.0f : 0.0f, 0.0f);
}

static int create(int n, void* dev, void* stream, qs_state** out, int prec = 128) {
  clear_error();
  if (!out) return fail(QS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_ERR_INVALID_ARG, "n=%d outside 1..%d", n, QS_MAX_QUBITS);
  if (dev && ((uintptr_t)dev & 15)) return fail(QS_ERR_INVALID_ARG, "external buffer not 16-byte aligned");
  qs_state* s = new (std::nothrow) qs_state;
  if (!s) return fail(QS_ERR_OOM, "host allocation failed");
  s->n = n;
  s->prec = prec;
  s->stream = (cudaStream_t)stream;
  cudaGetDevice(&s->device);
  size_t bytes = ((size_t)1 << n) * amp_bytes(s);
  if (dev) {
    s->amps = (double2*)dev;
    s->owns = false;
    s->bound = 0;
  } else {
    cudaError_t e = dmalloc(&s->amps, bytes);
    if (e != cudaSuccess) {
      delete s;
      return cuda_fail(e, "cudaMalloc(state)");
    }
    s->owns = true;
  }
  s->ws_bytes = workspace_bytes(n);
  cudaError_t e = dmalloc(&s->ws, s->ws_bytes);
  if (e != cudaSuccess) {
    if (s->owns) cudaFree(s->amps);
    delete s;
    return cuda_fail(e, "cudaMalloc(workspace)");
  }
  *out = s;
  return QS_OK;
}

extern "C" int qs_set_zero(qs_state* s) {
  QS_TRY(check_state(s));
  size_t N = (size_t)1 << s->n;
  int blocks = (int)std::min<size_t>((N + 255) / 256, 152 * 16);
  KTimer kt(s, QS_K_OTHER, 0, 0, 0, 0, (double)N, 0.0);
  with_amps(s, [&](auto* a) {
    k_set_zero<<<blocks, 256, 0, s->stream>>>(a, N);
    return QS_OK;
  });
  s->bound = 1;
  return launch_check("set_zero");
}

extern "C" int qs_set_arith(qs_state* s, int mode) {
  QS_TRY(check_state(s));
  if (mode != QS_ARITH_AUTO && mode != QS_ARITH_FP64 && mode != QS_ARITH_FIXED)
    return fail(QS_ERR_INVALID_ARG, "arith mode %d", mode);
  if (s->prec == 64 && mode == QS_ARITH_FIXED)
    return fail(QS_ERR_UNSUPPORTED, "complex64 states compute in FP32 (no Q60 engine)");
  s->arith = mode;
  return QS_OK;
}

extern "C" int qs_state_modified(qs_state* s) {
  QS_TRY(check_state(s));
  s->bound = 0;
  return QS_OK;
}

namespace qs {
int choose_fixed(qs_state* s, bool* fixed) {
  *fixed = false;
  if (s->arith == QS_ARITH_FP64 || s->prec == 64) return QS_OK;
  if (s->bound == 0) {
    double norm2 = 0.0;
    QS_TRY(qs_probs(s, nullptr, 0, &norm2, 0));
    // every component is at most the norm; unitary gates keep the norm
    s->bound = (norm2 <= Q60_MAX_ABS * Q60_MAX_ABS) ? 1 : 2;
  }
  if (s->bound == 1) {
    *fixed = true;
    return QS_OK;
  }
  if (s->arith == QS_ARITH_FIXED)
    return fail(QS_ERR_UNSUPPORTED, "Q60 arithmetic needs a state of norm <= %.2f", Q60_MAX_ABS);
  return QS_OK;
}
}  // namespace qs

extern "C" int qs_alloc(int n, void* stream, qs_state** out) {
  QS_TRY(create(n, nullptr, stream, out));
  int rc = qs_set_zero(*out);
  if (rc) {
    qs_free(*out);
    *out = nullptr;
  }
  return rc;
}

extern "C" int qs_alloc_c64(int n, void* stream, qs_state** out) {
  QS_TRY(create(n, nullptr, stream, out, 64));
  int rc = qs_set_zero(*out);
  if (rc) {
    qs_free(*out);
    *out = nullptr;
  }
  return rc;
}

extern "C" int qs_state_precision(const qs_state* s, int* bits) {
  QS_TRY(check_state(s));
  if (!bits) return fail(QS_ERR_INVALID_ARG, "bits is NULL");
  *bits = s->prec;
  return QS_OK;
}

extern "C" int qs_alloc_external(int n, void* device_amps, void* stream, qs_state** out) {
  if (!device_amps) return fail(QS_ERR_INVALID_ARG, "device_amps is NULL");
  return create(n, device_amps, stream, out);
}

extern "C" int qs_free(qs_state* s) {
  if (!s) return QS_OK;
  cudaStreamSynchronize(s->stream);
  if (s->owns && s->amps) cudaFree(s->amps);
  if (s->ws) cudaFree(s->ws);
  if (s->pinned) cudaFreeHost(s->pinned);
  if (s->tables) cudaFree(s->tables);
  if (s->tables_pinned) cudaFreeHost(s->tables_pinned);
  if (s->tables_ev) cudaEventDestroy(s->tables_ev);
  for (auto& p : s->pending) {
    cudaEventDestroy(p.e0);
    cudaEventDestroy(p.e1);
  }
  for (auto e : s->event_pool) cudaEventDestroy(e);
  delete s;
  return QS_OK;
}

extern "C" int qs_num_qubits(const qs_state* s) {
  if (check_state(s)) return QS_ERR_INVALID_ARG;
  return s->n;
}

extern "C" int qs_device_ptr(const qs_state* s, void** out) {
  QS_TRY(check_state(s));
  if (!out) return fail(QS_ERR_INVALID_ARG, "out is NULL");
  *out = s->amps;
  return QS_OK;
}

extern "C" int qs_set_state(qs_state* s, const double* amps, int on_device) {
  QS_TRY(check_state(s));
  if (!amps) return fail(QS_ERR_INVALID_ARG, "amps is NULL");
  size_t bytes = ((size_t)1 << s->n) * amp_bytes(s);
  QS_CUDA(cudaMemcpyAsync(s->amps, amps, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          s->stream));
  if (!on_device) QS_CUDA(cudaStreamSynchronize(s->stream));
  s->bound = 0;
  return QS_OK;
}

extern "C" int qs_get_state(const qs_state* s, double* dst, int on_device) {
  QS_TRY(check_state(s));
  if (!dst) return fail(QS_ERR_INVALID_ARG, "dst is NULL");
  size_t bytes = ((size_t)1 << s->n) * amp_bytes(s);
  QS_CUDA(cudaMemcpyAsync(dst, s->amps, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          s->stream));
  if (!on_device) QS_CUDA(cudaStreamSynchronize(s->stream));
  return QS_OK;
}

extern "C" int qs_sync(const qs_state* s) {
  QS_TRY(check_state(s));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  return QS_OK;
}

extern "C" int qs_timing_enable(qs_state* s, int on) {
  QS_TRY(check_state(s));
  s->timing = on != 0;
  return QS_OK;
}

extern "C" int qs_timing_fetch(qs_state* s, qs_timing_record* out, size_t cap, size_t* count) {
  QS_TRY(check_state(s));
  if (!count || (cap && !out)) return fail(QS_ERR_INVALID_ARG, "NULL output");
  QS_CUDA(cudaStreamSynchronize(s->stream));
  size_t i = 0;
  for (auto& p : s->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.e0, p.e1);
    p.rec.ms = ms;
    if (i < cap) out[i] = p.rec;
    ++i;
    s->event_pool.push_back(p.e0);
    s->event_pool.push_back(p.e1);
  }
  *count = i;
  s->pending.clear();
  return QS_OK;
}

extern "C" uint64_t qs_launch_count(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

extern "C" int qs_gate_list_dagger(const qs_gate* in, size_t ng, qs_gate* out) {
  if (ng && (!in || !out)) return fail(QS_ERR_INVALID_ARG, "NULL gate list");
  if (ng && in == out) return fail(QS_ERR_INVALID_ARG, "out aliases in");
  for (size_t i = 0; i < ng; ++i) {
    out[i] = in[ng - 1 - i];
    out[i].dagger = !in[ng - 1 - i].dagger;
  }
  return QS_OK;
}
