// Internal declarations of libqsim (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qsim.h"

#define QS_MAX_QUBITS 34

struct qs_pending_timing {
  qs_timing_record rec;
  cudaEvent_t e0, e1;
};

struct qs_state {
  int n = 0;
  // 2^n amplitudes, device: complex128 (double2) when prec == 128, complex64
  // (float2, same pointer reinterpreted) when prec == 64
  double2* amps = nullptr;
  int prec = 128;
  bool owns = false;
  cudaStream_t stream = nullptr;
  int device = 0;
  // Reduction / sampling workspace (device), sized at creation for n.
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // Pinned host staging for small reduction results.
  void* pinned = nullptr;
  size_t pinned_bytes = 0;
  // Arithmetic of the gate kernels (QS_ARITH_*) and what is known about the
  // magnitude of the amplitudes: 1 = every |re|, |im| <= 1.5 (the Q60 engine is
  // safe), 2 = possibly larger, 0 = unknown (checked on the next apply).
  int arith = 0;
  int bound = 1;
  // Per-kernel timing log (qs_timing_enable / qs_timing_fetch).
  bool timing = false;
  std::vector<qs_pending_timing> pending;
  std::vector<cudaEvent_t> event_pool;
  // Phase tables of tile passes: device copy, pinned staging, and the event of the
  // last upload (the staging buffer is rewritten only after that copy ran).
  void* tables = nullptr;
  size_t tables_bytes = 0;
  void* tables_pinned = nullptr;
  size_t tables_pinned_bytes = 0;
  cudaEvent_t tables_ev = nullptr;
};

namespace qs {

// SplitMix64 output number s (0-based) of the stream seeded `seed`, in counter
// form state = seed + (s + 1) * gamma (Steele, Lea & Flood, OOPSLA 2014), and its
// mapping to [0, 1): the random draws of sampling and of measurement.
__host__ __device__ inline uint64_t splitmix64(uint64_t seed, uint64_t s) {
  uint64_t z = seed + (s + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ inline double u01_of(uint64_t z) { return (double)(z >> 11) * (1.0 / 9007199254740992.0); }


// Amplitude access for kernels templated on the stored element type: complex128
// or complex64, read as a double2 (float -> double is exact).
__device__ __forceinline__ double2 ld_amp(const double2* a, uint64_t i) { return a[i]; }
__device__ __forceinline__ double2 ld_amp(const float2* a, uint64_t i) {
  const float2 v = a[i];
  return make_double2((double)v.x, (double)v.y);
}
inline size_t amp_bytes(const qs_state* s) { return s->prec == 64 ? sizeof(float2) : sizeof(double2); }
// Calls f with the state's amplitude pointer typed by its precision.
template <class F>
int with_amps(const qs_state* s, F&& f) {
  if (s->prec == 64) return f(reinterpret_cast<float2*>(s->amps));
  return f(s->amps);
}

// ---- errors -------------------------------------------------------------------
int fail(int code, const char* fmt, ...);
// Marginal probabilities of `qubits` into host memory (qs_probs); allow_exact =
// false forces the FP64 reduction kernels.
int marginal_host(qs_state* s, const int* qubits, int nq, double* out, bool allow_exact);
int cuda_fail(cudaError_t e, const char* what);
void clear_error();
#define QS_CUDA(call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return ::qs::cuda_fail(e_, #call); \
  } while (0)
#define QS_TRY(expr)          \
  do {                        \
    int rc_ = (expr);         \
    if (rc_ != QS_OK) return rc_; \
  } while (0)

int check_state(const qs_state* s);
int launch_check(const char* what);  // cudaGetLastError after a launch

// ---- host-side fault injection (qs_fault_set, QS_FAULT) --------------------------
// True when the armed fault of `kind` (QS_FAULT_ALLOC or QS_FAULT_LAUNCH) fires at
// this event; the next cuda_fail on this thread then marks its message as injected.
bool fault_fire(int kind);
// Every device and pinned-host allocation of the library goes through these, so
// that an armed allocation fault fails it as cudaErrorMemoryAllocation would.
template <class T>
inline cudaError_t dmalloc(T** p, size_t bytes) {
  if (fault_fire(QS_FAULT_ALLOC)) return cudaErrorMemoryAllocation;
  return cudaMalloc((void**)p, bytes);
}
template <class T>
inline cudaError_t dmalloc_async(T** p, size_t bytes, cudaStream_t st) {
  if (fault_fire(QS_FAULT_ALLOC)) return cudaErrorMemoryAllocation;
  return cudaMallocAsync((void**)p, bytes, st);
}
template <class T>
inline cudaError_t hmalloc_pinned(T** p, size_t bytes) {
  if (fault_fire(QS_FAULT_ALLOC)) return cudaErrorMemoryAllocation;
  return cudaMallocHost((void**)p, bytes);
}

// ---- complex helpers (host) ---------------------------------------------------
struct C2 {
  double re, im;
};
struct Mat2 {
  C2 m[4];  // row-major: m[0]=U00 m[1]=U01 m[2]=U10 m[3]=U11
};

// Target qubit and full control mask of a record; validates indices.
int gate_qubits(const qs_gate& g, int n, int* target, uint64_t* cmask);
// 2x2 matrix of a record (dagger applied); params may be NULL if param_idx < 0.
int gate_matrix(const qs_gate& g, const double* params, Mat2* out);
int validate_gates(const qs_gate* gates, size_t ng, int n, const double* params);

// ---- one resolved one-qubit op (target + control mask + matrix + class) ---------
enum OpClass : int {
  OP_IDENTITY = 0,
  OP_PHASE1 = 1,   // diag(1, d1): touches the |1> half only
  OP_DIAG = 2,     // diag(d0, d1)
  OP_ANTI = 3,     // [[0, b], [c, 0]]
  OP_REAL = 4,     // real 2x2
  OP_GENERAL = 5,  // complex 2x2
};
// Multiplier codes for diagonal / anti-diagonal entries: exact unit phases are
// applied with sign flips and swaps (no floating-point instruction).
enum UnitCode : int { U_ONE = 0, U_I = 1, U_MINUS_ONE = 2, U_MINUS_I = 3, U_GENERAL = 4 };

struct Op1 {
  int cls;
  int target;
  uint64_t cmask;
  Mat2 m;
  int code0, code1;  // for PHASE1/DIAG: codes of d0,d1; ANTI: codes of b,c
};
Op1 classify(int target, uint64_t cmask, const Mat2& m);
int unit_code(const C2& z);

// ---- kernels (launchers) --------------------------------------------------------
// Whether the next gate kernels of this state run in Q60 fixed point (may
// synchronise once to bound an unknown state's magnitude).
int choose_fixed(qs_state* s, bool* fixed);
int launch_op1(qs_state* s, const Op1& op, bool fixed);  // complex64 states: FP32 arithmetic
int launch_dense(qs_state* s, const int* targets, int k, uint64_t cmask, const C2* mat);

// ---- planning ------------------------------------------------------------------
// One greedy fusion pass over `remaining` (indices in program order): `pass`
// receives the gates that run in a tile of at most m qubits containing `low`,
// `rest` the others (still in order); returns the tile's qubit mask.
uint64_t greedy_pass(const qs_gate* gates, const std::vector<int>& tgt, const std::vector<uint64_t>& cms,
                     const std::vector<uint32_t>& remaining, int m, uint64_t low, int max_ops,
                     std::vector<uint32_t>& pass, std::vector<uint32_t>& rest);
// The same scan starting from the qubit set `init` (it grows while it has fewer
// than m qubits, never by a qubit of `forbid`).
uint64_t greedy_pass_from(const qs_gate* gates, const std::vector<int>& tgt, const std::vector<uint64_t>& cms,
                          const std::vector<uint32_t>& remaining, int m, uint64_t init, int max_ops,
                          std::vector<uint32_t>& pass, std::vector<uint32_t>& rest, uint64_t forbid = 0);
// A starting qubit set for a pass: `low`, the first runnable gate's target and
// the most frequent targets among the next `window` runnable gates (m qubits).
uint64_t seed_qubits(const qs_gate* gates, const std::vector<int>& tgt, const std::vector<uint64_t>& cms,
                     const std::vector<uint32_t>& remaining, int m, uint64_t low, int window);

// Inputs of a cost model (0 for NULL).
int mlp_inputs(const qs_mlp* m);

// ---- instrumentation -------------------------------------------------------------
void note_launch(int count = 1);
// Brackets the kernels queued during its lifetime with timing events (if the
// state's log is enabled) and counts one launch.
struct KTimer {
  qs_state* s;
  qs_pending_timing pt;
  bool on;
  KTimer(qs_state* s, int kind, int k, int n_ops, uint64_t qmask, uint64_t cmask, double items, double flops,
         double int_ops = 0.0);
  ~KTimer();
};

// ---- workspace ------------------------------------------------------------------
size_t workspace_bytes(int n);
int ensure_pinned(qs_state* s, size_t bytes);

}  // namespace qs
