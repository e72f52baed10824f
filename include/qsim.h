/*
 * qsim.h -- C ABI of libqsim, a GB300 (sm_103a) full-amplitude state-vector
 * simulator for the hot path of QPanda's full-amplitude virtual machine
 * (arXiv 2212.14201): allocate n qubits, apply a gate program (optionally fused),
 * read probabilities, expectations and measurement samples, and take adjoint
 * gradients of parametrised circuits.
 *
 * Conventions
 *   - Qubit q is bit q of the basis index (qubit 0 = least significant bit).
 *   - A state is 2^n complex128 amplitudes, interleaved (re, im), 16 bytes each,
 *     contiguous in device memory.
 *   - Every call is asynchronous on the CUDA stream the state was created with,
 *     except where it returns results into host memory: those synchronise that
 *     stream before returning.
 *   - Host arrays passed in are owned by the caller and only read during the call.
 *   - Every entry point returns an int status: QS_OK (0) or a negative QS_ERR_*.
 *     Nothing aborts or exits the process.  qs_last_error() gives a message for
 *     the last failing call on the calling thread.
 *   - No entry point reads or writes memory the caller did not pass or the
 *     library did not allocate.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define QS_OK 0
#define QS_ERR_INVALID_ARG (-1)  /* bad qubit index, overlapping targets/controls, size out of range */
#define QS_ERR_OOM (-2)          /* a device or host allocation failed */
#define QS_ERR_CUDA (-3)         /* a CUDA runtime call or kernel launch failed */
#define QS_ERR_TIMEOUT (-4)      /* a bounded wait or loop gave up */
#define QS_ERR_UNSUPPORTED (-5)  /* well-formed request outside what is implemented */

/* ---- gate codes: the paper's gate set (API keyword list and the "Performance
 * of basic gates" experiment) plus P, the phase gate that CR controls.
 *   H = [[1,1],[1,-1]]/sqrt2          X = [[0,1],[1,0]]     Y = [[0,-i],[i,0]]
 *   Z = diag(1,-1)  S = diag(1,i)  T = diag(1,e^{i pi/4})  P(t) = diag(1,e^{it})
 *   RX(t) = exp(-i t X/2)  RY(t) = exp(-i t Y/2)  RZ(t) = exp(-i t Z/2)
 *   U3(t,f,l) = [[cos t/2, -e^{il} sin t/2], [e^{if} sin t/2, e^{i(f+l)} cos t/2]]
 *   CNOT(c,t) = X on t controlled by c; CZ(c,t) = Z on t controlled by c;
 *   CR(c,t,th) = P(th) on t controlled by c.                                    */
enum {
  QS_I = 0, QS_H = 1, QS_X = 2, QS_Y = 3, QS_Z = 4, QS_S = 5, QS_T = 6,
  QS_RX = 7, QS_RY = 8, QS_RZ = 9, QS_U3 = 10, QS_P = 11,
  QS_CNOT = 12, QS_CZ = 13, QS_CR = 14
};

/* One gate of a program (56 bytes).  The paper's ".control" form (Section
 * "A variety of convenient tools") is ctrl_mask; its set_dagger is `dagger`.
 *   q0         target of a one-qubit gate; the control of CNOT / CZ / CR
 *   q1         target of CNOT / CZ / CR; ignored (use -1) otherwise
 *   param_idx  >= 0: theta is params[param_idx] of the call; -1: theta is p[0]
 *   ctrl_mask  extra control qubits: the gate acts where all these bits are 1
 *   p          theta, phi, lambda (radians)
 *   dagger     nonzero: apply the conjugate transpose                          */
typedef struct qs_gate {
  int32_t type;
  int32_t q0;
  int32_t q1;
  int32_t param_idx;
  uint64_t ctrl_mask;
  double p[3];
  int32_t dagger;
  int32_t reserved;
} qs_gate;

/* One Pauli string with a real coefficient: qubit q carries X if only bit q of
 * xmask is set, Z if only bit q of zmask is set, Y if both are set.  A Pauli
 * sum is an array of these (the paper's Pauli operator, Section "Structure of
 * QPanda"; qop expectation, Section "Variational quantum circuit").           */
typedef struct qs_pauli {
  double coef;
  uint64_t xmask;
  uint64_t zmask;
} qs_pauli;

typedef struct qs_state qs_state; /* opaque */
typedef struct qs_plan qs_plan;   /* opaque */

/* ---- library ----------------------------------------------------------------- */

/* Message of the last failing call on this thread ("" if none).  The pointer
 * stays valid until the next call on this thread. */
const char* qs_last_error(void);

/* Largest qubit count a state may have in this build (34). */
int qs_max_qubits(void);

/* ---- host-side fault injection ---------------------------------------------------
 * Drives the library's error paths without a GPU fault.  One fault is armed per
 * process.  QS_FAULT_ALLOC fails device and pinned-host allocations (every
 * cudaMalloc / cudaMallocAsync / cudaMallocHost the library makes) before they
 * reach CUDA, as an out-of-memory would: the call returns QS_ERR_OOM.
 * QS_FAULT_LAUNCH fails the check that follows a kernel launch as a launch
 * failure would: the call returns QS_ERR_CUDA (that kernel has already been
 * queued; its stream and the context stay usable, as they do after a real
 * non-sticky launch error).  qs_last_error() then ends in "(injected by the
 * armed fault)".
 *
 * On error, every entry point frees what it allocated during the call.  A call
 * that only reads a state (reductions, sampling, copies out) leaves it unchanged.
 * A call that writes the state (qs_apply, qs_run_*, qs_measure, ...) may have run
 * some of its kernels before the failing allocation or launch, so the amplitudes
 * are then unspecified; the handle stays valid, and qs_set_zero / qs_set_state
 * make it usable again.
 *
 * qs_fault_set(kind, after, count): the first `after` events of `kind` pass, the
 * next `count` fail (count -1: all that follow); kind QS_FAULT_NONE disarms.
 * INVALID_ARG for an unknown kind, after < 0, count 0 or count < -1.
 * The environment variable QS_FAULT = "alloc" | "launch", optionally followed by
 * ":after" and ":count" (default 0 and 1), arms the same fault when the library
 * loads; an unparsable value arms nothing, and qs_fault_get's env_status holds
 * the parse result (QS_OK or INVALID_ARG).
 * qs_fault_get: the armed kind, events still to pass, failures still to inject
 * (-1: unlimited), failures injected so far; any pointer may be NULL. */
#define QS_FAULT_NONE 0
#define QS_FAULT_ALLOC 1
#define QS_FAULT_LAUNCH 2
int qs_fault_set(int kind, long long after, long long count);
int qs_fault_get(int* kind, long long* after, long long* left, long long* fired, int* env_status);

/* ---- states (qAlloc_many / init_qvm in the paper's listings) --------------------- */

/* Allocate an n-qubit state (1 <= n <= qs_max_qubits()) on the current CUDA
 * device, bound to `stream` (a cudaStream_t; NULL = the legacy default stream),
 * initialised to |0...0>.  The library owns the amplitude buffer and a small
 * reduction workspace; both are released by qs_free.
 * Errors: INVALID_ARG (n out of range), OOM, CUDA. */
int qs_alloc(int n, void* stream, qs_state** out);

/* Wrap an existing device buffer of 2^n complex128 amplitudes (16-byte aligned)
 * that the caller owns (for example a torch tensor).  Its contents are left as
 * they are.  The buffer must outlive the state; qs_free does not release it.
 * Errors: INVALID_ARG (n out of range, NULL or misaligned pointer), OOM, CUDA. */
int qs_alloc_external(int n, void* device_amps, void* stream, qs_state** out);

/* Allocate an n-qubit complex64 state (2^n interleaved float pairs, 8 bytes
 * per amplitude), initialised to |0...0>.  The complex64 variant of the path:
 * gates compute in FP32 (per-gate kernels and tile passes, matrices rounded to
 * float from their double form); probabilities, marginals, expectations, the
 * canonical sampler and measurement widen each component to double (exact) and
 * compute as for complex128, so sampling is the same definition on the stored
 * state.  qs_set_state / qs_get_state move float data for these states.
 * qs_apply_matrix, qs_adjoint_grad and QS_ARITH_FIXED return UNSUPPORTED.
 * Errors: INVALID_ARG, OOM, CUDA. */
int qs_alloc_c64(int n, void* stream, qs_state** out);

/* *bits = 128 (complex128 state) or 64 (complex64 state). */
int qs_state_precision(const qs_state* s, int* bits);

/* Release a state (waits for its stream first).  NULL is accepted. */
int qs_free(qs_state* s);

/* Qubit count, device pointer of the amplitudes, and the bound stream. */
int qs_num_qubits(const qs_state* s);
int qs_device_ptr(const qs_state* s, void** out);

/* Reset to |0...0>. */
int qs_set_zero(qs_state* s);

/* Copy 2^n interleaved amplitudes in from `amps` (device memory if on_device !=
 * 0, else host memory; synchronous for host memory): complex128 (double pairs),
 * or float pairs for a complex64 state (the pointer is then read as float). */
int qs_set_state(qs_state* s, const double* amps, int on_device);

/* Copy the 2^n amplitudes out to `dst` (device or host memory), in the state's
 * own precision (float pairs for a complex64 state). */
int qs_get_state(const qs_state* s, double* dst, int on_device);

/* Wait for all work queued on the state's stream. */
int qs_sync(const qs_state* s);

/* Arithmetic of the gate kernels.  The state is complex128 in memory either way.
 *   QS_ARITH_AUTO  (default) Q60 fixed point when every |re|, |im| is known to
 *                  be <= 1.25 (true for any state of norm <= 1.25), else FP64;
 *   QS_ARITH_FP64  IEEE double arithmetic on the FP64 pipe;
 *   QS_ARITH_FIXED Q60 fixed point on the integer pipe: each component is
 *                  rounded to a multiple of 2^-60 while a kernel holds it and
 *                  products are exact to 2^-60; a state whose norm exceeds 1.25
 *                  makes qs_apply return UNSUPPORTED.
 * The bound is known after qs_alloc / qs_set_zero and is kept by qs_apply
 * (unitary gates preserve the norm).  After qs_set_state, qs_alloc_external,
 * qs_apply_matrix or qs_state_modified it is re-established by the next
 * qs_apply from the squared norm (one reduction and one stream synchronisation). */
#define QS_ARITH_AUTO 0
#define QS_ARITH_FP64 1
#define QS_ARITH_FIXED 2
int qs_set_arith(qs_state* s, int mode);

/* Tell the library that the amplitudes were written outside its calls (for
 * example through the torch tensor of qs_alloc_external). */
int qs_state_modified(qs_state* s);

/* ---- gate application (directly_run; Section "High-performance simulation":
 * a circuit is an iteration of gates, each a map on the state vector) --------- */

/* Apply gates[0..ng-1] in order.  params (host, may be NULL if no record has
 * param_idx >= 0) supplies theta for parametrised records; param_idx must be
 * < the caller's params length (not checkable: the caller guarantees it).
 * plan == NULL: one kernel per gate (plain mode).  Otherwise the plan must have
 * been created from exactly this gate list and qubit count; its passes are run
 * (fused mode) with matrices computed from `params` at this call.
 * Every record is validated before any work is queued: a bad record returns
 * INVALID_ARG and leaves the state untouched. */
int qs_apply(qs_state* s, const qs_gate* gates, size_t ng, const double* params, const qs_plan* plan);

/* Dense k-qubit matrix gate, 1 <= k <= 5 (the "unitary matrix" gates of the
 * paper's basic-gate experiment).  targets[j] is bit j of the matrix's row and
 * column index; mat is 2^k x 2^k complex128, row-major, interleaved, in host
 * memory; it need not be unitary.  The gate acts where all ctrl_mask bits are 1. */
int qs_apply_matrix(qs_state* s, const int* targets, int k, uint64_t ctrl_mask, const double* mat);

/* out[i] = the adjoint of in[ng-1-i] (the paper's set_dagger on a circuit);
 * out may not alias in. */
int qs_gate_list_dagger(const qs_gate* in, size_t ng, qs_gate* out);

/* ---- fusion plans (Fusion.aggregate_operations; Section "Quantum circuit
 * fusion") ------------------------------------------------------------------ */

#define QS_PLAN_PLAIN 0   /* one pass per gate */
#define QS_PLAN_GREEDY 1  /* greedy grouping into tiled passes / dense blocks */
#define QS_PLAN_LEARNED 2 /* groupings scored by the trained cost model */

typedef struct qs_plan_stats {
  int64_t n_gates;       /* gates in the program */
  int64_t n_passes;      /* state sweeps the plan makes */
  int64_t n_tile_passes; /* of which shared-memory tile passes */
  int64_t n_dense;       /* dense-block ops (in tiles or standalone) */
  double est_seconds;    /* the planner's cost estimate (0 if none) */
  int64_t tile_qubits;   /* tile width the plan was built for (learned plans: the widest pass) */
  int64_t learned_fallback; /* learned plans: 1 if the model preferred the greedy plan (its passes kept) */
} qs_plan_stats;

/* Build a plan for n qubits from gates[0..ng-1] (host only; no device work).
 * kmax: widest dense block allowed (1..5).  mode: QS_PLAN_*.
 * Errors: INVALID_ARG, UNSUPPORTED (LEARNED without a loaded cost model), OOM. */
int qs_plan_create(int n, const qs_gate* gates, size_t ng, int mode, int kmax, qs_plan** out);
int qs_plan_free(qs_plan* p);
int qs_plan_get_stats(const qs_plan* p, qs_plan_stats* out);

/* Process-wide switch (default on) for gate aggregation inside tile passes (the
 * paper's Fusion.aggregate_operations, Section "Quantum circuit fusion"): when a
 * pass is applied, a one-qubit gate whose target and controls no other op of the
 * pass has touched since the previous op on the same target with the same
 * controls is multiplied into that op (later gate on the left), if the product's
 * limb products per amplitude do not exceed the two ops' plus one op's overhead
 * (6); an identity product is dropped.  Results agree with aggregation off
 * within rounding (the 2x2 products are formed in double).  Always QS_OK. */
int qs_set_aggregate(int on);

/* Process-wide switch (default on) for phase tables in Q60 tile passes.  An
 * uncontrolled general one-qubit op factors exactly as diag R diag with R real
 * (the ZYZ Euler form); within a pass the diagonal factors of many qubits, the
 * plain diagonal gates between them and the controlled diagonal gates among the
 * tile's qubits (CZ, CR, ...) commute into one table op a_j *= T[j], a diagonal
 * over the tile (2^m phases in device memory, one complex product per
 * amplitude), leaving real rotations: 12 instead of 18 limb products per
 * amplitude.  A table is built where the general ops it makes real and the
 * diagonals it absorbs outweigh its own cost.  The tables are staged through
 * pinned memory per pass, so a qs_apply with a plan is not stream-capturable
 * while this is on.  Results agree with the switch off within rounding (table
 * entries formed in double).  Always QS_OK. */
int qs_set_phase_tables(int on);

/* Process-wide switch (default on): in Q60 tile passes, consecutive real
 * one-qubit ops on different tile qubits (the real rotations the phase tables
 * leave, RY, ...) run together.  Two of them run on amplitude quads as two
 * complex products per quad and component (u = z0 + i z1 and v = z0 - i z1,
 * z_b the complex number formed along the first qubit: both rotations act on u
 * and v as multiplications), three on amplitude octets as four complex products
 * (the same basis change along each further qubit), four on one component of 16
 * amplitudes as eight: 8, 16 and 32 real products where the rotations apart take
 * 16, 24 and 64.  A phase table op just before a pair or triple runs inside its
 * loop.  Results agree with the switch off within the Q60 rounding.  For
 * measurement: on = 1 (default) groups of four, three and two, 4 groups of three
 * and two, 3 pairs only with tables fused, 2 pairs without table fusion, 0
 * none.  Always QS_OK. */
int qs_set_rotation_pairs(int on);


/* Greedy plan with an explicit tile width: tiles of tile_qubits (4..13) qubits,
 * the "block size" of the fusion (13: 128 KiB tiles, one 512-thread CTA per SM).
 * qs_plan_create(GREEDY) uses 12. */
int qs_plan_create_tiled(int n, const qs_gate* gates, size_t ng, int tile_qubits, qs_plan** out);

/* Pass `pass` of a plan (0 <= pass < n_passes): *kind (0 = one plain gate,
 * 1 = shared-memory tile pass), *qmask (tile qubits, or the gate's target),
 * and the indices of its gates into the program in execution order (up to cap
 * of them into `gates`; *ngates receives the count).  Running the passes in
 * order applies the same unitary as the program. */
int qs_plan_pass_info(const qs_plan* p, size_t pass, int* kind, uint64_t* qmask, uint32_t* gates, size_t cap,
                      size_t* ngates);

/* The op list a tile pass runs (introspection; host only, no device work): the
 * pass's gates after aggregation (qs_set_aggregate) and, when q60 != 0 and
 * phase tables are on (qs_set_phase_tables), after the general ops were split
 * into real rotations and phase tables.  Applying the ops in order is the pass's
 * gates in order (up to rounding).  Kind 0: the 2x2 matrix m (row-major,
 * interleaved complex) on `target` with controls ctrl_mask.  Kind 1: phase table
 * `table`, a diagonal over the pass's `bits` qubits: amplitude x gets T[j], j =
 * the bits of x at the pass's qubits in ascending order, times
 * (-1)^(x_{sign_q[i]} x_{sign_t[i]}) for i < nsigns (CZs between a qubit outside
 * the pass's qubits and one of them, absorbed by the table; sign_q and sign_t
 * are qubit numbers); the tables are written one after another, 2^bits complex
 * (interleaved) entries each (every table of a pass has the pass's tile width).
 * *count / *ntables receive the totals (only the first cap ops and table_cap
 * tables are written). */
typedef struct qs_pass_op {
  int32_t kind;
  int32_t target;
  uint64_t ctrl_mask;
  double m[8];
  int32_t table, bits;
  int32_t nsigns;
  uint8_t sign_q[16], sign_t[16];
} qs_pass_op;
int qs_plan_pass_ops(const qs_plan* p, size_t pass, const qs_gate* gates, size_t ng, const double* params,
                     int q60, qs_pass_op* ops, size_t cap, size_t* count, double* tables, size_t table_cap,
                     size_t* ntables);


/* ---- learned fusion cost model (not in the paper, whose fusion has no cost
 * model): a 3-layer tanh perceptron h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2),
 * y = w3 . h2 + b3 predicting log(milliseconds) of one pass from its features,
 * trained on the GPU by the library's own kernels from its own kernel timings.
 * Weights are flattened W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3 (doubles).
 * Every call below is synchronous and uses the model's private stream. ------ */

typedef struct qs_mlp qs_mlp; /* opaque */

/* n_in features (1..64), n_hidden units (1..128); weights (host) or NULL for a
 * seeded uniform +-1/sqrt(fan-in) initialisation (biases 0). */
int qs_mlp_create(int n_in, int n_hidden, const double* weights, uint64_t seed, qs_mlp** out);
int qs_mlp_free(qs_mlp* m);
int qs_mlp_num_weights(const qs_mlp* m, size_t* out);
int qs_mlp_get_weights(const qs_mlp* m, double* out);
int qs_mlp_set_weights(qs_mlp* m, const double* w);
/* y[s] for the B feature rows x[s*F .. s*F+F) (host arrays). */
int qs_mlp_forward(qs_mlp* m, const double* x, size_t B, double* y);
/* loss = (1/B) sum_s (y_s - t_s)^2 / 2 and its gradient for every weight. */
int qs_mlp_loss_grad(qs_mlp* m, const double* x, const double* t, size_t B, double* loss, double* grad);
/* `epochs` full-batch Adam steps (lr; beta 0.9 / 0.999) on the GPU; *final_loss
 * (may be NULL) receives the loss of the final weights. */
int qs_mlp_train(qs_mlp* m, const double* x, const double* t, size_t B, int epochs, double lr, double* final_loss);

/* Features of every pass of a plan (QS_PASS_FEATURES doubles per pass, in pass
 * order; `gates` must be the plan's program): pass kind (tile or plain gate),
 * tile qubits, state qubits, qubits outside the tile, gates by structural class
 * (general, real, general diagonal, unit factors), controlled gates, diagonal
 * gates with the target outside the tile, distinct non-diagonal targets, gates
 * that start a run on their target (the ops left after aggregation), controlled
 * non-diagonal gates, log2(1 + gates), and for a tile pass the kernel ops of
 * qs_plan_pass_kernel_ops (limb products per amplitude, phase tables, groups of
 * four, three and two real rotations, single rotations, general ops, phase and
 * diagonal ops, anti-diagonal ops, per-tile scalars, shared-memory sweeps).
 * Parametrised records are featurised with generic angles. */
#define QS_PASS_FEATURES 25
int qs_plan_features(const qs_plan* p, const qs_gate* gates, size_t ng, double* out);

/* Kernel ops of one pass of a plan as the Q60 tile engine would run it on a
 * complex128 state (host only, nothing launched; `params` as for qs_apply):
 * counts[k] (QS_KOP_KINDS entries) = ops of kind k: 1 one-qubit phase, 2
 * diagonal, 3 anti-diagonal, 4 real, 5 general 2x2, 9 diagonal on a qubit outside
 * the tile (a per-tile scalar), 10 phase tables (those fused into a rotation
 * group included), 11/13/14 groups of two/three/four real rotations; counts[0]
 * = the phase tables fused into a rotation group or into the tile's load or
 * store (no sweep of their own);
 * *int_ops_per_amp = the pass's limb products per amplitude of the state.  A
 * pass of plain per-gate kernels reports zeros.  Errors: INVALID_ARG. */
#define QS_KOP_KINDS 15
int qs_plan_pass_kernel_ops(const qs_plan* p, size_t pass, const qs_gate* gates, size_t ng, const double* params,
                            int64_t* counts, double* int_ops_per_amp);

/* Greedy plan with an explicit tile width (4..13) and pass construction:
 * strategy 0 takes the targets of the remaining gates in program order (as
 * qs_plan_create_tiled); strategy 1 starts each pass from the first runnable
 * gate's target and the most frequent targets among the next runnable gates;
 * strategy 2 (lookahead) takes the strategy-0 pass or a variant of it kept off
 * one of the qubits the strategy-0 scan added, whichever absorbs the most gates
 * together with the strategy-0 pass after it.  (The cost model's training
 * passes.)  Errors: INVALID_ARG. */
int qs_plan_create_variant(int n, const qs_gate* gates, size_t ng, int tile_qubits, int strategy, qs_plan** out);

/* Learned plan: the model chooses the groupings.  Pass by pass it scores
 * candidate tile passes over the remaining gates (widths 11 and 12; strategies
 * 0 and 1 of qs_plan_create_variant and every variant of strategy 2), each as
 * one tile pass and as plain per-gate kernels (exp of the predicted log ms),
 * together with the strategy-0 pass that would follow it, and takes the
 * candidate with the least predicted time per unit of work over the two passes
 * (the gates' touched fractions of the state), in the cheaper form.  The greedy
 * plan is the fallback and the judge: unless the model predicts the learned
 * plan faster by more than 5 %, the greedy passes are kept
 * (stats.learned_fallback = 1).  est_seconds is the model's prediction.  The
 * model needs QS_PASS_FEATURES inputs; its forward kernel runs on the GPU. */
int qs_plan_create_learned(int n, const qs_gate* gates, size_t ng, qs_mlp* model, qs_plan** out);

/* The same planner with a caller's cost model: score(ctx, x, B, y) writes the
 * predicted log(milliseconds) y[s] of the B passes whose features are the rows
 * x[s*QS_PASS_FEATURES ..] (host arrays, valid during the callback) and returns
 * 0, or non-zero to abandon the plan (INVALID_ARG).  Runs on the host only. */
typedef int (*qs_pass_scorer)(void* ctx, const double* x, size_t B, double* y);
int qs_plan_create_scored(int n, const qs_gate* gates, size_t ng, qs_pass_scorer score, void* ctx, qs_plan** out);

/* ---- reductions (prob_run_list / prob_run_dict, expectation tools) ------------- */

/* Marginal probabilities over qubits[0..nq-1] (0 <= nq <= n; qubits[j] is bit j
 * of the output index): out has 2^nq entries, out[k] = sum of |a_x|^2 over x
 * whose listed bits spell k.  nq = 0 gives the squared norm.  out is device
 * memory if on_device != 0 (asynchronous), else host memory (synchronous).
 * For nq <= 3 on a state known to satisfy the Q60 bound (reached from |0> by
 * unitary gates), the squares of the Q60-rounded components are summed exactly
 * in integers: absolute error below 2^-60 * sum_x |a_x| (2^-45 at n = 30);
 * otherwise FP64 sums in a fixed order.  Results are deterministic either way. */
int qs_probs(const qs_state* s, const int* qubits, int nq, double* out, int on_device);

/* Entries of the marginal over qubits[0..nq-1] with probability > threshold,
 * in increasing index order: idx[i], p[i] for i < min(count, cap) (host memory);
 * *count receives the total number of such entries. */
int qs_probs_dict(const qs_state* s, const int* qubits, int nq, double threshold, uint64_t* idx,
                  double* p, size_t cap, size_t* count);

/* <Z_i> for every qubit i into out[0..n-1] (host memory).  For 10 <= n <= 30 on
 * a state within the Q60 bound (norm <= 1.25; a state of unknown magnitude, e.g.
 * after qs_set_state, has its norm measured once), the squares of the Q60-rounded
 * components are summed exactly in integers: absolute error below
 * 2^-59 * sum_x |a_x| (about 2^-44 at n = 30).  Otherwise FP64 sums in a fixed
 * order.  Results are deterministic either way. */
int qs_expect_z_all(const qs_state* s, double* out);

/* <Z_i> for every qubit i, for callers that cannot allocate memory.  The paper
 * has no counterpart; this is a service entry point of this library.
 * Some callers cannot call cudaMalloc: code whose device memory all belongs to
 * another allocator (a framework's caching allocator, or a pool reserved at
 * start-up, where an extra allocation can fail or fragment it), and code on
 * latency-critical paths, where cudaMalloc / cudaFree would synchronise the
 * device.  This entry point allocates nothing, on the device or the host:
 *   device_amps  2^n complex128 amplitudes, interleaved, 16-byte aligned, device
 *                memory owned by the caller (read only);
 *   device_out   n doubles, device memory owned by the caller: out[i] = <Z_i>;
 *   stream       cudaStream_t the two kernels are queued on (NULL = legacy default);
 *   8 <= n <= 34, otherwise INVALID_ARG with a message naming the range.
 * Asynchronous: results are in device_out once `stream` reaches this point.
 * The partial sums live in one file-scope device array (25,600 doubles,
 * 200 KiB), which every GPU that loads the library holds until the process
 * exits.  Each call outside stream capture looks up that array's device address
 * (cudaGetSymbolAddress, which allocates nothing) with the device current;
 * during capture the address of the last call on that device is used, so make
 * a first call on each device before any stream capture (a call captured first
 * fails with UNSUPPORTED).  All calls share the array and it keeps the last call's
 * contents, which no call reads before rewriting; calls whose kernels overlap on
 * the GPU (other streams, other host threads) race on it and must be ordered by
 * the caller. */
int qs_expect_z_all_noalloc(const double* device_amps, int n, double* device_out, void* stream);

/* <psi| sum_k coef_k P_k |psi> into *out (host).  Each term's masks must lie
 * within the n qubits (else INVALID_ARG).  On a state within the Q60 bound (see
 * qs_expect_z_all) every term is an exact integer sum over the Q60-rounded
 * amplitudes (absolute error per term below 2^-59 * sum_x |a_x|): the terms are
 * grouped by X mask, and each pass reads the state once in tiles of up to 4096
 * amplitudes that serve every X mask in the span of the tile's basis (qubits
 * 0..3 and up to eight X masks).  Otherwise FP64, eight terms per pass.  The
 * weighted sum is formed on the host in term order; results are deterministic. */
int qs_expect_pauli(const qs_state* s, const qs_pauli* terms, size_t nterms, double* out);

/* Draw `shots` computational-basis samples (measure_all / run_with_configuration).
 * Canonical, bit-reproducible definition: u_s = ((SplitMix64 output number s of
 * the stream seeded `seed`) >> 11) * 2^-53; p_x = re*re + im*im rounded as two
 * products and a sum; blocks of L = min(1024, 2^n) amplitudes summed left to
 * right give the block totals T_b; superblocks of G = min(1024, blocks) blocks
 * give F_c(i) = T_cG + ... + T_cG+i (left to right) and P_0 = 0,
 * P_c+1 = P_c + F_c(G-1); E_0 = 0 and E_cG+i+1 = P_c + F_c(i) (for n <= 20 this
 * is the left-to-right prefix of the block totals); the sample is the smallest x
 * with E_b + (left-to-right partial sum of block b up to x) > u_s, or, when no x
 * qualifies, the largest x with p_x > 0.
 * The search within a block starts from the running sum kept after every 32
 * amplitudes (2^n / 32 doubles of stream-ordered scratch, freed when the call
 * returns), which continues the same left-to-right additions.
 * out[s] (uint64, device or host memory) receives the basis index of shot s. */
int qs_sample(const qs_state* s, uint64_t seed, uint64_t shots, uint64_t* out, int on_device);


/* ---- gradients (the paper's variational circuits and qop expectations, Section
 * "Variational quantum circuit"; the paper does not say how gradients are taken:
 * this is the adjoint recursion of Jones & Gacon, arXiv:2009.02823) ----------- */

/* Energy E = <psi|H|psi> of psi = U_G ... U_1 |0> (gates[0..ng-1] with angles
 * from params[0..np-1], host memory) for H = terms[0..nterms-1], and its gradient
 * dE/dparams[j] (host, np entries): the sum over every record with param_idx == j
 * of Im <lambda_k| G_k |psi_k>, lambda_k = U_{k+1}^dag ... U_G^dag H psi,
 * psi_k = U_k ... U_1 |0>, G_k the generator (U = exp(-i theta G / 2)):
 * RX -> X, RY -> Y, RZ -> Z, P and CR -> -2|1><1| on the target, times the
 * projector on the control qubits; a dagger record flips the sign.
 * The state `s` (n qubits) is used as the psi buffer and is overwritten; a
 * second vector and the partial sums are allocated on the state's stream for the
 * call.  Synchronous (returns results in host memory).
 * Errors: INVALID_ARG (bad record, param_idx >= np, term outside n),
 * UNSUPPORTED (a parametrised record other than RX, RY, RZ, P, CR), OOM, CUDA. */
int qs_adjoint_grad(qs_state* s, const qs_gate* gates, size_t ng, const double* params, size_t np,
                    const qs_pauli* terms, size_t nterms, double* energy, double* grad);

/* Process-wide choice of the backward sweep of qs_adjoint_grad under Q60
 * arithmetic: on (default) runs it as shared-memory tile passes over psi and
 * lambda together (the reversed, daggered program planned greedily); off runs one
 * fused kernel per gate.  Same results up to rounding; the switch is for
 * measurement. */
int qs_set_adjoint_fused(int on);

/* ---- mid-circuit measurement and classical control (QMeasure, QIf, QWhile and
 * ClassicalProg of Section "Core" and its QIf / QWhile listings; classical
 * operators per Section "Qif and QWhile") ----------------------------------- */

/* Projective measurement of `qubit` with the caller's draw u in [0, 1):
 * p0, p1 = squared norms of the parts of the state with the qubit 0 / 1;
 * *outcome = 0 if u (p0 + p1) < p0, else 1; the state collapses in place (the
 * other part set to 0, the kept part scaled by 1 / sqrt(p_outcome)).  *p1
 * (nullable) receives p1 / (p0 + p1).  Two passes over the state (reduction,
 * collapse; a third, FP64 reduction when the smaller branch is below 2^-20);
 * synchronous.  Errors: INVALID_ARG (qubit, u, zero state), CUDA. */
int qs_measure(qs_state* s, int qubit, double u, int* outcome, double* p1);

/* One instruction of a structured program (56 bytes).  Blocks nest by length:
 * an IF at index i owns the n_then instructions after it (then-block) and the
 * n_else after those (else-block); a WHILE owns the n_then after it (body).
 * Operands lhs / rhs name a classical register (int64), or -1 for `imm`.       */
typedef struct qs_pinstr {
  int32_t op;        /* QS_PI_* */
  int32_t qubit;     /* MEASURE: measured qubit */
  int32_t dst;       /* MEASURE / ASSIGN: register written */
  int32_t alu;       /* ASSIGN: QS_CA_* */
  int32_t lhs, rhs;  /* operands (register index or -1) */
  int64_t imm;       /* immediate operand */
  uint32_t n_then;   /* IF: then-block length; WHILE: body length */
  uint32_t n_else;   /* IF: else-block length; WHILE: 0 */
  uint64_t gate_begin, gate_end; /* GATES: gates[gate_begin .. gate_end) */
} qs_pinstr;

enum { QS_PI_GATES = 0, QS_PI_MEASURE = 1, QS_PI_ASSIGN = 2, QS_PI_IF = 3, QS_PI_WHILE = 4 };
/* ASSIGN: dst = lhs OP rhs.  ADD/SUB/MUL wrap (two's complement); DIV truncates
 * toward zero (division by zero or INT64_MIN / -1 is an error); AND/OR are
 * logical (result 0/1); XOR bitwise; comparisons give 0/1; NOT = (lhs == 0);
 * MOV = lhs.  IF and WHILE test lhs != 0, WHILE before every pass. */
enum {
  QS_CA_MOV = 0, QS_CA_ADD = 1, QS_CA_SUB = 2, QS_CA_MUL = 3, QS_CA_DIV = 4, QS_CA_AND = 5, QS_CA_OR = 6,
  QS_CA_XOR = 7, QS_CA_LT = 8, QS_CA_LE = 9, QS_CA_GT = 10, QS_CA_GE = 11, QS_CA_EQ = 12, QS_CA_NE = 13,
  QS_CA_NOT = 14
};

/* Run prog[0 .. nprog) on the current contents of s.  GATES applies a range of
 * `gates` (params as in qs_apply) per gate (fuse == 0) or through a greedy
 * fusion plan built on the instruction's first execution (fuse != 0).
 * Measurement k of the run (0-based, in execution order) uses the draw
 * u_k = (SplitMix64 output k of the stream seeded `seed` >> 11) * 2^-53, as
 * qs_measure does with that u, and writes the outcome (0/1) to register dst.
 * cbits: ncbits registers (host, in/out).  record (host, nullable): p1/(p0+p1)
 * of measurements 0 .. record_cap-1.  *nmeasured (nullable): measurements made
 * (also on error).  A WHILE that would start pass max_iters+1 stops the run with
 * TIMEOUT.  Synchronous.  Errors: INVALID_ARG (malformed program, register or
 * qubit out of range, bad division), TIMEOUT, the errors of qs_apply. */
int qs_run_program(qs_state* s, const qs_pinstr* prog, size_t nprog, const qs_gate* gates, size_t ngates,
                   const double* params, int fuse, uint64_t seed, uint64_t max_iters, int64_t* cbits,
                   size_t ncbits, double* record, size_t record_cap, uint64_t* nmeasured);

/* ---- noisy simulation by Monte-Carlo trajectories (NoiseQVM, Section
 * "Multi-simulation methods": Kraus operator noise models, set_noise_model,
 * set_readout_error, set_rotation_error) --------------------------------------- */

enum {
  QS_NOISE_DAMPING = 0, QS_NOISE_DEPHASING = 1, QS_NOISE_DECOHERENCE = 2, QS_NOISE_DEPOLARIZING = 3,
  QS_NOISE_BITFLIP = 4, QS_NOISE_BITPHASEFLIP = 5, QS_NOISE_PHASEFLIP = 6, QS_NOISE_PHASE_DAMPING = 7
};

/* A noise rule (48 bytes): after every gate of type gate_type (-1: every gate)
 * whose first qubit is q0 and second qubit q1 (-1: any; for CNOT/CZ/CR the
 * control and the target), the one-qubit channel `model` acts on each qubit the
 * gate touches.  Kraus sets as the paper prints them:
 *   DAMPING [[1,0],[0,sqrt(1-p)]], [[0,sqrt(p)],[0,0]];
 *   DEPHASING and PHASEFLIP sqrt(1-p) I, sqrt(p) Z;  BITFLIP sqrt(1-p) I, sqrt(p) X;
 *   BITPHASEFLIP sqrt(1-p) I, sqrt(p) Y;
 *   DEPOLARIZING sqrt(1-3p/4) I, sqrt(p)/2 {X, Y, Z};
 *   PHASE_DAMPING [[1,0],[0,sqrt(1-p)]], [[0,0],[0,sqrt(p)]];
 *   DECOHERENCE Kdamp_i Kdeph_j with p_damp = 1 - exp(-tgate/t1) and
 *   p_deph = (1 - exp(-(tgate/t2 - tgate/(2 t1)))) / 2 (p unused). */
typedef struct qs_noise_rule {
  int32_t model, gate_type, q0, q1;
  double p, t1, t2, tgate;
} qs_noise_rule;

/* One trajectory of the noisy circuit on the current contents of s.  Gate by
 * gate: a rotation (RX, RY, RZ, U3, P, CR) gets theta += rotation_error (2u - 1)
 * (one draw, if rotation_error > 0); the gate is applied; then for each matching
 * rule in order and each touched qubit in ascending order, one draw u picks the
 * smallest j with u W < w_1 + ... + w_j (w_j = ||K_j psi||^2, W their sum) and
 * psi <- K_j psi / sqrt(w_j).  Draw k is (SplitMix64 output k of the stream
 * seeded `seed` >> 11) * 2^-53; *ndraws (nullable) receives the count.
 * Stretches without damping-type channels run as one gate list (fused with a
 * greedy plan if fuse != 0); damping-type channels take one reduction pass for
 * their weights.  Synchronous.  Errors: INVALID_ARG (rule, probability,
 * decoherence times), the errors of qs_apply. */
int qs_run_noisy(qs_state* s, const qs_gate* gates, size_t ng, const double* params,
                 const qs_noise_rule* rules, size_t nrules, double rotation_error, uint64_t seed, int fuse,
                 uint64_t* ndraws);

/* Readout error on sampled basis indices (set_readout_error's confusion matrix
 * [[f0, 1-f0], [1-f1, f1]] on every qubit): bit i of shot s flips when
 * u = u01(SplitMix64 output s*n + i of the stream seeded `seed`) >= f0 (bit 0)
 * or f1 (bit 1).  samples: shots indices in device (on_device != 0, on
 * `stream`) or host memory, rewritten in place.  Synchronous.
 * Errors: INVALID_ARG, CUDA. */
int qs_readout_error(uint64_t* samples, size_t shots, int n, double f0, double f1, uint64_t seed, int on_device,
                     void* stream);

/* ---- partial amplitudes (PartialAmpQVM, Section "Multi-simulation methods":
 * cut the two-qubit gates across a bisection into sums of products and simulate
 * the two halves) ---------------------------------------------------------------- */

/* Amplitudes <x|U|0...0> of an n-qubit program (2 <= n <= 64) for the count
 * basis indices in `indices` (host), written to out (host, count interleaved
 * complex128), without the 2^n state.  Qubits 0 .. n_low-1 form the low block,
 * the rest the high block (each at most qs_max_qubits()).  Every gate with
 * qubits in both blocks is cut: with target t, controls C_t in t's block and C_o
 * in the other, it is P(C_o all 1) (x) [U on t, controls C_t] + (I - P(C_o all
 * 1)) (x) I.  k cuts give 2^k paths (k <= 30); each path simulates both blocks
 * (fused per uncut stretch if fuse != 0), and the amplitude is the sum over paths
 * of <x_low|lo> <x_high|hi>, added in a fixed path order.  Consecutive paths share
 * their early cuts, so a block resumes from a snapshot before its first changed
 * cut (device memory: one block state per cut item of that block).  *npaths
 * (nullable) receives 2^k.  Runs on `stream`; synchronous.
 * Errors: INVALID_ARG, UNSUPPORTED (block too large, more than 30 cuts), OOM, CUDA. */
int qs_partial_amplitudes(int n, const qs_gate* gates, size_t ng, const double* params, int n_low,
                          const uint64_t* indices, size_t count, double* out, int fuse, void* stream,
                          uint64_t* npaths);

/* ---- batched variational evaluation (the hybrid quantum-classical loop of
 * Sections "Support hybrid quantum-classical algorithm" and "Variational
 * quantum circuit": many parameter sets evaluated per optimiser step) -------- */

typedef struct qs_batch qs_batch; /* opaque */

/* Describe nsets independent energy+gradient problems, set s having:
 *   n_per_set[s] qubits (1..24);
 *   gates[gate_offsets[s] .. gate_offsets[s+1]) (param_idx relative to the set);
 *   params[param_offsets[s] .. param_offsets[s+1]) in the run's params array;
 *   terms[term_offsets[s] .. term_offsets[s+1]) its Pauli sum.
 * All arrays are host memory, read during the call (offset arrays have nsets+1
 * entries, non-decreasing).  The batch owns device copies, per-set psi and
 * lambda buffers (32 bytes x 2^n per set), pinned staging and a private stream.
 * Errors: INVALID_ARG, UNSUPPORTED (parametrised record other than RX, RY, RZ,
 * P, CR), OOM, CUDA. */
int qs_batch_create(size_t nsets, const int* n_per_set, const qs_gate* gates, const size_t* gate_offsets,
                    const size_t* param_offsets, const qs_pauli* terms, const size_t* term_offsets,
                    qs_batch** out);

/* Evaluate every set for params (param_offsets[nsets] values): energies[s] and
 * grads (same layout as params), each as qs_adjoint_grad defines them, in ONE
 * persistent kernel launch in thread-block clusters: each cluster takes work
 * items from a device counter, most expensive first; an item is one set with at
 * least as many 2^11-amplitude tiles per pass as the cluster has CTAs (the CTAs
 * share its tiles, with cluster barriers between passes) or up to one small set
 * per CTA.  No CTA waits on a CTA of another cluster.  Results are
 * deterministic for a given batch (fixed summation orders).  on_device == 0: host arrays; the
 * copy-in, the launch and the copy-out are a CUDA graph captured on the first
 * such call and replayed after.  on_device != 0: device arrays, no graph.
 * Synchronous. */
int qs_batch_run(qs_batch* b, const double* params, double* energies, double* grads, int on_device);

/* Device time (ms) of the persistent kernel in the last run; launch shape
 * (grid in CTAs); CTAs per cluster. */
int qs_batch_last_ms(const qs_batch* b, double* ms);
int qs_batch_info(const qs_batch* b, int* grid, int* threads, size_t* smem_bytes);
int qs_batch_cluster(const qs_batch* b, int* ctas);

/* Cluster size of batches created after the call: 1, 2, 4 or 8 CTAs, or 0
 * (default) to choose per batch the size whose longest-processing-time schedule
 * of the work items over the resident clusters has the shortest estimated
 * makespan (set cost ~ 2^n x gates).  Not thread-safe against a concurrent
 * qs_batch_create.  Errors: INVALID_ARG. */
int qs_set_batch_cluster(int ctas);
int qs_batch_free(qs_batch* b);

/* ---- instrumentation ---------------------------------------------------------------
 * Per-kernel timing log of one state: when enabled, every kernel the library
 * queues for the state is bracketed by CUDA events on the state's stream.
 * qs_timing_fetch synchronises the stream, converts the pending pairs to
 * milliseconds, returns up to `cap` records (host memory, in launch order),
 * stores the number available in *count and clears the log.  The log is the
 * training data of the fusion cost model and the live per-kernel timing of the
 * benchmark.                                                                   */
enum {
  QS_K_PHASE1 = 1, QS_K_DIAG = 2, QS_K_ANTI = 3, QS_K_REAL = 4, QS_K_GENERAL = 5, /* one-qubit op classes */
  QS_K_DENSE = 10,   /* dense k-qubit block */
  QS_K_TILE = 11,    /* shared-memory tile pass */
  QS_K_REDUCE = 20,  /* reductions and sampling */
  QS_K_ADJOINT = 30, /* adjoint-gradient kernels */
  QS_K_OTHER = 40
};

typedef struct qs_timing_record {
  int32_t kind;        /* QS_K_* */
  int32_t n;           /* qubits of the state */
  int32_t k;           /* block / tile width (qubits), 1 for one-qubit ops */
  int32_t n_ops;       /* gates or ops executed by the launch */
  uint64_t qubit_mask; /* qubits the launch acts on (targets; tile qubits) */
  uint64_t ctrl_mask;  /* control qubits */
  double items;        /* amplitudes the launch reads (and writes) */
  double flops;        /* floating-point operations the launch's arithmetic needs (FP64 engine) */
  double int_ops;      /* 32x32->64 integer multiply-adds it needs (Q60 engine: 3 per real product) */
  double ms;           /* device time between the bracketing events */
} qs_timing_record;

int qs_timing_enable(qs_state* s, int on);
int qs_timing_fetch(qs_state* s, qs_timing_record* out, size_t cap, size_t* count);

/* Number of kernels this library has launched in this process so far. */
uint64_t qs_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* QSIM_H */
