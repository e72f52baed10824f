/*
 * Plain CPU oracle for the full-amplitude (Schroedinger) state-vector method of
 * QPanda (arXiv 2212.14201).  TEST INFRASTRUCTURE ONLY: the product library never
 * links, loads or calls this file; only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg do.
 *
 * Everything here is written to be checked against the paper by eye: one gate is
 * one pass over the amplitude array with the textbook 2x2 (or 2^k x 2^k) matrix, in
 * IEEE double precision, with no fusion, tiling or reordering.  It shares no code,
 * header or constant table with the CUDA library.
 *
 * Conventions (the paper is silent on them; the readings are listed in the design
 * notes): qubit q is bit q of the basis index (qubit 0 = least significant); a
 * state is 2^n complex doubles stored interleaved (re, im); CNOT/CZ/CR take
 * (control, target) in that order, as in the paper's listings.
 *
 * Compile with -ffp-contract=off: probabilities are re*re + im*im with two
 * separately rounded products, which the canonical sampler relies on.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2
#define OR_EUNSUPPORTED -5
#define OR_ELIMIT -4

enum {
  OR_I = 0, OR_H = 1, OR_X = 2, OR_Y = 3, OR_Z = 4, OR_S = 5, OR_T = 6,
  OR_RX = 7, OR_RY = 8, OR_RZ = 9, OR_U3 = 10, OR_P = 11,
  OR_CNOT = 12, OR_CZ = 13, OR_CR = 14
};

typedef struct {
  int32_t type, q0, q1, param_idx;
  uint64_t ctrl_mask;
  double p[3];
  int32_t dagger, reserved;
} or_gate;

typedef struct {
  double coef;
  uint64_t xmask, zmask;
} or_pauli;

typedef struct {
  double re, im;
} cplx;

static cplx c_make(double re, double im) { cplx z = {re, im}; return z; }
static cplx c_add(cplx a, cplx b) { return c_make(a.re + b.re, a.im + b.im); }
static cplx c_mul(cplx a, cplx b) { return c_make(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
static cplx c_conj(cplx a) { return c_make(a.re, -a.im); }
static cplx c_expi(double t) { return c_make(cos(t), sin(t)); }

/* ------------------------------------------------------------------------- */
/* Gate matrices (the paper's gate set: the keyword list of the API and the   */
/* "Performance of basic gates" experiment).  Textbook forms (Nielsen &       */
/* Chuang); U3 in the OpenQASM form.  m is row-major: m[0]=U00 m[1]=U01        */
/* m[2]=U10 m[3]=U11.                                                          */
/* ------------------------------------------------------------------------- */
static int gate_matrix_1q(int type, double th, double ph, double la, cplx m[4]) {
  const double r = 1.0 / sqrt(2.0);
  double c = cos(th / 2.0), s = sin(th / 2.0);
  switch (type) {
    case OR_I: m[0] = c_make(1, 0); m[1] = c_make(0, 0); m[2] = c_make(0, 0); m[3] = c_make(1, 0); break;
    case OR_H: m[0] = c_make(r, 0); m[1] = c_make(r, 0); m[2] = c_make(r, 0); m[3] = c_make(-r, 0); break;
    case OR_X: case OR_CNOT:
      m[0] = c_make(0, 0); m[1] = c_make(1, 0); m[2] = c_make(1, 0); m[3] = c_make(0, 0); break;
    case OR_Y: m[0] = c_make(0, 0); m[1] = c_make(0, -1); m[2] = c_make(0, 1); m[3] = c_make(0, 0); break;
    case OR_Z: case OR_CZ:
      m[0] = c_make(1, 0); m[1] = c_make(0, 0); m[2] = c_make(0, 0); m[3] = c_make(-1, 0); break;
    case OR_S: m[0] = c_make(1, 0); m[1] = c_make(0, 0); m[2] = c_make(0, 0); m[3] = c_make(0, 1); break;
    case OR_T: m[0] = c_make(1, 0); m[1] = c_make(0, 0); m[2] = c_make(0, 0); m[3] = c_expi(M_PI / 4.0); break;
    case OR_RX: /* exp(-i th X / 2) */
      m[0] = c_make(c, 0); m[1] = c_make(0, -s); m[2] = c_make(0, -s); m[3] = c_make(c, 0); break;
    case OR_RY: /* exp(-i th Y / 2) */
      m[0] = c_make(c, 0); m[1] = c_make(-s, 0); m[2] = c_make(s, 0); m[3] = c_make(c, 0); break;
    case OR_RZ: /* exp(-i th Z / 2) */
      m[0] = c_expi(-th / 2.0); m[1] = c_make(0, 0); m[2] = c_make(0, 0); m[3] = c_expi(th / 2.0); break;
    case OR_U3: {
      cplx el = c_expi(la), ep = c_expi(ph), epl = c_expi(ph + la);
      m[0] = c_make(c, 0);
      m[1] = c_make(-el.re * s, -el.im * s);
      m[2] = c_make(ep.re * s, ep.im * s);
      m[3] = c_make(epl.re * c, epl.im * c);
      break;
    }
    case OR_P: case OR_CR:
      m[0] = c_make(1, 0); m[1] = c_make(0, 0); m[2] = c_make(0, 0); m[3] = c_expi(th); break;
    default: return OR_EINVAL;
  }
  return OR_OK;
}

static int is_two_qubit(int type) { return type == OR_CNOT || type == OR_CZ || type == OR_CR; }

/* Target qubit and full control mask of one record (CNOT/CZ/CR: q0 is the
 * control, q1 the target). */
static int qubits_of(const or_gate* g, int n, int* target, uint64_t* cmask) {
  if (g->type < OR_I || g->type > OR_CR) return OR_EINVAL;
  if (g->q0 < 0 || g->q0 >= n) return OR_EINVAL;
  uint64_t full = (n >= 64) ? ~0ull : ((1ull << n) - 1);
  if (g->ctrl_mask & ~full) return OR_EINVAL;
  uint64_t cm = g->ctrl_mask;
  int t;
  if (is_two_qubit(g->type)) {
    if (g->q1 < 0 || g->q1 >= n || g->q1 == g->q0) return OR_EINVAL;
    t = g->q1;
    cm |= 1ull << g->q0;
  } else {
    t = g->q0;
  }
  if (cm & (1ull << t)) return OR_EINVAL;
  *target = t;
  *cmask = cm;
  return OR_OK;
}

/* Resolve one record into (target, control mask, 2x2 matrix); dagger gives the
 * conjugate transpose (the paper's set_dagger, Section "Quantum circuit
 * visualization" listing). */
static int resolve(const or_gate* g, int n, const double* params, int* target, uint64_t* cmask, cplx m[4]) {
  int rc = qubits_of(g, n, target, cmask);
  if (rc) return rc;
  double th = g->p[0];
  if (g->param_idx >= 0) {
    if (!params) return OR_EINVAL;
    th = params[g->param_idx];
  }
  rc = gate_matrix_1q(g->type, th, g->p[1], g->p[2], m);
  if (rc) return rc;
  if (g->dagger) {
    cplx a = m[0], b = m[1], c = m[2], d = m[3];
    m[0] = c_conj(a); m[1] = c_conj(c); m[2] = c_conj(b); m[3] = c_conj(d);
  }
  return OR_OK;
}

int or_gate_matrix(const or_gate* g, int n, const double* params, int* target, uint64_t* cmask, double* m8) {
  cplx m[4];
  int rc = resolve(g, n, params, target, cmask, m);
  if (rc) return rc;
  for (int i = 0; i < 4; ++i) { m8[2 * i] = m[i].re; m8[2 * i + 1] = m[i].im; }
  return OR_OK;
}

/* One gate = one sweep over the state (Section "High-performance simulation":
 * the circuit is an iteration of gates; Section "Multi-simulation methods": the
 * Schroedinger method updates the state vector by each gate).  Every pair
 * (x, x | 2^t) with bit t of x clear and all control bits of x set is replaced by
 * U applied to it.  A gate with controls is the paper's ".control" form. */
static void apply_2x2(cplx* psi, int n, int t, uint64_t cmask, const cplx m[4]) {
  const int64_t N = (int64_t)1 << n;
  const int64_t tb = (int64_t)1 << t;
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < N; ++x) {
    if ((x & tb) != 0) continue;
    if (((uint64_t)x & cmask) != cmask) continue;
    cplx a0 = psi[x], a1 = psi[x | tb];
    psi[x] = c_add(c_mul(m[0], a0), c_mul(m[1], a1));
    psi[x | tb] = c_add(c_mul(m[2], a0), c_mul(m[3], a1));
  }
}

int or_apply_gate(double* state, int n, const or_gate* g, const double* params) {
  int t; uint64_t cm; cplx m[4];
  int rc = resolve(g, n, params, &t, &cm, m);
  if (rc) return rc;
  apply_2x2((cplx*)state, n, t, cm, m);
  return OR_OK;
}

int or_apply_circuit(double* state, int n, const or_gate* gates, int64_t ng, const double* params) {
  for (int64_t k = 0; k < ng; ++k) {
    int rc = or_apply_gate(state, n, &gates[k], params);
    if (rc) return rc;
  }
  return OR_OK;
}

/* Dense k-qubit matrix gate (the "unitary matrix" gates of 1-3 qubits timed in
 * "Performance of basic gates", and the unitary blocks that circuit fusion
 * produces, Section "Quantum circuit fusion").  targets[j] is bit j of the
 * matrix's row/column index; mat is 2^k x 2^k row-major, interleaved. */
int or_apply_matrix(double* state, int n, const int* targets, int k, uint64_t cmask, const double* mat) {
  if (k < 1 || k > 10 || k > n) return OR_EINVAL;
  uint64_t tmask = 0;
  for (int j = 0; j < k; ++j) {
    if (targets[j] < 0 || targets[j] >= n || (tmask >> targets[j]) & 1) return OR_EINVAL;
    tmask |= 1ull << targets[j];
  }
  uint64_t full = (n >= 64) ? ~0ull : ((1ull << n) - 1);
  if ((cmask & ~full) || (cmask & tmask)) return OR_EINVAL;
  const int64_t N = (int64_t)1 << n;
  const int d = 1 << k;
  const cplx* M = (const cplx*)mat;
  cplx* psi = (cplx*)state;
#pragma omp parallel
  {
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * d);
    cplx* v = (cplx*)malloc(sizeof(cplx) * d);
#pragma omp for schedule(static)
    for (int64_t x = 0; x < N; ++x) {
      if ((uint64_t)x & tmask) continue;
      if (((uint64_t)x & cmask) != cmask) continue;
      for (int j = 0; j < d; ++j) {
        int64_t y = x;
        for (int b = 0; b < k; ++b)
          if ((j >> b) & 1) y |= (int64_t)1 << targets[b];
        idx[j] = y;
        v[j] = psi[y];
      }
      for (int i = 0; i < d; ++i) {
        cplx acc = c_make(0, 0);
        for (int j = 0; j < d; ++j) acc = c_add(acc, c_mul(M[i * d + j], v[j]));
        psi[idx[i]] = acc;
      }
    }
    free(idx);
    free(v);
  }
  return OR_OK;
}

/* |0...0> (all initial states are |0>, Section "Compared with existing libs"). */
void or_init_zero(double* state, int n) {
  memset(state, 0, sizeof(double) * 2 * ((size_t)1 << n));
  state[0] = 1.0;
}

/* ------------------------------------------------------------------------- */
/* Reductions: probability list, marginal probabilities, <Z_i>, Pauli sums     */
/* (the paper's probability / expectation tools, Section "A variety of        */
/* convenient tools"; prob_run_list / prob_run_dict in the API keyword list). */
/* ------------------------------------------------------------------------- */
static double prob_of(cplx a) { return a.re * a.re + a.im * a.im; }

void or_probs(const double* state, int n, double* p) {
  const cplx* psi = (const cplx*)state;
  const int64_t N = (int64_t)1 << n;
  for (int64_t x = 0; x < N; ++x) p[x] = prob_of(psi[x]);
}

/* out[k] = sum of p_x over x whose bits at qubits[0..nq-1] spell k (qubits[j] is
 * bit j of k).  Summed in ascending x. */
int or_marginal(const double* state, int n, const int* qubits, int nq, double* out) {
  if (nq < 0 || nq > n) return OR_EINVAL;
  for (int j = 0; j < nq; ++j) {
    if (qubits[j] < 0 || qubits[j] >= n) return OR_EINVAL;
    for (int i = 0; i < j; ++i) if (qubits[i] == qubits[j]) return OR_EINVAL;
  }
  const cplx* psi = (const cplx*)state;
  const int64_t N = (int64_t)1 << n;
  memset(out, 0, sizeof(double) * ((size_t)1 << nq));
  for (int64_t x = 0; x < N; ++x) {
    int64_t k = 0;
    for (int j = 0; j < nq; ++j) k |= ((x >> qubits[j]) & 1) << j;
    out[k] += prob_of(psi[x]);
  }
  return OR_OK;
}

/* <Z_i> = sum_x p_x (1 - 2 x_i), for every qubit i. */
void or_expect_z(const double* state, int n, double* out) {
  const cplx* psi = (const cplx*)state;
  const int64_t N = (int64_t)1 << n;
  for (int i = 0; i < n; ++i) out[i] = 0.0;
  for (int64_t x = 0; x < N; ++x) {
    double p = prob_of(psi[x]);
    for (int i = 0; i < n; ++i) out[i] += ((x >> i) & 1) ? -p : p;
  }
}

/* Pauli string P = (x, z masks; a Y where both are set) acting on a basis state:
 * P|x> = i^{#Y} (-1)^{popcount(x & z)} |x ^ xmask>.  Uses Y|b> = i(-1)^b |1-b>. */
static cplx pauli_phase(const or_pauli* t, uint64_t x) {
  int ny = __builtin_popcountll(t->xmask & t->zmask) & 3;
  int neg = __builtin_popcountll(x & t->zmask) & 1;
  static const double ire[4] = {1, 0, -1, 0}, iim[4] = {0, 1, 0, -1};
  cplx ph = c_make(ire[ny], iim[ny]);
  if (neg) ph = c_make(-ph.re, -ph.im);
  return ph;
}

static int check_terms(int n, const or_pauli* terms, int64_t nt) {
  uint64_t full = (n >= 64) ? ~0ull : ((1ull << n) - 1);
  for (int64_t k = 0; k < nt; ++k)
    if ((terms[k].xmask | terms[k].zmask) & ~full) return OR_EINVAL;
  return OR_OK;
}

/* <psi|H|psi> for H = sum_k coef_k P_k (the paper's Pauli operator and qop
 * expectation, Sections "Structure of QPanda" and "Variational quantum circuit"):
 * sum_k coef_k Re sum_x conj(psi_{x^xmask}) phase_k(x) psi_x. */
int or_expect_pauli(const double* state, int n, const or_pauli* terms, int64_t nt, double* out) {
  int rc = check_terms(n, terms, nt);
  if (rc) return rc;
  const cplx* psi = (const cplx*)state;
  const int64_t N = (int64_t)1 << n;
  double e = 0.0;
  for (int64_t k = 0; k < nt; ++k) {
    cplx s = c_make(0, 0);
    for (int64_t x = 0; x < N; ++x) {
      cplx v = c_mul(pauli_phase(&terms[k], (uint64_t)x), psi[x]);
      s = c_add(s, c_mul(c_conj(psi[x ^ (int64_t)terms[k].xmask]), v));
    }
    e += terms[k].coef * s.re;
  }
  *out = e;
  return OR_OK;
}

/* out = H psi (out must not alias state). */
int or_apply_pauli_sum(const double* state, int n, const or_pauli* terms, int64_t nt, double* out) {
  int rc = check_terms(n, terms, nt);
  if (rc) return rc;
  const cplx* psi = (const cplx*)state;
  cplx* o = (cplx*)out;
  const int64_t N = (int64_t)1 << n;
  for (int64_t x = 0; x < N; ++x) o[x] = c_make(0, 0);
  for (int64_t k = 0; k < nt; ++k) {
    cplx cf = c_make(terms[k].coef, 0);
    for (int64_t x = 0; x < N; ++x) {
      cplx v = c_mul(cf, c_mul(pauli_phase(&terms[k], (uint64_t)x), psi[x]));
      int64_t y = x ^ (int64_t)terms[k].xmask;
      o[y] = c_add(o[y], v);
    }
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Measurement sampling (measure_all / run_with_configuration in the API      */
/* keyword list, the Measure gate of the QProg listings).                      */
/*                                                                             */
/* Canonical sampler (the paper fixes no algorithm; this is the reading both   */
/* sides implement):                                                           */
/*   u_s   = SplitMix64 output number s (0-based) of the stream seeded `seed`,  */
/*           mapped to [0,1) as (z >> 11) * 2^-53;                              */
/*   p_x   = re*re + im*im (two rounded products, one rounded sum);             */
/*   L     = min(1024, 2^n); block b holds x in [bL, bL + L);                   */
/*   S_b(j)= p_{bL} + ... + p_{bL+j}, summed left to right;                     */
/*   T_b   = S_b(L-1);  G = min(1024, N/L); superblock c holds blocks            */
/*           [cG, cG + G); F_c(i) = T_{cG} + ... + T_{cG+i} left to right;       */
/*   P_0 = 0, P_{c+1} = P_c + F_c(G-1)      (left to right over superblocks);   */
/*   E_0 = 0, E_{cG+i+1} = P_c + F_c(i)     (for N <= 2^20 there is one         */
/*           superblock and E_{b+1} = E_b + T_b);                               */
/*   C_x   = E_b + S_b(x - bL);                                                 */
/*   shot s -> the smallest x with C_x > u_s; if there is none (rounding left   */
/*   the total <= u_s) the largest x with p_x > 0.                              */
/* C is non-decreasing in x, so the block is the first b with E_{b+1} > u_s.    */
/* ------------------------------------------------------------------------- */
uint64_t or_splitmix64(uint64_t seed, uint64_t s) {
  uint64_t z = seed + (s + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static double u01(uint64_t z) { return (double)(z >> 11) * (1.0 / 9007199254740992.0); }

int or_block_prefix(const double* state, int n, double* E /* nblocks + 1 */) {
  const cplx* psi = (const cplx*)state;
  const int64_t N = (int64_t)1 << n;
  const int64_t L = N < 1024 ? N : 1024;
  const int64_t nb = N / L;
  const int64_t G = nb < 1024 ? nb : 1024;
  double P = 0.0; /* P_c */
  E[0] = 0.0;
  for (int64_t c = 0; c < nb / G; ++c) {
    double F = 0.0; /* F_c(i) */
    for (int64_t i = 0; i < G; ++i) {
      const int64_t b = c * G + i;
      double T = 0.0;
      for (int64_t j = 0; j < L; ++j) T += prob_of(psi[b * L + j]);
      F += T;
      E[b + 1] = P + F;
    }
    P = P + F;
  }
  return OR_OK;
}

int or_sample(const double* state, int n, uint64_t seed, int64_t shots, uint64_t* out) {
  const cplx* psi = (const cplx*)state;
  const int64_t N = (int64_t)1 << n;
  const int64_t L = N < 1024 ? N : 1024;
  const int64_t nb = N / L;
  double* E = (double*)malloc(sizeof(double) * (nb + 1));
  if (!E) return OR_ENOMEM;
  or_block_prefix(state, n, E);
  int64_t last_nz = 0;
  for (int64_t x = N - 1; x >= 0; --x)
    if (prob_of(psi[x]) > 0.0) { last_nz = x; break; }
  for (int64_t s = 0; s < shots; ++s) {
    double u = u01(or_splitmix64(seed, (uint64_t)s));
    /* first block b with E[b+1] > u (binary search over the non-decreasing E) */
    int64_t lo = 0, hi = nb;  /* answer in [lo, hi]; hi == nb means none */
    while (lo < hi) {
      int64_t mid = lo + (hi - lo) / 2;
      if (E[mid + 1] > u) hi = mid; else lo = mid + 1;
    }
    if (lo == nb) { out[s] = (uint64_t)last_nz; continue; }
    int64_t b = lo;
    double S = 0.0;
    int64_t pick = b * L + L - 1;
    for (int64_t j = 0; j < L; ++j) {
      S += prob_of(psi[b * L + j]);
      if (E[b] + S > u) { pick = b * L + j; break; }
    }
    out[s] = (uint64_t)pick;
  }
  free(E);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Adjoint differentiation for parametrised rotations (the paper's VQC /      */
/* VQG_RX..RZ / qop, Section "Variational quantum circuit", does not say how  */
/* gradients are taken; this is the adjoint recursion of Jones & Gacon,       */
/* arXiv:2009.02823).  For a gate with dU/dtheta = -(i/2) G U:                 */
/*   dE/dtheta_k = Im <lambda_k| G_k |psi_k>,                                  */
/* psi_k = U_k ... U_1 |0>, lambda_k = U_{k+1}^dag ... U_G^dag H psi_G.        */
/* Generators: RX -> X, RY -> Y, RZ -> Z, P / CR -> -2|1><1| on the target,    */
/* each times the projector onto the control bits; a dagger flips the sign.    */
/* ------------------------------------------------------------------------- */
static int generator_of(const or_gate* g, int n, int* target, uint64_t* cmask, cplx G[4]) {
  int rc = qubits_of(g, n, target, cmask);
  if (rc) return rc;
  double sgn = g->dagger ? -1.0 : 1.0;
  switch (g->type) {
    case OR_RX: G[0] = c_make(0, 0); G[1] = c_make(sgn, 0); G[2] = c_make(sgn, 0); G[3] = c_make(0, 0); break;
    case OR_RY: G[0] = c_make(0, 0); G[1] = c_make(0, -sgn); G[2] = c_make(0, sgn); G[3] = c_make(0, 0); break;
    case OR_RZ: G[0] = c_make(sgn, 0); G[1] = c_make(0, 0); G[2] = c_make(0, 0); G[3] = c_make(-sgn, 0); break;
    case OR_P: case OR_CR:
      G[0] = c_make(0, 0); G[1] = c_make(0, 0); G[2] = c_make(0, 0); G[3] = c_make(-2.0 * sgn, 0); break;
    default: return OR_EUNSUPPORTED;
  }
  return OR_OK;
}

/* <a| G_(target, cmask) |b>, G acting on pairs whose control bits are all set and
 * as 0 elsewhere (the generator of a controlled rotation). */
static cplx braket_gen(const cplx* a, const cplx* b, int n, int t, uint64_t cmask, const cplx G[4]) {
  const int64_t N = (int64_t)1 << n;
  const int64_t tb = (int64_t)1 << t;
  cplx s = c_make(0, 0);
  for (int64_t x = 0; x < N; ++x) {
    if ((x & tb) != 0) continue;
    if (((uint64_t)x & cmask) != cmask) continue;
    cplx b0 = b[x], b1 = b[x | tb];
    cplx g0 = c_add(c_mul(G[0], b0), c_mul(G[1], b1));
    cplx g1 = c_add(c_mul(G[2], b0), c_mul(G[3], b1));
    s = c_add(s, c_mul(c_conj(a[x]), g0));
    s = c_add(s, c_mul(c_conj(a[x | tb]), g1));
  }
  return s;
}

int or_adjoint_grad(int n, const or_gate* gates, int64_t ng, const double* params, int64_t np,
                    const or_pauli* terms, int64_t nt, double* energy, double* grad) {
  const int64_t N = (int64_t)1 << n;
  int rc = check_terms(n, terms, nt);
  if (rc) return rc;
  for (int64_t k = 0; k < ng; ++k) {
    if (gates[k].param_idx >= np) return OR_EINVAL;
    if (gates[k].param_idx >= 0 && gates[k].type != OR_RX && gates[k].type != OR_RY &&
        gates[k].type != OR_RZ && gates[k].type != OR_P && gates[k].type != OR_CR)
      return OR_EUNSUPPORTED;
  }
  cplx* psi = (cplx*)malloc(sizeof(cplx) * N);
  cplx* lam = (cplx*)malloc(sizeof(cplx) * N);
  if (!psi || !lam) { free(psi); free(lam); return OR_ENOMEM; }
  or_init_zero((double*)psi, n);
  rc = or_apply_circuit((double*)psi, n, gates, ng, params);
  if (rc) { free(psi); free(lam); return rc; }
  or_apply_pauli_sum((const double*)psi, n, terms, nt, (double*)lam);
  double e = 0.0;
  for (int64_t x = 0; x < N; ++x) e += c_mul(c_conj(psi[x]), lam[x]).re;
  *energy = e;
  for (int64_t j = 0; j < np; ++j) grad[j] = 0.0;
  for (int64_t k = ng - 1; k >= 0; --k) {
    const or_gate* g = &gates[k];
    if (g->param_idx >= 0) {
      int t; uint64_t cm; cplx G[4];
      rc = generator_of(g, n, &t, &cm, G);
      if (rc) { free(psi); free(lam); return rc; }
      cplx s = braket_gen(lam, psi, n, t, cm, G);
      grad[g->param_idx] += s.im;
    }
    /* step both vectors back through U_k: apply U_k^dagger */
    or_gate inv = *g;
    inv.dagger = !g->dagger;
    or_apply_gate((double*)psi, n, &inv, params);
    or_apply_gate((double*)lam, n, &inv, params);
  }
  free(psi);
  free(lam);
  return OR_OK;
}

/* Energy only (used for parameter-shift and finite-difference pins). */
int or_energy(int n, const or_gate* gates, int64_t ng, const double* params,
              const or_pauli* terms, int64_t nt, double* energy) {
  const int64_t N = (int64_t)1 << n;
  double* psi = (double*)malloc(sizeof(double) * 2 * N);
  if (!psi) return OR_ENOMEM;
  or_init_zero(psi, n);
  int rc = or_apply_circuit(psi, n, gates, ng, params);
  if (!rc) rc = or_expect_pauli(psi, n, terms, nt, energy);
  free(psi);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Fusion cost model: a 3-layer perceptron (not in the paper; the learned      */
/* planner's network).  Inputs x (F features), hidden width H, tanh:           */
/*   h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = w3 . h2 + b3.            */
/* Weights flattened as W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3.           */
/* Loss over a batch of B samples: (1/B) sum_s (y_s - t_s)^2 / 2.              */
/* ------------------------------------------------------------------------- */
int64_t or_mlp_nweights(int F, int H) { return (int64_t)H * F + H + (int64_t)H * H + H + H + 1; }

static void mlp_layers(int F, int H, const double* w, const double* x, double* z1, double* h1, double* z2,
                       double* h2, double* y) {
  const double* W1 = w;
  const double* b1 = W1 + (int64_t)H * F;
  const double* W2 = b1 + H;
  const double* b2 = W2 + (int64_t)H * H;
  const double* w3 = b2 + H;
  const double b3 = w3[H];
  for (int i = 0; i < H; ++i) {
    double s = b1[i];
    for (int j = 0; j < F; ++j) s += W1[(int64_t)i * F + j] * x[j];
    z1[i] = s;
    h1[i] = tanh(s);
  }
  for (int i = 0; i < H; ++i) {
    double s = b2[i];
    for (int j = 0; j < H; ++j) s += W2[(int64_t)i * H + j] * h1[j];
    z2[i] = s;
    h2[i] = tanh(s);
  }
  double s = b3;
  for (int i = 0; i < H; ++i) s += w3[i] * h2[i];
  *y = s;
}

int or_mlp_forward(int F, int H, const double* w, const double* x, int64_t B, double* y) {
  if (F < 1 || H < 1) return OR_EINVAL;
  double* buf = (double*)malloc(sizeof(double) * 4 * H);
  if (!buf) return OR_ENOMEM;
  for (int64_t s = 0; s < B; ++s) mlp_layers(F, H, w, x + s * F, buf, buf + H, buf + 2 * H, buf + 3 * H, &y[s]);
  free(buf);
  return OR_OK;
}

/* Loss and its gradient with respect to every weight (same layout), by the
 * chain rule through the three layers, summed over the batch in sample order. */
int or_mlp_loss_grad(int F, int H, const double* w, const double* x, const double* t, int64_t B, double* loss,
                     double* grad) {
  if (F < 1 || H < 1 || B < 1) return OR_EINVAL;
  const int64_t NW = or_mlp_nweights(F, H);
  double* z1 = (double*)malloc(sizeof(double) * 6 * H);
  if (!z1) return OR_ENOMEM;
  double *h1 = z1 + H, *z2 = z1 + 2 * H, *h2 = z1 + 3 * H, *d2 = z1 + 4 * H, *d1 = z1 + 5 * H;
  const double* W2 = w + (int64_t)H * F + H;
  const double* w3 = W2 + (int64_t)H * H + H;
  double* gW1 = grad;
  double* gb1 = gW1 + (int64_t)H * F;
  double* gW2 = gb1 + H;
  double* gb2 = gW2 + (int64_t)H * H;
  double* gw3 = gb2 + H;
  double* gb3 = gw3 + H;
  for (int64_t k = 0; k < NW; ++k) grad[k] = 0.0;
  double L = 0.0;
  for (int64_t s = 0; s < B; ++s) {
    const double* xs = x + s * F;
    double y;
    mlp_layers(F, H, w, xs, z1, h1, z2, h2, &y);
    const double r = y - t[s];
    L += 0.5 * r * r;
    const double dy = r / (double)B;
    *gb3 += dy;
    for (int i = 0; i < H; ++i) {
      gw3[i] += dy * h2[i];
      d2[i] = dy * w3[i] * (1.0 - h2[i] * h2[i]);
    }
    for (int i = 0; i < H; ++i) {
      gb2[i] += d2[i];
      for (int j = 0; j < H; ++j) gW2[(int64_t)i * H + j] += d2[i] * h1[j];
    }
    for (int j = 0; j < H; ++j) {
      double s2 = 0.0;
      for (int i = 0; i < H; ++i) s2 += W2[(int64_t)i * H + j] * d2[i];
      d1[j] = s2 * (1.0 - h1[j] * h1[j]);
    }
    for (int i = 0; i < H; ++i) {
      gb1[i] += d1[i];
      for (int j = 0; j < F; ++j) gW1[(int64_t)i * F + j] += d1[i] * xs[j];
    }
  }
  *loss = L / (double)B;
  free(z1);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Mid-circuit measurement and classical control (the paper's QMeasure,      */
/* QIf, QWhile and ClassicalProg nodes, Section "Core" with its QIf / QWhile  */
/* listings, and Section "Qif and QWhile": classical bits take +, -, *, /,   */
/* XOR, logical and/or and comparisons).  The paper fixes neither the random */
/* draw nor the decision rule; the readings shared with the GPU library:     */
/*   draw k (0-based count of measurements in one run) u_k = u01(SplitMix64  */
/*   number k of the stream seeded `seed`), the sampler's mapping;           */
/*   p0, p1 = sums of |a_x|^2 over x with bit q = 0 / 1;                     */
/*   outcome = 0 if u_k * (p0 + p1) < p0, else 1;                            */
/*   collapse: a_x = 0 where bit q != outcome, a_x *= 1 / sqrt(p_outcome)    */
/*   elsewhere (Born rule and projective collapse, Nielsen & Chuang 2.2.3).  */
/* ------------------------------------------------------------------------- */
int or_measure(double* state, int n, int q, double u, int* outcome, double* p1_out) {
  if (q < 0 || q >= n) return OR_EINVAL;
  cplx* psi = (cplx*)state;
  const int64_t N = (int64_t)1 << n;
  double p0 = 0.0, p1 = 0.0;
  for (int64_t x = 0; x < N; ++x) {
    if ((x >> q) & 1) p1 += prob_of(psi[x]);
    else p0 += prob_of(psi[x]);
  }
  if (!(p0 + p1 > 0.0)) return OR_EINVAL;
  const int o = (u * (p0 + p1) < p0) ? 0 : 1;
  const double scale = 1.0 / sqrt(o ? p1 : p0);
  for (int64_t x = 0; x < N; ++x) {
    if ((int)((x >> q) & 1) == o) {
      psi[x].re *= scale;
      psi[x].im *= scale;
    } else {
      psi[x].re = 0.0;
      psi[x].im = 0.0;
    }
  }
  *outcome = o;
  if (p1_out) *p1_out = p1 / (p0 + p1);
  return OR_OK;
}

enum { OR_PI_GATES = 0, OR_PI_MEASURE = 1, OR_PI_ASSIGN = 2, OR_PI_IF = 3, OR_PI_WHILE = 4 };
enum {
  OR_CA_MOV = 0, OR_CA_ADD, OR_CA_SUB, OR_CA_MUL, OR_CA_DIV, OR_CA_AND, OR_CA_OR, OR_CA_XOR,
  OR_CA_LT, OR_CA_LE, OR_CA_GT, OR_CA_GE, OR_CA_EQ, OR_CA_NE, OR_CA_NOT
};

typedef struct {
  int32_t op, qubit, dst, alu, lhs, rhs;
  int64_t imm;
  uint32_t n_then, n_else;
  uint64_t gate_begin, gate_end;
} or_pinstr;

typedef struct {
  double* state;
  int n;
  const or_pinstr* prog;
  const or_gate* gates;
  int64_t ng;
  const double* params;
  uint64_t seed, max_iters, nmeas;
  int64_t* cbits;
  int64_t ncbits;
  double* record;
  int64_t record_cap;
} or_run;

static int operand(const or_run* r, int32_t idx, int64_t imm, int64_t* v) {
  if (idx < 0) { *v = imm; return OR_OK; }
  if (idx >= r->ncbits) return OR_EINVAL;
  *v = r->cbits[idx];
  return OR_OK;
}

/* two's-complement wrap for + - * (computed in unsigned arithmetic) */
static int alu_eval(int alu, int64_t a, int64_t b, int64_t* out) {
  switch (alu) {
    case OR_CA_MOV: *out = a; return OR_OK;
    case OR_CA_ADD: *out = (int64_t)((uint64_t)a + (uint64_t)b); return OR_OK;
    case OR_CA_SUB: *out = (int64_t)((uint64_t)a - (uint64_t)b); return OR_OK;
    case OR_CA_MUL: *out = (int64_t)((uint64_t)a * (uint64_t)b); return OR_OK;
    case OR_CA_DIV:
      if (b == 0 || (a == INT64_MIN && b == -1)) return OR_EINVAL;
      *out = a / b;
      return OR_OK;
    case OR_CA_AND: *out = (a != 0) && (b != 0); return OR_OK;
    case OR_CA_OR: *out = (a != 0) || (b != 0); return OR_OK;
    case OR_CA_XOR: *out = a ^ b; return OR_OK;
    case OR_CA_LT: *out = a < b; return OR_OK;
    case OR_CA_LE: *out = a <= b; return OR_OK;
    case OR_CA_GT: *out = a > b; return OR_OK;
    case OR_CA_GE: *out = a >= b; return OR_OK;
    case OR_CA_EQ: *out = a == b; return OR_OK;
    case OR_CA_NE: *out = a != b; return OR_OK;
    case OR_CA_NOT: *out = a == 0; return OR_OK;
    default: return OR_EINVAL;
  }
}

/* Runs instructions [begin, end) of the program; blocks nest by length. */
static int run_block(or_run* r, int64_t begin, int64_t end) {
  int64_t i = begin;
  while (i < end) {
    const or_pinstr* in = &r->prog[i];
    int rc = OR_OK;
    switch (in->op) {
      case OR_PI_GATES:
        if (in->gate_begin > in->gate_end || (int64_t)in->gate_end > r->ng) return OR_EINVAL;
        rc = or_apply_circuit(r->state, r->n, r->gates + in->gate_begin,
                              (int64_t)(in->gate_end - in->gate_begin), r->params);
        if (rc) return rc;
        ++i;
        break;
      case OR_PI_MEASURE: {
        if (in->dst < 0 || in->dst >= r->ncbits) return OR_EINVAL;
        const double u = u01(or_splitmix64(r->seed, r->nmeas));
        int o;
        double p1;
        rc = or_measure(r->state, r->n, in->qubit, u, &o, &p1);
        if (rc) return rc;
        if ((int64_t)r->nmeas < r->record_cap && r->record) r->record[r->nmeas] = p1;
        r->nmeas++;
        r->cbits[in->dst] = o;
        ++i;
        break;
      }
      case OR_PI_ASSIGN: {
        int64_t a, b, v;
        if (in->dst < 0 || in->dst >= r->ncbits) return OR_EINVAL;
        if ((rc = operand(r, in->lhs, in->imm, &a)) || (rc = operand(r, in->rhs, in->imm, &b))) return rc;
        if ((rc = alu_eval(in->alu, a, b, &v))) return rc;
        r->cbits[in->dst] = v;
        ++i;
        break;
      }
      case OR_PI_IF: {
        const int64_t t0 = i + 1, t1 = t0 + in->n_then, e1 = t1 + in->n_else;
        if (e1 > end) return OR_EINVAL;
        int64_t c;
        if ((rc = operand(r, in->lhs, in->imm, &c))) return rc;
        rc = c != 0 ? run_block(r, t0, t1) : run_block(r, t1, e1);
        if (rc) return rc;
        i = e1;
        break;
      }
      case OR_PI_WHILE: {
        const int64_t b0 = i + 1, b1 = b0 + in->n_then;
        if (b1 > end || in->n_else != 0) return OR_EINVAL;
        uint64_t iters = 0;
        for (;;) {
          int64_t c;
          if ((rc = operand(r, in->lhs, in->imm, &c))) return rc;
          if (c == 0) break;
          if (iters++ >= r->max_iters) return OR_ELIMIT;
          if ((rc = run_block(r, b0, b1))) return rc;
        }
        i = b1;
        break;
      }
      default:
        return OR_EINVAL;
    }
  }
  return OR_OK;
}

/* Runs a program with classical control on `state` (in place).  cbits (ncbits
 * int64 values, in/out) are the classical register; record[k] receives
 * p1 / (p0 + p1) of measurement k (up to record_cap); *nmeasured the count. */
int or_run_program(double* state, int n, const or_pinstr* prog, int64_t nprog, const or_gate* gates, int64_t ng,
                   const double* params, uint64_t seed, uint64_t max_iters, int64_t* cbits, int64_t ncbits,
                   double* record, int64_t record_cap, uint64_t* nmeasured) {
  or_run r;
  r.state = state;
  r.n = n;
  r.prog = prog;
  r.gates = gates;
  r.ng = ng;
  r.params = params;
  r.seed = seed;
  r.max_iters = max_iters;
  r.nmeas = 0;
  r.cbits = cbits;
  r.ncbits = ncbits;
  r.record = record;
  r.record_cap = record_cap;
  const int rc = run_block(&r, 0, nprog);
  if (nmeasured) *nmeasured = r.nmeas;
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Noise (the paper's NoiseQVM, Section "Multi-simulation methods", noise     */
/* simulation method): one-qubit Kraus channels attached to gate types, a     */
/* readout confusion matrix and a rotation error.                             */
/* Kraus sets, as printed in the paper (row-major 2x2):                       */
/*   DAMPING       K1 = [[1,0],[0,sqrt(1-p)]], K2 = [[0,sqrt(p)],[0,0]]        */
/*   DEPHASING     K1 = sqrt(1-p) I, K2 = sqrt(p) Z                            */
/*   DECOHERENCE   K_ij = Kdamp_i Kdeph_j (i, j = 1, 2; K1 = K11, K2 = K12,    */
/*                 K3 = K21, K4 = K22) with p_damp = 1 - exp(-tg/T1) and       */
/*                 p_deph = (1 - exp(-(tg/T2 - tg/(2 T1)))) / 2                */
/*   DEPOLARIZING  sqrt(1 - 3p/4) I, sqrt(p)/2 X, sqrt(p)/2 Y, sqrt(p)/2 Z      */
/*   BITFLIP       sqrt(1-p) I, sqrt(p) X                                      */
/*   BITPHASEFLIP  sqrt(1-p) I, sqrt(p) Y   (the matrix the paper prints for    */
/*                 its "bit or phase flip" operator)                           */
/*   PHASEFLIP     sqrt(1-p) I, sqrt(p) Z                                      */
/*   PHASE_DAMPING K1 = [[1,0],[0,sqrt(1-p)]], K2 = [[0,0],[0,sqrt(p)]]        */
/* ------------------------------------------------------------------------- */
enum {
  OR_NOISE_DAMPING = 0, OR_NOISE_DEPHASING = 1, OR_NOISE_DECOHERENCE = 2, OR_NOISE_DEPOLARIZING = 3,
  OR_NOISE_BITFLIP = 4, OR_NOISE_BITPHASEFLIP = 5, OR_NOISE_PHASEFLIP = 6, OR_NOISE_PHASE_DAMPING = 7
};

typedef struct {
  int32_t model, gate_type, q0, q1;
  double p, t1, t2, tgate;
} or_noise_rule;

static void set2(cplx K[4], double a, double b, double c, double d) {
  K[0] = c_make(a, 0); K[1] = c_make(b, 0); K[2] = c_make(c, 0); K[3] = c_make(d, 0);
}

static void mul2(const cplx A[4], const cplx B[4], cplx C[4]) {
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      C[2 * i + j] = c_add(c_mul(A[2 * i], B[j]), c_mul(A[2 * i + 1], B[2 + j]));
}

/* Kraus operators of a rule into K (up to 4 x 4 entries); returns their count,
 * or 0 for a bad rule.  *unital: 1 when every operator is a scaled unitary (the
 * choice weights are the squared scales, independent of the state). */
int or_kraus(int model, double p, double t1, double t2, double tg, double* K8x4, int* unital) {
  cplx* K = (cplx*)K8x4;
  const double s = sqrt(p), r = sqrt(1.0 - p);
  *unital = 1;
  switch (model) {
    case OR_NOISE_DAMPING:
      set2(K, 1, 0, 0, r); set2(K + 4, 0, s, 0, 0); *unital = 0; return 2;
    case OR_NOISE_PHASE_DAMPING:
      set2(K, 1, 0, 0, r); set2(K + 4, 0, 0, 0, s); *unital = 0; return 2;
    case OR_NOISE_DEPHASING:
    case OR_NOISE_PHASEFLIP:
      set2(K, r, 0, 0, r); set2(K + 4, s, 0, 0, -s); return 2;
    case OR_NOISE_BITFLIP:
      set2(K, r, 0, 0, r); set2(K + 4, 0, s, s, 0); return 2;
    case OR_NOISE_BITPHASEFLIP:
      set2(K, r, 0, 0, r);
      K[4] = c_make(0, 0); K[5] = c_make(0, -s); K[6] = c_make(0, s); K[7] = c_make(0, 0);
      return 2;
    case OR_NOISE_DEPOLARIZING: {
      const double a = sqrt(1.0 - 0.75 * p), h = 0.5 * s;
      set2(K, a, 0, 0, a);
      set2(K + 4, 0, h, h, 0);
      K[8] = c_make(0, 0); K[9] = c_make(0, -h); K[10] = c_make(0, h); K[11] = c_make(0, 0);
      set2(K + 12, h, 0, 0, -h);
      return 4;
    }
    case OR_NOISE_DECOHERENCE: {
      if (!(t1 > 0) || !(t2 > 0) || !(tg >= 0)) return 0;
      const double pa = 1.0 - exp(-tg / t1), pd = 0.5 * (1.0 - exp(-(tg / t2 - tg / (2.0 * t1))));
      cplx D[2][4], P[2][4];
      set2(D[0], 1, 0, 0, sqrt(1.0 - pa)); set2(D[1], 0, sqrt(pa), 0, 0);
      set2(P[0], sqrt(1.0 - pd), 0, 0, sqrt(1.0 - pd)); set2(P[1], sqrt(pd), 0, 0, -sqrt(pd));
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) mul2(D[i], P[j], K + 4 * (2 * i + j));
      *unital = 0;
      return 4;
    }
    default:
      return 0;
  }
}

/* The weights w_j = || K_j psi ||^2 on qubit q (from the state), or the squared
 * scales of a scaled-unitary set (independent of the state). */
static void kraus_weights(const cplx* psi, int n, int q, const cplx* K, int m, int unital, double* w) {
  for (int j = 0; j < m; ++j) {
    if (unital) {
      const cplx* k = K + 4 * j;
      /* a scaled unitary c U has |column|^2 = c^2 */
      w[j] = k[0].re * k[0].re + k[0].im * k[0].im + k[2].re * k[2].re + k[2].im * k[2].im;
      continue;
    }
    double s = 0.0;
    const int64_t N = (int64_t)1 << n, b = (int64_t)1 << q;
    for (int64_t x = 0; x < N; ++x) {
      if (x & b) continue;
      const cplx a0 = psi[x], a1 = psi[x | b];
      const cplx y0 = c_add(c_mul(K[4 * j], a0), c_mul(K[4 * j + 1], a1));
      const cplx y1 = c_add(c_mul(K[4 * j + 2], a0), c_mul(K[4 * j + 3], a1));
      s += prob_of(y0) + prob_of(y1);
    }
    w[j] = s;
  }
}

static int is_rotation(int type) {
  return type == OR_RX || type == OR_RY || type == OR_RZ || type == OR_U3 || type == OR_P || type == OR_CR;
}

/* One Monte-Carlo trajectory.  For every gate in order:
 *   1. a rotation gate's theta gets e * (2u - 1) added (one draw, if e > 0);
 *   2. the gate is applied;
 *   3. for every rule that matches it (gate type, or -1 for all; q0/q1 the
 *      gate's first / second qubit, -1 = any), in rule order, and every qubit
 *      the gate acts on (controls, then target, ascending), one draw u picks
 *      the smallest j with u * W < w_1 + ... + w_j (W = sum of weights), and
 *      psi <- K_j psi / sqrt(w_j).
 * Draw k of the trajectory is u01(SplitMix64 output k of the stream seeded
 * `seed`).  *ndraws receives the draws used. */
int or_run_noisy(double* state, int n, const or_gate* gates, int64_t ng, const double* params,
                 const or_noise_rule* rules, int64_t nrules, double rot_err, uint64_t seed, uint64_t* ndraws) {
  cplx* psi = (cplx*)state;
  uint64_t k = 0;
  double* pv = NULL;
  int64_t np = 0;
  for (int64_t g = 0; g < ng; ++g)
    if (gates[g].param_idx >= 0 && gates[g].param_idx + 1 > np) np = gates[g].param_idx + 1;
  if (np) {
    pv = (double*)malloc(sizeof(double) * np);
    if (!pv) return OR_ENOMEM;
  }
  int rc = OR_OK;
  for (int64_t g = 0; g < ng && rc == OR_OK; ++g) {
    or_gate gate = gates[g];
    const double* prm = params;
    if (rot_err > 0.0 && is_rotation(gate.type)) {
      const double d = rot_err * (2.0 * u01(or_splitmix64(seed, k++)) - 1.0);
      if (gate.param_idx >= 0) {
        memcpy(pv, params, sizeof(double) * np);
        pv[gate.param_idx] += d;
        prm = pv;
      } else {
        gate.p[0] += d;
      }
    }
    if ((rc = or_apply_gate(state, n, &gate, prm)) != OR_OK) break;
    int t;
    uint64_t cm;
    if ((rc = qubits_of(&gate, n, &t, &cm)) != OR_OK) break;
    const int first = gate.q0;
    const int second = is_two_qubit(gate.type) ? gate.q1 : -1;
    for (int64_t r = 0; r < nrules && rc == OR_OK; ++r) {
      const or_noise_rule* R = &rules[r];
      if (R->gate_type >= 0 && R->gate_type != gate.type) continue;
      if (R->q0 >= 0 && R->q0 != first) continue;
      if (R->q1 >= 0 && R->q1 != second) continue;
      double K8[32];
      int unital = 0;
      const int m = or_kraus(R->model, R->p, R->t1, R->t2, R->tgate, K8, &unital);
      if (!m) { rc = OR_EINVAL; break; }
      const uint64_t touched = cm | (1ull << t);
      for (int q = 0; q < n; ++q) {
        if (!((touched >> q) & 1)) continue;
        double w[4] = {0.0, 0.0, 0.0, 0.0}, W = 0.0;
        kraus_weights(psi, n, q, (const cplx*)K8, m, unital, w);
        for (int j = 0; j < m; ++j) W += w[j];
        const double u = u01(or_splitmix64(seed, k++));
        int pick = m - 1;
        double c = 0.0;
        for (int j = 0; j < m; ++j) {
          c += w[j];
          if (u * W < c) { pick = j; break; }
        }
        if (!(w[pick] > 0.0)) { rc = OR_EINVAL; break; }
        const cplx* Kp = (const cplx*)K8 + 4 * pick;
        const double sc = 1.0 / sqrt(w[pick]);
        const int64_t N = (int64_t)1 << n, b = (int64_t)1 << q;
        for (int64_t x = 0; x < N; ++x) {
          if (x & b) continue;
          const cplx a0 = psi[x], a1 = psi[x | b];
          const cplx y0 = c_add(c_mul(Kp[0], a0), c_mul(Kp[1], a1));
          const cplx y1 = c_add(c_mul(Kp[2], a0), c_mul(Kp[3], a1));
          psi[x] = c_make(y0.re * sc, y0.im * sc);
          psi[x | b] = c_make(y1.re * sc, y1.im * sc);
        }
      }
    }
  }
  free(pv);
  if (ndraws) *ndraws = k;
  return rc;
}

/* Readout error on sampled basis indices: bit i of shot s reads wrong with
 * probability 1 - f0 (true bit 0) or 1 - f1 (true bit 1), the confusion matrix
 * [[f0, 1-f0], [1-f1, f1]] of the paper's set_readout_error; draw
 * u = u01(SplitMix64 output s*n + i of the stream seeded `seed`) flips the bit
 * when u >= f_bit. */
void or_readout(uint64_t* samples, int64_t shots, int n, double f0, double f1, uint64_t seed) {
  for (int64_t s = 0; s < shots; ++s)
    for (int i = 0; i < n; ++i) {
      const int bit = (int)((samples[s] >> i) & 1);
      const double u = u01(or_splitmix64(seed, (uint64_t)s * (uint64_t)n + (uint64_t)i));
      if (u >= (bit ? f1 : f0)) samples[s] ^= 1ull << i;
    }
}

/* ---- density-matrix reference (n <= 8): rho -> U rho U^dag per gate, then
 * rho -> sum_j K_j rho K_j^dag for every matching rule and touched qubit, as
 * above but averaged instead of sampled (no rotation error). rho is 2^n x 2^n
 * complex, row-major, interleaved. ------------------------------------------ */
static void dm_left(cplx* rho, int n, int q, uint64_t cm, const cplx M[4]) {  /* rho <- M_q rho */
  const int64_t N = (int64_t)1 << n, b = (int64_t)1 << q;
  for (int64_t c = 0; c < N; ++c)
    for (int64_t x = 0; x < N; ++x) {
      if ((x & b) || (x & cm) != (int64_t)cm) continue;
      const cplx a0 = rho[x * N + c], a1 = rho[(x | b) * N + c];
      rho[x * N + c] = c_add(c_mul(M[0], a0), c_mul(M[1], a1));
      rho[(x | b) * N + c] = c_add(c_mul(M[2], a0), c_mul(M[3], a1));
    }
}

static void dm_right(cplx* rho, int n, int q, uint64_t cm, const cplx M[4]) {  /* rho <- rho M_q^dag */
  const int64_t N = (int64_t)1 << n, b = (int64_t)1 << q;
  const cplx Mc[4] = {c_conj(M[0]), c_conj(M[1]), c_conj(M[2]), c_conj(M[3])};
  for (int64_t r = 0; r < N; ++r)
    for (int64_t x = 0; x < N; ++x) {
      if ((x & b) || (x & cm) != (int64_t)cm) continue;
      const cplx a0 = rho[r * N + x], a1 = rho[r * N + (x | b)];
      rho[r * N + x] = c_add(c_mul(a0, Mc[0]), c_mul(a1, Mc[1]));
      rho[r * N + (x | b)] = c_add(c_mul(a0, Mc[2]), c_mul(a1, Mc[3]));
    }
}

int or_dm_run(double* rho_out, int n, const or_gate* gates, int64_t ng, const double* params,
              const or_noise_rule* rules, int64_t nrules) {
  if (n < 1 || n > 8) return OR_EINVAL;
  const int64_t N = (int64_t)1 << n;
  cplx* rho = (cplx*)rho_out;
  cplx* acc = (cplx*)malloc(sizeof(cplx) * N * N);
  cplx* tmp = (cplx*)malloc(sizeof(cplx) * N * N);
  if (!acc || !tmp) { free(acc); free(tmp); return OR_ENOMEM; }
  for (int64_t i = 0; i < N * N; ++i) rho[i] = c_make(0, 0);
  rho[0] = c_make(1, 0);
  int rc = OR_OK;
  for (int64_t g = 0; g < ng && rc == OR_OK; ++g) {
    int t;
    uint64_t cm;
    cplx U[4];
    if ((rc = resolve(&gates[g], n, params, &t, &cm, U)) != OR_OK) break;
    dm_left(rho, n, t, cm, U);
    dm_right(rho, n, t, cm, U);
    const int first = gates[g].q0;
    const int second = is_two_qubit(gates[g].type) ? gates[g].q1 : -1;
    for (int64_t r = 0; r < nrules && rc == OR_OK; ++r) {
      const or_noise_rule* R = &rules[r];
      if (R->gate_type >= 0 && R->gate_type != gates[g].type) continue;
      if (R->q0 >= 0 && R->q0 != first) continue;
      if (R->q1 >= 0 && R->q1 != second) continue;
      double K8[32];
      int unital = 0;
      const int m = or_kraus(R->model, R->p, R->t1, R->t2, R->tgate, K8, &unital);
      if (!m) { rc = OR_EINVAL; break; }
      const uint64_t touched = cm | (1ull << t);
      for (int q = 0; q < n; ++q) {
        if (!((touched >> q) & 1)) continue;
        for (int64_t i = 0; i < N * N; ++i) acc[i] = c_make(0, 0);
        for (int j = 0; j < m; ++j) {
          memcpy(tmp, rho, sizeof(cplx) * N * N);
          dm_left(tmp, n, q, 0, (const cplx*)K8 + 4 * j);
          dm_right(tmp, n, q, 0, (const cplx*)K8 + 4 * j);
          for (int64_t i = 0; i < N * N; ++i) acc[i] = c_add(acc[i], tmp[i]);
        }
        memcpy(rho, acc, sizeof(cplx) * N * N);
      }
    }
  }
  free(acc);
  free(tmp);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Partial amplitudes (the paper's PartialAmpQVM, Section "Multi-simulation   */
/* methods", noise-free simulation method): the qubits are split into a low   */
/* block (0 .. n_low-1) and a high block; every gate with qubits in both      */
/* blocks is cut.  A controlled gate with target t, controls C_t in t's block */
/* and C_o in the other block is                                              */
/*   P(C_o all 1) (x) [U on t controlled by C_t]  +  (I - P(C_o all 1)) (x) I */
/* so k cut gates turn the circuit into 2^k products of block circuits; path  */
/* bit i = 1 takes the first term of cut i.  <x|psi> = sum over paths of      */
/* <x_low|lo_path> <x_high|hi_path>.                                          */
/* ------------------------------------------------------------------------- */
static void project_ones(cplx* psi, int n, uint64_t mask, int keep_all_ones) {
  const int64_t N = (int64_t)1 << n;
  for (int64_t x = 0; x < N; ++x) {
    const int all = ((uint64_t)x & mask) == mask;
    if (all != keep_all_ones) psi[x] = c_make(0, 0);
  }
}

int or_partial_amplitudes(int n, const or_gate* gates, int64_t ng, const double* params, int n_low,
                          const uint64_t* idx, int64_t count, double* out_amps, uint64_t* npaths) {
  if (n_low < 1 || n_low >= n || n > 24) return OR_EINVAL;
  const int nh = n - n_low;
  const uint64_t lowmask = ((uint64_t)1 << n_low) - 1;
  /* cut gates */
  int64_t k = 0;
  for (int64_t g = 0; g < ng; ++g) {
    int t;
    uint64_t cm;
    int rc = qubits_of(&gates[g], n, &t, &cm);
    if (rc) return rc;
    const uint64_t all = cm | ((uint64_t)1 << t);
    if ((all & lowmask) && (all & ~lowmask)) ++k;
  }
  if (k > 20) return OR_EUNSUPPORTED;
  cplx* lo = (cplx*)malloc(sizeof(cplx) << n_low);
  cplx* hi = (cplx*)malloc(sizeof(cplx) << nh);
  cplx* out = (cplx*)out_amps;
  if (!lo || !hi) { free(lo); free(hi); return OR_ENOMEM; }
  for (int64_t i = 0; i < count; ++i) out[i] = c_make(0, 0);
  int rc = OR_OK;
  for (uint64_t path = 0; path < ((uint64_t)1 << k) && rc == OR_OK; ++path) {
    or_init_zero((double*)lo, n_low);
    or_init_zero((double*)hi, nh);
    int64_t cut = 0;
    for (int64_t g = 0; g < ng && rc == OR_OK; ++g) {
      int t;
      uint64_t cm;
      cplx U[4];
      if ((rc = resolve(&gates[g], n, params, &t, &cm, U)) != OR_OK) break;
      const uint64_t all = cm | ((uint64_t)1 << t);
      const int t_low = t < n_low;
      if (!((all & lowmask) && (all & ~lowmask))) {     /* inside one block */
        if (t_low) apply_2x2(lo, n_low, t, cm, U);
        else apply_2x2(hi, nh, t - n_low, cm >> n_low, U);
        continue;
      }
      const int bit = (int)((path >> cut) & 1);
      ++cut;
      const uint64_t c_low = cm & lowmask, c_high = cm >> n_low;
      if (t_low) {
        if (bit) apply_2x2(lo, n_low, t, c_low, U);
        project_ones(hi, nh, c_high, bit);
      } else {
        if (bit) apply_2x2(hi, nh, t - n_low, c_high, U);
        project_ones(lo, n_low, c_low, bit);
      }
    }
    for (int64_t i = 0; i < count && rc == OR_OK; ++i) {
      const uint64_t x = idx[i];
      if (x >> n) { rc = OR_EINVAL; break; }
      out[i] = c_add(out[i], c_mul(lo[x & lowmask], hi[x >> n_low]));
    }
  }
  free(lo);
  free(hi);
  if (npaths) *npaths = (uint64_t)1 << k;
  return rc;
}
