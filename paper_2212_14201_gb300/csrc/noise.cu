// Noisy simulation by Monte-Carlo trajectories (the paper's NoiseQVM, Section
// "Multi-simulation methods", noise simulation method): one-qubit Kraus channels
// attached to gate types, a rotation error on rotation angles, and a readout
// confusion matrix on sampled bits.
//
// Kraus sets as the paper prints them (row-major 2x2):
//   DAMPING       [[1,0],[0,sqrt(1-p)]], [[0,sqrt(p)],[0,0]]
//   DEPHASING     sqrt(1-p) I, sqrt(p) Z           (PHASEFLIP: the same set)
//   DECOHERENCE   Kdamp_i Kdeph_j, i, j = 1, 2 (order 11, 12, 21, 22), with
//                 p_damp = 1 - exp(-tg/T1), p_deph = (1 - exp(-(tg/T2 - tg/(2 T1)))) / 2
//   DEPOLARIZING  sqrt(1 - 3p/4) I, sqrt(p)/2 X, sqrt(p)/2 Y, sqrt(p)/2 Z
//   BITFLIP       sqrt(1-p) I, sqrt(p) X
//   BITPHASEFLIP  sqrt(1-p) I, sqrt(p) Y
//   PHASE_DAMPING [[1,0],[0,sqrt(1-p)]], [[0,0],[0,sqrt(p)]]
// A trajectory, gate by gate: a rotation's theta gets e (2u - 1) (one draw);
// the gate; then for each matching rule and each qubit the gate touches
// (ascending) one draw u picks the smallest j with u W < w_1 + ... + w_j, and
// psi <- K_j psi / sqrt(w_j).  Weights w_j = ||K_j psi||^2 = tr(K_j^dag K_j G),
// G the 2x2 Gram matrix of the qubit's amplitude pairs (one reduction pass);
// for a set of scaled unitaries w_j is the squared scale (no pass), and the
// chosen Pauli joins the gate stream, so such stretches stay fusable.
#include <math.h>

#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "fixed.h"
#include "internal.h"

namespace qs {

// ---- Gram matrix of one qubit: g00 = sum |a0|^2, g11 = sum |a1|^2,
// g01 = sum a0 conj(a1), over the pairs (x, x | 2^q) -------------------------------
template <class A>
__global__ void __launch_bounds__(256) k_gram(const A* __restrict__ a, uint64_t pairs, int q,
                                               double* __restrict__ part) {
  __shared__ double sh[4][8];
  double g00 = 0.0, g11 = 0.0, gr = 0.0, gi = 0.0;
  const uint64_t b = 1ull << q;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < pairs; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t x0 = ((i >> q) << (q + 1)) | (i & (b - 1));
    const double2 a0 = ld_amp(a, x0), a1 = ld_amp(a, x0 | b);
    g00 = fma(a0.y, a0.y, fma(a0.x, a0.x, g00));
    g11 = fma(a1.y, a1.y, fma(a1.x, a1.x, g11));
    gr = fma(a0.y, a1.y, fma(a0.x, a1.x, gr));   // Re(a0 conj(a1))
    gi = fma(a0.y, a1.x, fma(-a0.x, a1.y, gi));  // Im(a0 conj(a1))
  }
  double v[4] = {g00, g11, gr, gi};
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (l == 0) sh[k][w] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += sh[threadIdx.x][i];
    part[(size_t)blockIdx.x * 4 + threadIdx.x] = t;
  }
}

// The same four sums exactly, for a state within the Q60 bound: components rounded
// once to Q60 and the products summed as 128-bit integers (units of 2^-120; every
// sum is at most the squared norm <= 1.5625 in magnitude).  Integer pipes instead
// of GB300's 1/74-rate FP64 pipe.
using i128 = __int128;

__device__ __forceinline__ i128 shfl_xor_i128(i128 v, int o) {
  const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)(uint64_t)v, o);
  const unsigned long long hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(uint64_t)((unsigned __int128)v >> 64), o);
  return (i128)(((unsigned __int128)hi << 64) | lo);
}

template <class A>
__global__ void __launch_bounds__(256) k_gram_exact(const A* __restrict__ a, uint64_t pairs, int q,
                                                     uint64_t* __restrict__ part) {
  __shared__ uint64_t sh[4][8][2];
  i128 v[4] = {0, 0, 0, 0};
  const uint64_t b = 1ull << q;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < pairs; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t x0 = ((i >> q) << (q + 1)) | (i & (b - 1));
    const double2 a0 = ld_amp(a, x0), a1 = ld_amp(a, x0 | b);
    const int64_t r0 = q60_from_double(a0.x), i0 = q60_from_double(a0.y);
    const int64_t r1 = q60_from_double(a1.x), i1 = q60_from_double(a1.y);
    v[0] += (i128)r0 * r0 + (i128)i0 * i0;
    v[1] += (i128)r1 * r1 + (i128)i1 * i1;
    v[2] += (i128)r0 * r1 + (i128)i0 * i1;  // Re(a0 conj(a1))
    v[3] += (i128)i0 * r1 - (i128)r0 * i1;  // Im(a0 conj(a1))
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += shfl_xor_i128(v[k], o);
    if (l == 0) {
      sh[k][w][0] = (uint64_t)v[k];
      sh[k][w][1] = (uint64_t)((unsigned __int128)v[k] >> 64);
    }
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    i128 t = 0;
    for (int i = 0; i < 8; ++i) t += (i128)(((unsigned __int128)sh[threadIdx.x][i][1] << 64) | sh[threadIdx.x][i][0]);
    part[((size_t)blockIdx.x * 4 + threadIdx.x) * 2] = (uint64_t)t;
    part[((size_t)blockIdx.x * 4 + threadIdx.x) * 2 + 1] = (uint64_t)((unsigned __int128)t >> 64);
  }
}

__global__ void k_gram_exact_finish(const uint64_t* __restrict__ part, int nblocks, double* __restrict__ out) {
  const int k = threadIdx.x;
  if (k >= 4) return;
  i128 t = 0;
  for (int c = 0; c < nblocks; ++c)
    t += (i128)(((unsigned __int128)part[((size_t)c * 4 + k) * 2 + 1] << 64) | part[((size_t)c * 4 + k) * 2]);
  const bool neg = t < 0;
  const unsigned __int128 m = neg ? (unsigned __int128)(-t) : (unsigned __int128)t;
  const double d = (double)(uint64_t)(m >> 64) * 18446744073709551616.0 + (double)(uint64_t)m;
  out[k] = (neg ? -d : d) * 0x1p-120;
}

__global__ void k_gram_finish(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  const int k = threadIdx.x;
  if (k >= 4) return;
  double t = 0.0;
  for (int c = 0; c < nblocks; ++c) t += part[(size_t)c * 4 + k];
  out[k] = t;
}

// ---- readout error on sampled indices ----------------------------------------------
__global__ void k_readout(uint64_t* __restrict__ samples, uint64_t shots, int n, double f0, double f1,
                          uint64_t seed) {
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < shots; s += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t x = samples[s];
    for (int i = 0; i < n; ++i) {
      const int bit = (int)((x >> i) & 1);
      const double u = u01_of(splitmix64(seed, s * (uint64_t)n + (uint64_t)i));
      if (u >= (bit ? f1 : f0)) x ^= 1ull << i;
    }
    samples[s] = x;
  }
}

// ---- Kraus sets ---------------------------------------------------------------------
struct KrausSet {
  int m = 0;
  bool unital = true;  // every operator c_j U_j with U_j in {I, X, Y, Z}
  Mat2 K[4];
  int pauli[4];        // unital sets: 0 = I, 1 = X, 2 = Y, 3 = Z
  double w[4];         // unital sets: c_j^2
};

static Mat2 m2(double a, double b, double c, double d) {
  Mat2 r;
  r.m[0] = {a, 0};
  r.m[1] = {b, 0};
  r.m[2] = {c, 0};
  r.m[3] = {d, 0};
  return r;
}

static Mat2 m2mul(const Mat2& A, const Mat2& B) {
  Mat2 r;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      const C2 x = A.m[2 * i], y = B.m[j], u = A.m[2 * i + 1], v = B.m[2 + j];
      r.m[2 * i + j] = {x.re * y.re - x.im * y.im + u.re * v.re - u.im * v.im,
                        x.re * y.im + x.im * y.re + u.re * v.im + u.im * v.re};
    }
  return r;
}

static int kraus_set(const qs_noise_rule& r, KrausSet* ks) {
  const double p = r.p;
  if (r.model != QS_NOISE_DECOHERENCE && !(p >= 0.0 && p <= 1.0))
    return fail(QS_ERR_INVALID_ARG, "noise probability %g outside [0, 1]", p);
  const double s = sqrt(p), c = sqrt(1.0 - p);
  auto pauli_set = [&](int P, double scale) {
    ks->m = 2;
    ks->unital = true;
    ks->pauli[0] = 0;
    ks->w[0] = c * c;
    ks->pauli[1] = P;
    ks->w[1] = scale * scale;
    ks->K[0] = m2(c, 0, 0, c);
  };
  switch (r.model) {
    case QS_NOISE_DAMPING:
      ks->m = 2;
      ks->unital = false;
      ks->K[0] = m2(1, 0, 0, c);
      ks->K[1] = m2(0, s, 0, 0);
      return QS_OK;
    case QS_NOISE_PHASE_DAMPING:
      ks->m = 2;
      ks->unital = false;
      ks->K[0] = m2(1, 0, 0, c);
      ks->K[1] = m2(0, 0, 0, s);
      return QS_OK;
    case QS_NOISE_DEPHASING:
    case QS_NOISE_PHASEFLIP: pauli_set(3, s); return QS_OK;
    case QS_NOISE_BITFLIP: pauli_set(1, s); return QS_OK;
    case QS_NOISE_BITPHASEFLIP: pauli_set(2, s); return QS_OK;
    case QS_NOISE_DEPOLARIZING: {
      ks->m = 4;
      ks->unital = true;
      const double a = sqrt(1.0 - 0.75 * p), h = 0.5 * s;
      ks->w[0] = a * a;
      for (int j = 1; j < 4; ++j) ks->w[j] = h * h;
      for (int j = 0; j < 4; ++j) ks->pauli[j] = j;
      return QS_OK;
    }
    case QS_NOISE_DECOHERENCE: {
      if (!(r.t1 > 0.0) || !(r.t2 > 0.0) || !(r.tgate >= 0.0))
        return fail(QS_ERR_INVALID_ARG, "decoherence needs T1 > 0, T2 > 0, tgate >= 0");
      const double pa = 1.0 - exp(-r.tgate / r.t1);
      const double pd = 0.5 * (1.0 - exp(-(r.tgate / r.t2 - r.tgate / (2.0 * r.t1))));
      if (!(pd >= 0.0 && pd <= 1.0)) return fail(QS_ERR_INVALID_ARG, "decoherence: T2 > 2 T1 gives no valid dephasing");
      const Mat2 D[2] = {m2(1, 0, 0, sqrt(1.0 - pa)), m2(0, sqrt(pa), 0, 0)};
      const Mat2 P[2] = {m2(sqrt(1.0 - pd), 0, 0, sqrt(1.0 - pd)), m2(sqrt(pd), 0, 0, -sqrt(pd))};
      ks->m = 4;
      ks->unital = false;
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) ks->K[2 * i + j] = m2mul(D[i], P[j]);
      return QS_OK;
    }
    default: return fail(QS_ERR_INVALID_ARG, "unknown noise model %d", r.model);
  }
}

static bool is_rotation(int type) {
  return type == QS_RX || type == QS_RY || type == QS_RZ || type == QS_U3 || type == QS_P || type == QS_CR;
}

static bool two_qubit(int type) { return type == QS_CNOT || type == QS_CZ || type == QS_CR; }

// ---- the trajectory driver -----------------------------------------------------------
struct Trajectory {
  qs_state* s;
  bool fuse;
  uint64_t seed, k = 0;
  std::vector<qs_gate> pending;  // parameter-free records (angles resolved)

  double draw() { return u01_of(splitmix64(seed, k++)); }

  int flush() {
    if (pending.empty()) return QS_OK;
    int rc = QS_OK;
    if (fuse && pending.size() > 1) {
      qs_plan* p = nullptr;
      rc = qs_plan_create(s->n, pending.data(), pending.size(), QS_PLAN_GREEDY, 5, &p);
      if (rc == QS_OK) rc = qs_apply(s, pending.data(), pending.size(), nullptr, p);
      if (p) qs_plan_free(p);
    } else {
      rc = qs_apply(s, pending.data(), pending.size(), nullptr, nullptr);
    }
    pending.clear();
    return rc;
  }

  int gram(int q, double G[4]) {
    const uint64_t pairs = 1ull << (s->n - 1);
    const int nblocks = (int)std::min<uint64_t>(608, std::max<uint64_t>(1, pairs / 512));
    double* part = (double*)s->ws;
    double* dres = part + (size_t)nblocks * 4;
    KTimer kt(s, QS_K_REDUCE, 1, 1, 1ull << q, 0, (double)(pairs * 2), 8.0 * (double)pairs);
    if (s->bound == 1) {  // components known to lie within the Q60 bound: exact integer sums
      uint64_t* ipart = (uint64_t*)s->ws;
      dres = (double*)(ipart + (size_t)nblocks * 8);
      with_amps(s, [&](auto* a) {
        using T = std::remove_cv_t<std::remove_pointer_t<decltype(a)>>;
        k_gram_exact<<<nblocks, 256, 0, s->stream>>>((const T*)a, pairs, q, ipart);
        return QS_OK;
      });
      QS_TRY(launch_check("gram"));
      k_gram_exact_finish<<<1, 32, 0, s->stream>>>(ipart, nblocks, dres);
      QS_TRY(launch_check("gram finish"));
    } else {
      with_amps(s, [&](auto* a) {
        using T = std::remove_cv_t<std::remove_pointer_t<decltype(a)>>;
        k_gram<<<nblocks, 256, 0, s->stream>>>((const T*)a, pairs, q, part);
        return QS_OK;
      });
      QS_TRY(launch_check("gram"));
      k_gram_finish<<<1, 32, 0, s->stream>>>(part, nblocks, dres);
      QS_TRY(launch_check("gram finish"));
    }
    QS_TRY(ensure_pinned(s, 4 * sizeof(double)));
    QS_CUDA(cudaMemcpyAsync(s->pinned, dres, 4 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    QS_CUDA(cudaStreamSynchronize(s->stream));
    memcpy(G, s->pinned, 4 * sizeof(double));
    return QS_OK;
  }

  int channel(const KrausSet& ks, int q) {
    double w[4] = {0, 0, 0, 0};
    if (ks.unital) {
      for (int j = 0; j < ks.m; ++j) w[j] = ks.w[j];
    } else {
      QS_TRY(flush());
      double G[4];
      QS_TRY(gram(q, G));
      // w_j = tr(K^dag K G), G = [[g00, g01], [conj(g01), g11]]
      for (int j = 0; j < ks.m; ++j) {
        const Mat2& K = ks.K[j];
        const double a00 = K.m[0].re * K.m[0].re + K.m[0].im * K.m[0].im + K.m[2].re * K.m[2].re + K.m[2].im * K.m[2].im;
        const double a11 = K.m[1].re * K.m[1].re + K.m[1].im * K.m[1].im + K.m[3].re * K.m[3].re + K.m[3].im * K.m[3].im;
        // (K^dag K)_{01} = conj(K00) K01 + conj(K10) K11
        const double br = K.m[0].re * K.m[1].re + K.m[0].im * K.m[1].im + K.m[2].re * K.m[3].re + K.m[2].im * K.m[3].im;
        const double bi = K.m[0].re * K.m[1].im - K.m[0].im * K.m[1].re + K.m[2].re * K.m[3].im - K.m[2].im * K.m[3].re;
        // tr(B G) = B00 g00 + B11 g11 + 2 Re(B01 conj(g01))
        w[j] = a00 * G[0] + a11 * G[1] + 2.0 * (br * G[2] + bi * G[3]);
      }
    }
    double W = 0.0;
    for (int j = 0; j < ks.m; ++j) W += w[j];
    const double u = draw();
    int pick = ks.m - 1;
    double c = 0.0;
    for (int j = 0; j < ks.m; ++j) {
      c += w[j];
      if (u * W < c) {
        pick = j;
        break;
      }
    }
    if (!(w[pick] > 0.0)) return fail(QS_ERR_INVALID_ARG, "noise channel picked an operator of zero weight");
    if (ks.unital) {
      static const int codes[4] = {QS_I, QS_X, QS_Y, QS_Z};
      if (ks.pauli[pick] != 0) {
        qs_gate g{};
        g.type = codes[ks.pauli[pick]];
        g.q0 = q;
        g.q1 = -1;
        g.param_idx = -1;
        pending.push_back(g);
      }
      return QS_OK;
    }
    Mat2 M = ks.K[pick];
    const double sc = 1.0 / sqrt(w[pick]);
    for (int e = 0; e < 4; ++e) M.m[e] = {M.m[e].re * sc, M.m[e].im * sc};
    // A renormalised Kraus operator is not unitary, but the state it produces is
    // normalised: the Q60 kernel applies it when every entry has |re| + |im| < 1.9
    // (its Gauss-form sums then stay below 2, the limb range), e.g. the usual
    // no-decay operator of amplitude damping; otherwise (the rare jump operators,
    // scaled by 1 / sqrt(p)) the FP64 kernel.
    bool fixed = false;
    QS_TRY(choose_fixed(s, &fixed));
    for (int e = 0; e < 4 && fixed; ++e)
      if (fabs(M.m[e].re) + fabs(M.m[e].im) >= 1.9) fixed = false;
    return launch_op1(s, classify(q, 0, M), fixed);
  }
};

}  // namespace qs

using namespace qs;

extern "C" int qs_run_noisy(qs_state* s, const qs_gate* gates, size_t ng, const double* params,
                            const qs_noise_rule* rules, size_t nrules, double rotation_error, uint64_t seed, int fuse,
                            uint64_t* ndraws) {
  clear_error();
  QS_TRY(check_state(s));
  QS_TRY(validate_gates(gates, ng, s->n, params));
  if (nrules && !rules) return fail(QS_ERR_INVALID_ARG, "rules is NULL");
  if (!(rotation_error >= 0.0)) return fail(QS_ERR_INVALID_ARG, "rotation_error must be >= 0");
  std::vector<KrausSet> sets(nrules);
  for (size_t r = 0; r < nrules; ++r) {
    QS_TRY(kraus_set(rules[r], &sets[r]));
    if (rules[r].gate_type < -1 || rules[r].gate_type > QS_CR)
      return fail(QS_ERR_INVALID_ARG, "rule %zu: gate type %d", r, rules[r].gate_type);
  }
  Trajectory tr;
  tr.s = s;
  tr.fuse = fuse != 0;
  tr.seed = seed;
  int rc = QS_OK;
  for (size_t k = 0; k < ng && rc == QS_OK; ++k) {
    qs_gate g = gates[k];
    if (g.param_idx >= 0) {  // resolve the angle into the record
      g.p[0] = params[g.param_idx];
      g.param_idx = -1;
    }
    if (rotation_error > 0.0 && is_rotation(g.type)) g.p[0] += rotation_error * (2.0 * tr.draw() - 1.0);
    tr.pending.push_back(g);
    int t;
    uint64_t cm;
    if ((rc = gate_qubits(g, s->n, &t, &cm)) != QS_OK) break;
    const int first = g.q0, second = two_qubit(g.type) ? g.q1 : -1;
    const uint64_t touched = cm | (1ull << t);
    for (size_t r = 0; r < nrules && rc == QS_OK; ++r) {
      const qs_noise_rule& R = rules[r];
      if (R.gate_type >= 0 && R.gate_type != g.type) continue;
      if (R.q0 >= 0 && R.q0 != first) continue;
      if (R.q1 >= 0 && R.q1 != second) continue;
      for (uint64_t b = touched; b && rc == QS_OK; b &= b - 1) rc = tr.channel(sets[r], __builtin_ctzll(b));
    }
  }
  if (rc == QS_OK) rc = tr.flush();
  if (ndraws) *ndraws = tr.k;
  if (rc == QS_OK) QS_CUDA(cudaStreamSynchronize(s->stream));
  return rc;
}

extern "C" int qs_readout_error(uint64_t* samples, size_t shots, int n, double f0, double f1, uint64_t seed,
                                int on_device, void* stream) {
  clear_error();
  if (shots && !samples) return fail(QS_ERR_INVALID_ARG, "samples is NULL");
  if (n < 1 || n > 64) return fail(QS_ERR_INVALID_ARG, "n=%d outside 1..64", n);
  if (!(f0 >= 0.0 && f0 <= 1.0 && f1 >= 0.0 && f1 <= 1.0)) return fail(QS_ERR_INVALID_ARG, "fidelities outside [0, 1]");
  if (!shots) return QS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  uint64_t* d = samples;
  if (!on_device) QS_CUDA(dmalloc_async(&d, shots * sizeof(uint64_t), st));
  int rc = QS_OK;
  cudaError_t e = cudaSuccess;
  if (!on_device) e = cudaMemcpyAsync(d, samples, shots * sizeof(uint64_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const uint64_t grid = std::min<uint64_t>((shots + 255) / 256, (uint64_t)std::max(1, sms) * 8);
    note_launch(1);
    k_readout<<<(unsigned)grid, 256, 0, st>>>(d, shots, n, f0, f1, seed);
    rc = launch_check("readout kernel");
    if (rc == QS_OK && !on_device) e = cudaMemcpyAsync(samples, d, shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && rc == QS_OK) e = cudaStreamSynchronize(st);
  }
  if (!on_device) cudaFreeAsync(d, st);
  if (rc != QS_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "readout error");
  return QS_OK;
}
