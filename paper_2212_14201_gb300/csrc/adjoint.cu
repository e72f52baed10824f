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
    QAcc re{0, 0}, im{0, 0};
    qacc_add(re, u.re, ar);
    qacc_add(re, u.nim, ai);
    qacc_add(im, u.re, ai);
    qacc_add(im, u.im, ar);
    return make_double2(q60_to_double(qacc_result(re)), q60_to_double(qacc_result(im)));
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
      QAcc re{0, 0}, im{0, 0};
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
      out[2 * row] = qacc_result(re);
      out[2 * row + 1] = qacc_result(im);
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
  int imag[HMAX];   // ... placed in the imaginary part when ny is odd
};

__global__ void __launch_bounds__(256) k_apply_h(const double2* __restrict__ psi, double2* __restrict__ lam,
                                                 const __grid_constant__ HArgs h) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t y = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; y < h.N; y += stride) {
    double2 out = h.accumulate ? lam[y] : make_double2(0.0, 0.0);
    for (int gi = 0; gi < h.ngroups; ++gi) {
      const uint64_t x = y ^ h.gxm[gi];
      double dre = 0.0, dim = 0.0;
      for (int k = h.gstart[gi]; k < h.gstart[gi + 1]; ++k) {
        double v = (__popcll(x & h.zm[k]) & 1) ? -h.c[k] : h.c[k];
        if (h.imag[k]) dim += v;
        else dre += v;
      }
      const double2 p = psi[x];
      out.x += dre * p.x - dim * p.y;
      out.y += dre * p.y + dim * p.x;
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
  QS_CUDA(cudaMallocAsync((void**)&lam, bytes, s->stream));
  const int nblocks = 608;
  double* part = nullptr;
  double* sums = nullptr;
  int rc = QS_OK;
  auto cleanup = [&]() {
    if (lam) cudaFreeAsync(lam, s->stream);
    if (part) cudaFreeAsync(part, s->stream);
    if (sums) cudaFreeAsync(sums, s->stream);
  };
  cudaError_t e = cudaMallocAsync((void**)&part, sizeof(double) * nblocks * (nslots + 1), s->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&sums, sizeof(double) * (nslots + 1), s->stream);
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
  for (size_t kk = ng; rc == QS_OK && kk-- > 0;) {
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
