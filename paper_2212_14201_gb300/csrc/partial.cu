// Partial amplitudes (the paper's PartialAmpQVM, Section "Multi-simulation
// methods", noise-free simulation method): selected amplitudes of an n-qubit
// circuit without the 2^n state.  The qubits split into a low block (0 ..
// n_low-1) and a high block; a gate with qubits in both blocks is cut.  With
// target t, controls C_t in t's block and C_o in the other block,
//   controlled-U = P(C_o all 1) (x) [U on t, controls C_t]
//                + (I - P(C_o all 1)) (x) I,
// so k cuts give 2^k paths, each a product of two block circuits (bit i of the
// path = 1 takes the first term of cut i), and
//   <x|psi> = sum over paths of <x_low|lo_path> <x_high|hi_path>.
// Each path runs both blocks on library states (per-gate kernels, or a greedy
// plan per uncut stretch), the projectors as one masking pass, and adds its
// products into the requested amplitudes in a fixed path order (deterministic).
// Paths are enumerated so that consecutive ones share their early cuts, and each
// block resumes from a snapshot taken before its first changed cut.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace qs {

// zero the amplitudes whose bits under `mask` are all 1 (keep = 0) or not all 1 (keep = 1)
__global__ void k_project(double2* __restrict__ a, uint64_t N, uint64_t mask, int keep_all_ones) {
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x)
    if ((((x & mask) == mask) ? 1 : 0) != keep_all_ones) a[x] = make_double2(0.0, 0.0);
}

// out[i] += lo[x_i & lowmask] * hi[x_i >> n_low]
__global__ void k_pa_accum(double2* __restrict__ out, const uint64_t* __restrict__ idx, uint64_t count,
                           const double2* __restrict__ lo, const double2* __restrict__ hi, int n_low) {
  const uint64_t lowmask = (1ull << n_low) - 1;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t x = idx[i];
    const double2 u = lo[x & lowmask], v = hi[x >> n_low];
    double2 o = out[i];
    o.x = fma(u.x, v.x, fma(-u.y, v.y, o.x));
    o.y = fma(u.x, v.y, fma(u.y, v.x, o.y));
    out[i] = o;
  }
}

struct PaItem {
  int kind = 0;                  // 0: gate stretch, 1: cut gate (applied on path bit 1), 2: projector
  std::vector<qs_gate> gates;    // kind 0
  qs_gate gate{};                // kind 1
  uint64_t mask = 0;             // kind 2
  int cut = 0;                   // kinds 1 and 2: index of the cut
  qs_plan* plan = nullptr;
};

// The record of a gate restricted to one block: qubits re-indexed by -base, the
// controls outside the block dropped; a cut two-qubit gate becomes its one-qubit
// target gate (CNOT -> X, CZ -> Z, CR -> P) controlled by the block's controls.
static qs_gate block_record(const qs_gate& g, int t, uint64_t cm_block, int base, bool cut) {
  qs_gate r = g;
  if (cut && (g.type == QS_CNOT || g.type == QS_CZ || g.type == QS_CR)) {
    r.type = g.type == QS_CNOT ? QS_X : g.type == QS_CZ ? QS_Z : QS_P;
    r.q0 = t - base;
    r.q1 = -1;
    r.ctrl_mask = cm_block >> base;
    return r;
  }
  if (g.type == QS_CNOT || g.type == QS_CZ || g.type == QS_CR) {
    r.q0 = g.q0 - base;
    r.q1 = g.q1 - base;
    // the record's own control is q0; the extra mask excludes it
    r.ctrl_mask = (g.ctrl_mask >> base);
    return r;
  }
  r.q0 = g.q0 - base;
  r.ctrl_mask = cm_block >> base;
  return r;
}

// One block's circuit: gate stretches and cut items in circuit order.  The block
// keeps the state before each of its cut items; a path that differs from the
// previous one first at cut c resumes from the snapshot before the block's first
// item of cut >= c (and a block with no such item keeps its final state).
struct PaBlock {
  int nq = 0;
  qs_state* s = nullptr;
  std::vector<PaItem> items;
  std::vector<double2*> snap;  // per item: the state before it (cut items only)
  bool started = false;

  void add_gate(const qs_gate& g) {
    if (items.empty() || items.back().kind != 0) items.emplace_back();
    items.back().gates.push_back(g);
  }

  // path bit of cut c: bits[c]
  int run(const std::vector<int>& bits, int first_cut, const double* params, bool fuse) {
    size_t start = 0;
    if (started) {
      size_t j = 0;
      while (j < items.size() && !(items[j].kind != 0 && items[j].cut >= first_cut)) ++j;
      if (j == items.size()) return QS_OK;  // nothing of this block changed
      QS_CUDA(cudaMemcpyAsync(s->amps, snap[j], sizeof(double2) << nq, cudaMemcpyDeviceToDevice, s->stream));
      start = j;
    } else {
      QS_TRY(qs_set_zero(s));
      snap.assign(items.size(), nullptr);
      started = true;
    }
    const size_t bytes = sizeof(double2) << nq;
    for (size_t j = start; j < items.size(); ++j) {
      PaItem& it = items[j];
      if (it.kind != 0) {
        if (!snap[j]) QS_CUDA(dmalloc_async(&snap[j], bytes, s->stream));
        QS_CUDA(cudaMemcpyAsync(snap[j], s->amps, bytes, cudaMemcpyDeviceToDevice, s->stream));
      }
      if (it.kind == 0) {
        if (fuse && it.gates.size() > 1) {
          if (!it.plan) QS_TRY(qs_plan_create(nq, it.gates.data(), it.gates.size(), QS_PLAN_GREEDY, 5, &it.plan));
          QS_TRY(qs_apply(s, it.gates.data(), it.gates.size(), params, it.plan));
        } else {
          QS_TRY(qs_apply(s, it.gates.data(), it.gates.size(), params, nullptr));
        }
      } else if (it.kind == 1) {
        if (bits[it.cut]) QS_TRY(qs_apply(s, &it.gate, 1, params, nullptr));
      } else {
        const uint64_t N = 1ull << nq;
        const int grid = (int)std::min<uint64_t>((N + 255) / 256, 152 * 16);
        KTimer kt(s, QS_K_OTHER, 0, 1, it.mask, 0, (double)N, 0.0);
        k_project<<<grid, 256, 0, s->stream>>>(s->amps, N, it.mask, bits[it.cut]);
        QS_TRY(launch_check("projector kernel"));
      }
    }
    return QS_OK;
  }

  ~PaBlock() {
    for (PaItem& it : items)
      if (it.plan) qs_plan_free(it.plan);
    if (s) {
      for (double2* p : snap)
        if (p) cudaFreeAsync(p, s->stream);
      qs_free(s);
    }
  }
};

}  // namespace qs

using namespace qs;

extern "C" int qs_partial_amplitudes(int n, const qs_gate* gates, size_t ng, const double* params, int n_low,
                                     const uint64_t* indices, size_t count, double* out, int fuse, void* stream,
                                     uint64_t* npaths) {
  clear_error();
  if (n < 2 || n > 64) return fail(QS_ERR_INVALID_ARG, "n=%d outside 2..64", n);
  if (n_low < 1 || n_low >= n) return fail(QS_ERR_INVALID_ARG, "n_low=%d outside 1..n-1", n_low);
  if (n_low > QS_MAX_QUBITS || n - n_low > QS_MAX_QUBITS)
    return fail(QS_ERR_UNSUPPORTED, "a block of more than %d qubits", QS_MAX_QUBITS);
  if ((count && (!indices || !out)) || (ng && !gates)) return fail(QS_ERR_INVALID_ARG, "NULL argument");
  QS_TRY(validate_gates(gates, ng, n, params));
  for (size_t i = 0; i < count; ++i)
    if (n < 64 && (indices[i] >> n)) return fail(QS_ERR_INVALID_ARG, "index %zu outside 2^n", i);
  const uint64_t lowmask = (1ull << n_low) - 1;
  PaBlock lo, hi;
  lo.nq = n_low;
  hi.nq = n - n_low;
  int k = 0;
  for (size_t i = 0; i < ng; ++i) {
    int t;
    uint64_t cm;
    QS_TRY(gate_qubits(gates[i], n, &t, &cm));
    const uint64_t all = cm | (1ull << t);
    const bool in_lo = (all & ~lowmask) == 0, in_hi = (all & lowmask) == 0;
    if (in_lo) {
      lo.add_gate(block_record(gates[i], t, cm, 0, false));
      continue;
    }
    if (in_hi) {
      hi.add_gate(block_record(gates[i], t, cm, n_low, false));
      continue;
    }
    // a cut: the target's block applies the gate on path bit 1, the other block projects
    const bool t_lo = t < n_low;
    PaBlock& tb = t_lo ? lo : hi;
    PaBlock& ob = t_lo ? hi : lo;
    PaItem g1;
    g1.kind = 1;
    g1.cut = k;
    g1.gate = block_record(gates[i], t, t_lo ? (cm & lowmask) : (cm & ~lowmask), t_lo ? 0 : n_low, true);
    tb.items.push_back(g1);
    PaItem pr;
    pr.kind = 2;
    pr.cut = k;
    pr.mask = t_lo ? (cm >> n_low) : (cm & lowmask);
    ob.items.push_back(pr);
    ++k;
  }
  if (k > 30) return fail(QS_ERR_UNSUPPORTED, "%d cut gates (at most 30)", k);
  if (npaths) *npaths = 1ull << k;
  if (!count) return QS_OK;
  QS_TRY(qs_alloc(lo.nq, stream, &lo.s));
  QS_TRY(qs_alloc(hi.nq, stream, &hi.s));
  cudaStream_t st = (cudaStream_t)stream;
  uint64_t* didx = nullptr;
  double2* dout = nullptr;
  const size_t cnt = std::max<size_t>(count, 1);
  QS_CUDA(dmalloc_async(&didx, cnt * sizeof(uint64_t), st));
  cudaError_t e = dmalloc_async(&dout, cnt * sizeof(double2), st);
  int rc = e == cudaSuccess ? QS_OK : cuda_fail(e, "cudaMallocAsync(out)");
  if (rc == QS_OK && count) {
    e = cudaMemcpyAsync(didx, indices, count * sizeof(uint64_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dout, 0, count * sizeof(double2), st);
    if (e != cudaSuccess) rc = cuda_fail(e, "partial amplitudes set-up");
  }
  // paths in the order of a counter whose lowest bit is the last cut, so that
  // consecutive paths share every block state up to the first changed cut
  const int grid = (int)std::min<uint64_t>((count + 255) / 256, 152 * 8);
  std::vector<int> bits(std::max(k, 1), 0);
  for (uint64_t c = 0; rc == QS_OK && c < (1ull << k); ++c) {
    int first = 0;
    if (c) first = k - 1 - (63 - __builtin_clzll(c ^ (c - 1)));
    for (int i = 0; i < k; ++i) bits[i] = (int)((c >> (k - 1 - i)) & 1);
    rc = lo.run(bits, first, params, fuse != 0);
    if (rc == QS_OK) rc = hi.run(bits, first, params, fuse != 0);
    if (rc == QS_OK) {
      note_launch(1);
      k_pa_accum<<<std::max(1, grid), 256, 0, st>>>(dout, didx, count, lo.s->amps, hi.s->amps, n_low);
      rc = launch_check("partial amplitude accumulation");
    }
  }
  if (rc == QS_OK && count) {
    e = cudaMemcpyAsync(out, dout, count * sizeof(double2), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "partial amplitudes read-back");
  }
  cudaFreeAsync(didx, st);
  if (dout) cudaFreeAsync(dout, st);
  cudaStreamSynchronize(st);
  return rc;
}
