// Batched variational evaluation: energy and adjoint gradient of many parameter
// sets of possibly different qubit counts in ONE persistent launch (the
// hybrid quantum-classical loop of the paper, Sections "Support hybrid
// quantum-classical algorithm" and "Variational quantum circuit"; the batching
// itself is this library's design, not the paper's).
//
// The kernel runs in clusters of c CTAs (c = 1, 2, 4 or 8, chosen per batch).
// Each cluster repeatedly takes the next work item from a device counter (items
// pre-sorted by decreasing cost): one large set (at least c tiles of 2^11
// amplitudes per pass), whose tiles the c CTAs share with hardware cluster
// barriers between passes, or up to c small sets, one per CTA.  No CTA waits on
// a CTA outside its own cluster.  Per set:
//   1. gate matrices of the set from its parameters (forward and adjoint);
//   2. forward sweep psi = U_G ... U_1 |0> as greedy tile passes (<= 11 tile
//      qubits, Q60 arithmetic in shared memory);
//   3. lambda = (H / S) psi and E = S Re<psi|lambda> (FP64 gather);
//   4. backward sweep over the passes in reverse: for every op in reverse, the
//      generator inner product Im<lambda|G|psi> over the tile (Q60 products,
//      FP64 accumulation, fixed reduction order), then U^dag on both tiles.
// The host side of a run (parameters in, energies and gradients out) is
// captured once in a CUDA graph and replayed.
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include <cooperative_groups.h>

#include "q60tile.cuh"

namespace cg = cooperative_groups;

namespace qs {

constexpr int BT_CLUSTER = 8;  // largest cluster (portable size); the launch uses 1, 2, 4 or 8
static_assert(BT_CLUSTER <= BT_THREADS / 32, "cluster rows must fit the warp-row accumulator");
static_assert(BT_MAX_OPS <= BT_THREADS, "one thread per gradient slot");

struct BItem {
  int cluster;               // 1: sets[0] on the whole cluster; 0: sets[r] on CTA r
  int nsets;
  int sets[BT_CLUSTER];
};


struct BSet {
  int n, pass_begin, npasses, gate_begin, ngates, group_begin, ngroups, param_begin, nparams;
  int dg_begin, ndg;  // diagonal groups (BK_DGROUP heads) of the set's passes
  long long amp_off;
  double S;
};

struct BGate {
  int type, param, dagger;
  double p[3];
};

struct BGroup {
  uint64_t xm;
  int tbegin, tend;
};

struct BTerm {
  double c;       // coef / S, with the real sign of i^ny
  int64_t cq;     // the same in Q60 (|c| <= 1)
  uint64_t zm;
  int imag;       // i^ny is imaginary
};

struct BatchArgs {
  const BSet* sets;
  const BItem* items;
  int nitems;
  int csize;   // CTAs per cluster
  const BPass* passes;
  const BOp* ops;
  const BGate* gates;
  const BGroup* groups;
  const BTerm* terms;
  const double* params;
  double* grads;
  double* energies;
  double2* psi;
  double2* lam;
  QC* matf;   // 4 per gate (Gauss form)
  QC* matb;   // 4 per gate (Gauss form)
  const int* dghead;  // per diagonal group: global index of its head op
  QC* dgf;    // 16 per diagonal group (Gauss form), forward
  QC* dgb;    // 16 per diagonal group, adjoint
  int* counter;
};

// ---- device helpers ------------------------------------------------------------------

__device__ void bt_gate_matrix(const BGate& g, const double* params, bool flip, double2 m[4]) {
  double th = g.param >= 0 ? params[g.param] : g.p[0];
  double s, c;
  sincos(0.5 * th, &s, &c);
  const double r = 0.70710678118654752440;
  const double2 z = make_double2(0, 0), one = make_double2(1, 0);
  switch (g.type) {
    case QS_H: m[0] = make_double2(r, 0); m[1] = make_double2(r, 0); m[2] = make_double2(r, 0); m[3] = make_double2(-r, 0); break;
    case QS_X: case QS_CNOT: m[0] = z; m[1] = one; m[2] = one; m[3] = z; break;
    case QS_Y: m[0] = z; m[1] = make_double2(0, -1); m[2] = make_double2(0, 1); m[3] = z; break;
    case QS_Z: case QS_CZ: m[0] = one; m[1] = z; m[2] = z; m[3] = make_double2(-1, 0); break;
    case QS_S: m[0] = one; m[1] = z; m[2] = z; m[3] = make_double2(0, 1); break;
    case QS_T: m[0] = one; m[1] = z; m[2] = z; m[3] = make_double2(r, r); break;
    case QS_RX: m[0] = make_double2(c, 0); m[1] = make_double2(0, -s); m[2] = make_double2(0, -s); m[3] = make_double2(c, 0); break;
    case QS_RY: m[0] = make_double2(c, 0); m[1] = make_double2(-s, 0); m[2] = make_double2(s, 0); m[3] = make_double2(c, 0); break;
    case QS_RZ: m[0] = make_double2(c, -s); m[1] = z; m[2] = z; m[3] = make_double2(c, s); break;
    case QS_U3: {
      double sl, cl, sp, cp, spl, cpl;
      sincos(g.p[2], &sl, &cl);
      sincos(g.p[1], &sp, &cp);
      sincos(g.p[1] + g.p[2], &spl, &cpl);
      m[0] = make_double2(c, 0);
      m[1] = make_double2(-cl * s, -sl * s);
      m[2] = make_double2(cp * s, sp * s);
      m[3] = make_double2(cpl * c, spl * c);
      break;
    }
    case QS_P: case QS_CR: {
      double st, ct;
      sincos(th, &st, &ct);
      m[0] = one; m[1] = z; m[2] = z; m[3] = make_double2(ct, st);
      break;
    }
    default: m[0] = one; m[1] = z; m[2] = z; m[3] = one; break;
  }
  if ((g.dagger != 0) != flip) {
    double2 a = m[0], b = m[1], cc = m[2], d = m[3];
    m[0] = make_double2(a.x, -a.y);
    m[1] = make_double2(cc.x, -cc.y);
    m[2] = make_double2(b.x, -b.y);
    m[3] = make_double2(d.x, -d.y);
  }
}


// Cluster barrier that also publishes this CTA's global writes (psi, lambda,
// gradients) to the other CTAs of the cluster.  A hardware barrier: every CTA of
// the cluster is resident for the whole launch, and every CTA reaches the same
// sequence of these barriers (work items are taken per cluster, not per CTA).
__device__ __forceinline__ void bt_cluster_sync() {
  __threadfence();
  cg::this_cluster().sync();
}

// One pass over the tiles r = rank, rank + nr, ... of the set's state (nr CTAs
// of a cluster share the set; nr = 1: this CTA alone).  Forward: U on psi.
// Backward: for every op in reverse, the generator term then U^dag on psi and
// lambda; gradient contributions are added in backward op order, per slot the
// warps of a CTA in warp order, then the CTAs in rank order.
__device__ void bt_run_pass(const BatchArgs& d, const BPass& ps, double2* psi, double2* lam, const QC* matf,
                            const QC* matb, bool backward, longlong2* tP, longlong2* tL, uint64_t* offs, double* acc,
                            int rank, int nr) {
  const int m = ps.m;
  const int L = m - ps.nhigh;
  const uint32_t TS = 1u << m;
  const uint32_t H = 1u << ps.nhigh;
  const uint32_t lowmask = (1u << L) - 1;
  const uint64_t ntiles = 1ull << ps.nout;
  for (uint32_t h = threadIdx.x; h < H; h += BT_THREADS) {
    uint64_t o = 0;
    for (int b = 0; b < ps.nhigh; ++b) o |= (uint64_t)((h >> b) & 1u) << ps.qhigh[b];
    offs[h] = o;
  }
  for (int s = threadIdx.x; s < ps.nslots * (BT_THREADS / 32); s += BT_THREADS) acc[s] = 0.0;
  for (uint64_t r = rank; r < ntiles; r += nr) {
    uint64_t base = 0;
    for (int b = 0; b < ps.nout; ++b) base |= ((r >> b) & 1ull) << ps.outpos[b];
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < TS; j += BT_THREADS) {
      const uint64_t x = base + offs[j >> L] + (j & lowmask);
      const double2 a = psi[x];
      tP[j] = make_longlong2(q60_from_double(a.x), q60_from_double(a.y));
      if (backward) {
        const double2 b = lam[x];
        tL[j] = make_longlong2(q60_from_double(b.x), q60_from_double(b.y));
      }
    }
    __syncthreads();
    if (!backward) {
      for (int k = ps.op_begin; k < ps.op_end; ++k) {
        const BOp op = d.ops[k];
        if (op.kf == BK_MEMBER || (base & op.ext) != op.ext) continue;
        if (op.kf == BK_DGROUP) bt_apply_dgroup(tP, TS, d.ops + k + 1, op.nmem, d.dgf + 16 * op.gate);
        else bt_apply(tP, TS, op, op.kf, op.c0f, op.c1f, matf + 4 * op.gate, base);
        __syncthreads();
      }
    } else {
      for (int k = ps.op_end - 1; k >= ps.op_begin; --k) {
        const BOp op = d.ops[k];
        if (op.kb == BK_MEMBER || (base & op.ext) != op.ext) continue;
        // each thread reads and then rewrites only its own pairs (amplitudes) of this op
        if (op.kb == BK_DGROUP) {
          int64_t part[BT_DG_MAX];
          const BOp* mem = d.ops + k + 1;
          bt_back_dgroup(tP, tL, TS, mem, op.nmem, d.dgb + 16 * op.gate, part);
          for (int mm = 0; mm < op.nmem; ++mm)
            if (mem[mm].slot >= 0) bt_warp_accumulate(part[mm], acc, ps.nslots, mem[mm].slot);
          __syncthreads();
          continue;
        }
        if (op.slot < 0 && op.kb == OP_ANTI && op.c0b != U_GENERAL && op.c1b != U_GENERAL) {
          bt_anti_both(tP, tL, TS, op, op.c0b, op.c1b);  // psi and lambda in one sweep
          __syncthreads();
          continue;
        }
        if (op.slot >= 0 && op.kb == OP_REAL) {  // one pass over the pairs
          bt_warp_accumulate(bt_back_real(tP, tL, TS, op, matb + 4 * op.gate), acc, ps.nslots, op.slot);
          __syncthreads();
          continue;
        }
        if (op.slot >= 0) bt_warp_accumulate(bt_gen_partial(tP, tL, TS, op, base), acc, ps.nslots, op.slot);
        bt_apply(tP, TS, op, op.kb, op.c0b, op.c1b, matb + 4 * op.gate, base);
        bt_apply(tL, TS, op, op.kb, op.c0b, op.c1b, matb + 4 * op.gate, base);
        __syncthreads();
      }
    }
    for (uint32_t j = threadIdx.x; j < TS; j += BT_THREADS) {
      const uint64_t x = base + offs[j >> L] + (j & lowmask);
      psi[x] = make_double2(q60_to_double(tP[j].x), q60_to_double(tP[j].y));
      if (backward) lam[x] = make_double2(q60_to_double(tL[j].x), q60_to_double(tL[j].y));
    }
  }
  __syncthreads();
  if (nr == 1) {
    if (backward && threadIdx.x == 0) {
      for (int k = ps.op_end - 1; k >= ps.op_begin; --k) {
        const BOp& op = d.ops[k];
        if (op.slot >= 0) d.grads[op.param] += bt_warp_total(acc, ps.nslots, op.slot) * op.gsign;
      }
    }
    __syncthreads();
    return;
  }
  if (!backward) {
    bt_cluster_sync();  // the next pass reads tiles other CTAs wrote
    return;
  }
  // per-CTA slot totals -> rows [rank][slot] of rank 0's accumulator (distributed
  // shared memory), then rank 0 adds them in rank order
  const double v = threadIdx.x < ps.nslots ? bt_warp_total(acc, ps.nslots, threadIdx.x) : 0.0;
  bt_cluster_sync();
  if (threadIdx.x < ps.nslots) cg::this_cluster().map_shared_rank(acc, 0)[rank * ps.nslots + threadIdx.x] = v;
  bt_cluster_sync();
  if (rank == 0 && threadIdx.x == 0) {
    for (int k = ps.op_end - 1; k >= ps.op_begin; --k) {
      const BOp& op = d.ops[k];
      if (op.slot < 0) continue;
      double t = 0.0;
      for (int q = 0; q < nr; ++q) t += acc[q * ps.nslots + op.slot];
      d.grads[op.param] += t * op.gsign;
    }
  }
  __syncthreads();
}

// Energy and gradient of one set, by CTA `rank` of `nr` cooperating CTAs.
__device__ void bt_eval_set(const BatchArgs& d, int set_id, int rank, int nr, longlong2* tP, longlong2* tL,
                            uint64_t* offs, double* acc, double* red, double* epart) {
  const BSet st = d.sets[set_id];
  const uint64_t N = 1ull << st.n;
  double2* psi = d.psi + st.amp_off;
  double2* lam = d.lam + st.amp_off;
  QC* matf = d.matf + 4 * (size_t)st.gate_begin;
  QC* matb = d.matb + 4 * (size_t)st.gate_begin;
  const int t0 = rank * BT_THREADS + threadIdx.x, ts = nr * BT_THREADS;
  // 1. matrices (indices of ops are global gate indices; shift back by gate_begin)
  for (int g = t0; g < st.ngates; g += ts) {
    double2 m[4];
    const BGate gt = d.gates[st.gate_begin + g];
    bt_gate_matrix(gt, d.params, false, m);
    for (int e = 0; e < 4; ++e) matf[4 * g + e] = qc_make_gauss(m[e].x, m[e].y);
    bt_gate_matrix(gt, d.params, true, m);
    for (int e = 0; e < 4; ++e) matb[4 * g + e] = qc_make_gauss(m[e].x, m[e].y);
  }
  // diagonal groups: E = product of the members' diagonals (forward and adjoint)
  for (int gi = t0; gi < st.ndg; gi += ts) {
    const int head = d.dghead[st.dg_begin + gi];
    const int nm = d.ops[head].nmem;
    double2 df[BT_DG_MAX][2], db[BT_DG_MAX][2];
    for (int mm = 0; mm < nm; ++mm) {
      const BGate gt = d.gates[st.gate_begin + d.ops[head + 1 + mm].gate];
      double2 mt[4];
      bt_gate_matrix(gt, d.params, false, mt);
      df[mm][0] = mt[0];
      df[mm][1] = mt[3];
      bt_gate_matrix(gt, d.params, true, mt);
      db[mm][0] = mt[0];
      db[mm][1] = mt[3];
    }
    QC* ef = d.dgf + 16 * (size_t)(st.dg_begin + gi);
    QC* eb = d.dgb + 16 * (size_t)(st.dg_begin + gi);
    for (int idx = 0; idx < (1 << nm); ++idx) {
      double2 f = make_double2(1.0, 0.0), b = make_double2(1.0, 0.0);
      for (int mm = 0; mm < nm; ++mm) {
        const double2 u = df[mm][(idx >> mm) & 1], v = db[mm][(idx >> mm) & 1];
        f = make_double2(f.x * u.x - f.y * u.y, f.x * u.y + f.y * u.x);
        b = make_double2(b.x * v.x - b.y * v.y, b.x * v.y + b.y * v.x);
      }
      ef[idx] = qc_make_gauss(f.x, f.y);
      eb[idx] = qc_make_gauss(b.x, b.y);
    }
  }
  for (int j = t0; j < st.nparams; j += ts) d.grads[st.param_begin + j] = 0.0;
  // 2. psi = |0>, forward passes
  for (uint64_t x = t0; x < N; x += ts) psi[x] = make_double2(x == 0 ? 1.0 : 0.0, 0.0);
  if (nr == 1) __syncthreads();
  else bt_cluster_sync();
  for (int p = st.pass_begin; p < st.pass_begin + st.npasses; ++p)
    bt_run_pass(d, d.passes[p], psi, lam, matf, matb, false, tP, tL, offs, acc, rank, nr);
  // 3. lambda = (H/S) psi, energy, in Q60 integers (GB300's FP64 pipe would bound
  // this loop): per group of terms sharing an X mask the signed coefficient sums
  // d = sum_t (-1)^popc(x & zm_t) c_t are exact in int64 (sum |c_t| <= 1), the
  // group's product d * psi_x is rounded once, and lambda_y = sum over groups
  // (|lambda_y| <= |psi|_inf <= 1.25: every partial fits).
  double e = 0.0;
  for (uint64_t y = t0; y < N; y += ts) {
    int64_t ore = 0, oim = 0;
    for (int gi = st.group_begin; gi < st.group_begin + st.ngroups; ++gi) {
      const BGroup grp = d.groups[gi];
      const uint64_t x = y ^ grp.xm;
      int64_t dre = 0, dim = 0;
      for (int k = grp.tbegin; k < grp.tend; ++k) {
        const BTerm& t = d.terms[k];
        const int64_t v = (__popcll(x & t.zm) & 1) ? -t.cq : t.cq;
        if (t.imag) dim += v;
        else dre += v;
      }
      const double2 pv = psi[x];
      const QL px = q60_split(q60_from_double(pv.x)), py = q60_split(q60_from_double(pv.y));
      const QL qr = q60_split(dre), qi = q60_split(dim), nqi = q60_split(-dim);
      QAcc r = qacc_new(), i = qacc_new();
      qacc_add(r, qr, px);   // re: dre px - dim py
      qacc_add(r, nqi, py);
      qacc_add(i, qr, py);   // im: dre py + dim px
      qacc_add(i, qi, px);
      ore += qacc_round(r);
      oim += qacc_round(i);
    }
    const double lr = q60_to_double(ore), li = q60_to_double(oim);
    lam[y] = make_double2(lr, li);
    const double2 pyv = psi[y];
    e += pyv.x * lr + pyv.y * li;
  }
  const double E = bt_block_sum(e, red);
  if (nr == 1) {
    if (threadIdx.x == 0) d.energies[set_id] = E * st.S;
    __syncthreads();
  } else {
    if (threadIdx.x == 0) cg::this_cluster().map_shared_rank(epart, 0)[rank] = E;
    bt_cluster_sync();  // also publishes lambda
    if (rank == 0 && threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < nr; ++q) t += epart[q];
      d.energies[set_id] = t * st.S;
    }
  }
  // 4. backward
  for (int p = st.pass_begin + st.npasses - 1; p >= st.pass_begin; --p)
    bt_run_pass(d, d.passes[p], psi, lam, matf, matb, true, tP, tL, offs, acc, rank, nr);
  if (rank == 0 && threadIdx.x == 0)
    for (int j = 0; j < st.nparams; ++j) d.grads[st.param_begin + j] *= st.S;
}

// The persistent kernel, launched in clusters of d.csize CTAs.  Rank 0 of a
// cluster takes the next work item from the device counter (items pre-sorted by
// decreasing estimated cost); the item is either one large set shared by the whole
// cluster or up to d.csize small sets, one per CTA.
__global__ void __launch_bounds__(BT_THREADS, 3) k_batch(const BatchArgs d) {
  extern __shared__ __align__(16) unsigned char smem[];
  longlong2* tP = reinterpret_cast<longlong2*>(smem);
  longlong2* tL = tP + (1 << BT_M);
  uint64_t* offs = reinterpret_cast<uint64_t*>(tL + (1 << BT_M));
  double* acc = reinterpret_cast<double*>(offs + BT_OFFS);  // [warps][slots]; [rank][slot] across the cluster
  double* red = acc + BT_MAX_OPS * (BT_THREADS / 32);
  __shared__ int s_item;
  __shared__ double s_epart[BT_CLUSTER];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) s_item = atomicAdd(d.counter, 1);
    cl.sync();
    const int it = *cl.map_shared_rank(&s_item, 0);
    cl.sync();  // read by all before rank 0 may exit or take the next item
    if (it >= d.nitems) break;
    const BItem& item = d.items[it];
    int set_id = -1, r = 0, nr = 1;
    if (item.cluster) {
      set_id = item.sets[0];
      r = rank;
      nr = d.csize;
    } else if (rank < item.nsets) {
      set_id = item.sets[rank];
    }
    if (set_id >= 0) bt_eval_set(d, set_id, r, nr, tP, tL, offs, acc, red, s_epart);
  }
}

size_t batch_smem_bytes() {
  return 2 * sizeof(longlong2) * (1 << BT_M) + sizeof(uint64_t) * BT_OFFS +
         sizeof(double) * (BT_MAX_OPS * (BT_THREADS / 32) + 8);
}

static int bt_gen(int type) {
  switch (type) {
    case QS_RX: return BG_X;
    case QS_RY: return BG_Y;
    case QS_RZ: return BG_Z;
    case QS_P: case QS_CR: return BG_P;
    default: return BG_NONE;
  }
}

// Structural op class (valid for every angle) and unit codes; `adj` = adjoint.
static void bt_class(int type, bool adj, int8_t* kind, int8_t* c0, int8_t* c1) {
  auto conj = [&](int8_t c) -> int8_t { return adj ? (c == U_I ? U_MINUS_I : c == U_MINUS_I ? U_I : c) : c; };
  *c0 = U_GENERAL;
  *c1 = U_GENERAL;
  switch (type) {
    case QS_I: *kind = OP_IDENTITY; *c0 = U_ONE; *c1 = U_ONE; break;
    case QS_H: case QS_RY: *kind = OP_REAL; break;
    case QS_X: case QS_CNOT: *kind = OP_ANTI; *c0 = U_ONE; *c1 = U_ONE; break;
    case QS_Y: *kind = OP_ANTI; *c0 = conj(U_MINUS_I); *c1 = conj(U_I); break;
    case QS_Z: case QS_CZ: *kind = OP_PHASE1; *c0 = U_ONE; *c1 = U_MINUS_ONE; break;
    case QS_S: *kind = OP_PHASE1; *c0 = U_ONE; *c1 = conj(U_I); break;
    case QS_T: case QS_P: case QS_CR: *kind = OP_PHASE1; *c0 = U_ONE; break;
    case QS_RZ: *kind = OP_DIAG; break;
    default: *kind = OP_GENERAL; break;  // RX, U3
  }
}

}  // namespace qs

using namespace qs;

struct qs_batch {
  size_t nsets = 0;
  size_t total_params = 0;
  cudaStream_t stream = nullptr;
  BatchArgs args{};
  std::vector<void*> dev;      // device allocations
  double* h_params = nullptr;  // pinned staging
  double* h_grads = nullptr;
  double* h_energies = nullptr;
  double* d_params = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // bracket the persistent kernel
  int grid = 0;
  int csize = 1;
  size_t smem = 0;
};

static void batch_release(qs_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  for (void* p : b->dev) cudaFree(p);
  if (b->h_params) cudaFreeHost(b->h_params);
  if (b->h_grads) cudaFreeHost(b->h_grads);
  if (b->h_energies) cudaFreeHost(b->h_energies);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

template <class T>
static int upload(qs_batch* b, const std::vector<T>& v, const T** out) {
  void* p = nullptr;
  size_t bytes = std::max<size_t>(1, v.size()) * sizeof(T);
  QS_CUDA(dmalloc(&p, bytes));
  b->dev.push_back(p);
  if (!v.empty()) QS_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *out = (const T*)p;
  return QS_OK;
}

static int dev_alloc(qs_batch* b, size_t bytes, void** out) {
  QS_CUDA(dmalloc(out, std::max<size_t>(bytes, 16)));
  b->dev.push_back(*out);
  return QS_OK;
}

static int g_batch_cluster = 0;  // 0: chosen per batch

// Work items for clusters of c CTAs, most expensive first (longest-processing-time
// order), and the makespan of their greedy schedule over `nclusters` clusters in
// units of one CTA's time for one gate on 2^n amplitudes.  Cost of a set ~
// 2^n (gates + 1); a set with at least c tiles per pass is one item for a whole
// cluster (cost / c); smaller sets go c to an item (cost of the largest member).
static double plan_items(const std::vector<BSet>& sets, int c, int nclusters, std::vector<BItem>* out) {
  auto cost = [&](int i) { return std::ldexp((double)sets[i].ngates + 1.0, sets[i].n); };
  std::vector<int> small;
  std::vector<std::pair<double, BItem>> its;
  for (size_t i = 0; i < sets.size(); ++i) {
    if (c > 1 && sets[i].n >= BT_M && (1 << (sets[i].n - BT_M)) >= c) {
      BItem it{};
      it.cluster = 1;
      it.nsets = 1;
      it.sets[0] = (int)i;
      its.push_back({cost((int)i) / c, it});
    } else {
      small.push_back((int)i);
    }
  }
  std::stable_sort(small.begin(), small.end(), [&](int a, int b) { return cost(a) > cost(b); });
  for (size_t k = 0; k < small.size(); k += c) {
    BItem it{};
    it.cluster = 0;
    it.nsets = (int)std::min<size_t>(c, small.size() - k);
    for (int r = 0; r < it.nsets; ++r) it.sets[r] = small[k + r];
    its.push_back({cost(small[k]), it});
  }
  std::stable_sort(its.begin(), its.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  std::vector<double> finish(nclusters, 0.0);  // small heap-free scan: nclusters is a few hundred
  double span = 0.0;
  out->clear();
  for (auto& pr : its) {
    size_t k = std::min_element(finish.begin(), finish.end()) - finish.begin();
    finish[k] += pr.first;
    span = std::max(span, finish[k]);
    out->push_back(pr.second);
  }
  return span;
}

extern "C" int qs_set_batch_cluster(int ctas) {
  clear_error();
  if (ctas != 0 && ctas != 1 && ctas != 2 && ctas != 4 && ctas != 8)
    return fail(QS_ERR_INVALID_ARG, "cluster size %d not in {0, 1, 2, 4, 8}", ctas);
  g_batch_cluster = ctas;
  return QS_OK;
}

static void batch_config(const qs_batch* b, int grid, cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr) {
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = b->args.csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg->gridDim = dim3(grid);
  cfg->blockDim = dim3(BT_THREADS);
  cfg->dynamicSmemBytes = b->smem;
  cfg->stream = b->stream;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
}

extern "C" int qs_batch_create(size_t nsets, const int* n_per_set, const qs_gate* gates, const size_t* gate_offsets,
                               const size_t* param_offsets, const qs_pauli* terms, const size_t* term_offsets,
                               qs_batch** out) {
  clear_error();
  if (!out) return fail(QS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nsets == 0 || !n_per_set || !gate_offsets || !param_offsets || !term_offsets)
    return fail(QS_ERR_INVALID_ARG, "NULL argument or no sets");
  std::vector<BSet> sets(nsets);
  std::vector<BPass> passes;
  std::vector<BOp> ops;
  std::vector<BGate> bgates;
  std::vector<BGroup> groups;
  std::vector<BTerm> bterms;
  std::vector<int> dgheads, dgsrc;
  long long amp_off = 0;
  for (size_t si = 0; si < nsets; ++si) {
    const int n = n_per_set[si];
    if (n < 1 || n > BT_MAX_N) return fail(QS_ERR_INVALID_ARG, "set %zu: n=%d outside 1..%d", si, n, BT_MAX_N);
    const size_t g0 = gate_offsets[si], g1 = gate_offsets[si + 1];
    const size_t p0 = param_offsets[si], p1 = param_offsets[si + 1];
    const size_t t0 = term_offsets[si], t1 = term_offsets[si + 1];
    if (g1 < g0 || p1 < p0 || t1 < t0) return fail(QS_ERR_INVALID_ARG, "set %zu: offsets decrease", si);
    const size_t ng = g1 - g0, np = p1 - p0;
    BSet& st = sets[si];
    st.n = n;
    st.gate_begin = (int)bgates.size();
    st.ngates = (int)ng;
    st.param_begin = (int)p0;
    st.nparams = (int)np;
    st.amp_off = amp_off;
    amp_off += 1ll << n;
    std::vector<int> tgt(ng);
    std::vector<uint64_t> cms(ng);
    for (size_t k = 0; k < ng; ++k) {
      const qs_gate& g = gates[g0 + k];
      int rc = gate_qubits(g, n, &tgt[k], &cms[k]);
      if (rc) return fail(rc, "set %zu gate %zu: %s", si, k, qs_last_error());
      if (g.param_idx >= 0) {
        if ((size_t)g.param_idx >= np) return fail(QS_ERR_INVALID_ARG, "set %zu gate %zu: param_idx >= set size", si, k);
        if (bt_gen(g.type) == BG_NONE)
          return fail(QS_ERR_UNSUPPORTED, "set %zu gate %zu: gradients need RX, RY, RZ, P or CR", si, k);
      }
      BGate bg;
      bg.type = g.type;
      bg.param = g.param_idx >= 0 ? (int)(p0 + g.param_idx) : -1;
      bg.dagger = g.dagger != 0;
      bg.p[0] = g.p[0];
      bg.p[1] = g.p[1];
      bg.p[2] = g.p[2];
      bgates.push_back(bg);
    }
    // Hamiltonian: groups of terms sharing an X mask, scaled by S
    double csum = 0.0;
    const uint64_t full = (1ull << n) - 1;
    for (size_t k = t0; k < t1; ++k) {
      if ((terms[k].xmask | terms[k].zmask) & ~full) return fail(QS_ERR_INVALID_ARG, "set %zu term %zu exceeds n", si, k - t0);
      csum += fabs(terms[k].coef);
    }
    st.S = csum > 0 ? exp2(ceil(log2(csum))) : 1.0;
    st.group_begin = (int)groups.size();
    std::vector<uint64_t> xms;
    for (size_t k = t0; k < t1; ++k)
      if (std::find(xms.begin(), xms.end(), terms[k].xmask) == xms.end()) xms.push_back(terms[k].xmask);
    for (uint64_t xm : xms) {
      BGroup grp;
      grp.xm = xm;
      grp.tbegin = (int)bterms.size();
      for (size_t k = t0; k < t1; ++k) {
        if (terms[k].xmask != xm) continue;
        const int ny = __builtin_popcountll(terms[k].xmask & terms[k].zmask) & 3;
        BTerm bt;
        bt.c = (ny >= 2 ? -terms[k].coef : terms[k].coef) / st.S;
        bt.cq = q60_from_double(bt.c);
        bt.zm = terms[k].zmask;
        bt.imag = ny & 1;
        bterms.push_back(bt);
      }
      grp.tend = (int)bterms.size();
      groups.push_back(grp);
    }
    st.ngroups = (int)xms.size();
    // greedy tile passes
    const int dg_first = (int)dgheads.size();
    const int m = std::min(n, BT_M);
    const uint64_t low = (1ull << std::min(n, 3)) - 1;
    std::vector<uint32_t> remaining(ng), pass, rest;
    for (size_t k = 0; k < ng; ++k) remaining[k] = (uint32_t)k;
    st.pass_begin = (int)passes.size();
    while (!remaining.empty()) {
      uint64_t Q = greedy_pass(gates + g0, tgt, cms, remaining, m, low, BT_MAX_OPS, pass, rest);
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
      for (uint32_t k : pass) {
        const qs_gate& g = gates[g0 + k];
        BOp op;
        memset(&op, 0, sizeof op);
        op.gate = (int)k;  // index within the set's matrix tables
        op.param = g.param_idx >= 0 ? (int)(p0 + g.param_idx) : -1;
        bt_class(g.type, g.dagger != 0, &op.kf, &op.c0f, &op.c1f);
        bt_class(g.type, g.dagger == 0, &op.kb, &op.c0b, &op.c1b);
        if (op.kf == OP_IDENTITY && g.param_idx < 0) continue;
        uint32_t lcm = 0;
        uint64_t ext = 0;
        for (int b = 0; b < n; ++b)
          if ((cms[k] >> b) & 1) {
            if (local[b] >= 0) lcm |= 1u << local[b];
            else ext |= 1ull << b;
          }
        op.lcm = lcm;
        op.ext = ext;
        if (local[tgt[k]] >= 0) {
          op.tb = (int8_t)local[tgt[k]];
        } else {
          // a diagonal op whose target lies outside the tile: a per-tile scalar
          op.tb = (int8_t)tgt[k];
          op.kf = BK_SCALAR;
          op.kb = BK_SCALAR;
        }
        op.gen = g.param_idx >= 0 ? (int8_t)bt_gen(g.type) : BG_NONE;
        op.gsign = g.dagger ? -1.0 : 1.0;
        op.slot = -1;
        if (op.gen != BG_NONE) op.slot = (int16_t)slot++;
        ops.push_back(op);
      }
      // (no real pairs here: their quad code alone pushes the batch kernel past its
      // 80-register budget for three CTAs per SM; measured 847 -> 879 ms)
      group_diagonals(ops, bp.op_begin, &dgheads, &dgsrc, nullptr);
      bp.op_end = (int)ops.size();
      bp.nslots = slot;
      passes.push_back(bp);
      remaining.swap(rest);
    }
    st.npasses = (int)passes.size() - st.pass_begin;
    st.dg_begin = dg_first;
    st.ndg = (int)dgheads.size() - dg_first;
  }
  qs_batch* b = new (std::nothrow) qs_batch;
  if (!b) return fail(QS_ERR_OOM, "host allocation failed");
  int rc = QS_OK;
  auto chk = [&](int r) {
    if (rc == QS_OK) rc = r;
    return rc == QS_OK;
  };
  b->nsets = nsets;
  b->total_params = param_offsets[nsets];
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
  if (e != cudaSuccess) chk(cuda_fail(e, "cudaStreamCreate / cudaEventCreate"));
  BatchArgs& a = b->args;
  void* p0dg = nullptr;
  if (rc == QS_OK) chk(upload(b, sets, &a.sets));
  if (rc == QS_OK) chk(upload(b, passes, &a.passes));
  if (rc == QS_OK) chk(upload(b, ops, &a.ops));
  if (rc == QS_OK) chk(upload(b, bgates, &a.gates));
  if (rc == QS_OK) chk(upload(b, groups, &a.groups));
  if (rc == QS_OK) chk(upload(b, bterms, &a.terms));
  if (rc == QS_OK) chk(upload(b, dgheads, &a.dghead));
  if (rc == QS_OK && chk(dev_alloc(b, std::max<size_t>(1, dgheads.size()) * 16 * sizeof(QC), &p0dg))) a.dgf = (QC*)p0dg;
  if (rc == QS_OK && chk(dev_alloc(b, std::max<size_t>(1, dgheads.size()) * 16 * sizeof(QC), &p0dg))) a.dgb = (QC*)p0dg;
  void* p = nullptr;
  const size_t np = std::max<size_t>(1, b->total_params);
  if (rc == QS_OK && chk(dev_alloc(b, np * sizeof(double), &p))) { a.params = (const double*)p; b->d_params = (double*)p; }
  if (rc == QS_OK && chk(dev_alloc(b, np * sizeof(double), &p))) a.grads = (double*)p;
  if (rc == QS_OK && chk(dev_alloc(b, nsets * sizeof(double), &p))) a.energies = (double*)p;
  if (rc == QS_OK && chk(dev_alloc(b, (size_t)amp_off * sizeof(double2), &p))) a.psi = (double2*)p;
  if (rc == QS_OK && chk(dev_alloc(b, (size_t)amp_off * sizeof(double2), &p))) a.lam = (double2*)p;
  if (rc == QS_OK && chk(dev_alloc(b, std::max<size_t>(1, bgates.size()) * 4 * sizeof(QC), &p))) a.matf = (QC*)p;
  if (rc == QS_OK && chk(dev_alloc(b, std::max<size_t>(1, bgates.size()) * 4 * sizeof(QC), &p))) a.matb = (QC*)p;
  if (rc == QS_OK && chk(dev_alloc(b, sizeof(int), &p))) a.counter = (int*)p;
  if (rc == QS_OK) {
    e = hmalloc_pinned(&b->h_params, np * sizeof(double));
    if (e == cudaSuccess) e = hmalloc_pinned(&b->h_grads, np * sizeof(double));
    if (e == cudaSuccess) e = hmalloc_pinned(&b->h_energies, nsets * sizeof(double));
    if (e != cudaSuccess) chk(cuda_fail(e, "cudaMallocHost"));
  }
  if (rc == QS_OK) {
    b->smem = batch_smem_bytes();
    e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    if (e != cudaSuccess) chk(cuda_fail(e, "batch kernel set-up"));
    // cluster size: the forced one, else the one whose LPT schedule of the items
    // over the resident clusters has the shortest estimated makespan
    std::vector<BItem> items;
    double best = 0.0;
    for (int c = BT_CLUSTER; c >= 1 && rc == QS_OK; c >>= 1) {
      if (g_batch_cluster && c != g_batch_cluster) continue;
      b->args.csize = c;
      cudaLaunchConfig_t cfg{};
      cudaLaunchAttribute attr[1];
      batch_config(b, c * std::max(1, sms), &cfg, attr);
      int nclusters = 0;
      e = cudaOccupancyMaxActiveClusters(&nclusters, k_batch, &cfg);
      if (e != cudaSuccess) {
        chk(cuda_fail(e, "cudaOccupancyMaxActiveClusters"));
        break;
      }
      if (nclusters < 1) continue;
      std::vector<BItem> its;
      const double span = plan_items(sets, c, nclusters, &its);
      if (items.empty() || span < best) {
        best = span;
        items.swap(its);
        b->grid = nclusters * c;
        b->csize = c;
      }
    }
    if (rc == QS_OK && items.empty()) chk(fail(QS_ERR_UNSUPPORTED, "no cluster of the batch kernel fits the device"));
    a.csize = b->csize;
    a.nitems = (int)items.size();
    if (rc == QS_OK) chk(upload(b, items, &a.items));
  }
  if (rc != QS_OK) {
    batch_release(b);
    return rc;
  }
  *out = b;
  return QS_OK;
}

// Queue one evaluation: params (device) -> energies/grads (device).
static int batch_enqueue(qs_batch* b) {
  const BatchArgs& a = b->args;
  QS_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(int), b->stream));
  // while capturing, external records become timing event nodes of the graph
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  QS_CUDA(cudaStreamIsCapturing(b->stream, &cs));
  const unsigned flags = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  QS_CUDA(cudaEventRecordWithFlags(b->ev0, b->stream, flags));
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  batch_config(b, b->grid, &cfg, attr);
  QS_CUDA(cudaLaunchKernelEx(&cfg, k_batch, a));
  QS_TRY(launch_check("batch kernel"));
  QS_CUDA(cudaEventRecordWithFlags(b->ev1, b->stream, flags));
  return QS_OK;
}

extern "C" int qs_batch_last_ms(const qs_batch* b, double* ms) {
  if (!b || !ms) return fail(QS_ERR_INVALID_ARG, "NULL argument");
  float f = 0.f;
  QS_CUDA(cudaEventElapsedTime(&f, b->ev0, b->ev1));
  *ms = f;
  return QS_OK;
}

extern "C" int qs_batch_cluster(const qs_batch* b, int* ctas) {
  if (!b || !ctas) return fail(QS_ERR_INVALID_ARG, "NULL argument");
  *ctas = b->csize;
  return QS_OK;
}

extern "C" int qs_batch_info(const qs_batch* b, int* grid, int* threads, size_t* smem_bytes) {
  if (!b || !grid || !threads || !smem_bytes) return fail(QS_ERR_INVALID_ARG, "NULL argument");
  *grid = b->grid;
  *threads = BT_THREADS;
  *smem_bytes = b->smem;
  return QS_OK;
}

extern "C" int qs_batch_run(qs_batch* b, const double* params, double* energies, double* grads, int on_device) {
  clear_error();
  if (!b || !params || !energies || (b->total_params && !grads)) return fail(QS_ERR_INVALID_ARG, "NULL argument");
  const size_t pb = b->total_params * sizeof(double), eb = b->nsets * sizeof(double);
  note_launch(1);
  if (on_device) {
    QS_CUDA(cudaMemcpyAsync(b->d_params, params, pb, cudaMemcpyDeviceToDevice, b->stream));
    QS_TRY(batch_enqueue(b));
    QS_CUDA(cudaMemcpyAsync(energies, b->args.energies, eb, cudaMemcpyDeviceToDevice, b->stream));
    if (pb) QS_CUDA(cudaMemcpyAsync(grads, b->args.grads, pb, cudaMemcpyDeviceToDevice, b->stream));
    QS_CUDA(cudaStreamSynchronize(b->stream));
    return QS_OK;
  }
  if (!b->exec) {
    // capture: staging -> device params, counter reset, the persistent kernel, results -> staging
    QS_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemcpyAsync(b->d_params, b->h_params, pb, cudaMemcpyHostToDevice, b->stream);
    int rc = e == cudaSuccess ? batch_enqueue(b) : cuda_fail(e, "capture params");
    if (rc == QS_OK) {
      e = cudaMemcpyAsync(b->h_energies, b->args.energies, eb, cudaMemcpyDeviceToHost, b->stream);
      if (e == cudaSuccess && pb) e = cudaMemcpyAsync(b->h_grads, b->args.grads, pb, cudaMemcpyDeviceToHost, b->stream);
      if (e != cudaSuccess) rc = cuda_fail(e, "capture results");
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (rc != QS_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    b->graph = g;
    QS_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
  }
  memcpy(b->h_params, params, pb);
  QS_CUDA(cudaGraphLaunch(b->exec, b->stream));
  QS_CUDA(cudaStreamSynchronize(b->stream));
  memcpy(energies, b->h_energies, eb);
  if (pb) memcpy(grads, b->h_grads, pb);
  return QS_OK;
}

extern "C" int qs_batch_free(qs_batch* b) {
  batch_release(b);
  return QS_OK;
}
