// Host-side planning of the exact Pauli-sum passes (k_pauli_tile in reduce.cu):
// the paper's expectation tool (qop, Section "Variational quantum circuit") as
// passes over tiles of the state.  Plain C++, no CUDA: the test suite compiles it
// on the host and checks every plan it makes.
//
// A term P = (xm, zm) with ny = popcount(xm & zm) pairs x0 with x1 = x0 ^ xm.  With
// w = conj(a_x1) a_x0 and s0 = (-1)^popcount(x0 & zm) a pair contributes
//   ny = 0: 2 s0 Re w,  1: -2 s0 Im w,  2: -2 s0 Re w,  3: 2 s0 Im w,
// and a term with xm = 0 contributes s0 |a_x0|^2 per index.  A slot (xm, zm, part)
// is one such sum restricted to pairs of sign +1 (pos); the term is
// mult * (2 pos - tot), tot being the slot of the same xm with zm = 0.
//
// A pass reads the state once, as tiles {base ^ span(basis)} of 2^T amplitudes
// (T = min(12, n)).  Its basis holds qubits 0..3 (so a tile is made of runs of 16
// consecutive amplitudes), X masks reduced to distinct leading bits, then further
// single qubits; every tile base has the leading bits clear.  Every X mask in the
// span is served by the pass; |a|^2 slots fill the free places (12 per pass).
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <map>
#include <tuple>
#include <utility>
#include <vector>

namespace qs {

constexpr int PT_TMAX = 12;  // tile coordinates
constexpr int PS_MAX = 12;   // slots per pass

struct PauliSlot {
  uint64_t xm, zm;
  int im;  // pair slots: 0 = Re w, 1 = Im w; |a|^2 slots: 0
};

struct PauliPass {
  std::vector<uint64_t> bm;  // basis vector of each coordinate, ascending leading bit
  std::vector<int> sl;       // slots: |a|^2 slots first, then pair slots ordered by (coordinates of xm, im)
};

struct PauliPlan {
  std::vector<PauliSlot> slots;
  std::vector<PauliPass> passes;
  std::vector<int> tslot, ttot, tmult;  // per term: its slot, the slot of its total, mult
};

inline int pp_lead(uint64_t m) { return 63 - __builtin_clzll(m); }

// v reduced by a basis in echelon form (distinct leading bits, any order): each
// basis vector's leading bit is cleared from v, highest leading bit first; *xc
// receives the coordinates used.  v is in the span iff the result is 0.
inline uint64_t pp_reduce(const std::vector<uint64_t>& B, uint64_t v, uint32_t* xc) {
  std::vector<int> order(B.size());
  for (size_t q = 0; q < B.size(); ++q) order[q] = (int)q;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return pp_lead(B[x]) > pp_lead(B[y]); });
  uint32_t c = 0;
  for (int q : order)
    if ((v >> pp_lead(B[q])) & 1) {
      v ^= B[q];
      c |= 1u << q;
    }
  if (xc) *xc = c;
  return v;
}

inline PauliPlan plan_pauli(int n, const uint64_t* xmask, const uint64_t* zmask, size_t nt) {
  PauliPlan R;
  std::map<std::tuple<uint64_t, uint64_t, int>, int> slot_of;
  auto get = [&](uint64_t xm, uint64_t zm, int im) {
    const auto key = std::make_tuple(xm, zm, im);
    const auto it = slot_of.find(key);
    if (it != slot_of.end()) return it->second;
    R.slots.push_back({xm, zm, im});
    return slot_of[key] = (int)R.slots.size() - 1;
  };
  R.tslot.resize(nt);
  R.ttot.resize(nt);
  R.tmult.resize(nt);
  std::vector<uint64_t> xms;  // distinct X masks, in order of first appearance
  for (size_t k = 0; k < nt; ++k) {
    const uint64_t xm = xmask[k], zm = zmask[k];
    const int ny = __builtin_popcountll(xm & zm) & 3;
    if (xm == 0) {
      R.tslot[k] = get(0, zm, 0);
      R.ttot[k] = get(0, 0, 0);
      R.tmult[k] = 1;
    } else {
      const int im = ny & 1;
      if (!slot_of.count(std::make_tuple(xm, 0ull, 0)) && !slot_of.count(std::make_tuple(xm, 0ull, 1)))
        xms.push_back(xm);
      R.tslot[k] = get(xm, zm, im);
      R.ttot[k] = get(xm, 0, im);
      R.tmult[k] = (ny == 0 || ny == 3) ? 2 : -2;
    }
  }
  const int Tmax = std::min(PT_TMAX, n);
  auto make_basis = [&](std::vector<uint64_t> B) {
    for (int b = 0; (int)B.size() < Tmax && b < n; ++b) {  // fill with single qubits
      bool is_lead = false;
      for (uint64_t v : B) is_lead |= pp_lead(v) == b;
      if (!is_lead) B.push_back(1ull << b);
    }
    std::sort(B.begin(), B.end(), [](uint64_t x, uint64_t y) { return pp_lead(x) < pp_lead(y); });
    return B;
  };
  std::map<uint64_t, std::vector<int>> by_xm;  // pair slots per X mask
  for (int k = 0; k < (int)R.slots.size(); ++k)
    if (R.slots[k].xm) by_xm[R.slots[k].xm].push_back(k);
  std::vector<char> done(xms.size(), 0);
  for (size_t i0 = 0; i0 < xms.size(); ++i0) {
    if (done[i0]) continue;
    std::vector<uint64_t> B;
    for (int b = 0; b < std::min(4, n); ++b) B.push_back(1ull << b);
    for (size_t q = i0; q < xms.size() && (int)B.size() < Tmax; ++q) {
      if (done[q]) continue;
      const uint64_t v = pp_reduce(B, xms[q], nullptr);
      if (v) B.push_back(v);
    }
    B = make_basis(B);
    std::vector<std::pair<uint64_t, int>> keyed;  // ((xc << 1) | im, slot)
    for (size_t q = i0; q < xms.size(); ++q) {
      if (done[q]) continue;
      uint32_t xc = 0;
      if (pp_reduce(B, xms[q], &xc)) continue;  // outside this span
      done[q] = 1;
      for (int k : by_xm[xms[q]]) keyed.push_back({((uint64_t)xc << 1) | (uint64_t)R.slots[k].im, k});
    }
    std::stable_sort(keyed.begin(), keyed.end(),
                     [](const std::pair<uint64_t, int>& x, const std::pair<uint64_t, int>& y) { return x.first < y.first; });
    for (size_t c = 0; c < keyed.size(); c += PS_MAX) {
      PauliPass P{B, {}};
      for (size_t q = c; q < std::min(keyed.size(), c + (size_t)PS_MAX); ++q) P.sl.push_back(keyed[q].second);
      R.passes.push_back(P);
    }
  }
  // |a|^2 slots: into free places, then passes over tiles of qubits 0..T-1
  std::vector<int> zs;
  for (int k = 0; k < (int)R.slots.size(); ++k)
    if (!R.slots[k].xm) zs.push_back(k);
  size_t zi = 0;
  for (auto& P : R.passes)
    while (zi < zs.size() && (int)P.sl.size() < PS_MAX) P.sl.insert(P.sl.begin(), zs[zi++]);
  while (zi < zs.size()) {
    PauliPass P{make_basis({}), {}};
    while (zi < zs.size() && (int)P.sl.size() < PS_MAX) P.sl.push_back(zs[zi++]);
    R.passes.push_back(P);
  }
  return R;
}

}  // namespace qs
