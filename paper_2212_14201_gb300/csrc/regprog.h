// Register programs of the Q60 tile pass (host side, no CUDA): the ops of one
// fusion pass (the paper's circuit fusion, Section "Quantum circuit fusion")
// grouped into register phases.
//
// A phase holds R = 4 tile bits in registers: each thread owns the 16 amplitudes
// of one group (the tile's other bits fixed) and runs every op of the phase on
// them before the next shared-memory exchange.  Diagonal ops (phase tables,
// diagonal gates, controls) run in any phase; an op that mixes amplitudes (real,
// general, antidiagonal) needs its target among the phase's register bits.
//
// Phases are built greedily over the pass's op list.  For a register set P, scan
// the remaining ops in order; an op joins the phase when it commutes with every
// op skipped so far and its mixing target lies in P; otherwise it is skipped.
// Two ops commute unless they share a qubit on which at least one of them acts
// non-diagonally.  The skipped ops, in order, form the rest.  P is chosen per
// phase among the sets that contain the target of the first op that can run:
// the one that lets the most mixing ops (then the most ops) join.  A phase that
// ends a layer therefore continues with the next layer's ops on its own register
// bits, so a layer of rotations over m tile qubits costs about m/R - 1 phases
// instead of m/R, and in light-cone passes a phase spans several short layers.
// Inside a phase, a real rotation that can be paired (uncontrolled, another
// register bit) is moved up next to an earlier unpaired one when it commutes with
// every op between them, so that the two run as one 4x4 on quads.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <vector>

namespace qs {

constexpr int RP_BITS = 4;  // register bits per phase: 16 amplitudes per thread

// Input op of the phase builder, in tile-local terms.
enum RpInKind : int { IK_TABLE = 0, IK_MIX = 1, IK_DIAG = 2 };
struct RpIn {
  int kind;       // IK_TABLE (diagonal over the whole tile), IK_MIX (mixes its target), IK_DIAG
  int tb;         // tile bit of the target, -1 when it lies outside the tile (IK_DIAG only)
  uint32_t lcm;   // controls inside the tile (tile-bit mask)
  bool pairable;  // an uncontrolled real rotation (may join another as a 4x4 pair)
};

struct RpPhase {
  uint32_t P = 0;          // register tile bits (exactly RP_BITS of them, or m if m < RP_BITS)
  std::vector<int> ops;    // indices into the input list, in application order
};

inline int rp_popc(uint32_t x) { return __builtin_popcount(x); }

// Tile bits an op mixes (N) and touches diagonally (D).
inline void rp_touch(const RpIn& o, uint32_t full, uint32_t* N, uint32_t* D) {
  if (o.kind == IK_TABLE) {
    *N = 0;
    *D = full;
  } else if (o.kind == IK_MIX) {
    *N = 1u << o.tb;
    *D = o.lcm;
  } else {
    *N = 0;
    *D = o.lcm | (o.tb >= 0 ? 1u << o.tb : 0u);
  }
}

// Ops of `rem` that a phase with register set P takes (in order), the rest in
// `rest`; returns the number of mixing ops taken.
inline int rp_take(const std::vector<RpIn>& ops, const std::vector<int>& rem, uint32_t P, uint32_t full,
                   std::vector<int>* take, std::vector<int>* rest) {
  uint32_t defN = 0, defD = 0;
  int mix = 0;
  for (int i : rem) {
    uint32_t N, D;
    rp_touch(ops[i], full, &N, &D);
    const bool blocked = (N & (defN | defD)) || (D & defN);
    if (!blocked && (N & ~P) == 0) {
      if (take) take->push_back(i);
      mix += N != 0;
      continue;
    }
    if (rest) rest->push_back(i);
    defN |= N;
    defD |= D;
  }
  return mix;
}

inline bool rp_commute(const RpIn& a, const RpIn& b, uint32_t full) {
  uint32_t Na, Da, Nb, Db;
  rp_touch(a, full, &Na, &Da);
  rp_touch(b, full, &Nb, &Db);
  return !(Na & (Nb | Db)) && !(Nb & Da);
}

// Moves pairable rotations next to an earlier unpaired partner (see above).
inline void rp_pair_order(const std::vector<RpIn>& ops, uint32_t full, std::vector<int>* list) {
  std::vector<int>& L = *list;
  size_t i = 0;
  while (i < L.size()) {
    const RpIn& a = ops[L[i]];
    if (!a.pairable) {
      ++i;
      continue;
    }
    if (i + 1 < L.size() && ops[L[i + 1]].pairable && ops[L[i + 1]].tb != a.tb) {
      i += 2;
      continue;
    }
    size_t found = 0;
    for (size_t j = i + 1; j < L.size(); ++j) {
      const RpIn& b = ops[L[j]];
      if (b.pairable && b.tb != a.tb) {
        bool ok = true;
        for (size_t k = i + 1; k < j && ok; ++k) ok = rp_commute(b, ops[L[k]], full);
        if (ok) found = j;
        break;  // only the first candidate: later ones would have to pass it
      }
    }
    if (found) {
      const int b = L[found];
      L.erase(L.begin() + (long)found);
      L.insert(L.begin() + (long)i + 1, b);
      i += 2;
    } else {
      ++i;
    }
  }
}

inline std::vector<RpPhase> rp_build_phases(const std::vector<RpIn>& ops, int m) {
  const int R = std::min(m, RP_BITS);
  const uint32_t full = m >= 32 ? ~0u : ((1u << m) - 1);
  std::vector<RpPhase> phases;
  std::vector<int> rem(ops.size()), rest, take;
  for (size_t i = 0; i < ops.size(); ++i) rem[i] = (int)i;
  while (!rem.empty()) {
    // the target of the first op that can run, and the mixing targets of the rest
    uint32_t first = 0, bits = 0;
    {
      uint32_t defN = 0, defD = 0;
      for (int i : rem) {
        uint32_t N, D;
        rp_touch(ops[i], full, &N, &D);
        bits |= N;
        const bool blocked = (N & (defN | defD)) || (D & defN);
        if (!blocked && !N) continue;  // a diagonal op every phase takes
        if (!blocked && !first) {
          first = N;
          continue;
        }
        defN |= N;
        defD |= D;
      }
    }
    uint32_t bestP = first;
    if (first) {
      int cand[32], nc = 0;
      for (int b = 0; b < m; ++b)
        if (((bits & ~first) >> b) & 1) cand[nc++] = b;
      const int need = std::min(R - 1, nc);
      int best_mix = -1, best_all = -1;
      // every choice of `need` further bits (nc <= m - 1 <= 11, need <= 3)
      int idx[3] = {0, 1, 2};
      for (int k = 0; k < need; ++k) idx[k] = k;
      while (true) {
        uint32_t P = first;
        for (int k = 0; k < need; ++k) P |= 1u << cand[idx[k]];
        take.clear();
        const int mix = rp_take(ops, rem, P, full, &take, nullptr);
        const int all = (int)take.size();
        if (mix > best_mix || (mix == best_mix && all > best_all)) {
          best_mix = mix;
          best_all = all;
          bestP = P;
        }
        int k = need - 1;
        while (k >= 0 && idx[k] == nc - need + k) --k;
        if (k < 0) break;
        ++idx[k];
        for (int j = k + 1; j < need; ++j) idx[j] = idx[j - 1] + 1;
      }
    }
    RpPhase ph;
    ph.P = bestP;
    rest.clear();
    rp_take(ops, rem, ph.P, full, &ph.ops, &rest);
    rp_pair_order(ops, full, &ph.ops);
    // pad the register set to R bits with the highest unused tile bits
    for (int b = m - 1; b >= 0 && rp_popc(ph.P) < R; --b) ph.P |= 1u << b;
    phases.push_back(std::move(ph));
    rem.swap(rest);
  }
  return phases;
}

// Shared-memory swizzle of the tile (element j of 16 bytes): the physical index
// is j XOR sw(j), where sw folds the bits at and above 3 into bits 0..2 with the
// vectors below.  It is linear over GF(2), so the physical index of a sum of
// disjoint bit sets is the XOR of theirs.  The vectors give every bit 0..2 of
// the bank quad a contribution from several tile bits: for any choice of four
// register bits the remaining tile bits span GF(2)^3, so some three of them
// (the low lane bits of a warp) reach eight different bank quads.
constexpr uint8_t RP_SWZ[16] = {1, 2, 4, 3, 5, 6, 7, 1, 2, 4, 3, 5, 6, 7, 1, 2};

inline uint32_t rp_swz(uint32_t j) {
  uint32_t s = 0;
  for (int b = 3; b < 16; ++b)
    if ((j >> b) & 1) s ^= RP_SWZ[b];
  return j ^ s;
}

// Group bits of a phase: the tile bits outside its register set, ordered so
// that the three lowest (lanes 0..7 of a warp) have independent bank vectors
// (RP_SWZ, with bits 0..2 as themselves), the rest ascending.  Returns the count.
inline int rp_group_bits(uint32_t P, int m, uint8_t* gl) {
  int cand[32], nc = 0;
  for (int b = 0; b < m; ++b)
    if (!((P >> b) & 1)) cand[nc++] = b;
  auto vec = [](int b) -> uint32_t { return b < 3 ? (1u << b) : RP_SWZ[b]; };
  int pick[3] = {-1, -1, -1};
  bool found = false;
  for (int a = 0; a < nc && !found; ++a)
    for (int b = a + 1; b < nc && !found; ++b)
      for (int c = b + 1; c < nc && !found; ++c) {
        const uint32_t x = vec(cand[a]), y = vec(cand[b]), z = vec(cand[c]);
        if (x && y && z && x != y && x != z && y != z && (x ^ y) != z) {
          pick[0] = a;
          pick[1] = b;
          pick[2] = c;
          found = true;
        }
      }
  int k = 0;
  if (found)
    for (int i = 0; i < 3; ++i) gl[k++] = (uint8_t)cand[pick[i]];
  for (int i = 0; i < nc; ++i)
    if (!found || (i != pick[0] && i != pick[1] && i != pick[2])) gl[k++] = (uint8_t)cand[i];
  return k;
}

}  // namespace qs
