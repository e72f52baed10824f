// Host-side harness for the Pauli pass planner of the CUDA library (compiled by
// the test suite with g++; runs the same inline planner the library uses).
#include <cstring>

#include "pauli_plan.h"

extern "C" {
// Plans nt terms on n qubits.  Outputs (caller-sized):
//   slots:  3 int64 per slot (xm, zm, part);
//   passes: 2 + 2 * PT_TMAX int64 per pass (T, slot count, basis[PT_TMAX], slot[PS_MAX]);
//   terms:  3 int32 per term (slot, total slot, mult).
// Returns 0, or -1 when a capacity is too small (counts are still written).
int pp_plan(int n, const unsigned long long* xm, const unsigned long long* zm, size_t nt, long long* slots,
            size_t slot_cap, long long* passes, size_t pass_cap, int* terms, size_t* nslots, size_t* npasses) {
  static_assert(qs::PS_MAX <= qs::PT_TMAX, "pass record layout");
  const qs::PauliPlan P = qs::plan_pauli(n, (const uint64_t*)xm, (const uint64_t*)zm, nt);
  *nslots = P.slots.size();
  *npasses = P.passes.size();
  if (P.slots.size() > slot_cap || P.passes.size() > pass_cap) return -1;
  for (size_t k = 0; k < P.slots.size(); ++k) {
    slots[3 * k] = (long long)P.slots[k].xm;
    slots[3 * k + 1] = (long long)P.slots[k].zm;
    slots[3 * k + 2] = P.slots[k].im;
  }
  const size_t W = 2 + 2 * qs::PT_TMAX;
  for (size_t p = 0; p < P.passes.size(); ++p) {
    long long* o = passes + p * W;
    std::memset(o, 0, W * sizeof(long long));
    o[0] = (long long)P.passes[p].bm.size();
    o[1] = (long long)P.passes[p].sl.size();
    for (size_t i = 0; i < P.passes[p].bm.size() && i < (size_t)qs::PT_TMAX; ++i) o[2 + i] = (long long)P.passes[p].bm[i];
    for (size_t i = 0; i < P.passes[p].sl.size() && i < (size_t)qs::PT_TMAX; ++i) o[2 + qs::PT_TMAX + i] = P.passes[p].sl[i];
  }
  for (size_t k = 0; k < nt; ++k) {
    terms[3 * k] = P.tslot[k];
    terms[3 * k + 1] = P.ttot[k];
    terms[3 * k + 2] = P.tmult[k];
  }
  return 0;
}
}
