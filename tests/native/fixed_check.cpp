// Host-side harness for the Q60 helpers of the CUDA library (compiled by the
// test suite with g++; exercises the same inline functions the kernels use).
#include "fixed.h"

extern "C" {
long long fc_from_double(double v) { return (long long)qs::q60_from_double(v); }
long long fc_from_double_nb(double v) { return (long long)qs::q60_from_double_nb(v); }
// x1 y1 + x2 y2 of Q60 integers through the split-column exact product, as two words
void fc_dot2_exact(long long x1, long long y1, long long x2, long long y2, unsigned long long* out) {
  const unsigned __int128 r = qs::dot2_exact(qs::split31(x1), qs::split31(y1), qs::split31(x2), qs::split31(y2));
  out[0] = (unsigned long long)r;
  out[1] = (unsigned long long)(r >> 64);
}
double fc_to_double(long long V) { return qs::q60_to_double((int64_t)V); }
// out = u0 * a0 + u1 * a1 for Q60 reals given as int64, via the limb accumulator
long long fc_dot2(long long u0, long long a0, long long u1, long long a1) {
  qs::QAcc acc{0, 0};
  qs::qacc_add(acc, qs::q60_split(u0), qs::q60_split(a0));
  qs::qacc_add(acc, qs::q60_split(u1), qs::q60_split(a1));
  return (long long)qs::qacc_result(acc);
}
// the same sum through the pre-biased accumulator the kernels use
long long fc_dot4_kernel(const long long* u, const long long* a) {
  qs::QAcc acc = qs::qacc_new();
  for (int i = 0; i < 4; ++i) qs::qacc_add(acc, qs::q60_split(u[i]), qs::q60_split(a[i]));
  return (long long)qs::qacc_round(acc);
}
// out = u0 a0 + u1 a1 for complex Q60 values (u given as doubles, a as Q60
// integer pairs) through the Gauss-form row of the tile kernels
void fc_gauss_row(const double* u, const long long* a, long long* out) {
  const qs::QC u0 = qs::qc_make_gauss(u[0], u[1]), u1 = qs::qc_make_gauss(u[2], u[3]);
  int64_t re, im;
  qs::q60_gauss_row(u0, u1, qs::q60_split(a[0]), qs::q60_split(a[1]), qs::q60_split(a[0] + a[1]),
                    qs::q60_split(a[2]), qs::q60_split(a[3]), qs::q60_split(a[2] + a[3]), &re, &im);
  out[0] = re;
  out[1] = im;
}
long long fc_dot4_full(const long long* u, const long long* a) {
  qs::QAccF acc{0, 0, 0};
  for (int i = 0; i < 4; ++i) qs::qaccf_add(acc, qs::q60_split(u[i]), qs::q60_split(a[i]));
  return (long long)qs::qaccf_result(acc);
}
long long fc_dot4(const long long* u, const long long* a) {
  qs::QAcc acc{0, 0};
  for (int i = 0; i < 4; ++i) qs::qacc_add(acc, qs::q60_split(u[i]), qs::q60_split(a[i]));
  return (long long)qs::qacc_result(acc);
}
}
