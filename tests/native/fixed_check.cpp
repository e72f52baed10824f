// Host-side harness for the Q60 helpers of the CUDA library (compiled by the
// test suite with g++; exercises the same inline functions the kernels use).
#include "fixed.h"
#include "ieee_sq.h"
#include "q60pair.cuh"

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
double fc_to_double_nb(long long V) { return qs::q60_to_double_nb((int64_t)V); }
// the coefficients of the pair form as Q60 integers (P.re, P.im, -P.im, Q.re,
// Q.im, -Q.im) and the reflection flags
int fc_pair_coef(const double* ra, const double* rb, long long* c) {
  qs::QL q[6];
  int flags = 0;
  qs::q60_pair_coef(ra, rb, q, &flags);
  for (int k = 0; k < 6; ++k) c[k] = (long long)q[k].h * (1ll << 30) + q[k].l;
  return flags;
}
// three real orthogonal 2x2 ops on one component of an octet x[8] (Q60 integers,
// index bit(a) + 2 bit(b) + 4 bit(c)) through the four-complex-product form;
// coefficients (re, im of U+, U-, V+, V-) as Q60 integers into c[8]
int fc_triple_comp(const double* ra, const double* rb, const double* rc, long long* x, long long* c) {
  qs::QL q[8];
  int flags = 0;
  qs::q60_triple_coef(ra, rb, rc, q, &flags);
  for (int k = 0; k < 8; ++k) c[k] = (long long)q[k].h * (1ll << 30) + q[k].l;
  qs::Q3 P[4][3];
  qs::q60_triple_q3(q, P);
  int64_t v[8];
  for (int k = 0; k < 8; ++k) v[k] = (__builtin_popcount(k & flags) & 1) ? -x[k] : x[k];
  qs::q60_triple_comp(v, P);
  for (int k = 0; k < 8; ++k) x[k] = v[k];
  return flags;
}
// four real orthogonal 2x2 ops on one component of 16 amplitudes x[16] (Q60
// integers, index bit(a) + 2 bit(b) + 4 bit(c) + 8 bit(d)) through the
// eight-complex-product form; coefficients (re, im of channel k) into c[16]
int fc_quad4_comp(const double* ra, const double* rb, const double* rc, const double* rd, long long* x,
                  long long* c) {
  qs::Q3 P[24];
  int flags = 0;
  qs::q60_quad4_coef(ra, rb, rc, rd, P, &flags);
  for (int k = 0; k < 8; ++k) {
    c[2 * k] = (long long)P[3 * k].h * (1ll << 30) + P[3 * k].l2 / 2;
    c[2 * k + 1] = (long long)P[3 * k + 1].h * (1ll << 30) + P[3 * k + 1].l2 / 2;
  }
  int64_t v[16];
  for (int k = 0; k < 16; ++k) v[k] = (__builtin_popcount(k & flags) & 1) ? -x[k] : x[k];
  qs::q60_quad4_comp(v, P, P + 8, P + 16);
  for (int k = 0; k < 16; ++k) x[k] = v[k];
  return flags;
}
// two real orthogonal 2x2 ops (ra on quad bit a, rb on bit b; row-major) on one
// component of a quad x[4] (Q60 integers, index bit(a) + 2 bit(b)), through the
// two-complex-product form of the pair kernels
void fc_pair_comp(const double* ra, const double* rb, long long* x) {
  qs::QL c[6];
  int flags = 0;
  qs::q60_pair_coef(ra, rb, c, &flags);
  int64_t x0 = x[0], x1 = x[1], x2 = x[2], x3 = x[3];
  switch (flags) {
    case 0: qs::q60_pair_comp<0>(x0, x1, x2, x3, c); break;
    case 1: qs::q60_pair_comp<1>(x0, x1, x2, x3, c); break;
    case 2: qs::q60_pair_comp<2>(x0, x1, x2, x3, c); break;
    default: qs::q60_pair_comp<3>(x0, x1, x2, x3, c); break;
  }
  x[0] = x0;
  x[1] = x1;
  x[2] = x2;
  x[3] = x3;
}
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

// fl(x * x) from integer operations (the sampler's squares); *ok as the helper sets it
extern "C" double fc_sq_rn(double x, int* ok) {
  bool o = false;
  const double r = qs::sq_rn_int(x, &o);
  *ok = o ? 1 : 0;
  return r;
}
// fl(a + b) for a, b >= 0 from integer operations (the sampler's p = re^2 + im^2)
extern "C" double fc_add_rn_pos(double a, double b, int* ok) {
  bool o = false;
  const double r = qs::add_rn_pos_int(a, b, &o);
  *ok = o ? 1 : 0;
  return r;
}
