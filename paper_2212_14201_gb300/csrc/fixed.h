// Q60 fixed-point arithmetic for gate application on the integer pipe.
//
// GB300 issues FP64 at 1/74 of its FP32 rate (measured: 5.0e11 DFMA/s against
// 1.8e13 32x32->64 integer multiply-adds/s), so a complex128 2x2 gate costs
// ~3x its HBM time in FP64.  The state stays complex128 in memory; inside a
// kernel each real component v (|v| <= 1.25) is converted to V = round(v * 2^60),
// a signed 64-bit integer, and gate matrices (|u| <= 1) likewise.  A product
// U*A is formed from limbs V = h * 2^30 + l with 0 <= l < 2^30:
//   U*A * 2^-60 = Uh*Ah + (Uh*Al + Ul*Ah) * 2^-30 + Ul*Al * 2^-60,
// the first two terms accumulated exactly in two int64 registers with
// mad.wide.s32, the last (< 2^-60 per product) dropped.  One output
// component of a 2x2 complex matvec (four products) carries at most
// 4 * 2^-60 + 2^-61 absolute error before the final rounding back to double
// (which adds the same <= 2^-53 relative error an FP64 kernel has).
// Bounds: the real and imaginary parts of one row of a unitary 2x2 sum to at
// most 2 in absolute value, so with |components| <= 1.25 the hi accumulator
// stays below 2.5 * 2^60 and the mid accumulator below 7 * 2^60 < 2^63.
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define QS_HD __host__ __device__ __forceinline__
#else
#define QS_HD inline
#endif

namespace qs {

constexpr double Q60_MAX_ABS = 1.25;  // component bound under which the accumulators cannot overflow

QS_HD uint64_t q_bits(double v) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t b;
  memcpy(&b, &v, 8);
  return b;
#endif
}

QS_HD double q_from_bits(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double v;
  memcpy(&v, &b, 8);
  return v;
#endif
}

QS_HD int q_clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

// round(v * 2^60), ties away from zero; |v| must be < 8.  Integer operations only.
QS_HD int64_t q60_from_double(double v) {
  const uint64_t b = q_bits(v);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return 0;  // zero or subnormal (< 2^-1022): rounds to 0
  const uint64_t mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = e - 1015;  // V = mant * 2^(e - 1075 + 60)
  uint64_t mag;
  if (sh >= 0) {
    mag = mant << sh;  // exact (sh <= 9 for |v| < 8)
  } else if (sh > -54) {
    mag = (mant + (1ull << (-sh - 1))) >> (-sh);
  } else {
    mag = 0;
  }
  return (b >> 63) ? -(int64_t)mag : (int64_t)mag;
}

// The same value as q60_from_double without branches, for kernels that decode
// many amplitudes per thread: with X = mant * 2^10 (< 2^63) and k = 1025 - e,
// V = (X + 2^(k-1)) >> k for k < 64 (X exactly for k = 0) and 0 for k >= 64
// (zero, subnormal or below 2^-62).  |v| must be < 8 (e <= 1025).
QS_HD int64_t q60_from_double_nb(double v) {
  const uint64_t b = q_bits(v);
  const int e = (int)((b >> 52) & 0x7ff);
  const uint64_t X = ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 10;
  const int k = 1025 - e;
  const int kk = k < 0 ? 0 : (k > 63 ? 63 : k);
  uint64_t mag = (X + ((1ull << kk) >> 1)) >> kk;
  mag = k > 63 ? 0 : mag;
  const uint64_t s = 0ull - (b >> 63);  // all ones when negative
  return (int64_t)((mag ^ s) - s);
}

// Exact 128-bit sums of products of Q60 values (the exact reductions): a value
// splits as v = h 2^31 + l with |l| <= 2^30, so for |v| < 2^61 also |h| <= 2^30,
// and x1 y1 + x2 y2 = A 2^62 + B 2^31 + C with |A| <= 2^61, |B| <= 2^62,
// |C| <= 2^61: three int64 column sums of 32 x 32 -> 64-bit products, combined
// modulo 2^128 (two's complement).
struct Sp {
  int32_t h, l;
};
QS_HD Sp split31(int64_t v) {
  const int64_t h = (v + (1ll << 30)) >> 31;
  return {(int32_t)h, (int32_t)(v - h * (1ll << 31))};
}
QS_HD Sp sp_neg(Sp v) { return {-v.h, -v.l}; }
QS_HD unsigned __int128 dot2_exact(Sp x1, Sp y1, Sp x2, Sp y2) {
  using u128 = unsigned __int128;
  const int64_t A = (int64_t)x1.h * y1.h + (int64_t)x2.h * y2.h;
  const int64_t B = (int64_t)x1.h * y1.l + (int64_t)x1.l * y1.h + (int64_t)x2.h * y2.l + (int64_t)x2.l * y2.h;
  const int64_t C = (int64_t)x1.l * y1.l + (int64_t)x2.l * y2.l;
  return ((u128)A << 62) + ((u128)B << 31) + (u128)C;
}

// Nearest double to V * 2^-60 (round half to even).  Integer operations only.
QS_HD double q60_to_double(int64_t V) {
  if (V == 0) return 0.0;
  const uint64_t sign = (uint64_t)V >> 63;
  uint64_t a = sign ? (uint64_t)0 - (uint64_t)V : (uint64_t)V;
  int msb = 63 - q_clz64(a);
  uint64_t mant;
  if (msb <= 52) {
    mant = a << (52 - msb);
  } else {
    const int sh = msb - 52;
    mant = a >> sh;
    const uint64_t rem = a & ((1ull << sh) - 1);
    const uint64_t half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (mant & 1))) {
      ++mant;
      if (mant == (1ull << 53)) {
        mant >>= 1;
        ++msb;
      }
    }
  }
  const uint64_t e = (uint64_t)(msb - 60 + 1023);
  return q_from_bits((sign << 63) | (e << 52) | (mant & 0xFFFFFFFFFFFFFull));
}

// The same value as q60_to_double without branches (|V| < 2^62): normalise |V|
// so that its leading one is bit 63, keep 53 bits rounded half to even, and
// place the exponent so that a carry of the mantissa into bit 53 raises it.
QS_HD double q60_to_double_nb(int64_t V) {
  const uint64_t s = (uint64_t)(V >> 63);
  const uint64_t a = ((uint64_t)V ^ s) - s;
  const int lz = q_clz64(a);  // 64 for a == 0
  const uint64_t x = a << (lz & 63);
  uint64_t mant = x >> 11;
  const uint32_t rem = (uint32_t)x & 0x7FFu;
  mant += (uint64_t)((rem > 0x400u) | ((rem == 0x400u) & ((uint32_t)mant & 1u)));
  // leading bit 63 - lz: biased exponent 1026 - lz, one of which the mantissa's
  // leading one supplies
  const uint64_t bits = ((uint64_t)(1025 - lz) << 52) + mant;
  return a ? q_from_bits((s << 63) | bits) : 0.0;
}

// Limb split V = h * 2^30 + l with 0 <= l < 2^30 (h = floor(V / 2^30)).
struct QL {
  int32_t h, l;
};

QS_HD QL q60_split(int64_t V) {
  return {(int32_t)(V >> 30), (int32_t)(V & ((1ll << 30) - 1))};
}

QS_HD int64_t madw(int32_t a, int32_t b, int64_t c) {
#ifdef __CUDA_ARCH__
  long long d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"((long long)c));
  return (int64_t)d;
#else
  return c + (int64_t)a * (int64_t)b;
#endif
}

// Accumulator pair of a sum of products (see the header comment).
struct QAcc {
  int64_t hi, mid;
};

QS_HD void qacc_add(QAcc& acc, QL u, QL a) {
  acc.hi = madw(u.h, a.h, acc.hi);
  acc.mid = madw(u.h, a.l, acc.mid);
  acc.mid = madw(u.l, a.h, acc.mid);
}

QS_HD int64_t qacc_result(const QAcc& acc) {
  return acc.hi + ((acc.mid + (1ll << 29)) >> 30);
}

// The same result with the rounding half (2^29 in mid units) added up front:
// start from qacc_new(), finish with qacc_round() (one shift and one add fewer
// per result; identical value, since integer addition is associative).
QS_HD QAcc qacc_new() { return {0, 1ll << 29}; }
QS_HD int64_t qacc_round(const QAcc& acc) { return acc.hi + (acc.mid >> 30); }

// Accumulator that keeps the low x low limb products too (exact up to the final
// rounding, no bias): for sums that are later added up over a whole state
// vector, such as inner products, where a dropped non-negative term per product
// would accumulate.
struct QAccF {
  int64_t hi, mid;
  uint64_t lo;
};

QS_HD void qaccf_add(QAccF& acc, QL u, QL a) {
  acc.hi = madw(u.h, a.h, acc.hi);
  acc.mid = madw(u.h, a.l, acc.mid);
  acc.mid = madw(u.l, a.h, acc.mid);
  acc.lo += (uint64_t)(uint32_t)u.l * (uint64_t)(uint32_t)a.l;  // < 2^60 per product
}

QS_HD int64_t qaccf_result(const QAccF& acc) {
  return acc.hi + ((acc.mid + (int64_t)(acc.lo >> 30) + (1ll << 29)) >> 30);
}

// A Q60 complex number as limbs, plus its negated imaginary part (so that
// re = ur*ar - ui*ai needs only additions).
struct QC {
  QL re, im, nim;
};

QS_HD QC qc_make(double re, double im) {
  QC c;
  c.re = q60_split(q60_from_double(re));
  c.im = q60_split(q60_from_double(im));
  c.nim = q60_split(-q60_from_double(im));
  return c;
}

// Gauss (three-multiplication) form of an entry c + i d, for the product
// (a + i b)(c + i d) = [c (a + b) - b (c + d)] + i [c (a + b) + a (d - c)]:
// re = c, im = d - c, nim = c + d, each from the Q60-rounded c and d, so the
// represented matrix is exactly the one qc_make() gives.  |c +- d| <= sqrt(2)|u|.
QS_HD QC qc_make_gauss(double re, double im) {
  const int64_t c = q60_from_double(re), d = q60_from_double(im);
  QC q;
  q.re = q60_split(c);
  q.im = q60_split(d - c);
  q.nim = q60_split(c + d);
  return q;
}

// One output of a general 2x2 complex row in Gauss form:
//   out = u0 (r0 + i i0) + u1 (r1 + i i1),  s_e = r_e + i_e (as Q60, split),
// u_e from qc_make_gauss().  Needs |s_e| < 2 (true for |amplitude| <= 1.25).
// Six limb products (18 wide multiply-adds) instead of eight.
QS_HD void q60_gauss_row(const QC& u0, const QC& u1, QL r0, QL i0, QL s0, QL r1, QL i1, QL s1, int64_t* re,
                         int64_t* im) {
  QAcc k1 = qacc_new(), k2{0, 0}, k3{0, 0};
  qacc_add(k1, u0.re, s0);
  qacc_add(k1, u1.re, s1);
  qacc_add(k2, u0.im, r0);
  qacc_add(k2, u1.im, r1);
  qacc_add(k3, u0.nim, i0);
  qacc_add(k3, u1.nim, i1);
  *re = qacc_round(QAcc{k1.hi - k3.hi, k1.mid - k3.mid});
  *im = qacc_round(QAcc{k1.hi + k2.hi, k1.mid + k2.mid});
}

// One complex product u * a in Gauss form (u from qc_make_gauss), a = r + i i,
// s = r + i (split): three limb products.
QS_HD void q60_gauss_mul(const QC& u, QL r, QL i, QL s, int64_t* re, int64_t* im) {
  QAcc k1 = qacc_new(), k2{0, 0}, k3{0, 0};
  qacc_add(k1, u.re, s);
  qacc_add(k2, u.im, r);
  qacc_add(k3, u.nim, i);
  *re = qacc_round(QAcc{k1.hi - k3.hi, k1.mid - k3.mid});
  *im = qacc_round(QAcc{k1.hi + k2.hi, k1.mid + k2.mid});
}

}  // namespace qs
