// fl(x * x) for IEEE 754 binary64, round to nearest with ties to even, from
// integer operations.  The canonical sampler defines p_x = fl(fl(re^2) + fl(im^2))
// and its block totals as left-to-right sums; GB300's FP64 pipe runs at a small
// fraction of the integer pipes, so the two squares and their sum are formed here
// on the integer and multiply-add pipes (bit-identical to the FP64 operations),
// leaving the running sum to the FP64 pipe.
//
// With x = m 2^(e - 1075) (m the 53-bit significand with its leading one, e the
// biased exponent), x^2 = m^2 2^(2e - 2150), m^2 exactly in 106 bits.  Its leading
// one is bit 104 or 105 (top); the 53 bits from there down are the candidate
// significand, the next bit the round bit, everything below it the sticky bits.
// Rounding up happens when the round bit is set and either a sticky bit is set or
// the candidate is odd; a carry out of 53 bits renormalises.  The biased result
// exponent is 2e - 1023 + top (+ 1 after a carry).  Valid when the result is a
// normal number: biased e in 512..1533 (|x| in [2^-511, 2^511)), or x = +-0;
// *ok = false otherwise (the caller then takes the FP64 multiplication).
#pragma once

#include <stdint.h>

#include "fixed.h"

namespace qs {

QS_HD double sq_rn_int(double x, bool* ok) {
  const uint64_t b = q_bits(x) & 0x7FFFFFFFFFFFFFFFull;
  const int e = (int)(b >> 52);
  const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  uint64_t lo, hi;
#ifdef __CUDA_ARCH__
  lo = m * m;
  hi = __umul64hi(m, m);
#else
  const unsigned __int128 P = (unsigned __int128)m * m;
  lo = (uint64_t)P;
  hi = (uint64_t)(P >> 64);
#endif
  const int top = (int)((hi >> 41) & 1u);  // bit 105 of the product
  const int sh = 52 + top;                 // product bits below the kept 53
  uint64_t mant = (hi << (64 - sh)) | (lo >> sh);
  const uint64_t rbit = (lo >> (sh - 1)) & 1u;
  const uint64_t sticky = (lo & ((1ull << (sh - 1)) - 1u)) != 0 ? 1u : 0u;
  mant += rbit & (sticky | (mant & 1u));
  const int carry = (int)(mant >> 53);
  mant >>= carry;
  const uint64_t E = (uint64_t)(2 * e - 1023 + top + carry);
  *ok = (e >= 512 && e <= 1533) || b == 0;
  return b == 0 ? 0.0 : q_from_bits((E << 52) | (mant & 0xFFFFFFFFFFFFFull));
}

// fl(a + b) for IEEE 754 binary64 with a, b >= +0 (both normal or zero), round to
// nearest with ties to even, from integer operations.  With x >= y the larger and
// smaller operand (non-negative doubles order like their bit patterns), the
// significands carry 10 extra low bits; y's is shifted right by the exponent
// difference, the bits shifted out kept as one sticky bit; after the addition a
// carry out of bit 62 shifts the sum right once (its low bit joins the sticky
// bit).  The 53 bits from bit 62 down are the candidate, rounded up when the 10
// bits below exceed half, or equal half with a sticky bit or an odd candidate.
// *ok = false when an operand is negative, subnormal, not finite, or the result
// could overflow (the caller then takes the FP64 addition).
QS_HD double add_rn_pos_int(double a, double b, bool* ok) {
  const uint64_t ua = q_bits(a), ub = q_bits(b);
  const uint64_t x = ua > ub ? ua : ub, y = ua > ub ? ub : ua;
  const int ex = (int)(x >> 52), ey = (int)(y >> 52);
  *ok = (x >> 63) == 0 && (y >> 63) == 0 && (x == 0 || (ex >= 1 && ex <= 2045)) && (y == 0 || ey >= 1);
  const uint64_t MX = ((x & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 10;
  const uint64_t my = y == 0 ? 0 : (((y & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 10);
  const int d = ex - ey;
  uint64_t MY, sticky;
  if (d >= 64) {
    MY = 0;
    sticky = my != 0 ? 1u : 0u;
  } else {
    MY = my >> d;
    sticky = (d > 0 && (my & ((1ull << d) - 1u)) != 0) ? 1u : 0u;
  }
  uint64_t sum = MX + MY;  // < 2^64: both below 2^63
  const int c = (int)(sum >> 63);
  sticky |= sum & (uint64_t)c;
  sum >>= c;
  uint64_t mant = sum >> 10;
  const uint64_t rem = sum & 0x3FFu;
  const uint64_t up = (rem > 0x200u || (rem == 0x200u && (sticky | (mant & 1u)))) ? 1u : 0u;
  mant += up;
  const int c2 = (int)(mant >> 53);
  mant >>= c2;
  const uint64_t E = (uint64_t)(ex + c + c2);
  return x == 0 ? 0.0 : q_from_bits((E << 52) | (mant & 0xFFFFFFFFFFFFFull));
}

}  // namespace qs
