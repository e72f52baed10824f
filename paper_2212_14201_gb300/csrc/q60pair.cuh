// Two real one-qubit rotations on tile bits a and b, applied to an amplitude
// quad as two complex products (Q60 engine).
//
// On one real component, the quad (x00, x01, x10, x11) (index bit(a) + 2 bit(b))
// is two complex numbers z_b = x_b0 + i x_b1.  A rotation R_a = [[c, -s], [s, c]]
// multiplies each z_b by w_a = c + i s; R_b mixes z_0 and z_1 with real
// coefficients.  In the basis u = z_0 + i z_1, v = z_0 - i z_1 both act
// diagonally: R_b (x) R_a multiplies u by w_a w_b and v by w_a conj(w_b), and
// z_0 = (u + v) / 2, z_1 = -i (u - v) / 2.  With P = w_a w_b / 2 and
// Q = w_a conj(w_b) / 2 the quad costs 8 real products per component instead of
// the 16 of the 4x4 matrix.  (C[i] (x) C[j] with commuting i^2 = j^2 = -1 splits
// into two copies of C through the idempotents (1 +- ij) / 2.)
//
// A reflection F = [[c, s], [s, -c]] (a real orthogonal op with determinant -1)
// is R Z: the sign flip of its bit-1 half first, then the rotation; the flips are
// folded into the basis change (flag bit 0: a reflected, bit 1: b).
//
// Limb arithmetic (fixed.h): the basis change adds limb pairs, leaving redundant
// low limbs in (-2^31, 2^31) (a dropped low x low product then stays below 2 units
// of 2^-60); |u|, |v| <= sqrt(2) |quad component| <= 1.77 for a state of norm <=
// 1.25, so every high limb stays inside int32.  Each output carries at most about
// 10 units of 2^-60 of error.
#pragma once

#include <cmath>

#include "fixed.h"

namespace qs {

QS_HD QL ql_add(QL p, QL q) { return QL{p.h + q.h, p.l + q.l}; }
QS_HD QL ql_sub(QL p, QL q) { return QL{p.h - q.h, p.l - q.l}; }

// One component of the quad.  c: P.re, P.im, -P.im, Q.re, Q.im, -Q.im (limb pairs).
template <int FL>
QS_HD void q60_pair_comp(int64_t& x00, int64_t& x01, int64_t& x10, int64_t& x11,
                                              const QL* __restrict__ c) {
  const QL a00 = q60_split(x00), a01 = q60_split(x01), a10 = q60_split(x10), a11 = q60_split(x11);
  // with the reflections' sign flips s01 = sa, s10 = sb, s11 = sa sb:
  // u = (x00 - s11 x11) + i (s01 x01 + s10 x10), v = (x00 + s11 x11) + i (s01 x01 - s10 x10)
  QL ur, ui, vr, vi;
  if ((FL == 0) || (FL == 3)) {
    ur = ql_sub(a00, a11);
    vr = ql_add(a00, a11);
  } else {
    ur = ql_add(a00, a11);
    vr = ql_sub(a00, a11);
  }
  if (FL == 0) {
    ui = ql_add(a01, a10);
    vi = ql_sub(a01, a10);
  } else if (FL == 1) {  // -x01 + x10, -x01 - x10
    ui = ql_sub(a10, a01);
    vi = QL{-(a01.h + a10.h), -(a01.l + a10.l)};
  } else if (FL == 2) {  // x01 - x10, x01 + x10
    ui = ql_sub(a01, a10);
    vi = ql_add(a01, a10);
  } else {  // -x01 - x10, -x01 + x10
    ui = QL{-(a01.h + a10.h), -(a01.l + a10.l)};
    vi = ql_sub(a10, a01);
  }
  QAcc A = qacc_new(), B = qacc_new(), D = qacc_new(), E = qacc_new();
  qacc_add(A, c[0], ur);  // u'.re = P.re u.re - P.im u.im
  qacc_add(A, c[2], ui);
  qacc_add(B, c[1], ur);  // u'.im = P.im u.re + P.re u.im
  qacc_add(B, c[0], ui);
  qacc_add(D, c[3], vr);  // v'.re
  qacc_add(D, c[5], vi);
  qacc_add(E, c[4], vr);  // v'.im
  qacc_add(E, c[3], vi);
  const int64_t Ur = qacc_round(A), Ui = qacc_round(B), Vr = qacc_round(D), Vi = qacc_round(E);
  x00 = Ur + Vr;  // z_0 = u' + v'
  x01 = Ui + Vi;
  x10 = Ui - Vi;  // z_1 = -i (u' - v')
  x11 = Vr - Ur;
}

#ifdef __CUDACC__
template <int FL>
__device__ __forceinline__ void q60_pair_quad_t(longlong2& q0, longlong2& q1, longlong2& q2, longlong2& q3,
                                                const QL* __restrict__ c) {
  int64_t r0 = q0.x, r1 = q1.x, r2 = q2.x, r3 = q3.x;
  int64_t i0 = q0.y, i1 = q1.y, i2 = q2.y, i3 = q3.y;
  q60_pair_comp<FL>(r0, r1, r2, r3, c);
  q60_pair_comp<FL>(i0, i1, i2, i3, c);
  q0 = make_longlong2(r0, i0);
  q1 = make_longlong2(r1, i1);
  q2 = make_longlong2(r2, i2);
  q3 = make_longlong2(r3, i3);
}

// The quad (q0, q1, q2, q3) = indices bit(a) + 2 bit(b); flags as above.
__device__ __forceinline__ void q60_pair_quad(longlong2& q0, longlong2& q1, longlong2& q2, longlong2& q3,
                                              const QL* __restrict__ c, int flags) {
  switch (flags) {
    case 0: q60_pair_quad_t<0>(q0, q1, q2, q3, c); break;
    case 1: q60_pair_quad_t<1>(q0, q1, q2, q3, c); break;
    case 2: q60_pair_quad_t<2>(q0, q1, q2, q3, c); break;
    default: q60_pair_quad_t<3>(q0, q1, q2, q3, c); break;
  }
}
#endif

// Three real rotations on tile bits a, b, c, applied to an amplitude octet
// (index bit(a) + 2 bit(b) + 4 bit(c)) as four complex products.
//
// With z_cb = x_cb0 + i x_cb1, u_c = z_c0 + i z_c1, v_c = z_c0 - i z_c1 (the pair
// basis along b) and U+- = u_0 +- i u_1, V+- = v_0 +- i v_1 (the same along c),
// R_c (x) R_b (x) R_a multiplies U+ by w_a w_b w_c, U- by w_a w_b conj(w_c), V+ by
// w_a conj(w_b) w_c and V- by w_a conj(w_b) conj(w_c) (C (x) C (x) C splits into
// four copies of C).  The inverse is u_0 = (U+ + U-) / 2, u_1 = -i (U+ - U-) / 2,
// the same for v, then z_c0 = (u_c + v_c) / 2, z_c1 = -i (u_c - v_c) / 2; the 1/4
// goes into the four coefficients.  16 real products per octet and component,
// against 24 for a pair and a single rotation.
// |U+-|, |V+-| <= 2 |octet component| <= 2.5, so the products take the basis
// values split as h 2^31 + l (0 <= l < 2^31): U P / 2^60 = (2 Ph) h + (Ph l +
// (2 Pl) h) / 2^30, with Ph, Pl the 30-bit limbs of a coefficient (|P| <= 1/4).
struct Q3 {
  int32_t h2, h, l2;  // limbs of a coefficient for products with 31-bit-split values
};
QS_HD Q3 q3_of(QL p) { return Q3{p.h * 2, p.h, p.l * 2}; }
QS_HD Q3 q3_neg(Q3 p) { return Q3{-p.h2, -p.h, -p.l2}; }
QS_HD void q3_add(QAcc& A, Q3 p, int32_t yh, int32_t yl) {
  A.hi = madw(p.h2, yh, A.hi);
  A.mid = madw(p.h, yl, A.mid);
  A.mid = madw(p.l2, yh, A.mid);
}

// One component of the octet; P[k] = (re, im, -im) of coefficient k (U+, U-, V+, V-).
QS_HD void q60_triple_comp(int64_t (&x)[8], const Q3 (&P)[4][3]) {
  int64_t ur[2], ui[2], vr[2], vi[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int64_t z0r = x[4 * c], z0i = x[4 * c + 1], z1r = x[4 * c + 2], z1i = x[4 * c + 3];
    ur[c] = z0r - z1i;
    ui[c] = z0i + z1r;
    vr[c] = z0r + z1i;
    vi[c] = z0i - z1r;
  }
  const int64_t Y[8] = {ur[0] - ui[1], ui[0] + ur[1], ur[0] + ui[1], ui[0] - ur[1],
                        vr[0] - vi[1], vi[0] + vr[1], vr[0] + vi[1], vi[0] - vr[1]};
  int32_t yh[8], yl[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    yh[k] = (int32_t)(Y[k] >> 31);
    yl[k] = (int32_t)(Y[k] & 0x7FFFFFFF);
  }
  int64_t R[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    QAcc A = qacc_new(), B = qacc_new();
    q3_add(A, P[k][0], yh[2 * k], yl[2 * k]);  // re = P.re Y.re - P.im Y.im
    q3_add(A, P[k][2], yh[2 * k + 1], yl[2 * k + 1]);
    q3_add(B, P[k][1], yh[2 * k], yl[2 * k]);  // im = P.im Y.re + P.re Y.im
    q3_add(B, P[k][0], yh[2 * k + 1], yl[2 * k + 1]);
    R[2 * k] = qacc_round(A);
    R[2 * k + 1] = qacc_round(B);
  }
  const int64_t u0r = R[0] + R[2], u0i = R[1] + R[3], u1r = R[1] - R[3], u1i = R[2] - R[0];
  const int64_t v0r = R[4] + R[6], v0i = R[5] + R[7], v1r = R[5] - R[7], v1i = R[6] - R[4];
  x[0] = u0r + v0r;
  x[1] = u0i + v0i;
  x[2] = u0i - v0i;
  x[3] = v0r - u0r;
  x[4] = u1r + v1r;
  x[5] = u1i + v1i;
  x[6] = u1i - v1i;
  x[7] = v1r - u1r;
}

// The coefficients in the form the products take: P[k] = (re, im, -im) of
// coefficient k (U+, U-, V+, V-) as Q3 limbs, from (re, im) limb pairs.
QS_HD void q60_triple_q3(const QL* c, Q3 (&P)[4][3]) {
  for (int k = 0; k < 4; ++k) {
    P[k][0] = q3_of(c[2 * k]);
    P[k][1] = q3_of(c[2 * k + 1]);
    P[k][2] = q3_neg(P[k][1]);
  }
}

#ifdef __CUDACC__
// The octet v[0..7]; P: the Q3 coefficients; flags bit k: rotation k (a, b, c) is
// a reflection, whose sign flip of its bit-1 half comes first.
__device__ __forceinline__ void q60_triple_octet(longlong2 (&v)[8], const Q3 (&P)[4][3], int flags) {
  if (flags) {
#pragma unroll
    for (int k = 1; k < 8; ++k)
      if (__popc(k & flags) & 1) v[k] = make_longlong2(-v[k].x, -v[k].y);
  }
  int64_t r[8], im[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    r[k] = v[k].x;
    im[k] = v[k].y;
  }
  q60_triple_comp(r, P);
  q60_triple_comp(im, P);
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = make_longlong2(r[k], im[k]);
}
#endif

// Four real rotations on tile bits a, b, c, d, applied to ONE component of 16
// amplitudes x[k] (k = bit(a) + 2 bit(b) + 4 bit(c) + 8 bit(d)) as eight complex
// products.  The pairs along a are complex numbers z_j = x[2j] + i x[2j+1]
// (j = bit(b) + 2 bit(c) + 4 bit(d)); the basis change along each of b, c, d maps
// a pair (lo, hi) of complex values to (lo + i hi, lo - i hi), after which
// R_d (x) R_c (x) R_b (x) R_a multiplies channel j by w_a times, for each of b, c,
// d, its w or (when the channel's bit for it is set) conj(w) (C^(x)4 splits into
// eight copies of C).  The inverse maps (A, B) back to (A + B, -i (A - B)); its
// 1/8 is in the coefficients.  32 real products per 16 values of a component:
// two per value for four rotations, where triples spend two per value on three.
// Real and imaginary parts are independent under real rotations, so a thread
// can take one component of 16 amplitudes.
// Bounds: each channel is a signed sum of 8 of the 16 values, so by Cauchy-
// Schwarz |Y| <= sqrt(8) * 1.25 < 3.54 (< 2^61.83 in Q60 units) for a state of
// norm <= 1.25: the 31-bit split leaves |h| < 2^31; |P| <= 1/8 keeps the mid
// accumulator of two products of two limb pairs below 2^63.  Each output sums 8
// rounded products: at most 36 units of 2^-60 of error.
// The 24 coefficients come in three runs of 8 (P0, P1, P2: they sit in three
// consecutive op slots).
QS_HD Q3 q3_at(int i, const Q3* P0, const Q3* P1, const Q3* P2) {
  return i < 8 ? P0[i] : (i < 16 ? P1[i - 8] : P2[i - 16]);
}
QS_HD void q60_quad4_comp(int64_t (&x)[16], const Q3* P0, const Q3* P1, const Q3* P2) {
  int64_t zr[8], zi[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    zr[j] = x[2 * j];
    zi[j] = x[2 * j + 1];
  }
#pragma unroll
  for (int bit = 1; bit < 8; bit <<= 1)
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (!(j & bit)) {
        const int64_t lr = zr[j], li = zi[j], hr = zr[j | bit], hi = zi[j | bit];
        zr[j] = lr - hi;  // lo + i hi
        zi[j] = li + hr;
        zr[j | bit] = lr + hi;  // lo - i hi
        zi[j | bit] = li - hr;
      }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int32_t rh = (int32_t)(zr[k] >> 31), rl = (int32_t)(zr[k] & 0x7FFFFFFF);
    const int32_t ih = (int32_t)(zi[k] >> 31), il = (int32_t)(zi[k] & 0x7FFFFFFF);
    QAcc A = qacc_new(), B = qacc_new();
    const Q3 pr = q3_at(3 * k, P0, P1, P2), pi = q3_at(3 * k + 1, P0, P1, P2), pn = q3_at(3 * k + 2, P0, P1, P2);
    q3_add(A, pr, rh, rl);  // re = P.re Y.re - P.im Y.im
    q3_add(A, pn, ih, il);
    q3_add(B, pi, rh, rl);  // im = P.im Y.re + P.re Y.im
    q3_add(B, pr, ih, il);
    zr[k] = qacc_round(A);
    zi[k] = qacc_round(B);
  }
#pragma unroll
  for (int bit = 4; bit >= 1; bit >>= 1)
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (!(j & bit)) {
        const int64_t ar = zr[j], ai = zi[j], br = zr[j | bit], bi = zi[j | bit];
        zr[j] = ar + br;  // lo = A + B
        zi[j] = ai + bi;
        zr[j | bit] = ai - bi;  // hi = -i (A - B)
        zi[j | bit] = br - ar;
      }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    x[2 * j] = zr[j];
    x[2 * j + 1] = zi[j];
  }
}

// Host: rotation angle (c, s) of a real orthogonal 2x2 (row-major) and whether it
// is a reflection R Z.
inline int q60_orth_angle(const double* m, double* c, double* s) {
  const double det = m[0] * m[3] - m[1] * m[2];
  const double sg = det < 0.0 ? -1.0 : 1.0;
  double cc = 0.5 * (m[0] + sg * m[3]), ss = 0.5 * (m[2] - sg * m[1]);
  const double r = std::sqrt(cc * cc + ss * ss);
  if (r > 0.0) {
    cc /= r;
    ss /= r;
  } else {
    cc = 1.0;
    ss = 0.0;
  }
  *c = cc;
  *s = ss;
  return det < 0.0 ? 1 : 0;
}

// Host: the four coefficients (re, im limb pairs: U+, U-, V+, V-) and the flags
// of R_c (x) R_b (x) R_a.
inline void q60_triple_coef(const double* ra, const double* rb, const double* rc, QL out[8], int* flags) {
  double ca, sa, cb, sb, cc, sc;
  const int fa = q60_orth_angle(ra, &ca, &sa), fb = q60_orth_angle(rb, &cb, &sb), fc = q60_orth_angle(rc, &cc, &sc);
  *flags = fa | (fb << 1) | (fc << 2);
  // w_a w_b^(+-1) w_c^(+-1) / 4
  for (int k = 0; k < 4; ++k) {
    const double sbk = (k & 2) ? -sb : sb, sck = (k & 1) ? -sc : sc;
    const double abr = ca * cb - sa * sbk, abi = sa * cb + ca * sbk;
    const double re = 0.25 * (abr * cc - abi * sck), im = 0.25 * (abi * cc + abr * sck);
    out[2 * k] = q60_split(q60_from_double(re));
    out[2 * k + 1] = q60_split(q60_from_double(im));
  }
}

// Host: the eight coefficients of R_d (x) R_c (x) R_b (x) R_a for q60_quad4_comp
// as Q3 limbs (channel k: re, im, -im at P[3k..3k+2]) and the reflection flags
// (bit 0: a ... bit 3: d; a reflection's sign flip of its bit-1 half comes first).
inline void q60_quad4_coef(const double* ra, const double* rb, const double* rc, const double* rd, Q3 P[24],
                           int* flags) {
  double c[4], s[4];
  const double* r[4] = {ra, rb, rc, rd};
  *flags = 0;
  for (int q = 0; q < 4; ++q) *flags |= q60_orth_angle(r[q], &c[q], &s[q]) << q;
  for (int k = 0; k < 8; ++k) {
    double wr = c[0], wi = s[0];
    for (int q = 1; q < 4; ++q) {
      const double sq = ((k >> (q - 1)) & 1) ? -s[q] : s[q];
      const double tr = wr * c[q] - wi * sq, ti = wi * c[q] + wr * sq;
      wr = tr;
      wi = ti;
    }
    const QL re = q60_split(q60_from_double(0.125 * wr)), im = q60_split(q60_from_double(0.125 * wi));
    P[3 * k] = q3_of(re);
    P[3 * k + 1] = q3_of(im);
    P[3 * k + 2] = q3_neg(P[3 * k + 1]);
  }
}

// Host: the six limb pairs and the flags of R_b (x) R_a (a, b real orthogonal
// 2x2 matrices, row-major m[0..3]).
inline void q60_pair_coef(const double* ra, const double* rb, QL out[6], int* flags) {
  double ca, sa, cb, sb;
  const int fa = q60_orth_angle(ra, &ca, &sa), fb = q60_orth_angle(rb, &cb, &sb);
  *flags = fa | (fb << 1);
  const double pr = 0.5 * (ca * cb - sa * sb), pi = 0.5 * (sa * cb + ca * sb);
  const double qr = 0.5 * (ca * cb + sa * sb), qi = 0.5 * (sa * cb - ca * sb);
  const double v[6] = {pr, pi, -pi, qr, qi, -qi};
  for (int k = 0; k < 6; ++k) out[k] = q60_split(q60_from_double(v[k]));
}

}  // namespace qs
