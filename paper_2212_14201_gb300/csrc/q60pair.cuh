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

// Host: the six limb pairs and the flags of R_b (x) R_a (a, b real orthogonal
// 2x2 matrices, row-major m[0..3]).
inline void q60_pair_coef(const double* ra, const double* rb, QL out[6], int* flags) {
  auto angle = [](const double* m, double* c, double* s) {
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
  };
  double ca, sa, cb, sb;
  const int fa = angle(ra, &ca, &sa), fb = angle(rb, &cb, &sb);
  *flags = fa | (fb << 1);
  const double pr = 0.5 * (ca * cb - sa * sb), pi = 0.5 * (sa * cb + ca * sb);
  const double qr = 0.5 * (ca * cb + sa * sb), qi = 0.5 * (sa * cb - ca * sb);
  const double v[6] = {pr, pi, -pi, qr, qi, -qi};
  for (int k = 0; k < 6; ++k) out[k] = q60_split(q60_from_double(v[k]));
}

}  // namespace qs
