// Tile-pass kernel.  A pass has a qubit set Q (m qubits, always containing the
// contiguous low run 0..L-1).  For each assignment r of the n-m qubits outside Q
// (a "tile"), the 2^m amplitudes x = deposit(r, ~Q) | deposit(j, Q) are loaded
// into shared memory (runs of 2^L contiguous amplitudes), every op of the pass is
// applied there in program order, and the tile is written back once.
//   - one-qubit ops on a tile qubit: pairs (j, j | 2^b) with the in-tile controls set;
//   - controls outside the tile are constant within a tile: the op is skipped for
//     tiles where one of them is 0;
//   - a diagonal op whose target lies outside the tile is a scalar for the tile.
// Gate matrices travel in the kernel parameters (constant bank).
// Two arithmetic engines share the structure: FP64 (tile of double2) and Q60
// fixed point (tile of int64 pairs, converted once on load and once on store).
#include <algorithm>
#include <type_traits>

#include "q60pair.cuh"
#include "tile.h"

namespace qs {

// Shared-memory swizzle of the tile: element j (16 or 8 bytes) lives at
// j ^ sw(j), where sw folds tile bits 3, 4, 5 into bits 0..2 with the vectors 7,
// 3, 5 (a linear map, so the physical index of a sum of disjoint bit sets is the
// XOR of theirs).  An op on tile bits B enumerates its pairs, quads or octets with
// consecutive threads on the lowest tile bits outside B; without the swizzle a
// quarter-warp hits one bank group as soon as B contains bits 0..2 (up to 8-way
// conflicts).  With these vectors every op on at most three tile bits has its
// lanes on at least four distinct bank groups (the best a 3-bit swizzle of bits
// 3..5 allows; 18 of the 299 such bit sets keep a 2-way conflict).
__device__ __forceinline__ uint32_t tsw_bits(uint32_t j) { return (0x3958f8u >> (3u * ((j >> 3) & 7u))) & 7u; }
__device__ __forceinline__ uint32_t tsw(uint32_t j) { return j ^ tsw_bits(j); }
// In a loop over i = threadIdx.x + k * THREADS (THREADS >= 64) whose element index
// j inserts zero bits into i, bits 3..5 of j come from the low bits of i, i.e. from
// threadIdx.x alone: the swizzle is one XOR with a per-thread constant.

// Insert zero bits at the set positions of `fixed` (ascending), then OR `set`.
__device__ __forceinline__ uint32_t tile_expand(uint32_t i, uint32_t fixed, uint32_t set) {
  while (fixed) {
    int f = __ffs(fixed) - 1;
    fixed &= fixed - 1;
    i = ((i >> f) << (f + 1)) | (i & ((1u << f) - 1));
  }
  return i | set;
}

// The sign mask of table t in the tile at `base`: amplitude j takes the sign
// (-1)^popc(j & S), S = XOR over the terms (q, t) with x_q = 1 of bit t (two terms
// on the same tile bit cancel when both of their outside qubits are set).
__device__ __forceinline__ uint32_t table_sign_mask(const TileArgs& g, int t, uint64_t base) {
  if (t >= TILE_MAX_SIGNED_TABLES) return 0;
  const TileSigns& sg = g.signs[t];
  uint32_t S = 0;
  for (int i = 0; i < sg.n; ++i)
    if ((base >> sg.q[i]) & 1ull) S ^= 1u << sg.t[i];
  return S;
}

// ---- FP64 engine -------------------------------------------------------------------
// a * T (Q60), T = c + i d from a phase table entry {c.h, c.l, d.h, d.l} (16 bytes),
// negated when neg: four limb products (direct form: fewer integer-pipe
// instructions than the three-product Gauss form, and 16 instead of 24 bytes a
// table entry from L2).
__device__ __forceinline__ longlong2 table_mul(const int4 e, longlong2 a, bool neg) {
  const int32_t m = neg ? -1 : 0;
  const QL c{(e.x ^ m) - m, (e.y ^ m) - m}, d{(e.z ^ m) - m, (e.w ^ m) - m}, nd{-d.h, -d.l};
  const QL ar = q60_split(a.x), ai = q60_split(a.y);
  QAcc re = qacc_new(), im = qacc_new();
  qacc_add(re, c, ar);
  qacc_add(re, nd, ai);
  qacc_add(im, d, ar);
  qacc_add(im, c, ai);
  return make_longlong2(qacc_round(re), qacc_round(im));
}

struct EngF64 {
  using T = double2;  // shared-memory element
  using G = double2;  // global element
  static constexpr int kMinBlocks = 3;  // CTAs per SM the register budget must allow (256 threads; 64 KiB tiles)
  static __device__ __forceinline__ double neg(double x) {
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
  }
  static __device__ __forceinline__ T load(const double2& a) { return a; }
  static __device__ __forceinline__ double2 store(const T& a) { return a; }
  static __device__ __forceinline__ T unit(T a, int code) {
    switch (code) {
      case U_ONE: return a;
      case U_I: return make_double2(neg(a.y), a.x);
      case U_MINUS_ONE: return make_double2(neg(a.x), neg(a.y));
      default: return make_double2(a.y, neg(a.x));
    }
  }
  static __device__ __forceinline__ T mul(T a, int code, const TileOp& op, int e) {
    if (code != U_GENERAL) return unit(a, code);
    const double2 u = op.m[e];
    return make_double2(fma(u.x, a.x, -u.y * a.y), fma(u.x, a.y, u.y * a.x));
  }
  static __device__ __forceinline__ void real2(const TileOp& op, T a0, T a1, T& b0, T& b1) {
    b0 = make_double2(fma(op.m[0].x, a0.x, op.m[1].x * a1.x), fma(op.m[0].x, a0.y, op.m[1].x * a1.y));
    b1 = make_double2(fma(op.m[2].x, a0.x, op.m[3].x * a1.x), fma(op.m[2].x, a0.y, op.m[3].x * a1.y));
  }
  static __device__ __forceinline__ void general2(const TileOp& op, T a0, T a1, T& b0, T& b1) {
    const double2 u0 = op.m[0], u1 = op.m[1], u2 = op.m[2], u3 = op.m[3];
    b0.x = fma(u0.x, a0.x, fma(-u0.y, a0.y, fma(u1.x, a1.x, -u1.y * a1.y)));
    b0.y = fma(u0.x, a0.y, fma(u0.y, a0.x, fma(u1.x, a1.y, u1.y * a1.x)));
    b1.x = fma(u2.x, a0.x, fma(-u2.y, a0.y, fma(u3.x, a1.x, -u3.y * a1.y)));
    b1.y = fma(u2.x, a0.y, fma(u2.y, a0.x, fma(u3.x, a1.y, u3.y * a1.x)));
  }
};

// ---- Q60 fixed-point engine ----------------------------------------------------------
struct EngQ60 {
  using T = longlong2;
  using G = double2;
  static constexpr int kMinBlocks = 3;  // 64 KiB tiles: three per SM; registers must not cut that
  static __device__ __forceinline__ T load(const double2& a) {
    return make_longlong2(q60_from_double_nb(a.x), q60_from_double_nb(a.y));
  }
  static __device__ __forceinline__ double2 store(const T& a) {
    return make_double2(q60_to_double_nb(a.x), q60_to_double_nb(a.y));
  }
  static __device__ __forceinline__ T unit(T a, int code) {
    switch (code) {
      case U_ONE: return a;
      case U_I: return make_longlong2(-a.y, a.x);
      case U_MINUS_ONE: return make_longlong2(-a.x, -a.y);
      default: return make_longlong2(a.y, -a.x);
    }
  }
  static __device__ __forceinline__ T mul(T a, int code, const TileOp& op, int e) {
    if (code != U_GENERAL) return unit(a, code);
    const QC& u = op.q[e];
    const QL ar = q60_split(a.x), ai = q60_split(a.y);
    QAcc re = qacc_new(), im = qacc_new();
    qacc_add(re, u.re, ar);
    qacc_add(re, u.nim, ai);
    qacc_add(im, u.re, ai);
    qacc_add(im, u.im, ar);
    return make_longlong2(qacc_round(re), qacc_round(im));
  }
  static __device__ __forceinline__ void real2(const TileOp& op, T a0, T a1, T& b0, T& b1) {
    const QL r0 = q60_split(a0.x), i0 = q60_split(a0.y), r1 = q60_split(a1.x), i1 = q60_split(a1.y);
    QAcc x = qacc_new(), y = qacc_new(), z = qacc_new(), w = qacc_new();
    qacc_add(x, op.q[0].re, r0);
    qacc_add(x, op.q[1].re, r1);
    qacc_add(y, op.q[0].re, i0);
    qacc_add(y, op.q[1].re, i1);
    qacc_add(z, op.q[2].re, r0);
    qacc_add(z, op.q[3].re, r1);
    qacc_add(w, op.q[2].re, i0);
    qacc_add(w, op.q[3].re, i1);
    b0 = make_longlong2(qacc_round(x), qacc_round(y));
    b1 = make_longlong2(qacc_round(z), qacc_round(w));
  }
  static __device__ __forceinline__ void general2(const TileOp& op, T a0, T a1, T& b0, T& b1) {
    const QL r0 = q60_split(a0.x), i0 = q60_split(a0.y), r1 = q60_split(a1.x), i1 = q60_split(a1.y);
    // Gauss form: K1 = sum c (a + b), K2 = sum a (d - c), K3 = sum b (c + d);
    // re = K1 - K3, im = K1 + K2 (three limb products per complex product)
    const QL s0 = q60_split(a0.x + a0.y), s1 = q60_split(a1.x + a1.y);
    int64_t re, im;
    q60_gauss_row(op.q[0], op.q[1], r0, i0, s0, r1, i1, s1, &re, &im);
    b0 = make_longlong2(re, im);
    q60_gauss_row(op.q[2], op.q[3], r0, i0, s0, r1, i1, s1, &re, &im);
    b1 = make_longlong2(re, im);
  }
};

// ---- FP32 engine (complex64 states) -------------------------------------------------
// The op's matrix arrives rounded to float by the host (no conversion on the FP64 pipe).
struct EngF32 {
  using T = float2;
  using G = float2;
  static constexpr int kMinBlocks = 4;  // 32 KiB tiles; four per SM leave the 16-amplitude register groups unspilled
  static __device__ __forceinline__ T load(const float2& a) { return a; }
  static __device__ __forceinline__ float2 store(const T& a) { return a; }
  static __device__ __forceinline__ float2 u(const TileOp& op, int e) { return op.f[e]; }
  static __device__ __forceinline__ T unit(T a, int code) {
    switch (code) {
      case U_ONE: return a;
      case U_I: return make_float2(-a.y, a.x);
      case U_MINUS_ONE: return make_float2(-a.x, -a.y);
      default: return make_float2(a.y, -a.x);
    }
  }
  static __device__ __forceinline__ T mul(T a, int code, const TileOp& op, int e) {
    if (code != U_GENERAL) return unit(a, code);
    const float2 w = u(op, e);
    return make_float2(fmaf(w.x, a.x, -w.y * a.y), fmaf(w.x, a.y, w.y * a.x));
  }
  static __device__ __forceinline__ void real2(const TileOp& op, T a0, T a1, T& b0, T& b1) {
    const float m0 = op.f[0].x, m1 = op.f[1].x, m2 = op.f[2].x, m3 = op.f[3].x;
    b0 = make_float2(fmaf(m0, a0.x, m1 * a1.x), fmaf(m0, a0.y, m1 * a1.y));
    b1 = make_float2(fmaf(m2, a0.x, m3 * a1.x), fmaf(m2, a0.y, m3 * a1.y));
  }
  static __device__ __forceinline__ void general2(const TileOp& op, T a0, T a1, T& b0, T& b1) {
    const float2 u0 = u(op, 0), u1 = u(op, 1), u2 = u(op, 2), u3 = u(op, 3);
    b0.x = fmaf(u0.x, a0.x, fmaf(-u0.y, a0.y, fmaf(u1.x, a1.x, -u1.y * a1.y)));
    b0.y = fmaf(u0.x, a0.y, fmaf(u0.y, a0.x, fmaf(u1.x, a1.y, u1.y * a1.x)));
    b1.x = fmaf(u2.x, a0.x, fmaf(-u2.y, a0.y, fmaf(u3.x, a1.x, -u3.y * a1.y)));
    b1.y = fmaf(u2.x, a0.y, fmaf(u2.y, a0.x, fmaf(u3.x, a1.y, u3.y * a1.x)));
  }
};

// All pairs (j, j | tb) of one op in the tile, the op class fixed at compile time;
// unrolled so that a thread has several independent pairs in flight.
template <class E, int KIND, int THREADS>
__device__ __forceinline__ void pair_loop(typename E::T* tile, uint32_t cnt, uint32_t fixed, uint32_t lcm, uint32_t tb,
                                          const TileOp& op) {
  using T = typename E::T;
  const uint32_t tbp = tsw(tb);
  const uint32_t csw = tsw_bits(lcm ? tile_expand(threadIdx.x, fixed, lcm) : threadIdx.x + (threadIdx.x & ~(tb - 1)));
#pragma unroll 4
  for (uint32_t i = threadIdx.x; i < cnt; i += THREADS) {
    // without in-tile controls the insertion of one zero bit is a mask and an add
    const uint32_t j0 = (lcm ? tile_expand(i, fixed, lcm) : i + (i & ~(tb - 1))) ^ csw, j1 = j0 ^ tbp;
    const T a0 = tile[j0], a1 = tile[j1];
    T b0, b1;
    if (KIND == TOP_DIAG) {
      b0 = E::mul(a0, op.code0, op, 0);
      b1 = E::mul(a1, op.code1, op, 3);
    } else if (KIND == TOP_ANTI) {
      b0 = E::mul(a1, op.code0, op, 1);
      b1 = E::mul(a0, op.code1, op, 2);
    } else if (KIND == TOP_REAL) {
      E::real2(op, a0, a1, b0, b1);
    } else {
      E::general2(op, a0, a1, b0, b1);
    }
    tile[j0] = b0;
    tile[j1] = b1;
  }
}

// Two real rotations on tile bits a and b on the quads (j, j|a, j|b, j|a|b), as
// two complex products per quad and component (q60pair.cuh): 48 wide
// multiply-adds per quad where the 4x4 matrix takes 96.  With a phase table
// (tab != nullptr, the table op just before the pair): every amplitude of the
// quad is first multiplied by its table entry, which saves the table op's own
// shared-memory round trip, index arithmetic and barrier.
template <int THREADS>
__device__ __forceinline__ void quad_real(longlong2* tile, uint32_t TS, uint32_t ta, uint32_t tbb, const QL* m0,
                                          int flags, const int4* tab, uint32_t S) {
  const uint32_t lo = min(ta, tbb), hi = max(ta, tbb);
  const uint32_t pa = tsw(ta), pb = tsw(tbb);
  uint32_t csw;
  {
    uint32_t j = threadIdx.x + (threadIdx.x & ~(lo - 1));
    csw = tsw_bits(j + (j & ~(hi - 1)));
  }
  const uint32_t cnt = TS >> 2;
#pragma unroll 2
  for (uint32_t i = threadIdx.x; i < cnt; i += THREADS) {
    uint32_t j = i + (i & ~(lo - 1));  // insert a zero bit at lo, then at hi
    j = j + (j & ~(hi - 1));
    const uint32_t jj[4] = {j, j | ta, j | tbb, j | ta | tbb};
    const uint32_t pj = j ^ csw;
    const uint32_t pp[4] = {pj, pj ^ pa, pj ^ pb, pj ^ pa ^ pb};
    longlong2 v[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      v[c] = tile[pp[c]];
      if (tab) v[c] = table_mul(__ldg(tab + jj[c]), v[c], __popc(jj[c] & S) & 1);
    }
    q60_pair_quad(v[0], v[1], v[2], v[3], m0, flags);
#pragma unroll
    for (int c = 0; c < 4; ++c) tile[pp[c]] = v[c];
  }
}

// Three real rotations on tile bits ta, tb, tc on the octets (index bit(ta) +
// 2 bit(tb) + 4 bit(tc)) as four complex products per octet and component
// (q60pair.cuh): 16 real products per octet and component where a pair and a
// single rotation take 24.  With a phase table, as in quad_real.
template <int THREADS>
__device__ __forceinline__ void octet_real(longlong2* tile, uint32_t TS, uint32_t ta, uint32_t tb, uint32_t tc,
                                           const Q3 (&P)[4][3], int flags, const int4* tab, uint32_t S) {
  const uint32_t p0 = min(ta, min(tb, tc)), p2 = max(ta, max(tb, tc));
  const uint32_t p1 = (ta | tb | tc) & ~(p0 | p2);
  const uint32_t pa = tsw(ta), pb = tsw(tb), pc = tsw(tc);
  uint32_t csw;
  {
    uint32_t j = threadIdx.x + (threadIdx.x & ~(p0 - 1));
    j = j + (j & ~(p1 - 1));
    csw = tsw_bits(j + (j & ~(p2 - 1)));
  }
  const uint32_t cnt = TS >> 3;
  for (uint32_t i = threadIdx.x; i < cnt; i += THREADS) {
    uint32_t j = i + (i & ~(p0 - 1));  // insert zero bits at p0 < p1 < p2
    j = j + (j & ~(p1 - 1));
    j = j + (j & ~(p2 - 1));
    uint32_t jj[8], pp[8];
    const uint32_t pj = j ^ csw;
    longlong2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      jj[k] = j | ((k & 1) ? ta : 0u) | ((k & 2) ? tb : 0u) | ((k & 4) ? tc : 0u);
      pp[k] = pj ^ ((k & 1) ? pa : 0u) ^ ((k & 2) ? pb : 0u) ^ ((k & 4) ? pc : 0u);
      v[k] = tile[pp[k]];
      if (tab) v[k] = table_mul(__ldg(tab + jj[k]), v[k], __popc(jj[k] & S) & 1);
    }
    q60_triple_octet(v, P, flags);
#pragma unroll
    for (int k = 0; k < 8; ++k) tile[pp[k]] = v[k];
  }
}

// Four real rotations on tile bits ta < ... (any order) on one component of 16
// amplitudes per work item: item t takes group t >> 1 and component t & 1, so the
// two lanes of a pair read the two halves of the same 16-byte amplitudes.
template <int THREADS>
__device__ __forceinline__ void quad4_real(longlong2* tile, uint32_t TS, uint32_t ta, uint32_t tb, uint32_t tc,
                                           uint32_t td, const Q3* P0, const Q3* P1, const Q3* P2, int flags) {
  const uint32_t all = ta | tb | tc | td;
  uint32_t p[4], rest = all;
#pragma unroll
  for (int e = 0; e < 4; ++e) {  // the four bits in ascending order
    p[e] = rest & (0u - rest);
    rest ^= p[e];
  }
  const uint32_t pa = tsw(ta), pb = tsw(tb), pc = tsw(tc), pd = tsw(td);
  const uint32_t grp0 = threadIdx.x >> 1;
  uint32_t csw;
  {
    uint32_t j = grp0;
#pragma unroll
    for (int e = 0; e < 4; ++e) j = j + (j & ~(p[e] - 1));
    csw = tsw_bits(j);
  }
  int64_t* comp = reinterpret_cast<int64_t*>(tile) + (threadIdx.x & 1);
  const uint32_t cnt = TS >> 4;
  for (uint32_t g = grp0; g < cnt; g += THREADS / 2) {
    uint32_t j = g;
#pragma unroll
    for (int e = 0; e < 4; ++e) j = j + (j & ~(p[e] - 1));  // insert zero bits at p[0] < ... < p[3]
    const uint32_t pj = j ^ csw;
    uint32_t pp[16];
    int64_t x[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      pp[k] = pj ^ ((k & 1) ? pa : 0u) ^ ((k & 2) ? pb : 0u) ^ ((k & 4) ? pc : 0u) ^ ((k & 8) ? pd : 0u);
      x[k] = comp[2 * pp[k]];
    }
    if (flags) {
#pragma unroll
      for (int k = 1; k < 16; ++k)
        if (__popc(k & flags) & 1) x[k] = -x[k];
    }
    q60_quad4_comp(x, P0, P1, P2);
#pragma unroll
    for (int k = 0; k < 16; ++k) comp[2 * pp[k]] = x[k];
  }
}

// The same two ops for the FP32 engine (complex64 states): a real 4x4 on quads with
// its 16 entries as floats in f[] of the op's two slots, optionally after a phase
// table of float2 entries (one per amplitude of the tile).
template <int THREADS>
__device__ __forceinline__ void quad_real_f32(float2* tile, uint32_t TS, uint32_t ta, uint32_t tbb, const float* m0,
                                              const float* m1, const float2* tab, uint32_t S) {
  const uint32_t lo = min(ta, tbb), hi = max(ta, tbb);
  const uint32_t pa = tsw(ta), pb = tsw(tbb);
  uint32_t csw;
  {
    uint32_t j = threadIdx.x + (threadIdx.x & ~(lo - 1));
    csw = tsw_bits(j + (j & ~(hi - 1)));
  }
  const uint32_t cnt = TS >> 2;
#pragma unroll 2
  for (uint32_t i = threadIdx.x; i < cnt; i += THREADS) {
    uint32_t j = i + (i & ~(lo - 1));
    j = j + (j & ~(hi - 1));
    const uint32_t jj[4] = {j, j | ta, j | tbb, j | ta | tbb};
    const uint32_t pj = j ^ csw;
    const uint32_t pp[4] = {pj, pj ^ pa, pj ^ pb, pj ^ pa ^ pb};
    float2 v[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      v[c] = tile[pp[c]];
      if (tab) {
        float2 u = __ldg(tab + jj[c]);
        if (__popc(jj[c] & S) & 1) u = make_float2(-u.x, -u.y);
        v[c] = make_float2(fmaf(u.x, v[c].x, -u.y * v[c].y), fmaf(u.x, v[c].y, u.y * v[c].x));
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float xr = 0.0f, xi = 0.0f;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int e = 4 * k + c;
        const float u = e < 8 ? m0[e] : m1[e - 8];
        xr = fmaf(u, v[c].x, xr);
        xi = fmaf(u, v[c].y, xi);
      }
      tile[pp[k]] = make_float2(xr, xi);
    }
  }
}

// FP32 engine: four real rotations (row-major 2x2 each, r[4q..4q+3] for bits a, b,
// c, d) on groups of 16 amplitudes held in registers, one after another, after an
// optional phase table: one shared-memory round trip for up to five ops.
template <int THREADS>
__device__ __forceinline__ void quad4_f32(float2* tile, uint32_t TS, uint32_t ta, uint32_t tb, uint32_t tc,
                                          uint32_t td, const float* r, const float2* tab, uint32_t S) {
  const uint32_t all = ta | tb | tc | td;
  uint32_t p[4], rest = all;
#pragma unroll
  for (int e = 0; e < 4; ++e) {  // the four bits in ascending order
    p[e] = rest & (0u - rest);
    rest ^= p[e];
  }
  const uint32_t pa = tsw(ta), pb = tsw(tb), pc = tsw(tc), pd = tsw(td);
  uint32_t csw;
  {
    uint32_t j = threadIdx.x;
#pragma unroll
    for (int e = 0; e < 4; ++e) j = j + (j & ~(p[e] - 1));
    csw = tsw_bits(j);
  }
  const uint32_t cnt = TS >> 4;
  for (uint32_t g = threadIdx.x; g < cnt; g += THREADS) {
    uint32_t j = g;
#pragma unroll
    for (int e = 0; e < 4; ++e) j = j + (j & ~(p[e] - 1));  // insert zero bits at p[0] < ... < p[3]
    const uint32_t pj = j ^ csw;
    auto slot = [&](int k) {
      return pj ^ ((k & 1) ? pa : 0u) ^ ((k & 2) ? pb : 0u) ^ ((k & 4) ? pc : 0u) ^ ((k & 8) ? pd : 0u);
    };
    float2 v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      v[k] = tile[slot(k)];
      if (tab) {
        const uint32_t jk = j | ((k & 1) ? ta : 0u) | ((k & 2) ? tb : 0u) | ((k & 4) ? tc : 0u) | ((k & 8) ? td : 0u);
        float2 u = __ldg(tab + jk);
        if (__popc(jk & S) & 1) u = make_float2(-u.x, -u.y);
        v[k] = make_float2(fmaf(u.x, v[k].x, -u.y * v[k].y), fmaf(u.x, v[k].y, u.y * v[k].x));
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float m00 = r[4 * q], m01 = r[4 * q + 1], m10 = r[4 * q + 2], m11 = r[4 * q + 3];
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (!(k & (1 << q))) {
          const float2 x0 = v[k], x1 = v[k | (1 << q)];
          v[k] = make_float2(fmaf(m01, x1.x, m00 * x0.x), fmaf(m01, x1.y, m00 * x0.y));
          v[k | (1 << q)] = make_float2(fmaf(m11, x1.x, m10 * x0.x), fmaf(m11, x1.y, m10 * x0.y));
        }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) tile[slot(k)] = v[k];
  }
}

// Loads a tile into shared memory with eight global loads in flight per thread
// before their shared-memory stores (thread t takes j = t, t + THREADS, ...; the
// swizzle tsq depends only on bits the stride keeps).
template <int THREADS, class T, class S, class F>
__device__ __forceinline__ void load_tile(T* tile, const S* src, uint64_t base, const uint64_t* offs, int L,
                                          uint32_t lowmask, uint32_t TS, uint32_t tsq, F conv) {
  constexpr uint32_t U = 8;
  uint32_t j = threadIdx.x;
  for (; j + (U - 1) * THREADS < TS; j += U * THREADS) {
    S v[U];
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) {
      const uint32_t jj = j + u * THREADS;
      v[u] = src[base + offs[jj >> L] + (jj & lowmask)];
    }
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) tile[(j + u * THREADS) ^ tsq] = conv(v[u]);
  }
  for (; j < TS; j += THREADS) tile[j ^ tsq] = conv(src[base + offs[j >> L] + (j & lowmask)]);
}

// The same load with a phase table applied on the way in (the pass's first op):
// element j is multiplied by tab[j], negated where popc(j & S) is odd; four loads
// in flight (the table entries take the other registers).
template <int THREADS, class S, class F>
__device__ __forceinline__ void load_tile_table(longlong2* tile, const S* src, uint64_t base, const uint64_t* offs,
                                                int L, uint32_t lowmask, uint32_t TS, uint32_t tsq, F conv,
                                                const int4* tab, uint32_t Sg) {
  constexpr uint32_t U = 4;
  uint32_t j = threadIdx.x;
  for (; j + (U - 1) * THREADS < TS; j += U * THREADS) {
    S v[U];
    int4 e[U];
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) {
      const uint32_t jj = j + u * THREADS;
      v[u] = src[base + offs[jj >> L] + (jj & lowmask)];
      e[u] = __ldg(tab + jj);
    }
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) {
      const uint32_t jj = j + u * THREADS;
      tile[jj ^ tsq] = table_mul(e[u], conv(v[u]), __popc(jj & Sg) & 1);
    }
  }
  for (; j < TS; j += THREADS)
    tile[j ^ tsq] = table_mul(__ldg(tab + j), conv(src[base + offs[j >> L] + (j & lowmask)]), __popc(j & Sg) & 1);
}

// Stores a tile the same way, eight shared-memory reads before their global stores.
template <int THREADS, class T, class D, class F>
__device__ __forceinline__ void store_tile(const T* tile, D* dst, uint64_t base, const uint64_t* offs, int L,
                                           uint32_t lowmask, uint32_t TS, uint32_t tsq, F conv) {
  constexpr uint32_t U = 8;
  uint32_t j = threadIdx.x;
  for (; j + (U - 1) * THREADS < TS; j += U * THREADS) {
    T v[U];
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) v[u] = tile[(j + u * THREADS) ^ tsq];
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) {
      const uint32_t jj = j + u * THREADS;
      dst[base + offs[jj >> L] + (jj & lowmask)] = conv(v[u]);
    }
  }
  for (; j < TS; j += THREADS) dst[base + offs[j >> L] + (j & lowmask)] = conv(tile[j ^ tsq]);
}

// The same store with a phase table applied on the way out (the pass's last op).
template <int THREADS, class D, class F>
__device__ __forceinline__ void store_tile_table(const longlong2* tile, D* dst, uint64_t base, const uint64_t* offs,
                                                 int L, uint32_t lowmask, uint32_t TS, uint32_t tsq, F conv,
                                                 const int4* tab, uint32_t Sg) {
  constexpr uint32_t U = 4;
  uint32_t j = threadIdx.x;
  for (; j + (U - 1) * THREADS < TS; j += U * THREADS) {
    longlong2 v[U];
    int4 e[U];
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) {
      v[u] = tile[(j + u * THREADS) ^ tsq];
      e[u] = __ldg(tab + j + u * THREADS);
    }
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) {
      const uint32_t jj = j + u * THREADS;
      dst[base + offs[jj >> L] + (jj & lowmask)] = conv(table_mul(e[u], v[u], __popc(jj & Sg) & 1));
    }
  }
  for (; j < TS; j += THREADS)
    dst[base + offs[j >> L] + (j & lowmask)] = conv(table_mul(__ldg(tab + j), tile[j ^ tsq], __popc(j & Sg) & 1));
}

template <class E, int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS == 256 ? E::kMinBlocks : 1) k_tile(typename E::G* __restrict__ a, const __grid_constant__ TileArgs g) {
  using T = typename E::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = g.m;
  const int L = m - g.nhigh;
  const uint32_t TS = 1u << m;
  const uint32_t H = 1u << g.nhigh;
  uint64_t* offs = reinterpret_cast<uint64_t*>(smem_raw);  // [H] offsets of the high tile bits
  T* tile = reinterpret_cast<T*>(smem_raw + ((H * sizeof(uint64_t) + 15) & ~(size_t)15));
  for (uint32_t h = threadIdx.x; h < H; h += THREADS) {
    uint64_t o = 0;
    for (int b = 0; b < g.nhigh; ++b) o |= (uint64_t)((h >> b) & 1u) << g.qhigh[b];
    offs[h] = o;
  }
  const uint32_t lowmask = (1u << L) - 1;
  const uint32_t tsq = tsw_bits(threadIdx.x);  // swizzle of the sequential loops over j
  for (uint64_t r = blockIdx.x; r < g.ntiles; r += gridDim.x) {
    uint64_t base = 0;
    for (int b = 0; b < g.nout; ++b) base |= ((r >> b) & 1ull) << g.outpos[b];
    __syncthreads();  // offs ready / previous tile stored
    auto conv = [](const typename E::G& v) { return E::load(v); };
    if constexpr (std::is_same<E, EngQ60>::value) {
      const int lt = ((g.io >> 8) & 255) - 1;  // a phase table applied on load
      if (lt >= 0) {
        const int4* tab = reinterpret_cast<const int4*>(g.tables) + (size_t)lt * TS;
        const uint32_t Sg = table_sign_mask(g, lt, base);
        if (g.io & 1)
          load_tile_table<THREADS>(tile, reinterpret_cast<const longlong2*>(a), base, offs, L, lowmask, TS, tsq,
                                   [](const longlong2& v) { return v; }, tab, Sg);
        else
          load_tile_table<THREADS>(tile, a, base, offs, L, lowmask, TS, tsq, conv, tab, Sg);
      } else if (g.io & 1) {
        load_tile<THREADS>(tile, reinterpret_cast<const longlong2*>(a), base, offs, L, lowmask, TS, tsq,
                           [](const longlong2& v) { return v; });
      } else {
        load_tile<THREADS>(tile, a, base, offs, L, lowmask, TS, tsq, conv);
      }
    } else {
      load_tile<THREADS>(tile, a, base, offs, L, lowmask, TS, tsq, conv);
    }
    __syncthreads();
    for (int k = 0; k < g.nops; ++k) {
      const TileOp& op = g.ops[k];
      if ((base & op.ext_cmask) != op.ext_cmask) continue;  // uniform across the CTA
      const uint32_t lcm = op.lcmask;
      if constexpr (std::is_same<E, EngF32>::value) {
        if (op.kind == TOP_DTABLE) {
          const float2* tf = reinterpret_cast<const float2*>(g.tables) + (size_t)lcm * TS;
          const uint32_t S = table_sign_mask(g, (int)lcm, base);
#pragma unroll 8
          for (uint32_t j = threadIdx.x; j < TS; j += THREADS) {
            float2 u = __ldg(tf + j);
            const float2 v = tile[j ^ tsq];
            if (__popc(j & S) & 1) u = make_float2(-u.x, -u.y);
            tile[j ^ tsq] = make_float2(fmaf(u.x, v.x, -u.y * v.y), fmaf(u.x, v.y, u.y * v.x));
          }
          __syncthreads();
          continue;
        }
        if (op.kind == TOP_REAL4) {
          const float2* tab =
              op.code1 >= 0 ? reinterpret_cast<const float2*>(g.tables) + (size_t)op.code1 * TS : nullptr;
          quad4_f32<THREADS>(tile, TS, 1u << op.tb, 1u << op.code0, 1u << ((op.lcmask >> 8) & 31),
                             1u << ((op.lcmask >> 16) & 31), reinterpret_cast<const float*>(op.q), tab,
                             op.code1 >= 0 ? table_sign_mask(g, op.code1, base) : 0u);
          __syncthreads();
          continue;
        }
        if (op.kind == TOP_REAL2) {
          const float2* tab =
              op.code1 >= 0 ? reinterpret_cast<const float2*>(g.tables) + (size_t)op.code1 * TS : nullptr;
          quad_real_f32<THREADS>(tile, TS, 1u << op.tb, 1u << op.code0, reinterpret_cast<const float*>(op.f),
                                 reinterpret_cast<const float*>(g.ops[k + 1].f), tab,
                                 op.code1 >= 0 ? table_sign_mask(g, op.code1, base) : 0u);
          ++k;  // the continuation slot
          __syncthreads();
          continue;
        }
      }
      if constexpr (std::is_same<E, EngQ60>::value) {
        if (op.kind == TOP_DTABLE) {
          // one table entry per amplitude, read through the read-only path (every
          // tile reads the same table: it stays in L2)
          const int4* tab = reinterpret_cast<const int4*>(g.tables) + (size_t)lcm * TS;
          const uint32_t S = table_sign_mask(g, (int)lcm, base);
#pragma unroll 8
          for (uint32_t j = threadIdx.x; j < TS; j += THREADS)
            tile[j ^ tsq] = table_mul(__ldg(tab + j), tile[j ^ tsq], __popc(j & S) & 1);
          __syncthreads();
          continue;
        }
        if (op.kind == TOP_REAL4) {
          // 24 Q3 coefficients: 8 in q[] of this slot and of each of the next two
          quad4_real<THREADS>(tile, TS, 1u << op.tb, 1u << op.code0, 1u << ((op.lcmask >> 8) & 31),
                              1u << ((op.lcmask >> 16) & 31), reinterpret_cast<const Q3*>(op.q),
                              reinterpret_cast<const Q3*>(g.ops[k + 1].q), reinterpret_cast<const Q3*>(g.ops[k + 2].q),
                              (int)(op.lcmask & 15));
          k += 2;  // the continuation slots
          __syncthreads();
          continue;
        }
        if (op.kind == TOP_REAL3) {
          const int4* tab = op.code1 >= 0 ? reinterpret_cast<const int4*>(g.tables) + (size_t)op.code1 * TS : nullptr;
          // 12 Q3 coefficients: 8 in this slot's q[] (96 bytes), 4 in the next slot's
          const Q3* pq0 = reinterpret_cast<const Q3*>(op.q);
          const Q3* pq1 = reinterpret_cast<const Q3*>(g.ops[k + 1].q);
          Q3 P[4][3];
#pragma unroll
          for (int e = 0; e < 12; ++e) P[e / 3][e % 3] = e < 8 ? pq0[e] : pq1[e - 8];
          if (tab)
            octet_real<THREADS>(tile, TS, 1u << op.tb, 1u << op.code0, 1u << (op.lcmask >> 8), P,
                                (int)(op.lcmask & 7), tab, table_sign_mask(g, op.code1, base));
          else
            octet_real<THREADS>(tile, TS, 1u << op.tb, 1u << op.code0, 1u << (op.lcmask >> 8), P,
                                (int)(op.lcmask & 7), nullptr, 0u);
          ++k;  // the continuation slot
          __syncthreads();
          continue;
        }
        if (op.kind == TOP_REAL2) {
          const int4* tab = op.code1 >= 0 ? reinterpret_cast<const int4*>(g.tables) + (size_t)op.code1 * TS : nullptr;
          if (tab)
            quad_real<THREADS>(tile, TS, 1u << op.tb, 1u << op.code0, reinterpret_cast<const QL*>(op.q),
                               (int)op.lcmask, tab, table_sign_mask(g, op.code1, base));
          else
            quad_real<THREADS>(tile, TS, 1u << op.tb, 1u << op.code0, reinterpret_cast<const QL*>(op.q),
                               (int)op.lcmask, nullptr, 0u);
          ++k;  // the continuation slot
          __syncthreads();
          continue;
        }
      }
      if (op.kind == TOP_SCALAR) {
        const bool one = (base >> op.tb) & 1ull;
        const int code = one ? op.code1 : op.code0;
        if (code == U_ONE) continue;
        const int e = one ? 3 : 0;
        const uint32_t cnt = TS >> __popc(lcm);
        for (uint32_t i = threadIdx.x; i < cnt; i += THREADS) {
          const uint32_t j = tsw(tile_expand(i, lcm, lcm));
          tile[j] = E::mul(tile[j], code, op, e);
        }
      } else {
        const uint32_t tb = 1u << op.tb;
        const uint32_t fixed = lcm | tb;
        const uint32_t cnt = TS >> __popc(fixed);
        if (op.kind == TOP_PHASE1) {
          for (uint32_t i = threadIdx.x; i < cnt; i += THREADS) {
            const uint32_t j = tsw(tile_expand(i, fixed, lcm) | tb);
            tile[j] = E::mul(tile[j], op.code1, op, 3);
          }
        } else if (op.kind == TOP_GENERAL) {
          pair_loop<E, TOP_GENERAL, THREADS>(tile, cnt, fixed, lcm, tb, op);
        } else if (op.kind == TOP_REAL) {
          pair_loop<E, TOP_REAL, THREADS>(tile, cnt, fixed, lcm, tb, op);
        } else if (op.kind == TOP_ANTI) {
          pair_loop<E, TOP_ANTI, THREADS>(tile, cnt, fixed, lcm, tb, op);
        } else {
          pair_loop<E, TOP_DIAG, THREADS>(tile, cnt, fixed, lcm, tb, op);
        }
      }
      __syncthreads();
    }
    if constexpr (std::is_same<E, EngQ60>::value) {
      const int st = ((g.io >> 16) & 255) - 1;  // a phase table applied on store
      if (st >= 0) {
        const int4* tab = reinterpret_cast<const int4*>(g.tables) + (size_t)st * TS;
        const uint32_t Sg = table_sign_mask(g, st, base);
        if (g.io & 2)
          store_tile_table<THREADS>(tile, reinterpret_cast<longlong2*>(a), base, offs, L, lowmask, TS, tsq,
                                    [](const longlong2& v) { return v; }, tab, Sg);
        else
          store_tile_table<THREADS>(tile, a, base, offs, L, lowmask, TS, tsq,
                                    [](const longlong2& v) { return E::store(v); }, tab, Sg);
        continue;
      }
      if (g.io & 2) {
        store_tile<THREADS>(tile, reinterpret_cast<longlong2*>(a), base, offs, L, lowmask, TS, tsq,
                            [](const longlong2& v) { return v; });
        continue;
      }
    }
    store_tile<THREADS>(tile, a, base, offs, L, lowmask, TS, tsq, [](const T& v) { return E::store(v); });
  }
}

// In-place Q60 integer pairs -> complex128 (the same rounding as a tile pass's store).
__global__ void k_q60_release(double2* __restrict__ a, size_t N) {
  longlong2* v = reinterpret_cast<longlong2*>(a);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const longlong2 x = v[i];
    a[i] = make_double2(q60_to_double_nb(x.x), q60_to_double_nb(x.y));
  }
}

template <class E, int THREADS>
static int launch_engine_t(qs_state* s, const TileArgs& g, size_t smem) {
  static bool attr_set = false;
  static int sms = 0;
  if (!attr_set) {
    QS_CUDA(cudaFuncSetAttribute(k_tile<E, THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
    attr_set = true;
  }
  int per_sm = 0;
  QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile<E, THREADS>, THREADS, smem));
  const uint64_t grid = std::min<uint64_t>(g.ntiles, (uint64_t)std::max(1, sms) * std::max(1, per_sm));
  k_tile<E, THREADS><<<(unsigned)grid, THREADS, smem, s->stream>>>(reinterpret_cast<typename E::G*>(s->amps), g);
  return launch_check("tile kernel");
}

// 256 threads per CTA (measured at n=30, 12-qubit tiles: 512 threads with 2 CTAs
// per SM and 1024 with one are 2-6 % slower); a 13-qubit tile (one CTA per SM)
// runs 512 threads.
template <class E>
static int launch_engine(qs_state* s, const TileArgs& g) {
  const size_t H = (size_t)1 << g.nhigh;
  const size_t smem = ((H * sizeof(uint64_t) + 15) & ~(size_t)15) + (sizeof(typename E::T) << g.m);
  if (g.m >= 13) return launch_engine_t<E, 512>(s, g, smem);
  return launch_engine_t<E, 256>(s, g, smem);
}

int launch_q60_release(qs_state* s) {
  const size_t N = (size_t)1 << s->n;
  const int blocks = (int)std::min<size_t>((N + 255) / 256, 152 * 16);
  KTimer kt(s, QS_K_OTHER, 0, 0, 0, 0, (double)N, 0.0);
  k_q60_release<<<blocks, 256, 0, s->stream>>>(s->amps, N);
  return launch_check("q60 release");
}

int launch_tile(qs_state* s, const TileArgs& g, double flops, double int_ops, int ngates, bool fixed) {
  size_t H = (size_t)1 << g.nhigh;
  size_t smem = ((H * sizeof(uint64_t) + 15) & ~(size_t)15) + ((size_t)16 << g.m);
  uint64_t qmask = 0;
  for (int b = 0; b < g.m - g.nhigh; ++b) qmask |= 1ull << b;
  for (int b = 0; b < g.nhigh; ++b) qmask |= 1ull << g.qhigh[b];
  KTimer kt(s, QS_K_TILE, g.m, ngates, qmask, 0, (double)(1ull << g.n), flops, int_ops);
  if (s->prec == 64) return launch_engine<EngF32>(s, g);
  return fixed ? launch_engine<EngQ60>(s, g) : launch_engine<EngF64>(s, g);
}

}  // namespace qs
