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
#include <algorithm>

#include "tile.h"

namespace qs {

__device__ __forceinline__ double tneg(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

__device__ __forceinline__ double2 tmul_unit(double2 a, int code) {
  switch (code) {
    case U_ONE: return a;
    case U_I: return make_double2(tneg(a.y), a.x);
    case U_MINUS_ONE: return make_double2(tneg(a.x), tneg(a.y));
    default: return make_double2(a.y, tneg(a.x));
  }
}

__device__ __forceinline__ double2 tmul(double2 a, int code, double2 u) {
  if (code != U_GENERAL) return tmul_unit(a, code);
  return make_double2(fma(u.x, a.x, -u.y * a.y), fma(u.x, a.y, u.y * a.x));
}

// Insert zero bits at the set positions of `fixed` (ascending), then OR `set`.
__device__ __forceinline__ uint32_t tile_expand(uint32_t i, uint32_t fixed, uint32_t set) {
  while (fixed) {
    int f = __ffs(fixed) - 1;
    fixed &= fixed - 1;
    i = ((i >> f) << (f + 1)) | (i & ((1u << f) - 1));
  }
  return i | set;
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_tile_f64(double2* __restrict__ a, const __grid_constant__ TileArgs g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = g.m;
  const int L = m - g.nhigh;
  const uint32_t T = 1u << m;
  const uint32_t H = 1u << g.nhigh;
  uint64_t* offs = reinterpret_cast<uint64_t*>(smem_raw);  // [H] offsets of the high tile bits
  double2* tile = reinterpret_cast<double2*>(smem_raw + ((H * sizeof(uint64_t) + 15) & ~(size_t)15));
  for (uint32_t h = threadIdx.x; h < H; h += THREADS) {
    uint64_t o = 0;
    for (int b = 0; b < g.nhigh; ++b) o |= (uint64_t)((h >> b) & 1u) << g.qhigh[b];
    offs[h] = o;
  }
  const uint32_t lowmask = (1u << L) - 1;
  for (uint64_t r = blockIdx.x; r < g.ntiles; r += gridDim.x) {
    uint64_t base = 0;
    for (int b = 0; b < g.nout; ++b) base |= ((r >> b) & 1ull) << g.outpos[b];
    __syncthreads();  // offs ready / previous tile stored
    for (uint32_t j = threadIdx.x; j < T; j += THREADS) tile[j] = a[base + offs[j >> L] + (j & lowmask)];
    __syncthreads();
    for (int k = 0; k < g.nops; ++k) {
      const TileOp& op = g.ops[k];
      if ((base & op.ext_cmask) != op.ext_cmask) continue;  // uniform across the CTA
      const uint32_t lcm = op.lcmask;
      if (op.kind == TOP_SCALAR) {
        const bool one = (base >> op.tb) & 1ull;
        const int code = one ? op.code1 : op.code0;
        if (code == U_ONE) continue;
        const double2 d = one ? op.m[3] : op.m[0];
        const uint32_t cnt = T >> __popc(lcm);
        for (uint32_t i = threadIdx.x; i < cnt; i += THREADS) {
          uint32_t j = tile_expand(i, lcm, lcm);
          tile[j] = tmul(tile[j], code, d);
        }
      } else {
        const uint32_t tb = 1u << op.tb;
        const uint32_t fixed = lcm | tb;
        const uint32_t cnt = T >> __popc(fixed);
        if (op.kind == TOP_PHASE1) {
          for (uint32_t i = threadIdx.x; i < cnt; i += THREADS) {
            uint32_t j = tile_expand(i, fixed, lcm) | tb;
            tile[j] = tmul(tile[j], op.code1, op.m[3]);
          }
        } else {
          for (uint32_t i = threadIdx.x; i < cnt; i += THREADS) {
            uint32_t j0 = tile_expand(i, fixed, lcm), j1 = j0 | tb;
            double2 a0 = tile[j0], a1 = tile[j1], b0, b1;
            if (op.kind == TOP_DIAG) {
              b0 = tmul(a0, op.code0, op.m[0]);
              b1 = tmul(a1, op.code1, op.m[3]);
            } else if (op.kind == TOP_ANTI) {
              b0 = tmul(a1, op.code0, op.m[1]);
              b1 = tmul(a0, op.code1, op.m[2]);
            } else if (op.kind == TOP_REAL) {
              b0 = make_double2(fma(op.m[0].x, a0.x, op.m[1].x * a1.x), fma(op.m[0].x, a0.y, op.m[1].x * a1.y));
              b1 = make_double2(fma(op.m[2].x, a0.x, op.m[3].x * a1.x), fma(op.m[2].x, a0.y, op.m[3].x * a1.y));
            } else {
              const double2 u0 = op.m[0], u1 = op.m[1], u2 = op.m[2], u3 = op.m[3];
              b0.x = fma(u0.x, a0.x, fma(-u0.y, a0.y, fma(u1.x, a1.x, -u1.y * a1.y)));
              b0.y = fma(u0.x, a0.y, fma(u0.y, a0.x, fma(u1.x, a1.y, u1.y * a1.x)));
              b1.x = fma(u2.x, a0.x, fma(-u2.y, a0.y, fma(u3.x, a1.x, -u3.y * a1.y)));
              b1.y = fma(u2.x, a0.y, fma(u2.y, a0.x, fma(u3.x, a1.y, u3.y * a1.x)));
            }
            tile[j0] = b0;
            tile[j1] = b1;
          }
        }
      }
      __syncthreads();
    }
    for (uint32_t j = threadIdx.x; j < T; j += THREADS) a[base + offs[j >> L] + (j & lowmask)] = tile[j];
  }
}

int launch_tile(qs_state* s, const TileArgs& g, double flops, int ngates) {
  constexpr int THREADS = 256;
  size_t H = (size_t)1 << g.nhigh;
  size_t smem = ((H * sizeof(uint64_t) + 15) & ~(size_t)15) + ((size_t)sizeof(double2) << g.m);
  static bool attr_set = false;
  if (!attr_set) {
    QS_CUDA(cudaFuncSetAttribute(k_tile_f64<THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  int per_sm = (int)std::max<size_t>(1, (220 * 1024) / (smem + 1024));
  per_sm = std::min(per_sm, 8);
  uint64_t grid = std::min<uint64_t>(g.ntiles, (uint64_t)152 * per_sm);
  uint64_t qmask = 0;
  for (int b = 0; b < g.m - g.nhigh; ++b) qmask |= 1ull << b;
  for (int b = 0; b < g.nhigh; ++b) qmask |= 1ull << g.qhigh[b];
  KTimer kt(s, QS_K_TILE, g.m, ngates, qmask, 0, (double)(1ull << g.n), flops);
  k_tile_f64<THREADS><<<(unsigned)grid, THREADS, smem, s->stream>>>(s->amps, g);
  return launch_check("tile kernel");
}

}  // namespace qs
