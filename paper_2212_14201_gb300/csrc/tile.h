// Shared-memory tile pass: one HBM read and one write of the state runs every op
// of a fusion pass (the paper's circuit fusion, Section "Quantum circuit fusion";
// gate data in fast on-chip memory, Section "GPU optimization").
#pragma once

#include "fixed.h"
#include "internal.h"

namespace qs {

constexpr int TILE_MAX_M = 13;      // widest tile: 2^13 x 16 B = 128 KiB of shared memory per CTA
constexpr int TILE_DEFAULT_M = 12;  // greedy plans: 2^12 x 16 B = 64 KiB, 3 CTAs per SM
constexpr int TILE_LOW = 3;     // qubits 0..2 are always in a tile: 128-byte contiguous runs
constexpr int TILE_MAX_OPS = 256;
constexpr int TILE_MAX_SIGNED_TABLES = 32;  // tables of a pass that may carry sign terms
constexpr int TILE_MAX_SIGNS = 16;          // sign terms per table

// Sign terms of a phase table: (-1)^(x_q j_t) for each (q, t), with x_q the tile's
// bit q (a qubit outside the tile) and j_t tile bit t of the amplitude.
struct TileSigns {
  uint8_t n;
  uint8_t q[TILE_MAX_SIGNS], t[TILE_MAX_SIGNS];
};

enum TileOpKind : int8_t {
  TOP_PHASE1 = OP_PHASE1,
  TOP_DIAG = OP_DIAG,
  TOP_ANTI = OP_ANTI,
  TOP_REAL = OP_REAL,
  TOP_GENERAL = OP_GENERAL,
  TOP_SCALAR = 9,  // diagonal op whose target lies outside the tile: a per-tile scalar
  TOP_DTABLE = 10, // Q60 only: a_j *= T[j], a diagonal over the tile's 2^tb amplitudes
                   // (table index in lcmask; TileArgs::tables)
  TOP_REAL2 = 11,  // two real rotations on tile bits tb and code0 on amplitude quads (quad
                   // index 2*bit(code0) + bit(tb)): Q60, two complex products (q60pair.cuh,
                   // 6 limb pairs in q[], reflection flags in lcmask); FP32, the real 4x4
                   // (16 floats in f[] of this slot and the next); code1 >= 0: phase
                   // table code1 applied first (the op before the pair)
  TOP_CONT = 12,   // continuation slot of the op before it (never run on its own)
  TOP_REAL3 = 13,  // Q60 only: three real rotations on tile bits tb, code0 and lcmask >> 8 on
                   // amplitude octets (index bit(tb) + 2 bit(code0) + 4 bit(lcmask >> 8)) as
                   // four complex products (q60pair.cuh); the 12 Q3 coefficients (4 x re, im,
                   // -im): 8 in q[] of this slot, 4 in the next; reflection flags in
                   // lcmask & 7; code1 >= 0: phase table code1 applied first
  TOP_REAL4 = 14,  // four real rotations on tile bits tb, code0, (lcmask >> 8) & 31 and
                   // (lcmask >> 16) & 31.  Q60: one amplitude component of 16 at a time, as
                   // eight complex products (q60_quad4_comp); the 24 Q3 coefficients fill q[]
                   // of this slot and the next two; reflection flags in lcmask & 15.  FP32:
                   // 16 amplitudes in registers, the four row-major matrices as 16 floats in
                   // q[] of this one slot; code1 >= 0: phase table code1 applied first
};

struct TileOp {
  union {
    double2 m[4];      // FP64 engine: matrix (for SCALAR: m[0] = d0, m[3] = d1)
    QC q[4];           // Q60 engine: the same entries as limbs (GENERAL ops: Gauss form)
    float2 f[4];       // FP32 engine (complex64 states): the entries rounded to float
  };
  uint64_t ext_cmask;  // control qubits outside the tile (global bit positions)
  uint32_t lcmask;     // control qubits inside the tile (local bit positions)
  int8_t kind;
  int8_t tb;           // local target bit; global target bit for SCALAR
  int8_t code0, code1;
};

struct TileArgs {
  uint64_t ntiles;   // 2^(n - m)
  int n, m;          // state qubits, tile qubits
  int nhigh;         // tile qubits above the contiguous low run
  int qhigh[TILE_MAX_M];  // their global positions (ascending)
  int nout;          // qubits outside the tile
  int outpos[QS_MAX_QUBITS];  // their global positions (ascending)
  int nops;
  // Q60 engine: bit 0, the buffer holds Q60 integers (int64 pairs) left by the
  // previous tile pass instead of complex128; bit 1, store Q60 integers for the
  // next tile pass; bits 8..15, 1 + the phase table applied as each element is
  // loaded (0: none); bits 16..23, 1 + the phase table applied as each element is
  // stored (0: none).  0 for the other engines.
  int io;
  const QL* tables;  // DTABLE ops: per table 2^m entries, each the limb pairs of Re and Im (Q60)
  TileSigns signs[TILE_MAX_SIGNED_TABLES];  // sign terms of tables 0..31
  TileOp ops[TILE_MAX_OPS];
};
static_assert(sizeof(TileArgs) < 32000, "tile arguments must fit the kernel parameter space");

int launch_tile(qs_state* s, const TileArgs& args, double flops, double int_ops, int ngates, bool fixed);
// Converts a buffer of Q60 integer pairs (left by a tile pass with io bit 1) back
// to complex128 in place.
int launch_q60_release(qs_state* s);

}  // namespace qs
