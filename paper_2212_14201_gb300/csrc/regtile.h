// Register-phase Q60 tile pass: launch parameters shared by the host planner
// (plan.cu) and the kernel (tile_q60.cu).
//
// One launch applies a list of register phases (regprog.h) to every tile of the
// state: the tile (2^m amplitudes over the pass's qubit set) is read from HBM
// once, converted to Q60 and kept in shared memory (swizzled, regprog.h).  In a
// phase each thread owns the 16 amplitudes of its group (four register tile
// bits); no other thread touches them until the phase's closing barrier.  The
// phase's ops come in runs that share a quad structure (two of the four bits):
// for each of the group's four quads the thread loads the quad into registers,
// applies every op of the run to it and stores it back.  The tile is converted
// back and written once.
#pragma once

#include "fixed.h"
#include "internal.h"
#include "regprog.h"
#include "tile.h"

namespace qs {

constexpr int RT_MAX_PHASES = 96;
constexpr int RT_MAX_RUNS = 192;
constexpr int RT_MAX_OPS = 320;
constexpr int RT_MAX_COEF = 2200;  // limb pairs (QL) of op coefficients per launch
constexpr int RT_MIN_M = 4;
constexpr int RT_MAX_M = 12;       // 2^(m-4) <= 256 threads, one group of 16 amplitudes each

enum RtKind : uint8_t {
  RK_PAIR = 0,   // R1 (x) R0, two real orthogonal ops on the run's bits r0, r1, as two complex
                 // products (q60pair.cuh): 6 QL, reflection flags in `role`
  RK_REAL = 1,   // real 2x2 on quad bit `role` (0: the run's r0, 1: its r1): 4 QL (m00 m01 m10 m11)
  RK_GEN = 2,    // general 2x2 on quad bit `role`: 4 Gauss-form entries (qc_make_gauss), 12 QL
  RK_ANTI = 3,   // antidiagonal on quad bit `role` (codes code0 / code1 of entries 01 / 10)
  RK_DIAG = 4,   // diag(d0, d1) on quad bit `role` (codes code0 / code1)
  RK_PH1 = 5,    // diag(1, d1) on quad bit `role` (code1)
  RK_SCAL = 6,   // diag(d0, d1) whose target is not a register bit: a factor per group
                 // (sout = 0: tile bit sbit) or per tile (sout = 1: global qubit sbit)
  RK_TABLE = 7,  // a_j *= T[j] over the tile (table index `table`)
};
// REAL .. PH1, SCAL and TABLE take 12 QL of qc_make entries (SCAL, DIAG, PH1:
// entry 0 = d0, entry 3 = d1; ANTI: entries 1 and 2) except REAL (4 QL).

struct RtPhase {
  uint8_t rb[4];      // tile bits of register bits 0..3 (ascending)
  uint8_t gl[12];     // tile bit of bit i of the thread's group index
  uint16_t run_begin, run_end;
};

// Consecutive ops of a phase on the same quad structure: register bits r0, r1
// span the quad; the other two register bits enumerate the group's four quads.
struct RtRun {
  uint8_t r0, r1;
  uint16_t op_begin, op_end;
  uint16_t pad;
};

struct RtOp {
  uint64_t ext;       // controls outside the tile (global qubit mask): the op runs on tiles with all set
  uint16_t gmask;     // controls on group bits (tile-bit mask)
  uint16_t coef;      // index of the first coefficient limb pair
  uint8_t kind, role, cr, pad0;  // cr: controls among the register bits (mask over register indices)
  uint8_t code0, code1, sbit, sout;
  int16_t table;      // RK_TABLE, or a table applied at the start of a RK_PAIR (-1 none)
  uint16_t pad;
};
static_assert(sizeof(RtOp) == 24, "RtOp layout");

// Table entries as stored for the kernel: Q60 limbs of c + i d (c.h, c.l, d.h, d.l),
// thread-major (entry k of thread t at t * 16 + k: the amplitude whose tile index
// is the thread's group base with register index k in the table's phase).
struct RtArgs {
  uint64_t ntiles;
  const int4* tables;  // per table 2^m entries
  int n, m, nhigh, nout;
  int nphases, nruns, nops, ncoef;
  int qhigh[TILE_MAX_M];
  int outpos[QS_MAX_QUBITS];
  RtPhase phases[RT_MAX_PHASES];
  RtRun runs[RT_MAX_RUNS];
  RtOp ops[RT_MAX_OPS];
  QL coef[RT_MAX_COEF];
};
static_assert(sizeof(RtArgs) < 32000, "register-pass arguments must fit the kernel parameter space");

int launch_tile_q60(qs_state* s, const RtArgs& args, double int_ops, int ngates, uint64_t qmask);

}  // namespace qs
