// Internal plan format: plain structs written by the host planner (plan.cpp)
// and read by the tile-pass kernels (sv_kernels.cu).  Everything is POD so the
// whole plan uploads to the device with one copy per array.
//
// Index conventions inside the engine: a state of N (internal) qubits holds
// 2^N amplitudes; "position" p is a bit of the amplitude index counted from
// the least significant end, so user qubit q lives at position N-1-q (qubit 0
// is the most significant bit).  A pass stages a tile of 2^k amplitudes whose
// tile bits j = 0..k-1 sit at ascending positions pos[j]; pos[0..4] = 0..4 so
// a warp's 32 lanes always touch 32 consecutive amplitudes.  Inside a tile, a
// thread holds 2^RB amplitudes in registers ("register bits" S[0..RB-1] are
// tile bits); stages change S through a swizzled shared-memory transpose.
#pragma once
#include <stdint.h>

namespace tcb {

constexpr int kRB = 4;          // register bits per thread (16 amplitudes)
constexpr int kR = 1 << kRB;    // amplitudes per thread
constexpr int kLaneBits = 5;    // lowest tile bits mapped to warp lanes
constexpr int kMinQubits = kRB + kLaneBits;  // narrower circuits get idle low qubits
constexpr int kMaxK = 14;
constexpr int kMaxQubits = 30;

// Instruction kinds executed on the register tile.
enum : int8_t {
  IK_MAT2 = 0,      // 2x2 complex matrix on register bit j0 (table slot mslot)
  IK_CNOT = 1,      // flip register bit j0 where global position `pos` is 1
  IK_MAT4 = 2,      // 4x4 complex matrix on register bits (j0 = q0, j1 = q1)
  IK_DIAG = 3,      // diagonal group `aux` (phases from the full index)
  IK_GRADX = 4,     // gslot += scale * Im <lam|X_j0|psi>
  IK_GRADY = 5,     // gslot += scale * Im <lam|Y_j0|psi>
  IK_GRADDIAG = 6,  // gslot += scale * Im <lam|G|psi>, G(x) = T - 2 m(x) of group aux
  IK_SKIP = 7,      // no-op (identity noise outcome placeholder)
};

// Per-CTA matrix-table entries built from theta[b] at the start of a pass.
enum : int8_t {
  MT_H = 0,
  MT_X = 1,
  MT_RX = 2,
  MT_RY = 3,
  MT_U1 = 4,      // 2x2 from pool
  MT_U2 = 5,      // 4x4 from pool
  MT_DIAGTAB = 6, // phases exp(-i s theta/2 (T - 2m)), m = 0..T  (T+1 entries)
  MT_NOISE = 7,   // Pauli selected by the event's uniform number
  MT_CZTAB = 8,   // the two signs {+1, -1} (CZ parity groups)
};

struct DevInstr {
  int8_t kind;
  int8_t j0, j1;   // register-bit indices
  int8_t jc;       // CNOT: register bit of the control, or -1 (control from the thread base)
  int32_t pos;     // CNOT: global position of the control
  int32_t aux;     // IK_DIAG / IK_GRADDIAG: diagonal-group index
  int32_t mslot;   // first complex entry in the per-CTA table
  int32_t gslot;   // local gradient slot (-1 = none)
  float gscale;    // gradient scale s
};

struct DevMat {
  int8_t type;
  int8_t adj;      // 1 = build the adjoint (conjugate transpose)
  int16_t pad;
  int32_t param;   // -1 = none
  double scale;
  int32_t pool;    // MT_U1/MT_U2 offset (complex entries) into the pool
  int32_t dst;     // first complex entry in the per-CTA table
  int32_t T;       // MT_DIAGTAB: number of terms; MT_NOISE: event index
  int32_t pad2;
  double t1, t2, t3;  // MT_NOISE: interval ends of I, X, Y (left-closed)
};

// A diagonal group: m(x) = sum_e popc(op_e(x) & mask_e), with
//   op_e(x) = x ^ (x >> d_e)   (ZZ pairs at distance d_e; d_e = 0 means x: single Z)
//   op_e(x) = x & (x >> d_e)   (CZ pairs) when `sign_mode`.
// Phase mode: amplitude *= table[m]; sign mode: amplitude *= (-1)^m.
struct DevDiag {
  int32_t sign_mode;
  int32_t n_ent;
  int32_t ent_off;  // into DevDiagEnt array
  int32_t T;        // number of Z / ZZ terms (generator G(x) = T - 2 m(x))
  int32_t tab;      // table slot (phase mode)
  int32_t pad;
};
struct DevDiagEnt {
  uint32_t d;
  uint32_t mask;
};

struct DevStage {
  int8_t S[kRB];     // register tile bits
  int32_t n_instr;
  int32_t instr_off;
};

// Pauli-sum terms, compiled per Hamiltonian.
//  Diagonal terms: value(x) = w * (cnt - 2 popc((x ^ (x >> d)) & mask)) when d > 0,
//                  w * (-1)^popc(x & mask) when d == 0.
//  Flip group f:   h_f(x) = sum_t w_t * i^{ny_t} * (-1)^popc(x & sm_t), and
//                  (P psi)_y = h_f(y ^ f) psi_{y ^ f}.
struct DevHDiag {
  uint32_t d, mask;
  int32_t cnt, pad;
  double w;
};
struct DevHTerm {
  uint32_t sm;
  int32_t ny;
  double w;
};
struct DevHFlip {
  uint32_t f;        // flip mask (global positions)
  uint32_t f_tile;   // same mask in tile-local bits of its pass
  int32_t term_off, n_terms;
};

enum : int32_t {
  PF_INIT = 1,       // forward pass 0: synthesise the initial state instead of loading
  PF_LAM_LOAD = 2,   // Hamiltonian pass: accumulate into lambda (else start from 0)
  PF_LAM_STORE = 4,  // Hamiltonian pass: write lambda
};

struct DevPass {
  int32_t k;            // tile bits
  int32_t nfix;         // N - k
  uint8_t pos[32];      // tile bit -> global position
  uint8_t fixpos[32];   // fixed (per-tile) bits -> global position, ascending
  int32_t n_stages, stage_off;
  int32_t n_mats, mat_off;
  int32_t table_size;   // complex entries of the per-CTA table
  int32_t n_gslots;     // local gradient slots
  int32_t gslot_base;   // first global slot
  int32_t flags;
  // Hamiltonian passes
  int32_t n_hdiag, hdiag_off;
  int32_t n_hflip, hflip_off;
  int32_t epart_index;  // which energy partial this pass writes
  int32_t pad;
};

}  // namespace tcb
