// Internal plan format: plain structs written by the host planner (planner.cpp)
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
#ifdef __CUDACC_RTC__
typedef signed char int8_t;
typedef short int16_t;
typedef int int32_t;
typedef long long int64_t;
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
#else
#include <stdint.h>
#endif

namespace tcb {

constexpr int kRBFwd = 5;       // register bits per thread, complex64 forward passes (32 amplitudes)
constexpr int kRBBwd = 4;       // complex64 adjoint passes hold psi and lambda (2 x 16 amplitudes)
constexpr int kRBFwdC128 = 3;   // complex128: fewer amplitudes per thread, more threads per tile
constexpr int kRBBwdC128 = 4;
constexpr int kRBHam = 4;       // Pauli-sum passes
constexpr int kRBMax = 5;
constexpr int kRYEntries = 2;   // per-row table entries of one RY gate
constexpr int kHamStageBytes = 48 * 1024;  // Pauli-sum terms a pass stages in shared memory (soft cap)
constexpr int kLaneBits = 5;    // lowest tile bits mapped to warp lanes
constexpr int kIOLowBits = 3;   // positions every tile holds: loads and stores move runs of 8 amplitudes
constexpr int kMinQubits = kRBMax + kLaneBits;  // narrower circuits get idle low qubits
constexpr int kMaxK = 14;
constexpr int kMaxQubits = 30;
constexpr int kDefaultGateCapFactor = 0;  // default gates-per-pass cap = factor x tile qubits (0 = none)

// Instruction kinds executed on the register tile.
enum : int8_t {
  IK_MAT2 = 0,      // general 2x2 complex matrix on register bit j0 (table[slot..slot+3])
  IK_CNOT = 1,      // flip register bit j0 where the control (global position `pos`) is 1
  IK_MAT4 = 2,      // 4x4 complex matrix on register bits (j0 = q0, j1 = q1)
  IK_DIAG = 3,      // diagonal group `slot` (phases from the full index)
  IK_GRADDIAG = 4,  // gslot += gscale * Im <lam|G|psi>, G(x) = T - 2 m(x) of group `slot`
  IK_RX = 5,        // RX: table[slot] = (c, s), a0' = c a0 - i s a1, a1' = c a1 - i s a0
  IK_RY = 6,        // RY a0' = c a0 - s a1, a1' = s a0 + c a1 (planner-internal: emitted as IK_RYM)
  IK_H = 7,
  IK_X = 8,
  IK_PAULI = 9,     // noise outcome: table[slot].x = 0,1,2,3 (I, X, Y, Z)
  IK_RX_ADJ = 10,   // adjoint step of RX: gslot += gscale*Im<lam|X|psi>; then RX(-a) on psi, lam
  IK_RY_ADJ = 11,   // same for RY (planner-internal: emitted as IK_RYM_ADJ)
  IK_CHAN = 12,     // Pauli-channel superoperator on register bits (j0, j1): real 2x2 blocks on
                    // (00, 11) with table[slot] = (a, b) and on (01, 10) with table[slot + 1] = (c, d)
  IK_RSEL = 13,     // random-axis rotation: the row's 2x2 matrix at table[slot..slot+3], axis (1..3) in table[slot+4].x
  IK_RXM = 14,      // RX on several register bits: j0 = bit mask, entry of bit r = slot + rank of r in mask
  IK_RXM_ADJ = 15,  // adjoint of IK_RXM: all bits share gslot/gscale
  IK_DIAG_ADJ = 16, // IK_GRADDIAG then IK_DIAG of the same group, fused
  IK_RYM = 17,      // RY on the register bits of mask j0; bit r's kRYEntries entries at slot + kRYEntries * rank
  IK_RYM_ADJ = 18,  // adjoint of IK_RYM (gslot < 0: a fixed-angle rotation, uncompute only)
  IK_RSEL_ADJ = 19, // adjoint step of IK_RSEL: gslot += gscale * Im<lam|G|psi> for the row's axis G, then U^dagger
  IK_SPHASE = 20,   // quarter phases on several qubits: each amplitude times i^(s c), s = gscale (+1 or -1),
                    // c = its 1-bits among the register bits of mask j0 and the global positions of mask slot
};

constexpr int kLocalSlots = 32;  // gradient slots a pass accumulates per thread before one reduction

// Per-CTA table entries built from theta[b] at the start of a pass.
enum : int8_t {
  MT_H = 0,
  MT_X = 1,
  MT_RX = 2,      // 1 entry (c, s) of the effective angle
  MT_RY = 3,      // kRYEntries entries: complex64 (t, c_hi), (c_lo, 0); complex128 (c, s), (0, 0)
  MT_U1 = 4,      // 2x2 from pool (4 entries)
  MT_U2 = 5,      // 4x4 from pool (16 entries)
  MT_DIAGTAB = 6, // phases exp(-i s theta/2 (T - 2m)), m = 0..T  (T+1 entries)
  MT_NOISE = 7,   // 1 entry: selected Pauli code in .x
  MT_QUARTER = 8, // quarter phases (i^{s m}), m = 0..T  (T+1 entries; s = +1 for S, -1 for S^dagger)
  MT_CHAN = 9,    // 2 entries (a, b), (c, d) read from a channel-shaped 4x4 pool matrix
  MT_RSEL = 10,   // 5 entries: the row's rotation matrix (2x2) and its axis code
};

struct DevInstr {  // 16 bytes
  int8_t kind;
  int8_t j0, j1;   // register-bit indices
  int8_t jc;       // CNOT: register bit of the control, or -1 (control from the thread base);
                   // gradient instructions: 1 = the last of its gradient slot in the pass
  int16_t pos;     // CNOT: global position of the control
  int16_t gslot;   // local gradient slot (-1 = none)
  int32_t slot;    // table entry (or diagonal-group index for IK_DIAG / IK_GRADDIAG)
  float gscale;    // gradient scale s
};

struct DevMat {
  int8_t type;
  int8_t adj;      // 1 = build the adjoint (conjugate transpose)
  int16_t pad;
  int32_t param;   // -1 = none
  double scale;
  int32_t pool;    // MT_U1/MT_U2 offset (complex entries) into the pool
  int32_t dst;     // entry offset in the per-row table array of the schedule
  int32_t T;       // MT_DIAGTAB: number of terms; MT_NOISE, MT_RSEL: event index; MT_U1: event folded before (-1 none)
  int32_t T2;      // MT_U1: event folded after the matrix (-1 none)
  double t1, t2, t3;  // MT_NOISE (and MT_U1's event before): interval ends of I, X, Y (left-closed)
  double u1, u2, u3;  // MT_U1's event after: interval ends of I, X, Y
};
static_assert(sizeof(DevMat) == 80, "DevMat layout");

// A diagonal group: m(x) = sum_e popc(op_e(x) & mask_e), with
//   op_e(x) = x ^ (x >> d_e)   (ZZ pairs at distance d_e; d_e = 0 means x: single Z)
//   op_e(x) = x & (x >> d_e)   (CZ pairs) when `sign_mode`.
// Phase mode: amplitude *= table[tab + m]; sign mode: amplitude *= (-1)^m.
// Packed form (packed = 1, phase mode, at most 64 terms): the n_ent = N
// entries are 64-bit column words, col(p) = (mask << 32) | d, bit k of col(p)
// set when term k acts on position p; the term parities of index x are the
// XOR of col(p) over x's set bits p (a linear map over GF(2)), and m(x) is
// their popcount.
struct DevDiag {
  int32_t sign_mode;
  int32_t n_ent;
  int32_t ent_off;  // into DevDiagEnt array
  int32_t T;        // number of Z / ZZ terms (generator G(x) = T - 2 m(x))
  int32_t tab;      // table slot (phase mode)
  int32_t packed;   // 1: the entries are column words (above)
};
struct DevDiagEnt {
  uint32_t d;
  uint32_t mask;
};

// A run of consecutive thread-index (or tile-index) bits [b, b + len) that
// lands on consecutive tile bits [j, j + len) at consecutive global positions
// [p, p + len): the thread -> amplitude map of a stage is a few shift/mask
// steps, one per run.
struct DevRun {
  uint8_t b, len, j, p;
};

struct DevStage {    // 72 bytes
  int8_t S[8];       // register tile bits (first RB used)
  int8_t P[8];       // their global positions
  DevRun run[10];    // thread-index bits -> tile bits / global positions
  int32_t n_runs;
  int32_t n_instr;
  int32_t instr_off; // relative to the pass's first instruction
  int32_t pad;
};

// The kernels carve these out of shared memory back to back, ahead of a
// double-precision reduction buffer: every size keeps 8-byte alignment.
static_assert(sizeof(DevInstr) == 16, "DevInstr layout");
static_assert(sizeof(DevStage) == 72, "DevStage layout");
static_assert(sizeof(DevDiag) % 8 == 0, "DevDiag layout");
static_assert(sizeof(DevDiagEnt) == 8, "DevDiagEnt layout");

// Pauli-sum terms, compiled per Hamiltonian.
//  Diagonal terms: value(x) = w * (cnt - 2 popc((x ^ (x >> d)) & mask)) when cnt >= 0
//                  (d == 0: popc(x & mask)), w * (-1)^popc(x & mask) when cnt < 0.
//                  Packed (pad == 1): cnt ZZ terms of weight w, value(x) = w * (cnt - 2 popc64(W(x))),
//                  W(x) = XOR of the 64-bit column words of x's set positions, held by the
//                  N records that follow (pad == 2, word = (mask << 32) | d).
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
// staged back to back in shared memory after a double-precision buffer
static_assert(sizeof(DevHDiag) == 24 && sizeof(DevHTerm) == 16 && sizeof(DevHFlip) == 16, "Pauli-sum layouts");

enum : int32_t {
  PF_INIT = 1,       // forward pass 0: synthesise the initial state instead of loading
  PF_LAM_LOAD = 2,   // Hamiltonian pass: accumulate into lambda (else start from 0)
  PF_LAM_STORE = 4,  // Hamiltonian pass: write lambda
  PF_FULL = 8,       // the pass needs the full instruction set (CNOT, 4x4, multi-entry groups)
  PF_LEAN = 16,      // the pass needs more than rotation layers (RX, H, X, noise, 2x2, CZ groups)
  PF_MULTI = 32,     // the pass has an XOR-type diagonal group with several entries
  PF_SKIP_PSI = 64,  // adjoint pass: psi is not written back (the last pass of an adjoint sweep)
  PF_SKIP_LAM = 128, // adjoint pass: lambda is not written back (cleared at launch when lambda is still needed)
  PF_GFLUSH = 256,   // adjoint pass: each gradient slot's last instruction is marked (jc = 1); compiled passes
                     // reduce the slot there instead of at the end of the pass
};

struct DevPass {
  int32_t k;            // tile bits
  int32_t nfix;         // N - k
  int32_t rb;           // register bits of this pass's kernel
  uint8_t pos[32];      // tile bit -> global position
  uint8_t fixpos[32];   // fixed (per-tile) bits -> global position, ascending
  DevRun fixrun[32];    // the same map as runs (b = CTA tile-index bit, p = position; j unused)
  int32_t n_fixruns;
  int32_t n_stages, stage_off;
  int32_t n_instr, instr_off;  // all instructions of the pass (contiguous)
  int32_t n_mats, mat_off;
  int32_t n_diag, diag_off;    // diagonal groups of the pass (contiguous)
  int32_t n_dent, dent_off;    // their entries (contiguous)
  int32_t table_size;   // complex entries of the per-CTA table
  int32_t table_off;    // offset of this pass's table in the per-row table array
  int32_t n_gslots;     // local gradient slots
  int32_t gslot_base;   // first global slot
  int32_t flags;
  // Hamiltonian passes
  int32_t n_hdiag, hdiag_off;
  int32_t n_hflip, hflip_off;
  int32_t n_hterm, hterm_off;  // this pass's terms (contiguous), staged in shared memory with its groups
  int32_t epart_index;  // which energy partial this pass writes
  // Paired Pauli-sum pass (flip masks wider than a tile): every group of the
  // pass flips the same fixed bits pair_fout, so tile t's partners all lie in
  // tile t ^ pair_fout.  One CTA owns both tiles of a pair (the one whose
  // tile-index bit pair_bit is 0 and its partner), stages both in shared
  // memory and writes lambda and the energy partial of each.  pair_fout = 0:
  // an ordinary pass.
  uint32_t pair_fout;      // global positions
  uint32_t pair_fout_idx;  // the same bits as CTA tile-index bits
  int32_t pair_bit;        // highest bit of pair_fout_idx
  int32_t pad_pair;
};

}  // namespace tcb
