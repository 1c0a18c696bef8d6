// Host-side planner: op list -> fused tile passes (see plan.h for the format).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "plan.h"
#include "../../include/tc.h"

namespace tcb {

// A gate after validation, in internal positions.
struct HGate {
  int kind = 0;        // tc_opkind
  int p0 = -1, p1 = -1;
  int param = -1;
  double scale = 1.0;
  int pool = -1;
  int noise_event = -1;
  double t1 = 0, t2 = 0, t3 = 0;
  bool diag = false;
  bool sign_mode = false;  // CZ
  bool quarter = false;    // S (scale +1) or S^dagger (scale -1) on p0: phase i^{scale * bit}
  bool chan = false;       // U2 whose pool matrix has the Pauli-channel superoperator shape
  // U1 with Pauli-noise events folded in (fold_noise_into_u1): the row's
  // outcome of event pre_ev acts before the matrix, of post_ev after it
  int pre_ev = -1, post_ev = -1;
  double pre_t[3] = {0, 0, 0}, post_t[3] = {0, 0, 0};
};

// Fold each Pauli-noise event into the non-diagonal U1 on the same qubit
// right before it (or, failing that, right after it) when no other gate or
// event touches that qubit in between: the row's Pauli then multiplies the
// row's 2x2 matrix when the gate tables are built, and the event costs no
// instruction.  Events keep their numbers (the random streams do not change);
// events with no such neighbour stay as they are.
std::vector<HGate> fold_noise_into_u1(const std::vector<HGate>& gates);

// Rewrite every RX(a) as S^dagger RY(a) S (an exact identity).  The S phases
// are diagonal, commute with every diagonal gate and cancel between two RX on
// the same qubit, so each qubit carries a "frame" flag and S / S^dagger are
// emitted only where a non-diagonal, non-RX gate needs the plain frame (and
// at the end).  RY has real coefficients, which the kernels evaluate with
// packed FP32x2 arithmetic.
std::vector<HGate> rewrite_rx_frames(const std::vector<HGate>& gates, int N);

struct PlanArrays {
  std::vector<DevPass> passes;
  std::vector<DevStage> stages;
  std::vector<DevInstr> instrs;
  std::vector<DevMat> mats;
  std::vector<DevDiag> diags;
  std::vector<DevDiagEnt> dents;
};

struct Schedule {
  int first_pass = 0, n_passes = 0;
  int k = 0;
  int n_gslots = 0;               // global gradient slots (adjoint schedules)
  std::vector<int> slot_param;    // global slot -> parameter
  int n_stages = 0;
  int first_mat = 0, n_mats = 0;  // table-building records of the schedule
  int table_total = 0;            // table entries per batch row
};

struct HamPlan {
  std::vector<DevPass> passes;
  std::vector<DevHDiag> hdiag;
  std::vector<DevHTerm> hterms;
  std::vector<DevHFlip> hflips;
  int k = 0;
  int packed_groups = 0;  // packed diagonal groups (DevHDiag.pad == 1)
};

// Normalise and validate ops; returns false and sets err on bad input.
bool normalise_ops(int n_user, int n_internal, const tc_op* ops, int n_ops, int n_params, int n_pool,
                   std::vector<HGate>& out, std::string& err);

// Schedule gates (forward order, or reversed with adjoint=true) into passes.
// max_gates: cap on non-diagonal gates per pass (<= 0: no cap).
Schedule build_schedule(const std::vector<HGate>& gates, int N, int k, int rb, bool adjoint, bool first_init,
                        PlanArrays& A, int max_gates);

// Compile a Pauli sum (user structures) into Hamiltonian passes.
bool build_hamiltonian(int n_user, int N, int k, const uint8_t* structures, const double* weights, int T,
                       HamPlan& H, std::string& err);

// Unfused baseline: one pass per gate (k = N tile not required; uses kMinQubits-bit tiles).
Schedule build_plain_schedule(const std::vector<HGate>& gates, int N, int rb, PlanArrays& A);

}  // namespace tcb
