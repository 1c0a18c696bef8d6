// Device-visible launch arguments of the state-vector passes: plain structs
// shared by the library's kernels and the pass kernels generated at plan
// time (tc_options.specialize), so both read the same layout.
#pragma once
#include "plan.h"

namespace tcb {

enum KMode : int { KM_FWD = 0, KM_BWD = 1, KM_HAM = 2 };

struct KArgs {
  // circuit plan (device)
  const DevPass* passes;
  const DevStage* stages;
  const DevInstr* instrs;
  const DevMat* mats;
  const DevDiag* diags;
  const DevDiagEnt* dents;
  const double* pool;  // complex128, interleaved
  // Hamiltonian plan (device)
  const DevPass* hpasses;
  const DevHDiag* hdiag;
  const DevHTerm* hterms;
  const DevHFlip* hflips;
  int pass;   // index into passes (KM_FWD/KM_BWD) or hpasses (KM_HAM)
  int N;      // internal qubits
  int n_user; // user qubits (INIT_PLUS covers only these)
  int init;   // tc_init
  int synth_init;  // 1: a pass flagged PF_INIT synthesises the initial state
  // data
  void* psi;
  void* lam;
  const double* theta;
  int n_params;
  const float* status;
  int n_noise;
  uint64_t seed;
  int64_t row_offset;
  double* gpart;   // [rows][gslots_total][tiles]
  int gslots_total;
  double* epart;   // [rows][n_hpasses][tiles]
  int n_hpasses;
  int store_lambda;
  // per-row gate tables (built by launch_tables) and their row stride (entries)
  const void* tables;
  int table_stride;
  // Pauli-sum passes of an energy-only call: the flip groups of a pass are
  // split over hchunks blocks per tile (blockIdx.y), each writing its own
  // energy partial; 0 or 1 = one block per tile (required when lambda is kept)
  int hchunks;
  // grouped rows (serving): > 0 = `dents` (`hdiag`) hold one copy of the
  // plan's diagonal entries (Pauli-sum diagonal records) per row, this many
  // entries apart, so rows of one plan may differ in the column words of
  // packed groups and in diagonal weights; 0 = one copy shared by all rows
  int dent_row_stride;
  int hdiag_row_stride;
};

// The pass descriptor and its first stage, passed by value as a kernel
// parameter.
struct PassArgs {
  DevPass pass;
  DevStage st0;  // unused by Pauli-sum passes
};

}  // namespace tcb
