// Light-cone tensor-network plan (host) and its device kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tc.h"

namespace tcb {

// Input tensor slot of the doubled network <0|U^dagger O U|0>.
enum : int32_t { TS_KET = 0, TS_BRA = 1, TS_ZERO = 2, TS_Z = 3 };

struct TnInput {
  int32_t kind;   // TS_*
  int32_t gate;   // gate index for TS_KET / TS_BRA
  int32_t off;    // offset (complex entries) in the per-instance input buffer
  int32_t rank;
};

// One pairwise contraction: C[i][j] = sum_k A[fa[i] + sa[k]] * B[sb[k] + fb[j]],
// with the index tables (fa, sa, sb, fb) at the given offsets of a shared
// table array, and M = 2^|free A|, K = 2^|shared|, N = 2^|free B|.
struct TnStep {
  int32_t a, b, c;           // tensor ids (inputs < n_inputs)
  int32_t M, K, N;
  int32_t fa, sa, sb, fb;    // offsets into the index-table array
  int64_t a_off, b_off, c_off;  // offsets (complex entries) of the operands in the per-instance arena
};

struct TnPlan {
  int n_qubits = 0;
  int n_gates = 0;
  std::vector<int32_t> gate_q;          // [n_gates][2]
  std::vector<int> cone;                // gate indices in the cone (forward order)
  int cone_lo = 0, cone_hi = -1;        // qubit span of the cone
  std::vector<TnInput> inputs;
  int64_t in_total = 0;                 // complex entries of inputs per instance
  std::vector<TnStep> steps;
  std::vector<int32_t> tables;          // index tables
  int64_t arena_total = 0;              // complex entries of the per-instance arena (inputs + intermediates)
  int64_t result_off = 0;
  double flops = 0, write = 0, size = 0;  // path metrics (complex MACs, elements, elements)
  int max_rank = 0;
  // device state
  bool uploaded = false;
  int device = -1;
  int32_t* d_tables = nullptr;
  TnInput* d_inputs = nullptr;
  int32_t* d_gate_q = nullptr;
  void* d_arena = nullptr;  // float2 [B][arena_total]
  int arena_B = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_B = -1;
  const void* graph_gates = nullptr;
  void* graph_out = nullptr;
};

bool tn_build_lightcone(int n_qubits, const int32_t* gate_q, int n_gates, const int32_t* z_q, int n_z, int rank_cap,
                        const int32_t* path, int n_path, TnPlan& P, std::string& err);

cudaError_t tn_launch_assemble(const TnPlan& P, int B, const float* d_gates, float2* arena, cudaStream_t s);
cudaError_t tn_launch_step(const TnPlan& P, const TnStep& st, int B, float2* arena, cudaStream_t s);
cudaError_t tn_launch_result(const TnPlan& P, int B, const float2* arena, double* d_out, cudaStream_t s);

}  // namespace tcb
