// Light-cone tensor-network plan (host) and its device kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tc.h"

namespace tcb {

// Input tensor slot of the doubled network <0|U^dagger O U|0>.
//   TS_KET / TS_BRA   per-instance 4x4 gate matrix (light-cone plans), labels (o0, o1, i0, i1)
//   TS_ZERO / TS_PLUS initial one-qubit vector |0> or |+>
//   TS_Z              Z observable, labels (bra, ket)
//   TS_PAULI          Pauli observable of code `gate` (1..3 = X, Y, Z), labels (bra, ket)
//   TS_OP1            one-qubit gate of op `gate`, labels (out, in)
//   TS_OP2            two-qubit gate of op `gate`, labels (o0, o1, i0, i1)
//   TS_SPA / TS_SPB   the q0 / q1 half of a two-qubit gate of operator-Schmidt
//                     rank 2 (RZZ, CZ, CNOT), labels (out, in, k)
// Circuit-network tensors on the bra side carry conj = 1 (complex conjugate).
enum : int32_t {
  TS_KET = 0, TS_BRA = 1, TS_ZERO = 2, TS_Z = 3, TS_PLUS = 4, TS_PAULI = 5,
  TS_OP1 = 6, TS_OP2 = 7, TS_SPA = 8, TS_SPB = 9
};

struct TnInput {
  int32_t kind;   // TS_*
  int32_t gate;   // gate index (TS_KET / TS_BRA), op index (TS_OP*, TS_SP*) or Pauli code
  int32_t off;    // offset (complex entries) in the per-instance input buffer
  int32_t rank;
  int32_t conj;   // 1: complex-conjugate the entries (bra side of a circuit network)
  int32_t pad;
};

// Device copy of one circuit op for the circuit-network assembly kernel.
struct TnOp {
  int32_t kind;   // tc_opkind
  int32_t param;  // -1 = angle 0
  float scale;
  int32_t mat;    // offset (complex entries) into the plan's matrix pool
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

// Fused executor blob: the path's steps grouped by level of the contraction
// tree (a step's level is one more than its operands'), steps of one level
// being independent; a level too large for one staged block is cut into
// several groups run one after another.  Per group:
//   header (kTnGHdr ints): {n_steps, n_items, len, next_len, 0...}
//   per step (kTnSRec ints, 16-byte aligned): {item0, M, K, N, lgM, lgK, lgN,
//     tpo | rot_c << 8, a, b, c, fa, sa, sb, fb, 0}
//     item0 = first work item of the step (work items: M N tpo, each run of
//     equal tpo padded to a warp), a, b, c = live-tensor offsets (complex
//     entries), rot_c = swizzle of the output tensor (tn_swz), fa..fb =
//     offsets of the step's four tables from the group start; each group's
//     block is padded to a multiple of four ints
//   tables: per step fa, sa, sb, fb, each entry already swizzled with its
//     operand's rotation (a full k table, K <= 256, is stored as (sa[k], sb[k])
//     pairs at an even offset, sb = sa + 1 with stride 2); an index set of
//     g <= 8 bits as one full table, a
//     wider one split in two levels: lo = the lowest (g + 1) / 2 bits,
//     table(v) = lo[v & (2^lo - 1)] ^ hi[v >> lo].  The swizzle is linear over
//     XOR and the index sets of one operand scatter to disjoint bit positions,
//     so an operand's address is its offset plus the XOR of its table entries.
//   Shared memory holds entry x of a tensor at offset + tn_swz(x, rot): bits
//   4.. of x are XOR-folded into bits 0..3 (rotated by rot), so lanes whose
//   entries differ only in high bits fall on different bank pairs.  Each
//   tensor's rot (0..3) is chosen on the host for the lanes of the one step
//   that reads it; inputs carry theirs in bits 28..29 of their offset.
constexpr int kTnGHdr = 8;
constexpr int kTnFullTabBits = 8;
#ifdef __CUDACC__
#define TN_HD __host__ __device__
#else
#define TN_HD
#endif
// The fused executor's shared-memory swizzle of a tensor entry x (< 2^20).
TN_HD inline int32_t tn_swz(int32_t x, int rot) {
  const uint32_t u = (uint32_t)x;
  uint32_t f = ((u >> 4) ^ (u >> 8) ^ (u >> 12) ^ (u >> 16)) & 15u;
  f = ((f << rot) | (f >> ((4 - rot) & 3))) & 15u;
  return (int32_t)(u ^ f);
}
// Threads of a fused-executor CTA (work items of a group are spread over them).
constexpr int kTnFusedThreads = 1024;
// Fused executor, few instances: up to kTnMaxCluster CTAs (a portable cluster)
// share an instance while B x cluster fits on the GPU's SMs; groups of at
// least kTnSplitMinItems work items are split over the cluster.
constexpr int kTnMaxCluster = 8;
constexpr int kTnSplitMinItems = 2048;
constexpr int kTnSRec = 16;
// Longest group block staged in shared memory (ints).
constexpr int kTnBlobMax = 3072;

// Largest live-tensor layout the fused executor keeps in shared memory
// (bytes per CTA; the two staged step blocks take 2 x kTnBlobMax ints more).
constexpr int kTnFusedSmemMax = 200 * 1024;


// Precision of the dense path steps (tc_tn_precision): FP32 on CUDA cores, or
// tensor cores with split operands (tn_tc.cu).
enum : int { TN_FP32 = TC_TN_FP32, TN_TF32X3 = TC_TN_TF32X3, TN_BF16X6 = TC_TN_BF16X6 };
// Steps of at least this many complex multiply-adds per instance go to the
// tensor cores in the split-precision modes (tc_tn_set_tc_threshold).
constexpr double kTnTcMinCmacs = 32768.0;

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
  // circuit networks (tc_tn_circuit_create): the ops whose values the
  // assembly kernel evaluates from each instance's parameters
  bool circuit = false;
  int n_params = 0;
  std::vector<TnOp> ops;
  std::vector<float> mats;              // complex pool as interleaved floats
  int n_active = 0;                     // qubits with ket/bra chains
  // fused executor layout
  std::vector<int32_t> fblob;           // group blocks (see kTnGHdr)
  int n_groups = 0;
  bool fblob_ok = false;                // every group within kTnBlobMax
  std::vector<int32_t> in_soff;         // shared-memory offset of each input tensor
  int64_t smem_entries = 0;
  int32_t result_soff = 0;
  // device state
  bool uploaded = false;
  int device = -1;
  int32_t* d_tables = nullptr;
  TnInput* d_inputs = nullptr;
  int32_t* d_gate_q = nullptr;
  TnOp* d_ops = nullptr;
  float* d_mats = nullptr;
  int32_t* d_fblob = nullptr;
  int32_t* d_in_soff = nullptr;
  void* d_arena = nullptr;  // float2 [B][arena_total]
  int arena_B = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_B = -1;
  int graph_prec = -1;
  // the CUDA-core steps of the captured graph grouped by tree level (device;
  // rebuilt with the graph)
  TnStep* d_lsteps = nullptr;
  int* d_lstart = nullptr;
  // split-precision tensor-core steps: eligibility threshold and the
  // device error word of their bounded waits, read back after each call
  // (pinned h_err, event err_ev) and reported by the next call
  double tc_min_cmacs = kTnTcMinCmacs;
  // fused executor with few instances: cluster size per instance (1 = one
  // CTA) and the group size (work items) from which a group is split over it
  int max_cluster = kTnMaxCluster;
  int split_min = kTnSplitMinItems;
  int fused_B = -1, fused_cl = 1, fused_grid = 0;  // launch shape cached for the last B
  int* d_err = nullptr;
  int* h_err = nullptr;
  cudaEvent_t err_ev = nullptr;
  bool err_pending = false;
  const void* graph_gates = nullptr;
  void* graph_out = nullptr;
};

bool tn_build_lightcone(int n_qubits, const int32_t* gate_q, int n_gates, const int32_t* z_q, int n_z, int rank_cap,
                        int trials, const int32_t* path, int n_path, TnPlan& P, std::string& err);

bool tn_build_circuit(int n_qubits, int init, const tc_op* ops, int n_ops, int n_params, const double* mats,
                      int n_mats, const uint8_t* pauli, int prune, int split, int rank_cap, int trials,
                      const int32_t* path, int n_path, TnPlan& P, std::string& err);

// d_src: [B][n_gates][16] complex64 gates (light-cone plans) or [B][n_params]
// float parameters (circuit networks)
cudaError_t tn_launch_assemble(const TnPlan& P, int B, const float* d_src, float2* arena, cudaStream_t s);
constexpr int kTnGemmTile = 32;  // output tile (rows and columns) of the CUDA-core step kernel
cudaError_t tn_launch_step(const TnPlan& P, const TnStep& st, int B, float2* arena, cudaStream_t s);
// the CUDA-core steps of one tree level in one launch: d_steps [n], d_tile_start [n + 1] (device), tiles output
// tiles in all
cudaError_t tn_launch_level(const TnPlan& P, const TnStep* d_steps, const int* d_tile_start, int n, int tiles, int B,
                            float2* arena, cudaStream_t s);
// The whole contraction of B instances in one launch (one CTA per instance,
// grid-stride) with every live tensor in shared memory; taken when the
// plan's layout fits (else one GEMM launch per step, replayed as a graph).
bool tn_fused_ok(const TnPlan& P);
// CTAs per instance of the fused launch for B instances (1, or a cluster when
// B clusters fit on the GPU at once and the plan allows it)
int tn_fused_cluster(const TnPlan& P, int B);
int tn_fused_grid(const TnPlan& P, int B, int cl);
cudaError_t tn_launch_fused(const TnPlan& P, int B, const float* d_src, double* d_out, int grid, int cl,
                            cudaStream_t s);
cudaError_t tn_launch_result(const TnPlan& P, int B, const float2* arena, double* d_out, cudaStream_t s);
// Tensor-core step (tn_tc.cu): TF32X3 or BF16X6; the larger free side on the
// MMA's 128 rows.  Eligible: K >= 2 and M N K >= min_cmacs.
bool tn_step_tc_eligible(const TnStep& st, double min_cmacs);
cudaError_t tn_launch_step_tc(const TnPlan& P, const TnStep& st, int B, float2* arena, int prec, int* d_err,
                              cudaStream_t s);

}  // namespace tcb
