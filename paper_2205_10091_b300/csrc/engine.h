// Engine object behind the opaque tc_circuit handle.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "planner.h"
#include "sv_kernels.cuh"

namespace tcb {

void set_error(const std::string& msg);
tc_status fail(tc_status st, const std::string& msg);
tc_status cuda_fail(cudaError_t e, const char* where);

// Device copy of a vector (freed with dev_free).
template <typename T>
cudaError_t dev_upload(const std::vector<T>& v, T** out) {
  *out = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)out, v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}
void dev_free(void* p);

struct DevPlan {
  DevPass* passes = nullptr;
  DevStage* stages = nullptr;
  DevInstr* instrs = nullptr;
  DevMat* mats = nullptr;
  DevDiag* diags = nullptr;
  DevDiagEnt* dents = nullptr;
  void release();
  cudaError_t upload(const PlanArrays& A);
};

struct DevHam {
  DevPass* passes = nullptr;
  DevHDiag* hdiag = nullptr;
  DevHTerm* hterms = nullptr;
  DevHFlip* hflips = nullptr;
  void release();
  cudaError_t upload(const HamPlan& H);
};

}  // namespace tcb

struct tc_circuit;

namespace tcb {
struct SmallPlan;
void small_free(SmallPlan* p);
tc_status circuit_upload(tc_circuit* c);  // plan and matrix pool on the device (first compute call)
bool small_eligible(tc_circuit* c);
// Workspace of tc_expect_grad per row / for `chunk` rows, and its body with a
// caller-provided workspace (used by the serving loop).
size_t grad_row_bytes(const tc_circuit* c);
size_t grad_ws_bytes(const tc_circuit* c, int chunk);
// Per-row copies of the plan's diagonal entries and Pauli-sum diagonal
// records (device, row-major, `*_stride` entries a row): rows of one plan
// that differ only in those (serving-loop groups).
struct RowDiag {
  const DevDiagEnt* dents;
  int dent_stride;
  const DevHDiag* hdiag;
  int hdiag_stride;
};
tc_status expect_grad_run(tc_circuit* c, const double* d_params, int B, uint64_t seed, double* d_energy_out,
                          double* d_grad_out, int chunk, char* ws, cudaStream_t s, const RowDiag* rd = nullptr);
// Plan + compiled Pauli sum placed in caller-provided device memory.
size_t plan_dev_bytes(const tc_circuit* c);
size_t ham_dev_bytes(const HamPlan& H);
tc_status place_plan_and_ham(tc_circuit* c, const HamPlan& H, char* base, cudaStream_t s);
// Specialised pass kernels (jit.cpp): CUDA source of the circuit's forward and
// adjoint passes compiled with NVRTC; kernel pass i is jit_kernel_name(i).
bool jit_compile(const tc_circuit* c, std::vector<std::vector<char>>& cubins, std::string& err, double* seconds,
                 const std::vector<std::string>& extra_opts = {}, std::string* log_out = nullptr);
std::string jit_kernel_name(int pass);
std::string jit_pass_source(const PlanArrays& A, int pass, int mode, bool dbl, bool fence);
bool jit_compile_source(const std::string& src, std::vector<char>& cubin, std::string& err,
                        const std::vector<std::string>& extra_opts, std::string* log_out);
}  // namespace tcb

struct tc_circuit {
  int n = 0, N = 0;
  int dm_n = 0;  // density-matrix circuit: qubits of rho (n = 2 dm_n); 0 otherwise
  tc_dtype dtype = TC_C64;
  tc_init init = TC_INIT_ZERO;
  int n_ops = 0, n_params = 0, n_noise = 0;
  tc_options opt{};
  int k_fwd = 0, k_bwd = 0, k_ham = 0;
  std::vector<tcb::HGate> gates;       // as planned (RX rewritten to framed RY for complex64)
  std::vector<tcb::HGate> gates_orig;  // as given (the unfused baseline applies these)
  std::vector<double> pool;

  tcb::PlanArrays A;       // forward + adjoint schedules
  tcb::Schedule fwd, bwd;
  std::vector<int> csr_off, csr_slots;  // parameter -> adjoint gradient slots

  tcb::PlanArrays Ap;      // unfused baseline (built on first use)
  tcb::Schedule plain;
  bool plain_built = false;

  // device state (uploaded on first compute call)
  bool uploaded = false;
  bool external_dev = false;  // plan arrays live in caller-owned memory (serving loop)
  int device = -1;
  tcb::DevPlan dplan, dplain;
  double* d_pool = nullptr;
  int* d_csr_off = nullptr;
  int* d_csr_slots = nullptr;

  // Hamiltonian cache: the most recently used compiled Pauli sums
  struct HamEntry {
    std::vector<uint8_t> st;
    std::vector<double> w;
    int T = -1;
    tcb::HamPlan H;
    tcb::DevHam dev;
    uint64_t used = 0;
  };
  std::vector<HamEntry> hcache;
  uint64_t hclock = 0;
  tcb::HamPlan H;     // the selected entry's plan (host copy)
  tcb::DevHam dham;   // the selected entry's device arrays (owned by hcache)

  // pass kernels specialised at plan time (tc_options.specialize): per pass
  // index of A.passes its cubin (host), library and kernel (device)
  std::vector<std::vector<char>> jit_cubins;
  double jit_compile_s = 0;
  std::vector<cudaLibrary_t> jit_libs;
  std::vector<cudaKernel_t> jit_kern;

  // scratch workspace
  void* ws = nullptr;
  size_t ws_bytes = 0;

  // geometric tensor (tc_qgt): the op list as given and its plan (built on
  // first use): occurrence groups that share a generator insertion point, the
  // circuit segments between the points and the suffix after each point
  std::vector<tc_op> ops_in;
  struct QgtGroup {
    int point = 0;            // insertion point (op index)
    int first = 0, count = 0; // state slots [first, first + count)
    tc_circuit* seg = nullptr;    // ops from the previous point to this one (nullptr if none)
    tc_circuit* suffix = nullptr; // ops from this point to the end (nullptr if none)
  };
  std::vector<QgtGroup> qgt_groups;
  bool qgt_ready = false;
  int qgt_occ = 0;                 // parameterised gate occurrences (state slots before the last)
  int* d_qgt_occ_param = nullptr;  // [occ] parameter of each slot's occurrence
  double* d_qgt_occ_c = nullptr;   // [occ] scale / 2
  int* d_qgt_off = nullptr;        // [n_params + 1] CSR parameter -> slots
  int* d_qgt_occ = nullptr;        // [occ]
  uint32_t* d_qgt_pauli = nullptr; // [occ][3] generator: flip mask, sign mask, number of Y
  void* qgt_ws = nullptr;
  size_t qgt_ws_bytes = 0;

  // the one-launch path of tc_apply_expect (small.cu; built on first use)
  tcb::SmallPlan* small = nullptr;
  bool small_tried = false;
  std::string small_why;

  // checkpointed gradients (TC_GRAD_CHECKPOINT): the op list cut into
  // segments of ckpt_ops ops, each planned as a circuit of its own
  std::vector<tc_circuit*> ckpt_segs;
  int ckpt_ops = 0;

  ~tc_circuit();
};
