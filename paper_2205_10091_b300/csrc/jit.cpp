// Pass kernels specialised per circuit at plan time (tc_options.specialize).
//
// The library's tile-pass kernel interprets a plan: per stage and instruction
// it reads the instruction from shared memory, dispatches on its kind and on
// its register bits, and walks index runs read from the stage records.  For a
// circuit evaluated many times the same plan can instead be compiled: every
// forward and adjoint pass becomes one kernel whose program (pass
// descriptor, stages, instructions, diagonal groups and their entries) is a
// set of constexpr functions, and the kernel runs the library's own
// gate_pass body (sv_core.cuh) over it, so every loop over stages and
// instructions unrolls and every register bit, mask, table offset and index
// run is a constant.  The arithmetic is the interpreter's, instruction for
// instruction.  Compilation is NVRTC to one cubin per pass for sm_103a on the
// host at tc_circuit_create (the passes on several host threads); the cubins
// are loaded (cudaLibraryLoadData) on the first compute call on a device.
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <cstdio>
#include <sstream>
#include <string>
#include <vector>

#include "engine.h"
#include "jit_headers.inc"  // kJitHeaderNames / kJitHeaderSrcs: the device headers, embedded at build time

namespace tcb {

namespace {

void emit_pass(std::ostringstream& o, const DevPass& P) {
  o << "  __host__ __device__ static constexpr tcb::DevPass pass() {\n    tcb::DevPass p{};\n";
  o << "    p.k = " << P.k << "; p.nfix = " << P.nfix << "; p.rb = " << P.rb << ";\n";
  for (int j = 0; j < P.k; ++j) o << "    p.pos[" << j << "] = " << (int)P.pos[j] << ";\n";
  for (int f = 0; f < P.nfix; ++f) o << "    p.fixpos[" << f << "] = " << (int)P.fixpos[f] << ";\n";
  for (int q = 0; q < P.n_fixruns; ++q) {
    const DevRun& u = P.fixrun[q];
    o << "    p.fixrun[" << q << "] = tcb::DevRun{" << (int)u.b << ", " << (int)u.len << ", " << (int)u.j << ", "
      << (int)u.p << "};\n";
  }
  // offsets relative to the pass (the generated program holds only this pass)
  o << "    p.n_fixruns = " << P.n_fixruns << "; p.n_stages = " << P.n_stages << "; p.n_instr = " << P.n_instr
    << "; p.n_diag = " << P.n_diag << "; p.n_dent = " << P.n_dent << ";\n";
  o << "    p.table_size = " << P.table_size << "; p.table_off = " << P.table_off << "; p.n_gslots = " << P.n_gslots
    << "; p.gslot_base = " << P.gslot_base << "; p.flags = " << P.flags << ";\n";
  o << "    return p;\n  }\n";
}

void emit_stages(std::ostringstream& o, const PlanArrays& A, const DevPass& P, int rb) {
  o << "  static constexpr int kStages = " << P.n_stages << ";\n";
  o << "  __host__ __device__ static constexpr tcb::DevStage stage(int i) {\n    tcb::DevStage s{};\n"
       "    switch (i) {\n";
  for (int si = 0; si < P.n_stages; ++si) {
    const DevStage& S = A.stages[P.stage_off + si];
    o << "      case " << si << ":\n";
    for (int r = 0; r < rb; ++r) o << "        s.S[" << r << "] = " << (int)S.S[r] << "; s.P[" << r << "] = " << (int)S.P[r] << ";\n";
    for (int q = 0; q < S.n_runs; ++q) {
      const DevRun& u = S.run[q];
      o << "        s.run[" << q << "] = tcb::DevRun{" << (int)u.b << ", " << (int)u.len << ", " << (int)u.j << ", "
        << (int)u.p << "};\n";
    }
    o << "        s.n_runs = " << S.n_runs << "; s.n_instr = " << S.n_instr << "; s.instr_off = " << S.instr_off
      << ";\n        break;\n";
  }
  o << "      default: break;\n    }\n    return s;\n  }\n";
}

void emit_instrs(std::ostringstream& o, const PlanArrays& A, const DevPass& P) {
  o << "  __host__ __device__ static constexpr tcb::DevInstr instr(int i) {\n    tcb::DevInstr d{};\n"
       "    switch (i) {\n";
  for (int ii = 0; ii < P.n_instr; ++ii) {
    const DevInstr& in = A.instrs[P.instr_off + ii];
    char gs[64];
    snprintf(gs, sizeof(gs), "(float)%a", (double)in.gscale);  // exact (hexadecimal) value
    o << "      case " << ii << ": d.kind = " << (int)in.kind << "; d.j0 = " << (int)in.j0 << "; d.j1 = " << (int)in.j1
      << "; d.jc = " << (int)in.jc << "; d.pos = " << in.pos << "; d.gslot = " << in.gslot << "; d.slot = " << in.slot
      << "; d.gscale = " << gs << "; break;\n";
  }
  o << "      default: break;\n    }\n    return d;\n  }\n";
}

void emit_diags(std::ostringstream& o, const PlanArrays& A, const DevPass& P) {
  o << "  __host__ __device__ static constexpr tcb::DevDiag diag(int i) {\n    tcb::DevDiag d{};\n    switch (i) {\n";
  for (int di = 0; di < P.n_diag; ++di) {
    const DevDiag& d = A.diags[P.diag_off + di];
    o << "      case " << di << ": d.sign_mode = " << d.sign_mode << "; d.n_ent = " << d.n_ent << "; d.ent_off = "
      << d.ent_off << "; d.T = " << d.T << "; d.tab = " << d.tab << "; d.packed = " << d.packed << "; break;\n";
  }
  o << "      default: break;\n    }\n    return d;\n  }\n";
  o << "  __host__ __device__ static constexpr tcb::DevDiagEnt dent(int i) {\n    tcb::DevDiagEnt e{};\n"
       "    switch (i) {\n";
  for (int ei = 0; ei < P.n_dent; ++ei) {
    const DevDiagEnt& e = A.dents[P.dent_off + ei];
    o << "      case " << ei << ": e.d = " << e.d << "u; e.mask = " << e.mask << "u; break;\n";
  }
  o << "      default: break;\n    }\n    return e;\n  }\n";
}

}  // namespace

std::string jit_kernel_name(int pass) { return "tcj_pass_" + std::to_string(pass); }

// CUDA source of pass `pi` (of schedule mode `mode`: KM_FWD or KM_BWD).
std::string jit_pass_source(const PlanArrays& A, int pi, int mode, bool dbl, bool fence) {
  std::ostringstream o;
  o << "#include \"sv_core.cuh\"\n";
  const DevPass& P = A.passes[pi];
  o << "struct TcjProg" << pi << " {\n";
  emit_pass(o, P);
  emit_stages(o, A, P, P.rb);
  emit_instrs(o, A, P);
  emit_diags(o, A, P);
  o << "};\n";
  const char* T = dbl ? "double" : "float";
  const int minb = dbl ? (P.rb <= 3 ? 2 : 1) : (P.rb <= 3 ? 4 : 2);
  o << "extern \"C\" __global__ void __launch_bounds__(256, " << minb << ") " << jit_kernel_name(pi)
    << "(const __grid_constant__ tcb::KArgs a, const __grid_constant__ tcb::PassArgs pa) {\n"
    << "  tcb::gate_pass<" << T << ", " << mode << ", " << P.rb << ", 7, tcb::CtSrc<TcjProg" << pi << ", "
    << (fence ? "true" : "false") << ">>(a, pa);\n}\n";
  return o.str();
}

bool jit_compile_source(const std::string& src, std::vector<char>& cubin, std::string& err,
                        const std::vector<std::string>& extra_opts, std::string* log_out) {
  nvrtcProgram prog;
  nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "tc_pass.cu", kJitHeaderCount, kJitHeaderSrcs,
                                     kJitHeaderNames);
  if (r != NVRTC_SUCCESS) {
    err = std::string("nvrtcCreateProgram: ") + nvrtcGetErrorString(r);
    return false;
  }
  // -default-device: the unannotated lambdas of gate_pass are device code
  std::vector<const char*> opts = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo", "-default-device"};
  for (const auto& x : extra_opts) opts.push_back(x.c_str());
  r = nvrtcCompileProgram(prog, (int)opts.size(), opts.data());
  size_t n = 0;
  nvrtcGetProgramLogSize(prog, &n);
  std::string log(n, '\0');
  if (n) nvrtcGetProgramLog(prog, &log[0]);
  if (log_out) *log_out = log;
  if (r != NVRTC_SUCCESS) {
    err = "pass kernel did not compile: " + log.substr(0, 4000);
    nvrtcDestroyProgram(&prog);
    return false;
  }
  nvrtcGetCUBINSize(prog, &n);
  cubin.resize(n);
  nvrtcGetCUBIN(prog, cubin.data());
  nvrtcDestroyProgram(&prog);
  return true;
}

bool jit_compile(const tc_circuit* c, std::vector<std::vector<char>>& cubins, std::string& err, double* seconds,
                 const std::vector<std::string>& extra_opts, std::string* log_out) {
  const auto t0 = std::chrono::steady_clock::now();
  const bool dbl = c->dtype == TC_C128;
  std::vector<std::pair<int, int>> work;  // (pass index, mode)
  for (int p = c->fwd.first_pass; p < c->fwd.first_pass + c->fwd.n_passes; ++p) work.push_back({p, KM_FWD});
  for (int p = c->bwd.first_pass; p < c->bwd.first_pass + c->bwd.n_passes; ++p) work.push_back({p, KM_BWD});
  cubins.assign(c->A.passes.size(), {});
  std::vector<std::string> errs(work.size()), logs(work.size());
  std::vector<char> ok(work.size(), 0);
  // one NVRTC program per pass, compiled on a few host threads
  std::atomic<size_t> next{0};
  auto worker = [&]() {
    for (size_t w = next++; w < work.size(); w = next++)
      ok[w] = jit_compile_source(jit_pass_source(c->A, work[w].first, work[w].second, dbl, false), cubins[work[w].first],
                                 errs[w], extra_opts, &logs[w]);
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t nth = std::min<size_t>(work.size(), std::min(16u, hw));
  std::vector<std::thread> th;
  for (size_t i = 1; i < nth; ++i) th.emplace_back(worker);
  worker();
  for (auto& t : th) t.join();
  if (log_out) {
    log_out->clear();
    for (size_t w = 0; w < work.size(); ++w) *log_out += logs[w];
  }
  for (size_t w = 0; w < work.size(); ++w)
    if (!ok[w]) {
      err = errs[w];
      return false;
    }
  if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return true;
}

}  // namespace tcb
