// C-ABI entry points of libtc_b300.so (declared in include/tc.h).
#include <cmath>
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "dm.h"
#include "engine.h"

namespace tcb {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }
tc_status fail(tc_status st, const std::string& msg) {
  g_err = msg;
  return st;
}
tc_status cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? TC_E_NOMEM : TC_E_CUDA;
}
void dev_free(void* p) {
  if (p) cudaFree(p);
}

void DevPlan::release() {
  dev_free(passes);
  dev_free(stages);
  dev_free(instrs);
  dev_free(mats);
  dev_free(diags);
  dev_free(dents);
  *this = DevPlan{};
}
cudaError_t DevPlan::upload(const PlanArrays& A) {
  cudaError_t e;
  if ((e = dev_upload(A.passes, &passes)) != cudaSuccess) return e;
  if ((e = dev_upload(A.stages, &stages)) != cudaSuccess) return e;
  if ((e = dev_upload(A.instrs, &instrs)) != cudaSuccess) return e;
  if ((e = dev_upload(A.mats, &mats)) != cudaSuccess) return e;
  if ((e = dev_upload(A.diags, &diags)) != cudaSuccess) return e;
  return dev_upload(A.dents, &dents);
}
void DevHam::release() {
  dev_free(passes);
  dev_free(hdiag);
  dev_free(hterms);
  dev_free(hflips);
  *this = DevHam{};
}
cudaError_t DevHam::upload(const HamPlan& H) {
  cudaError_t e;
  if ((e = dev_upload(H.passes, &passes)) != cudaSuccess) return e;
  if ((e = dev_upload(H.hdiag, &hdiag)) != cudaSuccess) return e;
  if ((e = dev_upload(H.hterms, &hterms)) != cudaSuccess) return e;
  return dev_upload(H.hflips, &hflips);
}

}  // namespace tcb

using namespace tcb;

tc_circuit::~tc_circuit() {
  for (auto l : jit_libs)
    if (l) cudaLibraryUnload(l);
  if (uploaded && !external_dev) {
    dplan.release();
    dplain.release();
    for (auto& e : hcache) e.dev.release();
    dev_free(d_pool);
    dev_free(d_csr_off);
    dev_free(d_csr_slots);
  }
  dev_free(ws);
  for (auto& g : qgt_groups) {
    delete g.seg;
    delete g.suffix;
  }
  dev_free(d_qgt_pauli);
  dev_free(d_qgt_occ_param);
  dev_free(d_qgt_occ_c);
  dev_free(d_qgt_off);
  dev_free(d_qgt_occ);
  dev_free(qgt_ws);
  for (auto* sg : ckpt_segs) delete sg;
  small_free(small);
}

namespace {

bool is_dbl(const tc_circuit* c) { return c->dtype == TC_C128; }
size_t amp_bytes(const tc_circuit* c) { return is_dbl(c) ? 16 : 8; }

tc_status ensure_device(tc_circuit* c) {
  if (c->uploaded) {
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != c->device) return fail(TC_E_INVALID, "circuit was first used on another device");
    return TC_OK;
  }
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if ((e = c->dplan.upload(c->A)) != cudaSuccess) return cuda_fail(e, "plan upload");
  if ((e = dev_upload(c->pool, &c->d_pool)) != cudaSuccess) return cuda_fail(e, "pool upload");
  if ((e = dev_upload(c->csr_off, &c->d_csr_off)) != cudaSuccess) return cuda_fail(e, "csr upload");
  if ((e = dev_upload(c->csr_slots, &c->d_csr_slots)) != cudaSuccess) return cuda_fail(e, "csr upload");
  if (!c->jit_cubins.empty()) {
    // the specialised pass kernels of this circuit, on this device
    c->jit_libs.assign(c->A.passes.size(), nullptr);
    c->jit_kern.assign(c->A.passes.size(), nullptr);
    for (const Schedule* sc : {&c->fwd, &c->bwd})
      for (int p = sc->first_pass; p < sc->first_pass + sc->n_passes; ++p) {
        if ((e = cudaLibraryLoadData(&c->jit_libs[p], c->jit_cubins[p].data(), nullptr, nullptr, 0, nullptr, nullptr,
                                     0)) != cudaSuccess)
          return cuda_fail(e, "loading a specialised pass kernel");
        if ((e = cudaLibraryGetKernel(&c->jit_kern[p], c->jit_libs[p], jit_kernel_name(p).c_str())) != cudaSuccess)
          return cuda_fail(e, "specialised pass kernel lookup");
      }
  }
  c->uploaded = true;
  return TC_OK;
}

tc_status ensure_ham(tc_circuit* c, const uint8_t* structures, const double* weights, int T) {
  if (T < 0) return fail(TC_E_INVALID, "T < 0");
  if (T > 0 && (!structures || !weights)) return fail(TC_E_INVALID, "structures/weights are NULL");
  const size_t ns = (size_t)T * c->n;
  for (auto& e : c->hcache) {
    if (e.T == T && e.st.size() == ns && (ns == 0 || !memcmp(e.st.data(), structures, ns)) &&
        (T == 0 || !memcmp(e.w.data(), weights, T * sizeof(double)))) {
      e.used = ++c->hclock;
      c->H = e.H;
      c->dham = e.dev;
      return TC_OK;
    }
  }
  tc_circuit::HamEntry ent;
  std::string err;
  if (!build_hamiltonian(c->n, c->N, c->k_ham, structures, weights, T, ent.H, err))
    return fail(err.find("flips more") != std::string::npos ? TC_E_UNSUPPORTED : TC_E_INVALID, err);
  cudaError_t e = ent.dev.upload(ent.H);
  if (e != cudaSuccess) {
    ent.dev.release();
    return cuda_fail(e, "hamiltonian upload");
  }
  ent.st.assign(structures, structures + ns);
  ent.w.assign(weights, weights + T);
  ent.T = T;
  ent.used = ++c->hclock;
  constexpr size_t kMaxCached = 8;
  if (c->hcache.size() >= kMaxCached) {
    // evict the least recently used entry (its device arrays are no longer referenced)
    size_t lru = 0;
    for (size_t i = 1; i < c->hcache.size(); ++i)
      if (c->hcache[i].used < c->hcache[lru].used) lru = i;
    c->hcache[lru].dev.release();
    c->hcache.erase(c->hcache.begin() + lru);
  }
  c->hcache.push_back(std::move(ent));
  c->H = c->hcache.back().H;
  c->dham = c->hcache.back().dev;
  return TC_OK;
}

tc_status ensure_ws(tc_circuit* c, size_t bytes) {
  if (bytes <= c->ws_bytes) return TC_OK;
  dev_free(c->ws);
  c->ws = nullptr;
  c->ws_bytes = 0;
  cudaError_t e = cudaMalloc(&c->ws, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "workspace allocation");
  }
  c->ws_bytes = bytes;
  return TC_OK;
}

int64_t budget(const tc_circuit* c) {
  if (c->opt.mem_budget_bytes > 0) return c->opt.mem_budget_bytes;
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  return (int64_t)((double)(fr + c->ws_bytes) * 0.6);
}

KArgs base_args(const tc_circuit* c, const DevPlan& dp) {
  KArgs a{};
  a.passes = dp.passes;
  a.stages = dp.stages;
  a.instrs = dp.instrs;
  a.mats = dp.mats;
  a.diags = dp.diags;
  a.dents = dp.dents;
  a.pool = c->d_pool;
  a.hpasses = c->dham.passes;
  a.hdiag = c->dham.hdiag;
  a.hterms = c->dham.hterms;
  a.hflips = c->dham.hflips;
  a.N = c->N;
  a.n_user = c->n;
  a.init = (int)c->init;
  a.synth_init = 1;
  a.n_params = c->n_params;
  a.n_noise = c->n_noise;
  return a;
}

#define TC_CHECK_CUDA(expr, where)               \
  do {                                           \
    cudaError_t _e = (expr);                     \
    if (_e != cudaSuccess) return cuda_fail(_e, where); \
  } while (0)

// keep_lambda: the adjoint sweep's lambda is read afterwards (checkpoint segments)
tc_status run_schedule(tc_circuit* c, int mode, const Schedule& sc, const PlanArrays& A, KArgs a, void* tables,
                       int rows, cudaStream_t s, bool keep_lambda = false) {
  a.tables = tables;
  a.table_stride = sc.table_total;
  TC_CHECK_CUDA(launch_tables(is_dbl(c), a, sc.first_mat, sc.n_mats, rows, s), "gate tables");
  // the circuit's specialised kernels run its own schedules (not the unfused
  // baseline's) with the plan's own diagonal entries compiled in
  const bool spec = &A == &c->A && !c->jit_kern.empty() && a.dent_row_stride == 0;
  for (int p = 0; p < sc.n_passes; ++p) {
    a.pass = sc.first_pass + p;
    if (spec)
      TC_CHECK_CUDA(launch_pass_specialised(c->jit_kern[a.pass], mode, is_dbl(c), a, A.passes[a.pass], rows, s),
                    mode == KM_FWD ? "forward pass (specialised)" : "adjoint pass (specialised)");
    else {
      DevPass hp = A.passes[a.pass];
      if (keep_lambda) hp.flags &= ~PF_SKIP_LAM;
      TC_CHECK_CUDA(launch_pass(mode, is_dbl(c), a, hp, &A.stages[hp.stage_off], rows, s),
                    mode == KM_FWD ? "forward pass" : "adjoint pass");
    }
  }
  return TC_OK;
}

tc_status run_ham(tc_circuit* c, KArgs a, int rows, bool store_lambda, cudaStream_t s) {
  a.store_lambda = store_lambda ? 1 : 0;
  a.n_hpasses = (int)c->H.passes.size();
  for (int p = 0; p < (int)c->H.passes.size(); ++p) {
    a.pass = p;
    TC_CHECK_CUDA(launch_pass(KM_HAM, is_dbl(c), a, c->H.passes[p], nullptr, rows, s), "hamiltonian pass");
  }
  return TC_OK;
}

}  // namespace

namespace tcb {

tc_status circuit_upload(tc_circuit* c) { return ensure_device(c); }

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t grad_row_bytes(const tc_circuit* c) {
  const size_t per = ((size_t)1 << c->N) * amp_bytes(c);
  const size_t tiles_h = (size_t)1 << (c->N - c->k_ham);
  const size_t tiles_b = (size_t)1 << (c->N - c->k_bwd);
  const size_t tf = (size_t)c->fwd.table_total * amp_bytes(c), tb = (size_t)c->bwd.table_total * amp_bytes(c);
  return 2 * per + (size_t)c->H.passes.size() * tiles_h * 8 + (size_t)std::max(c->bwd.n_gslots, 1) * tiles_b * 8 + tf +
         tb + 64;
}

size_t grad_ws_bytes(const tc_circuit* c, int chunk) {
  const size_t per = ((size_t)1 << c->N) * amp_bytes(c);
  const size_t tiles_h = (size_t)1 << (c->N - c->k_ham);
  const size_t tiles_b = (size_t)1 << (c->N - c->k_bwd);
  const size_t tf = (size_t)c->fwd.table_total * amp_bytes(c), tb = (size_t)c->bwd.table_total * amp_bytes(c);
  return 2 * al256(per * chunk) + al256((size_t)chunk * c->H.passes.size() * tiles_h * 8) +
         al256((size_t)chunk * std::max(c->bwd.n_gslots, 1) * tiles_b * 8) + al256(tf * chunk) + al256(tb * chunk);
}

tc_status expect_grad_run(tc_circuit* c, const double* d_params, int B, uint64_t seed, double* d_energy_out,
                          double* d_grad_out, int chunk, char* w, cudaStream_t s, const RowDiag* rd) {
  const size_t per = ((size_t)1 << c->N) * amp_bytes(c);
  const int nh = (int)c->H.passes.size();
  const size_t tiles_h = (size_t)1 << (c->N - c->k_ham);
  const size_t tiles_b = (size_t)1 << (c->N - c->k_bwd);
  const int G = c->bwd.n_gslots;
  const size_t tf = (size_t)c->fwd.table_total * amp_bytes(c);
  const size_t o_lam = al256(per * chunk);
  const size_t o_ep = o_lam + al256(per * chunk);
  const size_t o_gp = o_ep + al256((size_t)chunk * nh * tiles_h * 8);
  const size_t o_tf = o_gp + al256((size_t)chunk * std::max(G, 1) * tiles_b * 8);
  const size_t o_tb = o_tf + al256(tf * chunk);
  tc_status st;
  for (int r0 = 0; r0 < B; r0 += chunk) {
    const int rows = std::min(chunk, B - r0);
    KArgs a = base_args(c, c->dplan);
    a.psi = w;
    a.lam = w + o_lam;
    a.epart = (double*)(w + o_ep);
    a.gpart = (double*)(w + o_gp);
    a.gslots_total = G;
    a.theta = d_params ? d_params + (size_t)r0 * c->n_params : nullptr;
    a.seed = seed;
    a.row_offset = r0;
    if (rd) {
      a.dents = rd->dents + (size_t)r0 * rd->dent_stride;
      a.dent_row_stride = rd->dent_stride;
      a.hdiag = rd->hdiag + (size_t)r0 * rd->hdiag_stride;
      a.hdiag_row_stride = rd->hdiag_stride;
    }
    if ((st = run_schedule(c, KM_FWD, c->fwd, c->A, a, w + o_tf, rows, s)) != TC_OK) return st;
    if ((st = run_ham(c, a, rows, true, s)) != TC_OK) return st;
    if ((st = run_schedule(c, KM_BWD, c->bwd, c->A, a, w + o_tb, rows, s)) != TC_OK) return st;
    TC_CHECK_CUDA(launch_finalize(a.epart, nh, (int)tiles_h, a.gpart, G, (int)tiles_b, c->d_csr_off,
                                  c->d_csr_slots, c->n_params, rows, d_energy_out + r0,
                                  c->n_params ? d_grad_out + (size_t)r0 * c->n_params : nullptr, s),
                  "finalize");
  }
  return TC_OK;
}

// ---- plan arrays in caller-provided device memory (serving loop) -----------
template <typename T>
static void place(std::vector<std::pair<const void*, size_t>>& cp, char*& cur, const std::vector<T>& v, T** dst) {
  *dst = v.empty() ? nullptr : (T*)cur;
  if (!v.empty()) cp.push_back({v.data(), v.size() * sizeof(T)});
  cur += al256(v.size() * sizeof(T));
}

size_t plan_dev_bytes(const tc_circuit* c) {
  const PlanArrays& A = c->A;
  return al256(A.passes.size() * sizeof(DevPass)) + al256(A.stages.size() * sizeof(DevStage)) +
         al256(A.instrs.size() * sizeof(DevInstr)) + al256(A.mats.size() * sizeof(DevMat)) +
         al256(A.diags.size() * sizeof(DevDiag)) + al256(A.dents.size() * sizeof(DevDiagEnt)) +
         al256(c->pool.size() * 8) + al256(c->csr_off.size() * 4) + al256(c->csr_slots.size() * 4);
}

size_t ham_dev_bytes(const HamPlan& H) {
  return al256(H.passes.size() * sizeof(DevPass)) + al256(H.hdiag.size() * sizeof(DevHDiag)) +
         al256(H.hterms.size() * sizeof(DevHTerm)) + al256(H.hflips.size() * sizeof(DevHFlip));
}

tc_status place_plan_and_ham(tc_circuit* c, const HamPlan& H, char* base, cudaStream_t s) {
  std::vector<std::pair<const void*, size_t>> cp;
  std::vector<char*> dst;
  char* cur = base;
  auto rec = [&](auto& v, auto** d) {
    char* at = cur;
    place(cp, cur, v, d);
    if (!v.empty()) dst.push_back(at);
  };
  const PlanArrays& A = c->A;
  rec(A.passes, &c->dplan.passes);
  rec(A.stages, &c->dplan.stages);
  rec(A.instrs, &c->dplan.instrs);
  rec(A.mats, &c->dplan.mats);
  rec(A.diags, &c->dplan.diags);
  rec(A.dents, &c->dplan.dents);
  rec(c->pool, &c->d_pool);
  rec(c->csr_off, &c->d_csr_off);
  rec(c->csr_slots, &c->d_csr_slots);
  c->H = H;
  rec(c->H.passes, &c->dham.passes);
  rec(c->H.hdiag, &c->dham.hdiag);
  rec(c->H.hterms, &c->dham.hterms);
  rec(c->H.hflips, &c->dham.hflips);
  for (size_t i = 0; i < cp.size(); ++i)
    TC_CHECK_CUDA(cudaMemcpyAsync(dst[i], cp[i].first, cp[i].second, cudaMemcpyHostToDevice, s), "plan copy");
  c->uploaded = true;
  c->external_dev = true;
  cudaGetDevice(&c->device);
  return TC_OK;
}

}  // namespace tcb

extern "C" {

const char* tc_last_error(void) { return g_err.c_str(); }
const char* tc_version(void) { return "tc_b300 0.1 (sm_103a)"; }

tc_status tc_circuit_create(int n_qubits, tc_dtype dtype, tc_init init, const tc_op* ops, int n_ops, int n_params,
                            const double* pool, int n_pool, const tc_options* opt, tc_circuit** out) {
  if (!out) return fail(TC_E_INVALID, "out is NULL");
  *out = nullptr;
  if (n_qubits < 1 || n_qubits > kMaxQubits) return fail(TC_E_INVALID, "n_qubits must be in 1..30");
  if (dtype != TC_C64 && dtype != TC_C128) return fail(TC_E_INVALID, "unknown dtype");
  if (init != TC_INIT_ZERO && init != TC_INIT_PLUS) return fail(TC_E_INVALID, "unknown init");
  if (n_ops < 0 || (n_ops > 0 && !ops)) return fail(TC_E_INVALID, "ops is NULL");
  if (n_params < 0) return fail(TC_E_INVALID, "n_params < 0");
  if (n_pool < 0 || (n_pool > 0 && !pool)) return fail(TC_E_INVALID, "pool is NULL");
  auto* c = new tc_circuit();
  c->n = n_qubits;
  c->N = n_qubits < kMinQubits ? kMinQubits : n_qubits;
  c->dtype = dtype;
  c->init = init;
  c->n_ops = n_ops;
  c->n_params = n_params;
  if (n_ops > 0) c->ops_in.assign(ops, ops + n_ops);
  if (opt) c->opt = *opt;
  const bool dbl = dtype == TC_C128;
  auto pick = [&](int want, int dflt, int maxk) {
    int k = want > 0 ? want : dflt;
    if (k > maxk) k = maxk;
    if (k < kMinQubits) k = kMinQubits;
    if (k > c->N) k = c->N;
    return k;
  };
  // at most 256 threads per tile: k <= 8 + register bits
  c->k_fwd = pick(c->opt.tile_qubits_fwd, dbl ? 12 : 13, 8 + (dbl ? kRBFwdC128 : kRBFwd));
  c->k_bwd = pick(c->opt.tile_qubits_bwd, dbl ? 11 : 12, 8 + (dbl ? kRBBwdC128 : kRBBwd));
  c->k_ham = pick(0, 8 + kRBHam, 8 + kRBHam);  // 256-thread Pauli-sum passes
  std::string err;
  if (!normalise_ops(n_qubits, c->N, ops, n_ops, n_params, n_pool, c->gates, err)) {
    delete c;
    return fail(TC_E_INVALID, err);
  }
  for (auto& g : c->gates)
    if (g.noise_event >= 0) c->n_noise++;
  c->gates_orig = c->gates;
  c->gates = fold_noise_into_u1(c->gates);
  if (dtype == TC_C64) c->gates = rewrite_rx_frames(c->gates, c->N);
  c->pool.assign(pool, pool + 2 * (size_t)n_pool);
  // 4x4 matrices of the Pauli-channel superoperator shape (real, two symmetric
  // 2x2 blocks on (00, 11) and (01, 10); density-matrix circuits make them)
  // run as two real 2x2 blocks instead of a dense complex 4x4
  auto channel_shaped = [&](int off) {
    auto re = [&](int r, int col) { return c->pool[2 * ((size_t)off + 4 * r + col)]; };
    for (int e = 0; e < 16; ++e)
      if (c->pool[2 * ((size_t)off + e) + 1] != 0.0) return false;
    for (int r = 0; r < 4; ++r)
      for (int col = 0; col < 4; ++col) {
        const bool block = (r == col) || (r + col == 3);
        if (!block && re(r, col) != 0.0) return false;
      }
    return re(0, 0) == re(3, 3) && re(0, 3) == re(3, 0) && re(1, 1) == re(2, 2) && re(1, 2) == re(2, 1);
  };
  for (auto& g : c->gates)
    if (g.kind == TC_OP_U2 && channel_shaped(g.pool)) g.chan = true;
  // cap on gates per pass: deep multi-layer passes need many register stages
  // whose mixed register-bit sets conflict in shared memory
  const int mg_f = c->opt.max_gates_per_pass > 0 ? c->opt.max_gates_per_pass
                                                 : (c->opt.max_gates_per_pass < 0 ? 0 : kDefaultGateCapFactor * c->k_fwd);
  const int mg_b = c->opt.max_gates_per_pass > 0 ? c->opt.max_gates_per_pass
                                                 : (c->opt.max_gates_per_pass < 0 ? 0 : kDefaultGateCapFactor * c->k_bwd);
  c->fwd = build_schedule(c->gates, c->N, c->k_fwd, dbl ? kRBFwdC128 : kRBFwd, false, true, c->A, mg_f);
  c->bwd = build_schedule(c->gates, c->N, c->k_bwd, dbl ? kRBBwdC128 : kRBBwd, true, false, c->A, mg_b);
  // parameter -> gradient slots (CSR)
  c->csr_off.assign(n_params + 1, 0);
  for (int p : c->bwd.slot_param) c->csr_off[p + 1]++;
  for (int p = 0; p < n_params; ++p) c->csr_off[p + 1] += c->csr_off[p];
  c->csr_slots.assign(c->bwd.slot_param.size(), 0);
  {
    std::vector<int> fillp(c->csr_off.begin(), c->csr_off.end() - 1);
    for (int s = 0; s < (int)c->bwd.slot_param.size(); ++s) c->csr_slots[fillp[c->bwd.slot_param[s]]++] = s;
  }
  if (c->csr_slots.empty()) c->csr_slots.push_back(0);
  if (c->opt.specialize) {
    std::string jerr;
    if (!jit_compile(c, c->jit_cubins, jerr, &c->jit_compile_s)) {
      delete c;
      return fail(TC_E_CUDA, jerr);
    }
  }
  *out = c;
  return TC_OK;
}

void tc_circuit_destroy(tc_circuit* c) { delete c; }

tc_status tc_dm_circuit_create(int n_qubits, tc_dtype dtype, tc_init init, const tc_op* ops, int n_ops,
                               int n_params, const double* pool, int n_pool, const tc_options* opt,
                               tc_circuit** out) {
  if (!out) return fail(TC_E_INVALID, "out is NULL");
  *out = nullptr;
  if (n_qubits < 1 || 2 * n_qubits > kMaxQubits) return fail(TC_E_INVALID, "n_qubits must be in 1..15");
  if (n_ops < 0 || (n_ops > 0 && !ops)) return fail(TC_E_INVALID, "ops is NULL");
  if (n_pool < 0 || (n_pool > 0 && !pool)) return fail(TC_E_INVALID, "pool is NULL");
  std::vector<tc_op> dops;
  std::vector<double> dpool;
  std::string err;
  if (!build_dm_ops(n_qubits, ops, n_ops, pool, n_pool, dops, dpool, err)) return fail(TC_E_INVALID, err);
  const tc_status st = tc_circuit_create(2 * n_qubits, dtype, init, dops.empty() ? nullptr : dops.data(),
                                         (int)dops.size(), n_params, dpool.empty() ? nullptr : dpool.data(),
                                         (int)(dpool.size() / 2), opt, out);
  if (st == TC_OK) (*out)->dm_n = n_qubits;
  return st;
}

tc_status tc_dm_expect_pauli_sum(tc_circuit* c, const void* d_rho, int B, const uint8_t* structures,
                                 const double* weights, int T, double* d_out, void* stream) {
  if (!c || (B != 0 && (!d_rho || !d_out))) return fail(TC_E_INVALID, "NULL argument");
  if (c->dm_n <= 0) return fail(TC_E_INVALID, "not a density-matrix circuit (tc_dm_circuit_create)");
  if (B < 0 || T < 0 || (T > 0 && (!structures || !weights))) return fail(TC_E_INVALID, "bad Pauli sum or B");
  if (B == 0) return TC_OK;
  std::vector<DmTerm> terms;
  std::string err;
  if (!build_dm_terms(c->dm_n, structures, weights, T, terms, err)) return fail(TC_E_INVALID, err);
  if (terms.empty()) terms.push_back(DmTerm{});  // H = 0: one zero-weight identity term
  cudaStream_t s = (cudaStream_t)stream;
  const int n = c->dm_n;
  const int nblk = std::max(1, std::min(64, (1 << n) / 256));
  const int chunk = std::min(B, 65535);
  const size_t tb = (terms.size() * sizeof(DmTerm) + 255) & ~(size_t)255;
  tc_status st = ensure_ws(c, tb + (size_t)chunk * nblk * sizeof(double));
  if (st != TC_OK) return st;
  DmTerm* d_terms = (DmTerm*)c->ws;
  double* partial = (double*)((char*)c->ws + tb);
  TC_CHECK_CUDA(cudaMemcpyAsync(d_terms, terms.data(), terms.size() * sizeof(DmTerm), cudaMemcpyHostToDevice, s),
                "term upload");
  const size_t rb = ((size_t)1 << (2 * n)) * amp_bytes(c);
  for (int r0 = 0; r0 < B; r0 += chunk) {
    const int rows = std::min(chunk, B - r0);
    TC_CHECK_CUDA(launch_dm_trace(is_dbl(c), (const char*)d_rho + (size_t)r0 * rb, n, rows, d_terms,
                                  (int)terms.size(), partial, nblk, s),
                  "density-matrix trace");
    TC_CHECK_CUDA(launch_finalize(partial, nblk, 1, nullptr, 0, 1, nullptr, nullptr, 0, rows, d_out + r0, nullptr, s),
                  "finalize");
  }
  return TC_OK;
}

tc_status tc_circuit_info(const tc_circuit* c, tc_plan_info* o) {
  if (!c || !o) return fail(TC_E_INVALID, "NULL argument");
  memset(o, 0, sizeof(*o));
  o->n_qubits = c->n;
  o->n_qubits_internal = c->N;
  o->n_ops = c->n_ops;
  o->n_params = c->n_params;
  o->n_noise = c->n_noise;
  o->fwd_passes = c->fwd.n_passes;
  o->bwd_passes = c->bwd.n_passes;
  o->fwd_stages = c->fwd.n_stages;
  o->bwd_stages = c->bwd.n_stages;
  o->tile_qubits_fwd = c->k_fwd;
  o->tile_qubits_bwd = c->k_bwd;
  auto instrs = [&](const Schedule& sc) {
    int n = 0;
    for (int p = sc.first_pass; p < sc.first_pass + sc.n_passes; ++p) n += c->A.passes[p].n_instr;
    return n;
  };
  o->fwd_instrs = instrs(c->fwd);
  o->bwd_instrs = instrs(c->bwd);
  for (const auto& cb : c->jit_cubins) o->specialized_passes += cb.empty() ? 0 : 1;
  for (const Schedule* sc : {&c->fwd, &c->bwd})
    for (int p = sc->first_pass; p < sc->first_pass + sc->n_passes; ++p) {
      const DevPass& P = c->A.passes[p];
      for (int d = 0; d < P.n_diag; ++d) o->packed_diag_groups += c->A.diags[P.diag_off + d].packed;
    }
  return TC_OK;
}

tc_status tc_pauli_sum_info(const tc_circuit* c, const uint8_t* structures, const double* weights, int T,
                            tc_pauli_sum_plan_info* o) {
  if (!c || !o) return fail(TC_E_INVALID, "NULL argument");
  if (T < 0 || (T > 0 && (!structures || !weights))) return fail(TC_E_INVALID, "bad Pauli sum");
  HamPlan H;
  std::string err;
  if (!build_hamiltonian(c->n, c->N, c->k_ham, structures, weights, T, H, err)) return fail(TC_E_INVALID, err);
  memset(o, 0, sizeof(*o));
  o->passes = (int)H.passes.size();
  for (const auto& P : H.passes) o->paired_passes += P.pair_fout ? 1 : 0;
  o->flip_groups = (int)H.hflips.size();
  o->diag_entries = (int)H.hdiag.size();
  o->tile_qubits = c->k_ham;
  o->packed_diag_groups = H.packed_groups;
  return TC_OK;
}

tc_status tc_apply_layers(const tc_circuit* cc, const double* d_params, int B, const void* d_init, uint64_t seed,
                          const float* d_status, int64_t row_offset, void* d_states_out, void* stream) {
  tc_circuit* c = const_cast<tc_circuit*>(cc);
  if (!c || (B != 0 && !d_states_out)) return fail(TC_E_INVALID, "NULL circuit or output");
  if (B < 0) return fail(TC_E_INVALID, "B < 0");
  if (c->n_params > 0 && !d_params && B > 0) return fail(TC_E_INVALID, "d_params is NULL");
  if (B == 0) return TC_OK;
  tc_status st = ensure_device(c);
  if (st != TC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const bool padded = c->N != c->n;
  const size_t per = ((size_t)1 << c->N) * amp_bytes(c);
  const size_t trow = (size_t)c->fwd.table_total * amp_bytes(c);
  const size_t row_ws = (padded ? per : 0) + trow;
  int chunk = (int)std::min<int64_t>(B, std::max<int64_t>(1, (int64_t)(256u << 20) / (int64_t)std::max<size_t>(row_ws, 1)));
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  if ((st = ensure_ws(c, al(padded ? per * chunk : 0) + al(trow * chunk) + 256)) != TC_OK) return st;
  void* work = padded ? c->ws : d_states_out;
  void* tables = (char*)c->ws + al(padded ? per * chunk : 0);
  for (int r0 = 0; r0 < B; r0 += chunk) {
    const int rows = std::min(chunk, B - r0);
    const size_t ub = ((size_t)1 << c->n) * amp_bytes(c);
    void* out_rows = (char*)d_states_out + (size_t)r0 * ub;
    KArgs a = base_args(c, c->dplan);
    a.psi = padded ? work : out_rows;
    a.theta = d_params ? d_params + (size_t)r0 * c->n_params : nullptr;
    a.status = d_status ? d_status + (size_t)r0 * c->n_noise : nullptr;
    a.seed = seed;
    a.row_offset = row_offset + r0;
    if (d_init) {
      a.synth_init = 0;
      const void* in_rows = (const char*)d_init + (size_t)r0 * ub;
      if (padded) {
        TC_CHECK_CUDA(launch_pad_states(is_dbl(c), in_rows, work, c->n, c->N, rows, true, s), "pad");
      } else if (in_rows != out_rows) {
        TC_CHECK_CUDA(cudaMemcpyAsync(out_rows, in_rows, ub * rows, cudaMemcpyDeviceToDevice, s), "init copy");
      }
    }
    if ((st = run_schedule(c, KM_FWD, c->fwd, c->A, a, tables, rows, s)) != TC_OK) return st;
    if (padded) TC_CHECK_CUDA(launch_pad_states(is_dbl(c), work, out_rows, c->n, c->N, rows, false, s), "unpad");
  }
  return TC_OK;
}

tc_status tc_expect_pauli_sum(tc_circuit* c, const void* d_states, int B, const uint8_t* structures,
                              const double* weights, int T, double* d_energy_out, void* stream) {
  if (!c || (B != 0 && (!d_states || !d_energy_out))) return fail(TC_E_INVALID, "NULL argument");
  if (B < 0) return fail(TC_E_INVALID, "B < 0");
  if (B == 0) return TC_OK;
  tc_status st = ensure_device(c);
  if (st != TC_OK) return st;
  if ((st = ensure_ham(c, structures, weights, T)) != TC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const bool padded = c->N != c->n;
  const size_t per = ((size_t)1 << c->N) * amp_bytes(c);
  const int nh = (int)c->H.passes.size();
  const size_t tiles_h = (size_t)1 << (c->N - c->k_ham);
  // few rows x tiles: split each pass's flip groups over several blocks
  // (~4 blocks per SM in all, at least two groups each), each adding its own
  // energy partial
  int max_flips = 1;
  for (const auto& P : c->H.passes) max_flips = std::max(max_flips, P.n_hflip);
  const int64_t blocks = (int64_t)B * (int64_t)tiles_h;
  const int hch = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)max_flips / 2, 256, 592 / std::max<int64_t>(blocks, 1)}));
  const size_t epb = (size_t)nh * hch * tiles_h * 8;
  int chunk = B;
  if (padded) chunk = (int)std::min<int64_t>(B, std::max<int64_t>(1, (int64_t)(256u << 20) / (int64_t)per));
  else chunk = (int)std::min<int64_t>(B, std::max<int64_t>(1, (int64_t)(256u << 20) / (int64_t)epb));
  const size_t need = (size_t)chunk * (epb + (padded ? per : 0)) + 256;
  if ((st = ensure_ws(c, need)) != TC_OK) return st;
  double* epart = (double*)c->ws;
  void* work = (char*)c->ws + (((size_t)chunk * epb + 255) & ~(size_t)255);
  const size_t ub = ((size_t)1 << c->n) * amp_bytes(c);
  for (int r0 = 0; r0 < B; r0 += chunk) {
    const int rows = std::min(chunk, B - r0);
    const void* in_rows = (const char*)d_states + (size_t)r0 * ub;
    KArgs a = base_args(c, c->dplan);
    if (padded) {
      TC_CHECK_CUDA(launch_pad_states(is_dbl(c), in_rows, work, c->n, c->N, rows, true, s), "pad");
      a.psi = work;
    } else {
      a.psi = const_cast<void*>(in_rows);
    }
    a.lam = nullptr;
    a.epart = epart;
    a.hchunks = hch;
    if ((st = run_ham(c, a, rows, false, s)) != TC_OK) return st;
    TC_CHECK_CUDA(launch_finalize(epart, nh * hch, (int)tiles_h, nullptr, 0, 1, c->d_csr_off, c->d_csr_slots, 0, rows,
                                  d_energy_out + r0, nullptr, s),
                  "finalize");
  }
  return TC_OK;
}

}  // extern "C"

namespace {

// Segments of `ops` ops each, planned as circuits of their own (built on
// first use and kept while the segment length stays the same).
tc_status ensure_segments(tc_circuit* c, int ops) {
  if (c->ckpt_ops == ops && !c->ckpt_segs.empty()) return TC_OK;
  for (auto* sg : c->ckpt_segs) delete sg;
  c->ckpt_segs.clear();
  c->ckpt_ops = 0;
  tc_options o = c->opt;
  o.specialize = 0;
  for (int from = 0; from < c->n_ops; from += ops) {
    tc_circuit* sg = nullptr;
    const int cnt = std::min(ops, c->n_ops - from);
    tc_status st = tc_circuit_create(c->n, c->dtype, c->init, c->ops_in.data() + from, cnt, c->n_params,
                                     c->pool.empty() ? nullptr : c->pool.data(), (int)(c->pool.size() / 2), &o, &sg);
    if (st == TC_OK) st = ensure_device(sg);
    if (st != TC_OK) {
      delete sg;
      for (auto* q : c->ckpt_segs) delete q;
      c->ckpt_segs.clear();
      return st;
    }
    c->ckpt_segs.push_back(sg);
  }
  c->ckpt_ops = ops;
  return TC_OK;
}

// Workspace of one row: the state after every segment, lambda, the
// Pauli-sum partials, the largest segment's gradient partials and tables.
size_t ckpt_row_bytes(const tc_circuit* c) {
  const size_t per = ((size_t)1 << c->N) * amp_bytes(c);
  const size_t tiles_h = (size_t)1 << (c->N - c->k_ham);
  size_t gp = 8, tab = 0;
  for (const tc_circuit* sg : c->ckpt_segs) {
    gp = std::max(gp, (size_t)std::max(sg->bwd.n_gslots, 1) * ((size_t)1 << (sg->N - sg->k_bwd)) * 8);
    tab = std::max(tab, (size_t)std::max(sg->fwd.table_total, sg->bwd.table_total) * amp_bytes(c));
  }
  return (c->ckpt_segs.size() + 1) * per + c->H.passes.size() * tiles_h * 8 + gp + tab + 64 * 8;
}

// Checkpointed energy + gradient: forward segment by segment, keeping the
// state after each; lambda = H psi; then the adjoint of each segment from
// last to first, starting from that segment's stored state (so the
// uncompute of psi never runs across a segment boundary) and adding its
// gradient partials to the rows' gradients.
tc_status expect_grad_ckpt_run(tc_circuit* c, const double* d_params, int B, uint64_t seed, double* d_e,
                               double* d_g, int chunk, char* w, cudaStream_t s) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int S = (int)c->ckpt_segs.size();
  const size_t per = ((size_t)1 << c->N) * amp_bytes(c);
  const int nh = (int)c->H.passes.size();
  const size_t tiles_h = (size_t)1 << (c->N - c->k_ham);
  size_t gp = 8, tab = 0;
  for (const tc_circuit* sg : c->ckpt_segs) {
    gp = std::max(gp, (size_t)std::max(sg->bwd.n_gslots, 1) * ((size_t)1 << (sg->N - sg->k_bwd)) * 8);
    tab = std::max(tab, (size_t)std::max(sg->fwd.table_total, sg->bwd.table_total) * amp_bytes(c));
  }
  const size_t o_lam = (size_t)S * al(per * chunk);
  const size_t o_ep = o_lam + al(per * chunk);
  const size_t o_gp = o_ep + al((size_t)chunk * nh * tiles_h * 8);
  const size_t o_tab = o_gp + al(gp * chunk);
  auto ckpt = [&](int k) { return w + (size_t)(k - 1) * al(per * chunk); };  // state after segment k-1 (k >= 1)
  tc_status st;
  for (int r0 = 0; r0 < B; r0 += chunk) {
    const int rows = std::min(chunk, B - r0);
    const double* th = d_params ? d_params + (size_t)r0 * c->n_params : nullptr;
    for (int k = 0; k < S; ++k) {
      tc_circuit* sg = c->ckpt_segs[k];
      KArgs a = base_args(sg, sg->dplan);
      a.psi = ckpt(k + 1);
      a.theta = th;
      a.seed = seed;
      a.row_offset = r0;
      if (k > 0) {
        TC_CHECK_CUDA(cudaMemcpyAsync(ckpt(k + 1), ckpt(k), per * rows, cudaMemcpyDeviceToDevice, s), "checkpoint copy");
        a.synth_init = 0;
      }
      if ((st = run_schedule(sg, KM_FWD, sg->fwd, sg->A, a, w + o_tab, rows, s)) != TC_OK) return st;
    }
    {
      KArgs a = base_args(c, c->dplan);
      a.psi = ckpt(S);
      a.lam = w + o_lam;
      a.epart = (double*)(w + o_ep);
      if ((st = run_ham(c, a, rows, true, s)) != TC_OK) return st;
    }
    for (int k = S - 1; k >= 0; --k) {
      tc_circuit* sg = c->ckpt_segs[k];
      KArgs a = base_args(sg, sg->dplan);
      a.psi = ckpt(k + 1);
      a.lam = w + o_lam;
      a.gpart = (double*)(w + o_gp);
      a.gslots_total = sg->bwd.n_gslots;
      a.theta = th;
      a.seed = seed;
      a.row_offset = r0;
      if ((st = run_schedule(sg, KM_BWD, sg->bwd, sg->A, a, w + o_tab, rows, s, k > 0)) != TC_OK) return st;
      const size_t tiles_b = (size_t)1 << (sg->N - sg->k_bwd);
      TC_CHECK_CUDA(launch_finalize((double*)(w + o_ep), nh, (int)tiles_h, (double*)(w + o_gp), sg->bwd.n_gslots,
                                    (int)tiles_b, sg->d_csr_off, sg->d_csr_slots, c->n_params, rows,
                                    k == S - 1 ? d_e + r0 : nullptr,
                                    c->n_params ? d_g + (size_t)r0 * c->n_params : nullptr, s, k != S - 1),
                    "finalize");
    }
  }
  return TC_OK;
}

}  // namespace

extern "C" {

tc_status tc_expect_grad(tc_circuit* c, const double* d_params, int B, const uint8_t* structures,
                         const double* weights, int T, uint64_t seed, double* d_energy_out, double* d_grad_out,
                         const tc_grad_options* gopt, void* stream) {
  if (!c || (B != 0 && !d_energy_out)) return fail(TC_E_INVALID, "NULL argument");
  if (B < 0) return fail(TC_E_INVALID, "B < 0");
  if (c->n_params > 0 && (!d_params || !d_grad_out) && B > 0) return fail(TC_E_INVALID, "d_params/d_grad_out NULL");
  if (gopt && gopt->mode != TC_GRAD_UNCOMPUTE && gopt->mode != TC_GRAD_CHECKPOINT)
    return fail(TC_E_UNSUPPORTED, "unknown gradient mode");
  const bool ck = gopt && gopt->mode == TC_GRAD_CHECKPOINT;
  if (ck && c->n_noise > 0) return fail(TC_E_UNSUPPORTED, "checkpointed gradients of circuits with noise events");
  if (ck && gopt->checkpoint_ops < 0) return fail(TC_E_INVALID, "checkpoint_ops < 0");
  if (B == 0) return TC_OK;
  tc_status st = ensure_device(c);
  if (st != TC_OK) return st;
  if ((st = ensure_ham(c, structures, weights, T)) != TC_OK) return st;
  if (ck) {
    const int ops = gopt->checkpoint_ops > 0 ? gopt->checkpoint_ops : std::max(1, (c->n_ops + 3) / 4);
    if (c->n_ops == 0) return fail(TC_E_UNSUPPORTED, "checkpointed gradients of an empty circuit");
    if ((st = ensure_segments(c, ops)) != TC_OK) return st;
    int64_t cap = budget(c) / (int64_t)ckpt_row_bytes(c);
    if (gopt->max_rows > 0) cap = std::min<int64_t>(cap, gopt->max_rows);
    if (cap < 1) return fail(TC_E_NOMEM, "one row of checkpoints does not fit the memory budget");
    const int chunk = (int)std::min<int64_t>(B, cap);
    if ((st = ensure_ws(c, ckpt_row_bytes(c) * chunk + 4096)) != TC_OK) return st;
    return expect_grad_ckpt_run(c, d_params, B, seed, d_energy_out, d_grad_out, chunk, (char*)c->ws,
                                (cudaStream_t)stream);
  }
  int64_t cap = budget(c) / (int64_t)grad_row_bytes(c);
  if (gopt && gopt->max_rows > 0) cap = std::min<int64_t>(cap, gopt->max_rows);
  if (cap < 1) return fail(TC_E_NOMEM, "one row of states does not fit the memory budget");
  const int chunk = (int)std::min<int64_t>(B, cap);
  if ((st = ensure_ws(c, grad_ws_bytes(c, chunk))) != TC_OK) return st;
  return expect_grad_run(c, d_params, B, seed, d_energy_out, d_grad_out, chunk, (char*)c->ws, (cudaStream_t)stream);
}

tc_status tc_expect_plain(tc_circuit* c, const double* d_params, int B, const uint8_t* structures,
                          const double* weights, int T, void* d_states_work, double* d_energy_out, void* stream) {
  if (!c || (B != 0 && (!d_states_work || !d_energy_out))) return fail(TC_E_INVALID, "NULL argument");
  if (B < 0 || T < 0) return fail(TC_E_INVALID, "B < 0 or T < 0");
  if (T > 0 && (!structures || !weights)) return fail(TC_E_INVALID, "structures/weights NULL");
  if (c->N != c->n) return fail(TC_E_UNSUPPORTED, "the unfused baseline needs n >= 9");
  if (B > 65535) return fail(TC_E_UNSUPPORTED, "the unfused baseline takes at most 65535 rows per call");
  if (B == 0) return TC_OK;
  tc_status st = ensure_device(c);
  if (st != TC_OK) return st;
  if (!c->plain_built) {
    c->plain = build_plain_schedule(c->gates_orig, c->N, c->dtype == TC_C128 ? kRBFwdC128 : kRBFwd, c->Ap);
    cudaError_t e = c->dplain.upload(c->Ap);
    if (e != cudaSuccess) return cuda_fail(e, "plain plan upload");
    c->plain_built = true;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t trow = (size_t)c->plain.table_total * amp_bytes(c);
  if ((st = ensure_ws(c, trow * B + 256)) != TC_OK) return st;
  KArgs a = base_args(c, c->dplain);
  a.psi = d_states_work;
  a.theta = d_params;
  a.seed = 0;
  // pass 0 of the unfused plan writes the initial state, then one pass per gate
  if ((st = run_schedule(c, KM_FWD, c->plain, c->Ap, a, c->ws, B, s)) != TC_OK) return st;
  TC_CHECK_CUDA(cudaMemsetAsync(d_energy_out, 0, sizeof(double) * B, s), "memset");
  for (int t = 0; t < T; ++t) {
    uint32_t f = 0, sm = 0;
    int ny = 0;
    for (int q = 0; q < c->n; ++q) {
      const uint8_t code = structures[(size_t)t * c->n + q];
      if (code > 3) return fail(TC_E_INVALID, "structure entry outside {0,1,2,3}");
      const uint32_t b = 1u << (c->N - 1 - q);
      if (code == 1 || code == 2) f |= b;
      if (code == 2 || code == 3) sm |= b;
      if (code == 2) ny++;
    }
    TC_CHECK_CUDA(launch_plain_term(is_dbl(c), d_states_work, c->N, B, f, sm, ny & 3, weights[t], d_energy_out, s),
                  "plain term");
  }
  return TC_OK;
}

tc_status tc_state_norms(tc_circuit* c, const void* d_states, int B, double* d_norm2_out, void* stream) {
  if (!c || (B != 0 && (!d_states || !d_norm2_out))) return fail(TC_E_INVALID, "NULL argument");
  if (B < 0) return fail(TC_E_INVALID, "B < 0");
  if (B == 0) return TC_OK;
  const bool dbl = is_dbl(c);
  // 16-byte words per row: 2^n (complex128) or 2^(n-1) (complex64)
  const size_t words = ((size_t)1 << c->n) >> (dbl ? 0 : 1);
  if (words == 0 || ((uintptr_t)d_states & 15)) return fail(TC_E_INVALID, "states must be 16-byte aligned, n >= 1");
  // blocks per row from the width alone (at least 8192 words = 128 KiB each,
  // at most 256), so a row's summation order does not depend on B
  const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)(words / 8192), 256));
  const int chunk = std::min(B, 65535);
  tc_status st = ensure_ws(c, (size_t)chunk * nblk * sizeof(double) + 256);
  if (st != TC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t rb = ((size_t)1 << c->n) * amp_bytes(c);
  for (int r0 = 0; r0 < B; r0 += chunk) {
    const int rows = std::min(chunk, B - r0);
    TC_CHECK_CUDA(launch_norm2(dbl, (const char*)d_states + (size_t)r0 * rb, c->n, rows, nblk, (double*)c->ws, s),
                  "norm");
    TC_CHECK_CUDA(launch_finalize((double*)c->ws, nblk, 1, nullptr, 0, 1, nullptr, nullptr, 0, rows,
                                  d_norm2_out + r0, nullptr, s),
                  "finalize");
  }
  return TC_OK;
}

tc_status tc_mean_stderr(const double* d_x, int n, double* d_out, void* stream) {
  if (!d_x || !d_out || n < 1) return fail(TC_E_INVALID, "NULL argument or n < 1");
  TC_CHECK_CUDA(launch_mean_stderr(d_x, n, d_out, (cudaStream_t)stream), "mean/stderr");
  return TC_OK;
}

tc_status tc_shard_moments(const double* d_x, int n, double* d_out, void* stream) {
  if (!d_x || !d_out || n < 1) return fail(TC_E_INVALID, "NULL argument or n < 1");
  TC_CHECK_CUDA(launch_mean_stderr(d_x, n, d_out, (cudaStream_t)stream, true), "shard moments");
  return TC_OK;
}

tc_status tc_merge_moments(const double* parts, int R, double* out) {
  if (!parts || !out || R < 1) return fail(TC_E_INVALID, "NULL argument or R < 1");
  // pairwise update of (count, mean, M2) in the given order (Chan, Golub and
  // LeVeque's combination of sample variances)
  double n = 0, mean = 0, m2 = 0;
  for (int r = 0; r < R; ++r) {
    const double nb = parts[3 * r], mb = parts[3 * r + 1], m2b = parts[3 * r + 2];
    if (!(nb >= 0) || !std::isfinite(mb) || !(m2b >= 0)) return fail(TC_E_INVALID, "bad shard moments");
    if (nb == 0) continue;
    const double t = n + nb, d = mb - mean;
    mean += d * (nb / t);
    m2 += m2b + d * d * (n * nb / t);
    n = t;
  }
  if (n < 1) return fail(TC_E_INVALID, "no samples in any shard");
  out[0] = mean;
  out[1] = n > 1 ? std::sqrt(m2 / (n - 1) / n) : 0.0;
  return TC_OK;
}

tc_status tc_profile_begin(void) {
  prof_begin();
  return TC_OK;
}

tc_status tc_profile_end(tc_kernel_stat* out, int max_out, int* n_out) {
  int launches[PK_COUNT];
  double ms[PK_COUNT], bytes[PK_COUNT];
  const bool ok = prof_end(launches, ms, bytes);
  int n = 0;
  for (int k = 0; k < PK_COUNT; ++k) {
    if (!launches[k]) continue;
    if (out && n < max_out) {
      out[n].kind = k;
      out[n].launches = launches[k];
      out[n].total_ms = ms[k];
      out[n].algo_bytes = bytes[k];
    }
    ++n;
  }
  if (n_out) *n_out = n;
  return ok ? TC_OK : fail(TC_E_CUDA, "event timing failed");
}

}  // extern "C"
