// Light-cone tensor-network contraction: host planning and C-ABI.
//
// Section "Tensor network engine" / "Custom contraction settings": an
// expectation <0|U^dagger O U|0> is a closed tensor network whose value does
// not depend on the contraction order.  Only the gates in the backward causal
// cone of O matter (every other gate meets its inverse), so the network holds
// the cone's gates (ket), their conjugates (bra), |0> vectors and the Z
// observable.  The path is found on the host by the greedy rule the paper's
// default contractor uses (contract the connected pair that removes the most
// elements), with a rank cap; every step is one complex GEMM after an index
// permutation, folded into gather tables.
#include "tn.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <set>
#include <string>

namespace tcb {

tc_status fail(tc_status st, const std::string& msg);
tc_status cuda_fail(cudaError_t e, const char* where);

namespace {

struct Ten {
  std::vector<int> labels;  // first label = most significant index bit
};

int64_t pow2(int r) { return (int64_t)1 << r; }

}  // namespace

bool tn_build_lightcone(int n_qubits, const int32_t* gate_q, int n_gates, const int32_t* z_q, int n_z, int rank_cap,
                        const int32_t* path, int n_path, TnPlan& P, std::string& err) {
  P = TnPlan{};
  P.n_qubits = n_qubits;
  P.n_gates = n_gates;
  P.gate_q.assign(gate_q, gate_q + 2 * (size_t)n_gates);
  for (int g = 0; g < n_gates; ++g) {
    const int a = gate_q[2 * g], b = gate_q[2 * g + 1];
    if (a < 0 || a >= n_qubits || b < 0 || b >= n_qubits || a == b) {
      err = "gate " + std::to_string(g) + ": qubits out of range or equal";
      return false;
    }
  }
  std::set<int> obs;
  for (int i = 0; i < n_z; ++i) {
    if (z_q[i] < 0 || z_q[i] >= n_qubits) {
      err = "observable qubit out of range";
      return false;
    }
    obs.insert(z_q[i]);
  }
  if (obs.empty()) {
    err = "empty observable";
    return false;
  }
  // ---- backward light cone ------------------------------------------------
  std::set<int> active(obs.begin(), obs.end());
  for (int g = n_gates - 1; g >= 0; --g) {
    const int a = gate_q[2 * g], b = gate_q[2 * g + 1];
    if (active.count(a) || active.count(b)) {
      P.cone.push_back(g);
      active.insert(a);
      active.insert(b);
    }
  }
  std::reverse(P.cone.begin(), P.cone.end());
  P.cone_lo = *active.begin();
  P.cone_hi = *active.rbegin();

  // ---- doubled network ------------------------------------------------------
  std::vector<Ten> T;
  int next_label = 0;
  std::map<int, int> ket, bra;
  auto add_input = [&](int kind, int gate, std::vector<int> labels) {
    TnInput in{};
    in.kind = kind;
    in.gate = gate;
    in.rank = (int)labels.size();
    in.off = (int32_t)P.in_total;
    P.in_total += pow2(in.rank);
    P.inputs.push_back(in);
    T.push_back({labels});
  };
  for (int q : active) {
    ket[q] = next_label++;
    add_input(TS_ZERO, -1, {ket[q]});
    bra[q] = next_label++;
    add_input(TS_ZERO, -1, {bra[q]});
  }
  for (int g : P.cone) {
    const int a = gate_q[2 * g], b = gate_q[2 * g + 1];
    const int ka = next_label++, kb = next_label++;
    add_input(TS_KET, g, {ka, kb, ket[a], ket[b]});
    ket[a] = ka;
    ket[b] = kb;
    const int ba = next_label++, bb = next_label++;
    add_input(TS_BRA, g, {ba, bb, bra[a], bra[b]});
    bra[a] = ba;
    bra[b] = bb;
  }
  for (int q : active) {
    if (obs.count(q)) {
      add_input(TS_Z, -1, {bra[q], ket[q]});
    } else {
      // identity: the bra leg and the ket leg are the same index
      for (auto& t : T)
        for (auto& l : t.labels)
          if (l == bra[q]) l = ket[q];
    }
  }
  const int n_inputs = (int)T.size();

  // ---- path -----------------------------------------------------------------
  std::vector<int> live(n_inputs);
  for (int i = 0; i < n_inputs; ++i) live[i] = i;
  auto out_labels = [&](const Ten& a, const Ten& b, std::vector<int>& fa, std::vector<int>& sh, std::vector<int>& fb) {
    fa.clear();
    sh.clear();
    fb.clear();
    for (int l : a.labels)
      (std::find(b.labels.begin(), b.labels.end(), l) != b.labels.end() ? sh : fa).push_back(l);
    for (int l : b.labels)
      if (std::find(a.labels.begin(), a.labels.end(), l) == a.labels.end()) fb.push_back(l);
  };
  std::vector<std::pair<int, int>> pairs;  // tensor ids
  if (path) {
    std::vector<int> list = live;
    for (int s = 0; s < n_path; ++s) {
      int i = path[2 * s], j = path[2 * s + 1];
      if (i == j || i < 0 || j < 0 || i >= (int)list.size() || j >= (int)list.size()) {
        err = "path step " + std::to_string(s) + " out of range";
        return false;
      }
      if (i > j) std::swap(i, j);
      const int a = list[i], b = list[j];
      list.erase(list.begin() + j);
      list.erase(list.begin() + i);
      list.push_back((int)T.size() + (int)pairs.size());
      pairs.push_back({a, b});
      // placeholder tensor to keep ids aligned; labels filled below
    }
    if (list.size() != 1) {
      err = "path does not contract the network to one tensor";
      return false;
    }
  }
  int64_t tab_total = 0;
  std::vector<int64_t> ten_off(n_inputs);
  for (int i = 0; i < n_inputs; ++i) ten_off[i] = P.inputs[i].off;
  int64_t arena = P.in_total;
  size_t pi = 0;
  while (live.size() > 1) {
    int best_a = -1, best_b = -1;
    if (path) {
      best_a = pairs[pi].first;
      best_b = pairs[pi].second;
      ++pi;
    } else {
      // greedy: connected pair minimising size(out) - size(a) - size(b); ties -> smallest ids
      int64_t best_cost = 0;
      bool found = false;
      std::vector<int> fa, sh, fb;
      for (size_t x = 0; x < live.size(); ++x)
        for (size_t y = x + 1; y < live.size(); ++y) {
          const Ten& A = T[live[x]];
          const Ten& B = T[live[y]];
          out_labels(A, B, fa, sh, fb);
          if (sh.empty()) continue;
          const int r = (int)(fa.size() + fb.size());
          if (r > rank_cap) continue;
          const int64_t cost = pow2(r) - pow2((int)A.labels.size()) - pow2((int)B.labels.size());
          const int ia = std::min(live[x], live[y]), ib = std::max(live[x], live[y]);
          if (!found || cost < best_cost || (cost == best_cost && (ia < best_a || (ia == best_a && ib < best_b)))) {
            found = true;
            best_cost = cost;
            best_a = ia;
            best_b = ib;
          }
        }
      if (!found) {
        err = "no contraction within the rank cap (or the network is disconnected)";
        return false;
      }
    }
    std::vector<int> fa, sh, fb;
    out_labels(T[best_a], T[best_b], fa, sh, fb);
    const int rc = (int)(fa.size() + fb.size());
    if (rc > rank_cap) {
      err = "path step exceeds the rank cap";
      return false;
    }
    TnStep st{};
    st.a = best_a;
    st.b = best_b;
    st.c = (int)T.size();
    st.M = (int)pow2((int)fa.size());
    st.K = (int)pow2((int)sh.size());
    st.N = (int)pow2((int)fb.size());
    // index tables: bit of label l in a tensor = rank - 1 - position
    auto bitpos = [](const Ten& t, int l) {
      const int p = (int)(std::find(t.labels.begin(), t.labels.end(), l) - t.labels.begin());
      return (int)t.labels.size() - 1 - p;
    };
    auto table = [&](const Ten& t, const std::vector<int>& ls) {
      const int64_t off = tab_total;
      const int nb = (int)ls.size();
      for (int64_t v = 0; v < pow2(nb); ++v) {
        int32_t idx = 0;
        for (int u = 0; u < nb; ++u)
          if ((v >> (nb - 1 - u)) & 1) idx |= 1 << bitpos(t, ls[u]);
        P.tables.push_back(idx);
      }
      tab_total += pow2(nb);
      return (int32_t)off;
    };
    st.fa = table(T[best_a], fa);
    st.sa = table(T[best_a], sh);
    st.sb = table(T[best_b], sh);
    st.fb = table(T[best_b], fb);
    st.a_off = ten_off[best_a];
    st.b_off = ten_off[best_b];
    st.c_off = arena;
    ten_off.push_back(arena);
    arena += (int64_t)st.M * st.N;
    P.flops += (double)st.M * st.K * st.N;
    P.write += (double)st.M * st.N;
    P.size = std::max(P.size, (double)st.M * st.N);
    P.max_rank = std::max(P.max_rank, rc);
    Ten c;
    c.labels = fa;
    c.labels.insert(c.labels.end(), fb.begin(), fb.end());
    T.push_back(c);
    P.steps.push_back(st);
    live.erase(std::remove(live.begin(), live.end(), best_a), live.end());
    live.erase(std::remove(live.begin(), live.end(), best_b), live.end());
    live.push_back(st.c);
  }
  if (!T[live[0]].labels.empty()) {
    err = "network is not closed";
    return false;
  }
  P.arena_total = arena;
  P.result_off = P.steps.empty() ? 0 : P.steps.back().c_off;
  return true;
}

}  // namespace tcb

using namespace tcb;

struct tc_tn : TnPlan {};

namespace {
void tn_release(tc_tn* t) {
  if (t->graph) cudaGraphExecDestroy(t->graph);
  if (t->d_tables) cudaFree(t->d_tables);
  if (t->d_inputs) cudaFree(t->d_inputs);
  if (t->d_gate_q) cudaFree(t->d_gate_q);
  if (t->d_arena) cudaFree(t->d_arena);
}
}  // namespace

extern "C" {

tc_status tc_tn_lightcone_create(int n_qubits, const int32_t* gate_qubits, int n_gates, const int32_t* z_qubits,
                                 int n_z, int rank_cap, const int32_t* path, int n_path_steps, tc_tn** out) {
  if (!out) return fail(TC_E_INVALID, "out is NULL");
  *out = nullptr;
  if (n_qubits < 2 || n_gates < 0 || (n_gates > 0 && !gate_qubits) || n_z < 1 || !z_qubits)
    return fail(TC_E_INVALID, "bad sizes or NULL arrays");
  if (rank_cap < 1 || rank_cap > 26) return fail(TC_E_INVALID, "rank_cap must be in 1..26");
  auto* t = new tc_tn();
  std::string err;
  if (!tn_build_lightcone(n_qubits, gate_qubits, n_gates, z_qubits, n_z, rank_cap, path, n_path_steps, *t, err)) {
    delete t;
    return fail(TC_E_INVALID, err);
  }
  *out = t;
  return TC_OK;
}

tc_status tc_tn_info(const tc_tn* t, tc_path_info* o) {
  if (!t || !o) return fail(TC_E_INVALID, "NULL argument");
  *o = tc_path_info{};
  o->flops = 8.0 * t->flops;  // real floating-point operations of the complex multiply-adds
  o->cmacs = t->flops;
  o->write = t->write;
  o->size = t->size;
  o->n_steps = (int32_t)t->steps.size();
  o->max_rank = t->max_rank;
  o->n_cone_gates = (int32_t)t->cone.size();
  o->cone_lo = t->cone_lo;
  o->cone_hi = t->cone_hi;
  o->n_inputs = (int32_t)t->inputs.size();
  return TC_OK;
}

tc_status tc_contract_path(tc_tn* t, int B, const float* d_gates, double* d_out, void* stream) {
  if (!t || !d_gates || !d_out) return fail(TC_E_INVALID, "NULL argument");
  if (B <= 0) return B == 0 ? TC_OK : fail(TC_E_INVALID, "B < 0");
  if (B > 65535) return fail(TC_E_UNSUPPORTED, "at most 65535 instances per call");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (!t->uploaded) {
    if ((e = cudaGetDevice(&t->device)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (!t->tables.empty()) {
      if ((e = cudaMalloc(&t->d_tables, t->tables.size() * 4)) != cudaSuccess) return cuda_fail(e, "tn tables");
      if ((e = cudaMemcpy(t->d_tables, t->tables.data(), t->tables.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "tn tables copy");
    }
    if ((e = cudaMalloc(&t->d_inputs, t->inputs.size() * sizeof(TnInput))) != cudaSuccess) return cuda_fail(e, "tn inputs");
    if ((e = cudaMemcpy(t->d_inputs, t->inputs.data(), t->inputs.size() * sizeof(TnInput), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return cuda_fail(e, "tn inputs copy");
    if (!t->gate_q.empty()) {
      if ((e = cudaMalloc(&t->d_gate_q, t->gate_q.size() * 4)) != cudaSuccess) return cuda_fail(e, "tn gates");
      if ((e = cudaMemcpy(t->d_gate_q, t->gate_q.data(), t->gate_q.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "tn gates copy");
    }
    t->uploaded = true;
  }
  if (B > t->arena_B) {
    if (t->d_arena) cudaFree(t->d_arena);
    t->d_arena = nullptr;
    t->arena_B = 0;
    if ((e = cudaMalloc(&t->d_arena, (size_t)B * t->arena_total * sizeof(float2))) != cudaSuccess)
      return cuda_fail(e, "tn arena");
    t->arena_B = B;
    if (t->graph) cudaGraphExecDestroy(t->graph);
    t->graph = nullptr;
  }
  float2* arena = (float2*)t->d_arena;
  // the whole contraction is one CUDA graph (steps are tiny and launch-bound);
  // it is captured once per (B, input, output) and replayed on `stream`
  if (!t->graph || t->graph_B != B || t->graph_gates != d_gates || t->graph_out != d_out) {
    if (t->graph) cudaGraphExecDestroy(t->graph);
    t->graph = nullptr;
    cudaStream_t cap;
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "stream");
    cudaGraph_t g;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = tn_launch_assemble(*t, B, d_gates, arena, cap);
    for (size_t i = 0; e == cudaSuccess && i < t->steps.size(); ++i) e = tn_launch_step(*t, t->steps[i], B, arena, cap);
    if (e == cudaSuccess) e = tn_launch_result(*t, B, arena, d_out, cap);
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) {
      e = cudaGraphInstantiate(&t->graph, g, 0);
      cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
      t->graph = nullptr;
      return cuda_fail(e, "tn graph capture");
    }
    t->graph_B = B;
    t->graph_gates = d_gates;
    t->graph_out = d_out;
  }
  if ((e = cudaGraphLaunch(t->graph, s)) != cudaSuccess) return cuda_fail(e, "tn graph launch");
  return TC_OK;
}

void tc_tn_destroy(tc_tn* t) {
  if (!t) return;
  tn_release(t);
  delete t;
}

}  // extern "C"
