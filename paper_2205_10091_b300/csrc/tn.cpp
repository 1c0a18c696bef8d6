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
#include <array>
#include <cmath>
#include <map>
#include <random>
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

// Pairwise path over a closed network whose every label joins exactly two
// tensors (all index dimensions 2).  T holds the input tensors (P.inputs
// already carries their offsets); steps, gather tables, arena layout and the
// path metrics are appended to P.  Without a user path the greedy rule picks
// the connected pair minimising size(out) - size(a) - size(b), ties to the
// smallest tensor ids, skipping pairs whose result exceeds rank_cap; with
// no connected pair left, disconnected parts are joined by outer products.
bool tn_plan_once(std::vector<Ten>& T, int rank_cap, const int32_t* path, int n_path, double temp, uint64_t seed,
                  TnPlan& P, std::string& err) {
  const int n_inputs = (int)T.size();
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> uni(1e-300, 1.0);
  int max_label = -1;
  for (const auto& t : T)
    for (int l : t.labels) max_label = std::max(max_label, l);
  // holders[l] = the two tensors carrying label l
  std::vector<std::array<int, 2>> holders((size_t)(max_label + 1), std::array<int, 2>{-1, -1});
  for (int i = 0; i < n_inputs; ++i)
    for (int l : T[i].labels) {
      auto& h = holders[l];
      if (h[0] < 0) {
        h[0] = i;
      } else if (h[1] < 0 && h[0] != i) {
        h[1] = i;
      } else {
        err = "label " + std::to_string(l) + " is not shared by exactly two tensors";
        return false;
      }
    }
  for (int l = 0; l <= max_label; ++l)
    if (holders[l][0] >= 0 && holders[l][1] < 0) {
      err = "network is not closed (label " + std::to_string(l) + " is open)";
      return false;
    }
  std::vector<int> live(n_inputs);
  for (int i = 0; i < n_inputs; ++i) live[i] = i;
  auto split_labels = [&](const Ten& a, const Ten& b, std::vector<int>& fa, std::vector<int>& sh,
                          std::vector<int>& fb) {
    fa.clear();
    sh.clear();
    fb.clear();
    for (int l : a.labels)
      (std::find(b.labels.begin(), b.labels.end(), l) != b.labels.end() ? sh : fa).push_back(l);
    for (int l : b.labels)
      if (std::find(a.labels.begin(), a.labels.end(), l) == a.labels.end()) fb.push_back(l);
  };
  std::vector<std::pair<int, int>> pairs;  // tensor ids of a user path
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
      list.push_back(n_inputs + (int)pairs.size());
      pairs.push_back({a, b});
    }
    if (list.size() != 1) {
      err = "path does not contract the network to one tensor";
      return false;
    }
  }
  int64_t tab_total = (int64_t)P.tables.size();
  std::vector<int64_t> ten_off(n_inputs);
  for (int i = 0; i < n_inputs; ++i) ten_off[i] = P.inputs[i].off;
  int64_t arena = P.in_total;
  size_t pi = 0;
  std::vector<int> fa, sh, fb;
  while (live.size() > 1) {
    int best_a = -1, best_b = -1;
    if (path) {
      best_a = pairs[pi].first;
      best_b = pairs[pi].second;
      ++pi;
    } else {
      double best_cost = 0;
      bool found = false, connected = false;
      for (int x : live)
        for (int l : T[x].labels) {
          const int y = holders[l][0] == x ? holders[l][1] : holders[l][0];
          if (y <= x) continue;  // each connected pair once, from its smaller id
          connected = true;
          split_labels(T[x], T[y], fa, sh, fb);
          const int r = (int)(fa.size() + fb.size());
          if (r > rank_cap) continue;
          const int64_t c = pow2(r) - pow2((int)T[x].labels.size()) - pow2((int)T[y].labels.size());
          double cost = (double)c;
          if (temp > 0) {  // randomised trial: Gumbel noise on a log-scaled cost
            cost = (c < 0 ? -1.0 : 1.0) * std::log2(1.0 + std::fabs((double)c)) - temp * std::log(-std::log(uni(rng)));
          }
          if (!found || cost < best_cost || (cost == best_cost && (x < best_a || (x == best_a && y < best_b)))) {
            found = true;
            best_cost = cost;
            best_a = x;
            best_b = y;
          }
        }
      if (!found && !connected) {
        // disconnected components: once each is contracted, join the two
        // smallest tensors by an outer product (scalars in a closed network)
        int best_r = 0;
        for (size_t x = 0; x < live.size(); ++x)
          for (size_t y = x + 1; y < live.size(); ++y) {
            const int a = std::min(live[x], live[y]), b = std::max(live[x], live[y]);
            split_labels(T[a], T[b], fa, sh, fb);
            if (!sh.empty()) continue;
            const int r = (int)(fa.size() + fb.size());
            if (r > rank_cap) continue;
            if (!found || r < best_r || (r == best_r && (a < best_a || (a == best_a && b < best_b)))) {
              found = true;
              best_r = r;
              best_a = a;
              best_b = b;
            }
          }
      }
      if (!found) {
        err = "no contraction within the rank cap";
        return false;
      }
    }
    split_labels(T[best_a], T[best_b], fa, sh, fb);
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
    if ((st.M + 31) / 32 > 65535 || (st.N + 31) / 32 > 65535) {
      err = "path step too large for one launch (free rank above 21 on one side)";
      return false;
    }
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
    for (int l : c.labels) {
      auto& h = holders[l];
      h[h[0] == best_a || h[0] == best_b ? 0 : 1] = st.c;
    }
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

// Layout for the fused executor.  Steps are grouped by tree level (see
// tn.h); live tensors get offsets first-fit: inputs first, then per group the
// results of all its steps while every operand of the group is still live,
// then the group's operands are released (the root result stays).
void tn_layout_fused(TnPlan& P) {
  const int n_inputs = (int)P.inputs.size();
  const int n_steps = (int)P.steps.size();
  const int n_ten = n_inputs + n_steps;
  std::vector<int64_t> off(n_ten, -1), size(n_ten, 0);
  std::vector<std::pair<int64_t, int64_t>> live;  // (offset, size), sorted by offset
  int64_t peak = 0;
  auto place = [&](int id, int64_t sz) {
    int64_t at = 0;
    size_t pos = 0;
    for (; pos < live.size(); ++pos) {
      if (live[pos].first - at >= sz) break;
      at = std::max(at, live[pos].first + live[pos].second);
    }
    live.insert(live.begin() + pos, {at, sz});
    off[id] = at;
    size[id] = sz;
    peak = std::max(peak, at + sz);
  };
  auto release = [&](int id) {
    for (size_t i = 0; i < live.size(); ++i)
      if (live[i].first == off[id] && live[i].second == size[id]) {
        live.erase(live.begin() + i);
        return;
      }
  };
  auto lg = [](int64_t x) {
    int r = 0;
    while (((int64_t)1 << r) < x) ++r;
    return r;
  };
  auto tab_len = [](int g) {
    return g <= kTnFullTabBits ? (1 << g) : (1 << ((g + 1) / 2)) + (1 << (g - (g + 1) / 2));
  };
  // levels
  std::vector<int> lvl_t(n_ten, 0), lvl(n_steps);
  for (int s = 0; s < n_steps; ++s) {
    const TnStep& st = P.steps[s];
    lvl[s] = 1 + std::max(lvl_t[st.a], lvl_t[st.b]);
    lvl_t[st.c] = lvl[s];
  }
  std::vector<int> order(n_steps);
  for (int s = 0; s < n_steps; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return lvl[x] < lvl[y]; });
  // lanes per output: enough to fill the CTA with a small result, but each
  // lane keeps at least four terms of the sum (a shorter share costs more in
  // shuffles and work units than it saves)
  auto tpo_of = [](const TnStep& st) {
    int t = kTnFusedThreads / std::max(1, st.M * st.N);
    t = std::max(1, std::min(32, t));
    while (t > 1 && 4 * t > st.K) t >>= 1;
    return t;
  };
  auto step_tabs = [&](const TnStep& st) {  // + 1: the pair table's alignment word
    return tab_len(lg(st.M)) + 2 * tab_len(lg(st.K)) + tab_len(lg(st.N)) + 1;
  };
  // paired steps (one lane per output, >= 64 outputs, full tables): a lane
  // computes outputs e and e + 32, which share A's row when rows hold >= 64
  // outputs (mode 1) and B's column otherwise (mode 2: e + 32 is row i + 32 / N)
  auto pair_mode = [&](const TnStep& st) {
    if (tpo_of(st) != 1 || (int64_t)st.M * st.N < 64 || lg(st.K) > kTnFullTabBits) return 0;
    return st.N >= 64 ? 1 : 2;
  };
  auto pair_of = [&](const TnStep& st) { return pair_mode(st) != 0; };
  auto items_of = [&](const TnStep& st) {
    return (int64_t)st.M * st.N * tpo_of(st) / (pair_of(st) ? 2 : 1);
  };
  // output index of a work item: e = item / tpo, or for a paired step the
  // first output of the pair (blocks of 64 outputs: lanes take j and j + 32)
  auto out_of = [&](const TnStep& st, int64_t item) -> int64_t {
    if (pair_of(st)) return ((item >> 5) << 6) | (item & 31);
    return item / tpo_of(st);
  };
  // shared-memory swizzle of every tensor (tn_swz), chosen for the lanes of
  // the one step that reads it: two sample warps (the step's first and middle
  // one), two k-iterations each; cost = wavefronts of the warp's loads (the
  // largest number of distinct entries on one bank pair)
  std::vector<int> rot(n_ten, 0);
  for (int s = 0; s < n_steps; ++s) {
    const TnStep& st = P.steps[s];
    const int tpo = tpo_of(st), lgN = lg(st.N);
    const int64_t n_items = items_of(st);
    const bool paired = pair_of(st);
    for (int side = 0; side < 2; ++side) {
      int best = 0;
      int64_t best_cost = -1;
      for (int r = 0; r < 4; ++r) {
        int64_t cost = 0;
        for (int64_t w0 : {(int64_t)0, (n_items / 64) * 32}) {
          for (int it = 0; it < (paired ? 4 : 2); ++it) {
            int32_t words[32];
            int nw = 0;
            for (int l = 0; l < 32; ++l) {
              const int64_t item = w0 + l;
              // a paired step loads for outputs e (it even) and e + 32 (it odd)
              const int64_t e = out_of(st, item) + (paired && (it & 1) ? 32 : 0);
              const int k = paired ? it >> 1 : (int)(item % tpo) + it * tpo;
              if (e >= (int64_t)st.M * st.N || k >= st.K) continue;
              const int64_t i = e >> lgN, j = e & (st.N - 1);
              const int32_t x = side == 0 ? P.tables[st.fa + i] + P.tables[st.sa + k]
                                          : P.tables[st.sb + k] + P.tables[st.fb + j];
              words[nw++] = tn_swz(x, r);
            }
            int worst = 0;
            for (int q = 0; q < nw; ++q) {  // distinct words on the bank pair of word q
              int cnt = 0;
              for (int u = 0; u < nw; ++u) {
                if ((words[u] & 15) != (words[q] & 15)) continue;
                bool first = true;
                for (int v = 0; v < u; ++v) first = first && words[v] != words[u];
                cnt += first ? 1 : 0;
              }
              worst = std::max(worst, cnt);
            }
            cost += worst;
          }
        }
        if (best_cost < 0 || cost < best_cost) {
          best_cost = cost;
          best = r;
        }
      }
      rot[side == 0 ? st.a : st.b] = best;
    }
  }
  for (int i = 0; i < n_inputs; ++i) place(i, pow2(P.inputs[i].rank));
  P.fblob.clear();
  P.fblob_ok = true;
  P.n_groups = 0;
  std::vector<size_t> starts;
  size_t g0 = 0;
  while (g0 < order.size()) {
    // a group: consecutive steps of one level while the block fits
    size_t g1 = g0;
    int len = kTnGHdr;
    while (g1 < order.size() && lvl[order[g1]] == lvl[order[g0]]) {
      const int add = kTnSRec + step_tabs(P.steps[order[g1]]);
      if (g1 > g0 && len + add + 3 > kTnBlobMax) break;  // + the alignment padding
      len += add;
      ++g1;
    }
    if (len > kTnBlobMax) P.fblob_ok = false;
    // steps of the group sorted by tpo so a warp never mixes tpo values
    std::vector<int> gs(order.begin() + g0, order.begin() + g1);
    auto run_key = [&](int x) { return 2 * tpo_of(P.steps[x]) + (pair_of(P.steps[x]) ? 1 : 0); };
    std::stable_sort(gs.begin(), gs.end(), [&](int x, int y) { return run_key(x) < run_key(y); });
    for (int s : gs) place(P.steps[s].c, (int64_t)P.steps[s].M * P.steps[s].N);
    const size_t gstart = P.fblob.size();
    starts.push_back(gstart);
    P.fblob.resize(gstart + kTnGHdr + kTnSRec * gs.size(), 0);
    int64_t items = 0;
    int prev_key = -1;
    for (size_t q = 0; q < gs.size(); ++q) {
      const TnStep& st = P.steps[gs[q]];
      const int tpo = tpo_of(st);
      const int key = run_key(gs[q]);
      if (key != prev_key) items = (items + 31) / 32 * 32;  // a warp never spans two tpo values (or pairings)
      prev_key = key;
      const int lgM = lg(st.M), lgK = lg(st.K), lgN = lg(st.N);
      if (lgM > 16 || lgK > 16 || lgN > 16) P.fblob_ok = false;
      int32_t* rec = P.fblob.data() + gstart + kTnGHdr + kTnSRec * q;
      rec[0] = (int32_t)items;
      rec[1] = st.M;
      rec[2] = st.K;
      rec[3] = st.N;
      rec[4] = lgM;
      rec[5] = lgK;
      rec[6] = lgN;
      rec[7] = tpo | (rot[st.c] << 8) | (pair_mode(st) << 16);
      rec[8] = (int32_t)off[st.a];
      rec[9] = (int32_t)off[st.b];
      rec[10] = (int32_t)off[st.c];
      auto split = [&](int32_t tab, int g, int r) {
        if (g <= kTnFullTabBits) {
          for (int v = 0; v < (1 << g); ++v) P.fblob.push_back(tn_swz(P.tables[tab + v], r));
          return;
        }
        const int lo = (g + 1) / 2, hi = g - lo;
        for (int v = 0; v < (1 << lo); ++v) P.fblob.push_back(tn_swz(P.tables[tab + v], r));
        for (int v = 0; v < (1 << hi); ++v) P.fblob.push_back(tn_swz(P.tables[tab + ((int64_t)v << lo)], r));
      };
      // (rec is re-taken after each push: the blob may reallocate)
      auto mark = [&](int field) {
        P.fblob[gstart + kTnGHdr + kTnSRec * q + field] = (int32_t)(P.fblob.size() - gstart);
      };
      mark(11);
      split(st.fa, lgM, rot[st.a]);
      if (lgK <= kTnFullTabBits) {
        // full k tables interleaved as (sa[k], sb[k]) pairs at an even offset:
        // one 8-byte load per k (the group block starts 16-byte aligned)
        if ((P.fblob.size() - gstart) & 1) P.fblob.push_back(0);
        mark(12);
        for (int v = 0; v < (1 << lgK); ++v) {
          P.fblob.push_back(tn_swz(P.tables[st.sa + v], rot[st.a]));
          P.fblob.push_back(tn_swz(P.tables[st.sb + v], rot[st.b]));
        }
        P.fblob[gstart + kTnGHdr + kTnSRec * q + 13] = P.fblob[gstart + kTnGHdr + kTnSRec * q + 12] + 1;
      } else {
        mark(12);
        split(st.sa, lgK, rot[st.a]);
        mark(13);
        split(st.sb, lgK, rot[st.b]);
      }
      mark(14);
      split(st.fb, lgN, rot[st.b]);
      items += items_of(st);
      if (items_of(st) > (1 << 26)) P.fblob_ok = false;
    }
    items = (items + 31) / 32 * 32;
    while (P.fblob.size() % 4) P.fblob.push_back(0);  // the next group's records stay 16-byte aligned
    P.fblob[gstart + 0] = (int32_t)gs.size();
    P.fblob[gstart + 1] = (int32_t)std::min<int64_t>(items, INT32_MAX);
    for (int s : gs) {
      release(P.steps[s].a);
      release(P.steps[s].b);
    }
    ++P.n_groups;
    g0 = g1;
  }
  starts.push_back(P.fblob.size());
  for (size_t i = 0; i + 1 < starts.size(); ++i) {
    const int32_t len = (int32_t)(starts[i + 1] - starts[i]);
    if (len > kTnBlobMax) P.fblob_ok = false;
    P.fblob[starts[i] + 2] = len;
    if (i > 0) P.fblob[starts[i - 1] + 3] = len;
  }
  P.in_soff.assign(n_inputs, 0);
  for (int i = 0; i < n_inputs; ++i) P.in_soff[i] = (int32_t)off[i] | (int32_t)(rot[i] << 28);
  P.smem_entries = peak;
  P.result_soff = n_steps == 0 ? 0 : (int32_t)off[P.steps.back().c];
}

// Path for T: the user's, else the deterministic greedy path, else (trials >
// 1) the best of that and trials - 1 randomised greedy runs (costs perturbed
// by Gumbel noise, seeds 1..trials-1): plans whose live tensors fit the fused
// executor first, then fewer FLOPs, then less WRITE.
bool tn_plan_path(std::vector<Ten>& T, int rank_cap, const int32_t* path, int n_path, int trials, TnPlan& P,
                  std::string& err) {
  if (path || trials <= 1) {
    if (!tn_plan_once(T, rank_cap, path, n_path, 0.0, 0, P, err)) return false;
    tn_layout_fused(P);
    return true;
  }
  TnPlan best;
  bool have = false;
  std::string first_err;
  for (int t = 0; t < trials; ++t) {
    std::vector<Ten> Tt = T;
    TnPlan Pt = P;
    std::string e;
    if (!tn_plan_once(Tt, rank_cap, nullptr, 0, t == 0 ? 0.0 : 1.0, (uint64_t)t, Pt, e)) {
      if (first_err.empty()) first_err = e;
      continue;
    }
    tn_layout_fused(Pt);
    const bool fits = tn_fused_ok(Pt), best_fits = have && tn_fused_ok(best);
    if (!have || (fits && !best_fits) ||
        (fits == best_fits && (Pt.flops < best.flops || (Pt.flops == best.flops && Pt.write < best.write)))) {
      best = std::move(Pt);
      have = true;
    }
  }
  if (!have) {
    err = first_err;
    return false;
  }
  P = std::move(best);
  return true;
}

bool tn_build_lightcone(int n_qubits, const int32_t* gate_q, int n_gates, const int32_t* z_q, int n_z, int rank_cap,
                        int trials, const int32_t* path, int n_path, TnPlan& P, std::string& err) {
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
  return tn_plan_path(T, rank_cap, path, n_path, trials, P, err);
}

// Circuit network <init| K^dagger P K |init> for a Pauli string P, K the ops
// that survive pruning (Section "Custom contraction settings": the testbed
// expectation computed as one network, two-qubit gates split in two tensors).
//   prune 0  every op and qubit (the whole doubled network)
//   prune 1  backward causal cone of P in circuit order
//   prune 2  cone with commuting diagonal gates removed: walking back from P
//            in the Heisenberg picture, each qubit's support is none, diagonal
//            (only I/Z factors) or full.  A diagonal gate commutes with the
//            operator unless one of its qubits is full, so it drops out
//            exactly; a kept diagonal gate makes its idle qubits diagonal (it
//            multiplies X/Y factors by Z on the partner).  A non-diagonal gate
//            on a supported qubit makes its qubits full.
//   split 1  RZZ, CZ and CNOT enter as two rank-3 tensors joined by a bond
//            of dimension 2 (their operator-Schmidt rank), else as one 4x4.
bool tn_build_circuit(int n, int init, const tc_op* ops, int n_ops, int n_params, const double* mats, int n_mats,
                      const uint8_t* pauli, int prune, int split, int rank_cap, int trials, const int32_t* path,
                      int n_path, TnPlan& P, std::string& err) {
  P = TnPlan{};
  P.circuit = true;
  P.n_qubits = n;
  P.n_params = n_params;
  auto is_diag_mat = [&](int off, int dim) {
    for (int r = 0; r < dim; ++r)
      for (int c = 0; c < dim; ++c)
        if (r != c && (mats[2 * (off + r * dim + c)] != 0.0 || mats[2 * (off + r * dim + c) + 1] != 0.0)) return false;
    return true;
  };
  std::vector<char> two(n_ops), diag(n_ops);
  for (int i = 0; i < n_ops; ++i) {
    const tc_op& o = ops[i];
    const bool q2 = o.kind == TC_OP_RZZ || o.kind == TC_OP_CNOT || o.kind == TC_OP_CZ || o.kind == TC_OP_U2;
    if (o.kind < TC_OP_H || o.kind > TC_OP_U2) {
      err = "op " + std::to_string(i) + ": kind not supported by tensor-network plans (noise and random-axis "
            "rotations need the state-vector engine)";
      return false;
    }
    if (o.q0 < 0 || o.q0 >= n || (q2 && (o.q1 < 0 || o.q1 >= n || o.q1 == o.q0))) {
      err = "op " + std::to_string(i) + ": qubit out of range";
      return false;
    }
    if (o.param >= n_params || o.param < -1) {
      err = "op " + std::to_string(i) + ": parameter index out of range";
      return false;
    }
    const int dim = o.kind == TC_OP_U1 ? 2 : 4;
    if ((o.kind == TC_OP_U1 || o.kind == TC_OP_U2) && (o.mat < 0 || (int64_t)o.mat + dim * dim > n_mats || !mats)) {
      err = "op " + std::to_string(i) + ": matrix offset out of range";
      return false;
    }
    two[i] = q2;
    diag[i] = o.kind == TC_OP_RZ || o.kind == TC_OP_RZZ || o.kind == TC_OP_CZ ||
              ((o.kind == TC_OP_U1 || o.kind == TC_OP_U2) && is_diag_mat(o.mat, dim));
  }
  std::vector<int> sup(n, 0);  // 0 none, 1 diagonal, 2 full
  bool any = false;
  for (int q = 0; q < n; ++q) {
    if (pauli[q] > 3) {
      err = "Pauli code out of range";
      return false;
    }
    sup[q] = pauli[q] == 0 ? 0 : (pauli[q] == 3 ? 1 : 2);
    any = any || pauli[q] != 0;
  }
  if (!any) {
    err = "empty observable";
    return false;
  }
  std::vector<char> keep(n_ops, 0);
  if (prune == 0) {
    std::fill(keep.begin(), keep.end(), 1);
    for (int q = 0; q < n; ++q) sup[q] = std::max(sup[q], 1);
  } else {
    for (int i = n_ops - 1; i >= 0; --i) {
      const tc_op& o = ops[i];
      const int a = o.q0, b = two[i] ? o.q1 : o.q0;
      if (prune == 1) {
        if (sup[a] || sup[b]) {
          keep[i] = 1;
          sup[a] = sup[b] = 2;
        }
      } else if (diag[i]) {
        if (sup[a] == 2 || sup[b] == 2) {
          keep[i] = 1;
          sup[a] = std::max(sup[a], 1);
          sup[b] = std::max(sup[b], 1);
        }
      } else if (sup[a] || sup[b]) {
        keep[i] = 1;
        sup[a] = sup[b] = 2;
      }
    }
  }
  P.cone_lo = n;
  P.cone_hi = -1;
  for (int q = 0; q < n; ++q)
    if (sup[q]) {
      P.cone_lo = std::min(P.cone_lo, q);
      P.cone_hi = std::max(P.cone_hi, q);
      ++P.n_active;
    }
  for (int i = 0; i < n_ops; ++i) {
    const tc_op& o = ops[i];
    P.ops.push_back(TnOp{o.kind, o.param, (float)o.scale, o.mat});
    if (keep[i]) P.cone.push_back(i);
  }
  if (mats)
    for (int i = 0; i < 2 * n_mats; ++i) P.mats.push_back((float)mats[i]);

  // ---- doubled network ------------------------------------------------------
  std::vector<Ten> T;
  int next_label = 0;
  std::vector<int> ket(n, -1), bra(n, -1);
  auto add_input = [&](int kind, int gate, int conj, std::vector<int> labels) {
    TnInput in{};
    in.kind = kind;
    in.gate = gate;
    in.conj = conj;
    in.rank = (int)labels.size();
    in.off = (int32_t)P.in_total;
    P.in_total += pow2(in.rank);
    P.inputs.push_back(in);
    T.push_back({std::move(labels)});
  };
  const int vec = init == TC_INIT_PLUS ? TS_PLUS : TS_ZERO;
  for (int q = 0; q < n; ++q)
    if (sup[q]) {
      ket[q] = next_label++;
      add_input(vec, -1, 0, {ket[q]});
      bra[q] = next_label++;
      add_input(vec, -1, 1, {bra[q]});
    }
  for (int i : P.cone) {
    const tc_op& o = ops[i];
    for (int side = 0; side < 2; ++side) {
      std::vector<int>& ch = side ? bra : ket;
      if (!two[i]) {
        const int out = next_label++;
        add_input(TS_OP1, i, side, {out, ch[o.q0]});
        ch[o.q0] = out;
      } else if (split && (o.kind == TC_OP_RZZ || o.kind == TC_OP_CZ || o.kind == TC_OP_CNOT)) {
        const int k = next_label++, oa = next_label++, ob = next_label++;
        add_input(TS_SPA, i, side, {oa, ch[o.q0], k});
        add_input(TS_SPB, i, side, {ob, ch[o.q1], k});
        ch[o.q0] = oa;
        ch[o.q1] = ob;
      } else {
        const int oa = next_label++, ob = next_label++;
        add_input(TS_OP2, i, side, {oa, ob, ch[o.q0], ch[o.q1]});
        ch[o.q0] = oa;
        ch[o.q1] = ob;
      }
    }
  }
  for (int q = 0; q < n; ++q) {
    if (!sup[q]) continue;
    if (pauli[q]) {
      add_input(TS_PAULI, pauli[q], 0, {bra[q], ket[q]});
    } else {
      for (auto& t : T)
        for (auto& l : t.labels)
          if (l == bra[q]) l = ket[q];
    }
  }
  return tn_plan_path(T, rank_cap, path, n_path, trials, P, err);
}

}  // namespace tcb

using namespace tcb;

struct tc_tn : TnPlan {};

namespace {
void tn_release(tc_tn* t) {
  if (t->graph) cudaGraphExecDestroy(t->graph);
  if (t->err_ev) cudaEventDestroy(t->err_ev);
  if (t->h_err) cudaFreeHost(t->h_err);
  if (t->d_err) cudaFree(t->d_err);
  if (t->d_tables) cudaFree(t->d_tables);
  if (t->d_inputs) cudaFree(t->d_inputs);
  if (t->d_gate_q) cudaFree(t->d_gate_q);
  if (t->d_ops) cudaFree(t->d_ops);
  if (t->d_mats) cudaFree(t->d_mats);
  if (t->d_fblob) cudaFree(t->d_fblob);
  if (t->d_in_soff) cudaFree(t->d_in_soff);
  if (t->d_arena) cudaFree(t->d_arena);
  if (t->d_lsteps) cudaFree(t->d_lsteps);
  if (t->d_lstart) cudaFree(t->d_lstart);
}
}  // namespace

extern "C" {

tc_status tc_tn_lightcone_create(int n_qubits, const int32_t* gate_qubits, int n_gates, const int32_t* z_qubits,
                                 int n_z, int rank_cap, int greedy_trials, const int32_t* path, int n_path_steps,
                                 tc_tn** out) {
  if (!out) return fail(TC_E_INVALID, "out is NULL");
  *out = nullptr;
  if (n_qubits < 2 || n_gates < 0 || (n_gates > 0 && !gate_qubits) || n_z < 1 || !z_qubits)
    return fail(TC_E_INVALID, "bad sizes or NULL arrays");
  if (rank_cap < 1 || rank_cap > 26) return fail(TC_E_INVALID, "rank_cap must be in 1..26");
  auto* t = new tc_tn();
  std::string err;
  if (greedy_trials < 0 || greedy_trials > 4096) {
    delete t;
    return fail(TC_E_INVALID, "greedy_trials must be in 0..4096");
  }
  if (!tn_build_lightcone(n_qubits, gate_qubits, n_gates, z_qubits, n_z, rank_cap, greedy_trials, path, n_path_steps,
                          *t, err)) {
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
  o->n_active = t->circuit ? t->n_active : t->cone_hi - t->cone_lo + 1;
  o->fused = tn_fused_ok(*t) ? 1 : 0;
  o->smem_bytes = (int32_t)std::min<int64_t>(t->smem_entries * 8, INT32_MAX);
  o->fused_groups = t->n_groups;
  o->n_inputs = (int32_t)t->inputs.size();
  for (const auto& st : t->steps)
    if (tn_step_tc_eligible(st, t->tc_min_cmacs)) {
      o->tc_steps++;
      o->tc_cmacs += (double)st.M * st.N * st.K;
    }
  o->blob_ints = tn_fused_ok(*t) ? (int32_t)t->fblob.size() : 0;
  o->max_cluster = t->max_cluster;
  o->split_min_items = t->split_min;
  if (tn_fused_ok(*t))
    for (size_t off = 0, gi = 0; gi < (size_t)t->n_groups && off + 2 < t->fblob.size(); ++gi) {
      if (t->fblob[off + 1] >= t->split_min) o->split_groups++;
      off += (size_t)t->fblob[off + 2];
    }
  return TC_OK;
}

tc_status tc_tn_set_cluster(tc_tn* t, int max_cluster, int split_min_items) {
  if (!t) return fail(TC_E_INVALID, "NULL plan");
  if (max_cluster < 1 || max_cluster > kTnMaxCluster || (max_cluster & (max_cluster - 1)))
    return fail(TC_E_INVALID, "max_cluster must be 1, 2, 4 or 8");
  if (split_min_items < 1) return fail(TC_E_INVALID, "split_min_items must be >= 1");
  t->max_cluster = max_cluster;
  t->split_min = split_min_items;
  t->fused_B = -1;  // the next call recomputes the launch shape
  return TC_OK;
}

tc_status tc_tn_set_tc_threshold(tc_tn* t, double min_cmacs) {
  if (!t) return fail(TC_E_INVALID, "NULL plan");
  if (!(min_cmacs >= 0.0)) return fail(TC_E_INVALID, "min_cmacs must be >= 0");
  t->tc_min_cmacs = min_cmacs;
  if (t->graph) cudaGraphExecDestroy(t->graph);  // the next call re-captures with the new split
  t->graph = nullptr;
  return TC_OK;
}

}  // extern "C"

namespace {
// Uploads the plan once.  A plan whose live tensors fit in shared memory runs
// as one fused launch (in the split-precision modes only when no step reaches
// the tensor-core threshold); otherwise the arena is sized for B instances
// and the whole contraction (assembly, every path step, result) replays as
// one CUDA graph, captured once per (B, source buffer, output buffer,
// precision).
tc_status tn_run(tc_tn* t, int B, const float* d_src, double* d_out, int prec, void* stream) {
  if (B > 65535) return fail(TC_E_UNSUPPORTED, "at most 65535 instances per call");
  if (prec != TN_FP32 && prec != TN_TF32X3 && prec != TN_BF16X6) return fail(TC_E_INVALID, "unknown precision");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  // an earlier call's tensor-core step reported a timed-out wait
  if (t->err_pending && cudaEventQuery(t->err_ev) == cudaSuccess) {
    t->err_pending = false;
    if (*t->h_err) {
      *t->h_err = 0;
      if ((e = cudaMemsetAsync(t->d_err, 0, sizeof(int), s)) != cudaSuccess) return cuda_fail(e, "tn status reset");
      return fail(TC_E_TIMEOUT, "an earlier contraction on this plan: a tensor-core step's wait timed out");
    }
  }
  bool use_tc = false;
  if (prec != TN_FP32)
    for (const auto& st : t->steps) use_tc = use_tc || tn_step_tc_eligible(st, t->tc_min_cmacs);
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
    if (!t->ops.empty()) {
      if ((e = cudaMalloc(&t->d_ops, t->ops.size() * sizeof(TnOp))) != cudaSuccess) return cuda_fail(e, "tn ops");
      if ((e = cudaMemcpy(t->d_ops, t->ops.data(), t->ops.size() * sizeof(TnOp), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "tn ops copy");
    }
    if (!t->mats.empty()) {
      if ((e = cudaMalloc(&t->d_mats, t->mats.size() * 4)) != cudaSuccess) return cuda_fail(e, "tn mats");
      if ((e = cudaMemcpy(t->d_mats, t->mats.data(), t->mats.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "tn mats copy");
    }
    if (tn_fused_ok(*t)) {
      if ((e = cudaMalloc(&t->d_fblob, t->fblob.size() * 4)) != cudaSuccess) return cuda_fail(e, "tn fused steps");
      if ((e = cudaMemcpy(t->d_fblob, t->fblob.data(), t->fblob.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "tn fused steps copy");
      if ((e = cudaMalloc(&t->d_in_soff, t->in_soff.size() * 4)) != cudaSuccess) return cuda_fail(e, "tn offsets");
      if ((e = cudaMemcpy(t->d_in_soff, t->in_soff.data(), t->in_soff.size() * 4, cudaMemcpyHostToDevice)) !=
          cudaSuccess)
        return cuda_fail(e, "tn offsets copy");
    }
    t->uploaded = true;
  }
  if (use_tc && !t->d_err) {
    if ((e = cudaMalloc(&t->d_err, sizeof(int))) != cudaSuccess) return cuda_fail(e, "tn status");
    if ((e = cudaMemset(t->d_err, 0, sizeof(int))) != cudaSuccess) return cuda_fail(e, "tn status");
    if ((e = cudaMallocHost(&t->h_err, sizeof(int))) != cudaSuccess) return cuda_fail(e, "tn status");
    *t->h_err = 0;
    if ((e = cudaEventCreateWithFlags(&t->err_ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "tn status event");
  }
  if (tn_fused_ok(*t) && !use_tc) {
    if (t->fused_B != B) {
      t->fused_cl = tn_fused_cluster(*t, B);
      t->fused_grid = tn_fused_grid(*t, B, t->fused_cl);
      t->fused_B = B;
    }
    if (t->fused_grid < 1) return fail(TC_E_CUDA, "tn fused launch: no valid grid");
    if ((e = tn_launch_fused(*t, B, d_src, d_out, t->fused_grid, t->fused_cl, s)) != cudaSuccess)
      return cuda_fail(e, "tn fused launch");
    return TC_OK;
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
  if (!t->graph || t->graph_B != B || t->graph_gates != d_src || t->graph_out != d_out || t->graph_prec != prec) {
    if (t->graph) cudaGraphExecDestroy(t->graph);
    t->graph = nullptr;
    // steps grouped by level of the contraction tree (one more than their
    // operands'): the steps of a level are independent and every step writes
    // its own arena region, so a level's CUDA-core steps run as one launch and
    // its tensor-core steps one launch each.  lstart holds, per level, the first
    // output tile of each of its CUDA-core steps and the level's tile count.
    std::vector<int> lev(t->steps.size());
    int maxl = 0;
    {
      std::vector<int> tlev;  // level of each tensor id (inputs 0)
      for (size_t i = 0; i < t->steps.size(); ++i) {
        const TnStep& st = t->steps[i];
        const int hi = std::max(std::max(st.a, st.b), st.c);
        if ((int)tlev.size() <= hi) tlev.resize(hi + 1, 0);
        lev[i] = 1 + std::max(tlev[st.a], tlev[st.b]);
        tlev[st.c] = lev[i];
        maxl = std::max(maxl, lev[i]);
      }
    }
    std::vector<TnStep> ls;
    std::vector<int> lstart, lfirst(maxl + 2, 0), lso(maxl + 2, 0);  // per level: first step, first lstart entry
    std::vector<std::vector<size_t>> tcs(maxl + 1);
    for (int l = 1; l <= maxl; ++l) {
      lfirst[l] = (int)ls.size();
      lso[l] = (int)lstart.size();
      int tiles = 0;
      for (size_t i = 0; i < t->steps.size(); ++i) {
        if (lev[i] != l) continue;
        const TnStep& st = t->steps[i];
        if (prec != TN_FP32 && tn_step_tc_eligible(st, t->tc_min_cmacs)) {
          tcs[l].push_back(i);
          continue;
        }
        ls.push_back(st);
        lstart.push_back(tiles);
        tiles += ((st.M + kTnGemmTile - 1) / kTnGemmTile) * ((st.N + kTnGemmTile - 1) / kTnGemmTile);
      }
      lstart.push_back(tiles);
    }
    lfirst[maxl + 1] = (int)ls.size();
    if (t->d_lsteps) cudaFree(t->d_lsteps);
    if (t->d_lstart) cudaFree(t->d_lstart);
    t->d_lsteps = nullptr;
    t->d_lstart = nullptr;
    if (!ls.empty()) {
      if ((e = cudaMalloc(&t->d_lsteps, ls.size() * sizeof(TnStep))) != cudaSuccess) return cuda_fail(e, "tn level steps");
      if ((e = cudaMalloc(&t->d_lstart, lstart.size() * sizeof(int))) != cudaSuccess) return cuda_fail(e, "tn levels");
      if ((e = cudaMemcpy(t->d_lsteps, ls.data(), ls.size() * sizeof(TnStep), cudaMemcpyHostToDevice)) != cudaSuccess ||
          (e = cudaMemcpy(t->d_lstart, lstart.data(), lstart.size() * sizeof(int), cudaMemcpyHostToDevice)) !=
              cudaSuccess)
        return cuda_fail(e, "tn level copy");
    }
    cudaStream_t cap;
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "stream");
    cudaGraph_t g;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = tn_launch_assemble(*t, B, d_src, arena, cap);
    for (int l = 1; e == cudaSuccess && l <= maxl; ++l) {
      const int n_l = lfirst[l + 1] - lfirst[l];
      if (n_l > 0)
        e = tn_launch_level(*t, t->d_lsteps + lfirst[l], t->d_lstart + lso[l], n_l, lstart[lso[l] + n_l], B, arena, cap);
      for (size_t q = 0; e == cudaSuccess && q < tcs[l].size(); ++q)
        e = tn_launch_step_tc(*t, t->steps[tcs[l][q]], B, arena, prec, t->d_err, cap);
    }
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
    t->graph_gates = d_src;
    t->graph_out = d_out;
    t->graph_prec = prec;
  }
  if ((e = cudaGraphLaunch(t->graph, s)) != cudaSuccess) return cuda_fail(e, "tn graph launch");
  if (use_tc) {
    // the error word comes back with the call's results; the next call reads it
    if ((e = cudaMemcpyAsync(t->h_err, t->d_err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaEventRecord(t->err_ev, s)) != cudaSuccess)
      return cuda_fail(e, "tn status copy");
    t->err_pending = true;
  }
  return TC_OK;
}
}  // namespace

extern "C" {

tc_status tc_contract_path(tc_tn* t, int B, const float* d_gates, tc_tn_precision precision, double* d_out,
                           void* stream) {
  if (!t || (B != 0 && (!d_gates || !d_out))) return fail(TC_E_INVALID, "NULL argument");
  if (t->circuit) return fail(TC_E_INVALID, "plan was built from a circuit: use tc_tn_circuit_expect");
  if (precision != TC_TN_FP32 && precision != TC_TN_TF32X3 && precision != TC_TN_BF16X6)
    return fail(TC_E_INVALID, "unknown precision");
  if (B <= 0) return B == 0 ? TC_OK : fail(TC_E_INVALID, "B < 0");
  return tn_run(t, B, d_gates, d_out, (int)precision, stream);
}

tc_status tc_tn_circuit_create(int n_qubits, tc_init init, const tc_op* ops, int n_ops, int n_params,
                               const double* const_mats, int n_mats, const uint8_t* pauli, int prune, int split,
                               int rank_cap, int greedy_trials, const int32_t* path, int n_path_steps, tc_tn** out) {
  if (!out) return fail(TC_E_INVALID, "out is NULL");
  *out = nullptr;
  if (n_qubits < 1 || n_ops < 0 || (n_ops > 0 && !ops) || !pauli || n_params < 0 || n_mats < 0)
    return fail(TC_E_INVALID, "bad sizes or NULL arrays");
  if (init != TC_INIT_ZERO && init != TC_INIT_PLUS) return fail(TC_E_INVALID, "init must be TC_INIT_ZERO or TC_INIT_PLUS");
  if (prune < 0 || prune > 2 || split < 0 || split > 1) return fail(TC_E_INVALID, "prune must be 0..2, split 0..1");
  if (rank_cap < 1 || rank_cap > 26) return fail(TC_E_INVALID, "rank_cap must be in 1..26");
  if (greedy_trials < 0 || greedy_trials > 4096) return fail(TC_E_INVALID, "greedy_trials must be in 0..4096");
  if (path && n_path_steps < 0) return fail(TC_E_INVALID, "n_path_steps < 0");
  auto* t = new tc_tn();
  std::string err;
  if (!tn_build_circuit(n_qubits, (int)init, ops, n_ops, n_params, const_mats, n_mats, pauli, prune, split, rank_cap,
                        greedy_trials, path, n_path_steps, *t, err)) {
    delete t;
    return fail(err.rfind("op ", 0) == 0 && err.find("not supported") != std::string::npos ? TC_E_UNSUPPORTED
                                                                                          : TC_E_INVALID,
                err);
  }
  *out = t;
  return TC_OK;
}

tc_status tc_tn_circuit_expect(tc_tn* t, int B, const float* d_params, tc_tn_precision precision, double* d_out,
                               void* stream) {
  if (!t || (B != 0 && !d_out)) return fail(TC_E_INVALID, "NULL argument");
  if (!t->circuit) return fail(TC_E_INVALID, "plan is a light-cone gate network: use tc_contract_path");
  if (precision != TC_TN_FP32 && precision != TC_TN_TF32X3 && precision != TC_TN_BF16X6)
    return fail(TC_E_INVALID, "unknown precision");
  if (t->n_params > 0 && B != 0 && !d_params) return fail(TC_E_INVALID, "d_params is NULL");
  if (B <= 0) return B == 0 ? TC_OK : fail(TC_E_INVALID, "B < 0");
  return tn_run(t, B, d_params, d_out, (int)precision, stream);
}

void tc_tn_destroy(tc_tn* t) {
  if (!t) return;
  tn_release(t);
  delete t;
}

}  // extern "C"
