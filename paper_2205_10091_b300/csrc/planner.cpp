// Host planner: op list -> fused shared-memory tile passes -> register stages.
//
// Fusion rule (the "preprocessing" idea of Section "Custom contraction
// settings", restated for a state vector): gates are taken in list order and
// a gate may move ahead of deferred gates only if it shares no qubit with any
// of them, so every reordering is between commuting gates.  A pass takes the
// gates whose non-diagonal qubits fit in k tile qubits; diagonal gates (RZ,
// RZZ, CZ) need no tile qubit because their phase depends only on the
// amplitude index, and those sharing (parameter, scale) merge into one
// phase-table lookup.  Inside a pass the same rule splits the gates into
// register stages of RB qubits.
#include "planner.h"

#include <algorithm>
#include <cmath>
#include <cmath>
#include <map>
#include <numeric>
#include <tuple>

namespace tcb {

static inline int popc(uint32_t x) { return __builtin_popcount(x); }
static inline uint32_t bit(int p) { return p >= 0 ? (1u << p) : 0u; }

bool normalise_ops(int n_user, int N, const tc_op* ops, int n_ops, int n_params, int n_pool,
                   std::vector<HGate>& out, std::string& err) {
  out.clear();
  int ev = 0;
  for (int i = 0; i < n_ops; ++i) {
    const tc_op& o = ops[i];
    auto bad = [&](const char* m) {
      err = "op " + std::to_string(i) + ": " + m;
      return false;
    };
    if (o.kind < TC_OP_H || o.kind > TC_OP_RSEL) return bad("unknown kind");
    const bool two = o.kind == TC_OP_RZZ || o.kind == TC_OP_CNOT || o.kind == TC_OP_CZ || o.kind == TC_OP_U2;
    if (o.q0 < 0 || o.q0 >= n_user) return bad("q0 out of range");
    if (two && (o.q1 < 0 || o.q1 >= n_user || o.q1 == o.q0)) return bad("q1 out of range or equal to q0");
    HGate g;
    g.kind = o.kind;
    g.p0 = N - 1 - o.q0;
    g.p1 = two ? N - 1 - o.q1 : -1;
    const bool rot = o.kind == TC_OP_RX || o.kind == TC_OP_RY || o.kind == TC_OP_RZ || o.kind == TC_OP_RZZ ||
                     o.kind == TC_OP_RSEL;
    if (rot) {
      if (o.param < -1 || o.param >= n_params) return bad("param out of range");
      if (!std::isfinite(o.scale)) return bad("scale not finite");
      g.param = o.param;
      g.scale = o.scale;
    }
    if (o.kind == TC_OP_U1 && (o.mat < 0 || (int64_t)o.mat + 4 > n_pool)) return bad("U1 matrix offset out of range");
    if (o.kind == TC_OP_U2 && (o.mat < 0 || (int64_t)o.mat + 16 > n_pool)) return bad("U2 matrix offset out of range");
    g.pool = o.mat;
    if (o.kind == TC_OP_PAULI_NOISE) {
      if (!(o.px >= 0 && o.py >= 0 && o.pz >= 0) || !(o.px + o.py + o.pz <= 1.0))
        return bad("noise probabilities must be >= 0 and sum to <= 1");
      // interval ends for [I, X, Y, Z]; the same arithmetic as the selection rule
      g.t1 = 1.0 - (o.px + o.py + o.pz);
      g.t2 = g.t1 + o.px;
      g.t3 = g.t2 + o.py;
      g.noise_event = ev++;
    }
    if (o.kind == TC_OP_RSEL) {
      if (!(o.px >= 0 && o.py >= 0 && o.pz >= 0) || std::fabs(o.px + o.py + o.pz - 1.0) > 1e-9)
        return bad("rotation probabilities must be >= 0 and sum to 1");
      // interval ends for [RX, RY, RZ], left-closed
      g.t1 = o.px;
      g.t2 = o.px + o.py;
      g.noise_event = ev++;
    }
    g.diag = o.kind == TC_OP_RZ || o.kind == TC_OP_RZZ || o.kind == TC_OP_CZ;
    g.sign_mode = o.kind == TC_OP_CZ;
    out.push_back(g);
  }
  return true;
}

std::vector<HGate> fold_noise_into_u1(const std::vector<HGate>& gates) {
  const int n = (int)gates.size();
  std::vector<HGate> g = gates;
  std::vector<char> gone(n, 0);
  auto touches = [&](int i, int p) { return g[i].p0 == p || g[i].p1 == p; };
  auto foldable = [&](int i) { return g[i].kind == TC_OP_U1 && !g[i].diag; };
  for (int i = 0; i < n; ++i) {
    if (g[i].kind != TC_OP_PAULI_NOISE) continue;
    const int p = g[i].p0;
    int prev = -1, next = -1;
    for (int j = i - 1; j >= 0 && prev < 0; --j)
      if (touches(j, p)) prev = j;
    for (int j = i + 1; j < n && next < 0; ++j)
      if (touches(j, p)) next = j;
    if (prev >= 0 && foldable(prev) && g[prev].post_ev < 0) {
      g[prev].post_ev = g[i].noise_event;
      g[prev].post_t[0] = g[i].t1;
      g[prev].post_t[1] = g[i].t2;
      g[prev].post_t[2] = g[i].t3;
      gone[i] = 1;
    } else if (next >= 0 && foldable(next) && g[next].pre_ev < 0) {
      g[next].pre_ev = g[i].noise_event;
      g[next].pre_t[0] = g[i].t1;
      g[next].pre_t[1] = g[i].t2;
      g[next].pre_t[2] = g[i].t3;
      gone[i] = 1;
    }
  }
  std::vector<HGate> out;
  for (int i = 0; i < n; ++i)
    if (!gone[i]) out.push_back(g[i]);
  return out;
}

std::vector<HGate> rewrite_rx_frames(const std::vector<HGate>& gates, int N) {
  std::vector<HGate> out;
  std::vector<char> frame(N, 0);
  auto sphase = [&](int p, double sign) {
    HGate g;
    g.kind = -1;
    g.p0 = p;
    g.diag = true;
    g.quarter = true;
    g.scale = sign;
    out.push_back(g);
  };
  for (const HGate& g : gates) {
    if (g.kind == TC_OP_RX) {
      if (!frame[g.p0]) {
        sphase(g.p0, +1.0);  // enter: S
        frame[g.p0] = 1;
      }
      HGate r = g;
      r.kind = TC_OP_RY;
      out.push_back(r);
      continue;
    }
    if (!g.diag) {
      // CNOT commutes with S on its control; every other qubit it touches
      // leaves the frame first
      for (int p : {g.p0, g.p1}) {
        if (p < 0 || !frame[p]) continue;
        if (g.kind == TC_OP_CNOT && p == g.p0) continue;
        sphase(p, -1.0);  // leave: S^dagger
        frame[p] = 0;
      }
    }
    out.push_back(g);
  }
  for (int p = 0; p < N; ++p)
    if (frame[p]) sphase(p, -1.0);
  return out;
}

// Thread -> amplitude runs of a stage (see DevRun), and the CTA -> fixed bits runs of a pass.
void fill_stage_runs(const DevPass& P, int rb, DevStage& ds) {
  uint32_t smask = 0;
  for (int r = 0; r < rb; ++r) {
    smask |= 1u << ds.S[r];
    ds.P[r] = (int8_t)P.pos[ds.S[r]];
  }
  int b = 0;
  ds.n_runs = 0;
  for (int j = 0; j < P.k; ++j) {
    if ((smask >> j) & 1u) continue;
    if (ds.n_runs > 0) {
      DevRun& u = ds.run[ds.n_runs - 1];
      if (u.b + u.len == b && u.j + u.len == j && u.p + u.len == P.pos[j]) {
        ++u.len;
        ++b;
        continue;
      }
    }
    ds.run[ds.n_runs++] = DevRun{(uint8_t)b, 1, (uint8_t)j, P.pos[j]};
    ++b;
  }
}

void fill_fix_runs(DevPass& P) {
  P.n_fixruns = 0;
  for (int f = 0; f < P.nfix; ++f) {
    if (P.n_fixruns > 0) {
      DevRun& u = P.fixrun[P.n_fixruns - 1];
      if (u.b + u.len == f && u.p + u.len == P.fixpos[f]) {
        ++u.len;
        continue;
      }
    }
    P.fixrun[P.n_fixruns++] = DevRun{(uint8_t)f, 1, 0, P.fixpos[f]};
  }
}

namespace {

struct Item {
  bool group = false;
  int gate = -1;
  std::vector<int> members;
  uint32_t touch = 0;
};

uint32_t gate_touch(const HGate& g) { return bit(g.p0) | bit(g.p1); }

// register-tile bits an item needs
uint32_t item_need(const Item& it, const std::vector<HGate>& gates, const int* tb) {
  if (it.group) return 0;
  const HGate& g = gates[it.gate];
  if (g.quarter) return 0;  // a phase: register bit or thread bit alike
  if (g.kind == TC_OP_CNOT) return 1u << tb[g.p1];
  if (g.kind == TC_OP_U2) return (1u << tb[g.p0]) | (1u << tb[g.p1]);
  return 1u << tb[g.p0];
}

// Merge each run of consecutive RX instructions (or adjoint RX steps with one
// shared gradient slot and scale) on distinct register bits into one multi-bit
// instruction; RY always becomes the multi-bit form (a run of one included),
// so the kernels carry one RY code path.  RX gates on different qubits commute, and Im<lam|X_q|psi> is
// unchanged by RX on other qubits, so the run may be reordered by bit index.
// Their per-row table entries are moved so that bit r reads entry
// slot + stride * rank(r) (rank among the run's bits; RY has kRYEntries
// entries per gate, RX one).
void merge_rx_runs(PlanArrays& A, int first, int rb, int table_base) {
  std::vector<DevInstr> out;
  const int end = (int)A.instrs.size();
  int i = first;
  while (i < end) {
    const DevInstr& in0 = A.instrs[i];
    const bool isy = in0.kind == IK_RY || in0.kind == IK_RY_ADJ;
    const bool fwd = in0.kind == IK_RX || in0.kind == IK_RY, adj = in0.kind == IK_RX_ADJ || in0.kind == IK_RY_ADJ;
    const int8_t mtype = isy ? MT_RY : MT_RX;
    if (!fwd && !adj) {
      out.push_back(in0);
      ++i;
      continue;
    }
    int j = i;
    uint32_t mask = 0;
    while (j < end && A.instrs[j].kind == in0.kind && !(mask & (1u << A.instrs[j].j0)) &&
           (!adj || (A.instrs[j].gslot == in0.gslot && A.instrs[j].gscale == in0.gscale))) {
      mask |= 1u << A.instrs[j].j0;
      ++j;
    }
    if (j - i < 2 && !isy) {
      out.push_back(in0);
      ++i;
      continue;
    }
    // table entries of the run, sorted by bit
    std::vector<std::pair<int, int>> bit_slot;
    for (int q = i; q < j; ++q) bit_slot.push_back({A.instrs[q].j0, A.instrs[q].slot});
    std::sort(bit_slot.begin(), bit_slot.end());
    int lo = bit_slot[0].second;
    for (auto& bs : bit_slot) lo = std::min(lo, bs.second);
    // move the DevMat records: the entries of the r-th smallest bit go to
    // lo + stride * r (the run's entries are one contiguous block)
    const int stride = isy ? kRYEntries : 1;
    std::vector<std::pair<int, int>> moves;  // (mat index, new local entry)
    for (size_t r = 0; r < bit_slot.size(); ++r) {
      const int old_local = bit_slot[r].second;
      for (int mi = (int)A.mats.size() - 1; mi >= 0; --mi)
        if (A.mats[mi].type == mtype && A.mats[mi].dst == table_base + old_local) {
          moves.push_back({mi, lo + stride * (int)r});
          break;
        }
    }
    for (auto& mv : moves) A.mats[mv.first].dst = table_base + mv.second;
    DevInstr mi = in0;
    mi.kind = isy ? (fwd ? IK_RYM : IK_RYM_ADJ) : (fwd ? IK_RXM : IK_RXM_ADJ);
    mi.j0 = (int8_t)mask;
    mi.slot = lo;
    out.push_back(mi);
    i = j;
  }
  (void)rb;
  A.instrs.resize(first);
  A.instrs.insert(A.instrs.end(), out.begin(), out.end());
}

}  // namespace

Schedule build_schedule(const std::vector<HGate>& gates, int N, int k, int rb, bool adjoint, bool first_init,
                        PlanArrays& A, int max_gates) {
  Schedule sc;
  sc.first_pass = (int)A.passes.size();
  sc.first_mat = (int)A.mats.size();
  sc.k = k;
  std::vector<int> remaining(gates.size());
  std::iota(remaining.begin(), remaining.end(), 0);
  if (adjoint) std::reverse(remaining.begin(), remaining.end());
  const uint32_t low = (1u << kLaneBits) - 1;      // lane tile bits of the load/store stages
  const uint32_t io_low = (1u << kIOLowBits) - 1;  // positions every tile holds
  bool first = true;

  while (!remaining.empty() || (first && first_init)) {
    // ---- choose the pass's gates and tile -------------------------------
    uint32_t tile = io_low, blocked = 0;
    int n_nondiag = 0;
    std::vector<int> taken, deferred;
    for (int gi : remaining) {
      const HGate& g = gates[gi];
      const uint32_t touch = gate_touch(g);
      if (touch & blocked) {
        deferred.push_back(gi);
        blocked |= touch;
        continue;
      }
      if (g.diag) {
        taken.push_back(gi);
        continue;
      }
      const uint32_t need = g.kind == TC_OP_CNOT ? bit(g.p1) : touch;
      if (popc(tile | need) <= k && (max_gates <= 0 || n_nondiag < max_gates)) {
        tile |= need;
        taken.push_back(gi);
        ++n_nondiag;
      } else {
        deferred.push_back(gi);
        blocked |= touch;
      }
    }
    for (int p = 0; popc(tile) < k && p < N; ++p) tile |= bit(p);  // fill with low positions

    DevPass P{};
    P.k = k;
    P.nfix = N - k;
    P.rb = rb;
    int tb[32];
    for (int p = 0; p < 32; ++p) tb[p] = -1;
    {
      int j = 0, f = 0;
      for (int p = 0; p < N; ++p) {
        if (tile & bit(p)) {
          P.pos[j] = (uint8_t)p;
          tb[p] = j++;
        } else {
          P.fixpos[f++] = (uint8_t)p;
        }
      }
    }
    fill_fix_runs(P);
    P.flags = (first && first_init && !adjoint) ? PF_INIT : 0;

    // ---- items: non-diagonal gates, and diagonal groups ------------------
    std::vector<Item> items;
    std::map<std::tuple<int, int, double>, int> open;  // key -> item index
    int last_touch[32];
    for (int p = 0; p < 32; ++p) last_touch[p] = -1;
    for (int gi : taken) {
      const HGate& g = gates[gi];
      if (g.diag && !g.quarter) {
        const int mode = g.sign_mode ? 1 : (g.quarter ? 2 : 0);
        auto key = std::make_tuple(mode, mode == 0 ? g.param : -1, mode == 1 ? 0.0 : g.scale);
        auto itk = open.find(key);
        bool joined = false;
        if (itk != open.end()) {
          const int gidx = itk->second;
          bool ok = true;
          for (int p : {g.p0, g.p1})
            if (p >= 0 && last_touch[p] > gidx) ok = false;
          if (ok) {
            items[gidx].members.push_back(gi);
            items[gidx].touch |= gate_touch(g);
            joined = true;
          }
        }
        if (!joined) {
          Item it;
          it.group = true;
          it.members.push_back(gi);
          it.touch = gate_touch(g);
          items.push_back(it);
          open[key] = (int)items.size() - 1;
        }
      } else {
        Item it;
        it.gate = gi;
        it.touch = gate_touch(g);
        items.push_back(it);
        for (int p : {g.p0, g.p1})
          if (p >= 0) last_touch[p] = (int)items.size() - 1;
      }
    }

    // ---- register stages ------------------------------------------------
    // Every stage is one linear scan that keeps list order between items on
    // shared qubits.  The first stage only takes items on high tile bits (so
    // it can load straight from HBM), the next ones first take items on the
    // lane bits 0..4 and then fill up; the pass ends on a high-bit stage.
    const uint32_t kmask = (k >= 32) ? 0xffffffffu : ((1u << k) - 1);
    const uint32_t high_tile = kmask & ~low;
    std::vector<std::pair<uint32_t, std::vector<int>>> stages;  // (S mask in tile bits, item ids)
    {
      std::vector<int> rem(items.size());
      std::iota(rem.begin(), rem.end(), 0);
      int si = 0;
      while (!rem.empty()) {
        uint32_t S = 0, blk = 0;
        std::vector<int> tk, df;
        std::vector<char> took(items.size(), 0);
        const bool prefer_low = si > 0;
        for (int scan = 0; scan < 2; ++scan) {
          blk = 0;
          for (int ii : rem) {
            if (took[ii]) continue;
            const Item& it = items[ii];
            if (it.touch & blk) {
              blk |= it.touch;
              continue;
            }
            const uint32_t need = item_need(it, gates, tb);
            bool allowed;
            if (si == 0) allowed = !(need & ~high_tile);
            else if (prefer_low && scan == 0) allowed = !need || (need & low);
            else allowed = true;
            if (allowed && popc(S | need) <= rb) {
              S |= need;
              took[ii] = 1;
              tk.push_back(ii);
            } else {
              blk |= it.touch;
            }
          }
          if (si == 0) break;
        }
        for (int ii : rem)
          if (!took[ii]) df.push_back(ii);
        if (tk.empty() && si == 0) {
          // nothing fits a high-bit stage: start with an empty load stage
          stages.push_back({0u, {}});
          ++si;
          continue;
        }
        // keep scan order inside the stage equal to list order where it matters:
        // scan-1 items first, then scan-2 items, each in list order (tk already is)
        stages.push_back({S, tk});
        rem = df;
        ++si;
      }
    }
    auto fill = [&](uint32_t S) {
      // complete S to rb bits, preferring high tile bits (keeps lanes on bits 0..4)
      for (int j = k - 1; popc(S) < rb && j >= kLaneBits; --j) S |= 1u << j;
      for (int j = 0; popc(S) < rb && j < k; ++j) S |= 1u << j;
      return S;
    };
    if (stages.empty()) stages.push_back({0u, {}});
    for (auto& st : stages) st.first = fill(st.first);
    if (stages.front().first & ~high_tile) stages.insert(stages.begin(), {fill(0u), {}});
    if (stages.back().first & ~high_tile) stages.push_back({fill(0u), {}});

    // ---- emit -----------------------------------------------------------
    P.stage_off = (int)A.stages.size();
    P.n_stages = (int)stages.size();
    P.instr_off = (int)A.instrs.size();
    P.mat_off = (int)A.mats.size();
    P.diag_off = (int)A.diags.size();
    P.dent_off = (int)A.dents.size();
    P.gslot_base = sc.n_gslots;
    int table = 0;
    std::map<int, int> local_slot;  // param -> local slot
    auto slot_of = [&](int param) {
      auto it = local_slot.find(param);
      if (it != local_slot.end()) return it->second;
      const int s = (int)local_slot.size();
      local_slot[param] = s;
      sc.slot_param.push_back(param);
      return s;
    };
    auto add_mat = [&](int8_t type, const HGate& g, int entries) {
      DevMat m{};
      m.type = type;
      m.adj = adjoint ? 1 : 0;
      m.param = g.param;
      m.scale = g.scale;
      m.pool = g.pool;
      m.dst = sc.table_total + table;
      if (type == MT_NOISE || type == MT_RSEL) {
        m.T = g.noise_event;
        m.t1 = g.t1;
        m.t2 = g.t2;
        m.t3 = g.t3;
      }
      if (type == MT_U1) {
        m.T = g.pre_ev;
        m.t1 = g.pre_t[0];
        m.t2 = g.pre_t[1];
        m.t3 = g.pre_t[2];
        m.T2 = g.post_ev;
        m.u1 = g.post_t[0];
        m.u2 = g.post_t[1];
        m.u3 = g.post_t[2];
      }
      A.mats.push_back(m);
      const int local = table;
      table += entries;
      return local;
    };
    for (auto& st : stages) {
      DevStage ds{};
      int jof[32];
      for (int j = 0; j < 32; ++j) jof[j] = -1;
      {
        int r = 0;
        for (int j = 0; j < k; ++j)
          if (st.first & (1u << j)) {
            ds.S[r] = (int8_t)j;
            jof[j] = r++;
          }
      }
      fill_stage_runs(P, rb, ds);
      ds.instr_off = (int)A.instrs.size() - P.instr_off;
      // Quarter phases (S, S^dagger of RX frames) commute with every item of
      // the stage except non-diagonal gates on their own qubit (and another
      // phase there), so each may sit at any insertion point between those
      // neighbours.  The fewest points that cover every phase's interval
      // (greedy on the interval ends) each get one IK_SPHASE per sign.
      const std::vector<int>& sitems = st.second;
      const int ns = (int)sitems.size();
      std::vector<int> q_at;  // stage positions of the quarter items
      std::vector<int> point_of;
      {
        auto q_of = [&](int t) -> const HGate* {
          const Item& it = items[sitems[t]];
          return (!it.group && gates[it.gate].quarter) ? &gates[it.gate] : nullptr;
        };
        auto blocks = [&](int t, int p) {
          const Item& it = items[sitems[t]];
          if (it.group) return false;  // diagonal groups commute with the phases
          const HGate& g = gates[it.gate];
          return g.p0 == p || g.p1 == p;
        };
        std::vector<std::pair<int, int>> iv;  // (lo, hi) insertion points of each quarter
        for (int t = 0; t < ns; ++t) {
          const HGate* g = q_of(t);
          if (!g) continue;
          int lo = t, hi = t;
          while (lo > 0 && !blocks(lo - 1, g->p0)) --lo;
          while (hi < ns - 1 && !blocks(hi + 1, g->p0)) ++hi;
          q_at.push_back(t);
          iv.push_back({lo, hi + 1});  // point t' = before item t' (ns = after the last)
        }
        point_of.assign(q_at.size(), -1);
        std::vector<int> order(q_at.size());
        std::iota(order.begin(), order.end(), 0);
        std::sort(order.begin(), order.end(), [&](int a, int b) { return iv[a].second < iv[b].second; });
        for (int a : order) {
          if (point_of[a] >= 0) continue;
          const int pt = iv[a].second;
          for (int b : order)
            if (point_of[b] < 0 && iv[b].first <= pt && pt <= iv[b].second) point_of[b] = pt;
        }
      }
      // the phases placed at point pt, one instruction per sign (a qubit
      // already in an instruction's masks starts a new one)
      auto emit_point = [&](int pt) {
        for (double sg : {1.0, -1.0}) {
          std::vector<const HGate*> mine;
          for (size_t a = 0; a < q_at.size(); ++a) {
            const HGate* g = &gates[items[sitems[q_at[a]]].gate];
            if (point_of[a] == pt && (g->scale > 0 ? 1.0 : -1.0) * (adjoint ? -1.0 : 1.0) == sg) mine.push_back(g);
          }
          while (!mine.empty()) {
            DevInstr q{};
            q.kind = IK_SPHASE;
            q.gslot = -1;
            q.jc = -1;
            q.gscale = (float)sg;
            uint32_t rmask = 0, pmask = 0, seen = 0;
            std::vector<const HGate*> rest;
            for (const HGate* g : mine) {
              if (seen & bit(g->p0)) {
                rest.push_back(g);
                continue;
              }
              seen |= bit(g->p0);
              const int r = tb[g->p0] >= 0 ? jof[tb[g->p0]] : -1;
              if (r >= 0) rmask |= 1u << r;
              else pmask |= bit(g->p0);
            }
            q.j0 = (int8_t)rmask;
            q.slot = (int32_t)pmask;
            A.instrs.push_back(q);
            mine = rest;
          }
        }
      };
      for (int t = 0; t < ns; ++t) {
        const int ii = sitems[t];
        emit_point(t);
        const Item& it = items[ii];
        if (!it.group && gates[it.gate].quarter) continue;
        DevInstr in{};
        in.gslot = -1;
        in.jc = -1;
        if (it.group) {
          const HGate& g0 = gates[it.members[0]];
          DevDiag dg{};
          dg.sign_mode = g0.sign_mode ? 1 : 0;
          dg.T = (int)it.members.size();
          dg.ent_off = (int)A.dents.size() - P.dent_off;
          std::vector<DevDiagEnt> ents;
          for (int gi : it.members) {
            const HGate& g = gates[gi];
            uint32_t d, m;
            if (g.p1 < 0) {
              d = 0;
              m = bit(g.p0);
            } else {
              const int a = std::min(g.p0, g.p1), b = std::max(g.p0, g.p1);
              d = (uint32_t)(b - a);
              m = bit(a);
            }
            bool placed = false;
            for (auto& e : ents)
              if (e.d == d && !(e.mask & m)) {
                e.mask |= m;
                placed = true;
                break;
              }
            if (!placed) ents.push_back({d, m});
          }
          if (!dg.sign_mode && ents.size() >= 2 && it.members.size() <= 64) {
            // several pair distances: one 64-bit column word per position
            // (term k = member k), counted by XOR walk and popcount
            std::vector<uint64_t> col(N, 0);
            for (size_t k = 0; k < it.members.size(); ++k) {
              const HGate& g = gates[it.members[k]];
              col[g.p0] |= 1ull << k;
              if (g.p1 >= 0) col[g.p1] |= 1ull << k;
            }
            ents.clear();
            for (int p = 0; p < N; ++p) ents.push_back({(uint32_t)(col[p] & 0xffffffffu), (uint32_t)(col[p] >> 32)});
            dg.packed = 1;
          }
          for (auto& e : ents) A.dents.push_back(e);
          dg.n_ent = (int)ents.size();
          dg.tab = dg.sign_mode ? -1 : add_mat(g0.quarter ? MT_QUARTER : MT_DIAGTAB, g0, dg.T + 1);
          if (!dg.sign_mode) A.mats.back().T = dg.T;
          const int di = (int)A.diags.size() - P.diag_off;
          A.diags.push_back(dg);
          in.kind = IK_DIAG;
          in.slot = di;
          if (adjoint && !dg.sign_mode && !g0.quarter && g0.param >= 0) {
            // gradient of the group's parameter, then the group's inverse phases
            in.kind = IK_DIAG_ADJ;
            in.gslot = (int16_t)slot_of(g0.param);
            in.gscale = (float)g0.scale;
          }
          A.instrs.push_back(in);
          continue;
        }
        const HGate& g = gates[it.gate];
        if (g.kind == TC_OP_CNOT) {
          in.kind = IK_CNOT;
          in.j0 = (int8_t)jof[tb[g.p1]];
          in.pos = (int16_t)g.p0;
          in.jc = (int8_t)((tb[g.p0] >= 0) ? jof[tb[g.p0]] : -1);
          A.instrs.push_back(in);
          continue;
        }
        in.j0 = (int8_t)jof[tb[g.p0]];
        switch (g.kind) {
          case TC_OP_U2:
            in.j1 = (int8_t)jof[tb[g.p1]];
            if (g.chan) {
              in.kind = IK_CHAN;
              in.slot = add_mat(MT_CHAN, g, 2);
            } else {
              in.kind = IK_MAT4;
              in.slot = add_mat(MT_U2, g, 16);
            }
            break;
          case TC_OP_U1:
            in.kind = IK_MAT2;
            in.slot = add_mat(MT_U1, g, 4);
            break;
          case TC_OP_H:
            in.kind = IK_H;
            break;
          case TC_OP_X:
            in.kind = IK_X;
            break;
          case TC_OP_PAULI_NOISE:
            in.kind = IK_PAULI;
            in.slot = add_mat(MT_NOISE, g, 1);
            break;
          case TC_OP_RSEL:
            in.slot = add_mat(MT_RSEL, g, 5);
            if (adjoint && g.param >= 0) {
              in.kind = IK_RSEL_ADJ;
              in.gslot = (int16_t)slot_of(g.param);
              in.gscale = (float)g.scale;
            } else {
              in.kind = IK_RSEL;
            }
            break;
          case TC_OP_RX:
          case TC_OP_RY: {
            const bool rx = g.kind == TC_OP_RX;
            in.slot = add_mat(rx ? MT_RX : MT_RY, g, rx ? 1 : kRYEntries);
            if (adjoint && g.param >= 0) {
              in.kind = rx ? IK_RX_ADJ : IK_RY_ADJ;
              in.gslot = (int16_t)slot_of(g.param);
              in.gscale = (float)g.scale;
            } else if (adjoint && !rx) {
              in.kind = IK_RY_ADJ;  // fixed angle: uncompute only (no gradient slot)
            } else {
              in.kind = rx ? IK_RX : IK_RY;
            }
          } break;
          default:
            in.kind = IK_X;
            break;
        }
        A.instrs.push_back(in);
      }
      emit_point(ns);
      merge_rx_runs(A, P.instr_off + ds.instr_off, rb, sc.table_total);
      ds.n_instr = (int)A.instrs.size() - P.instr_off - ds.instr_off;
      A.stages.push_back(ds);
    }
    P.n_instr = (int)A.instrs.size() - P.instr_off;
    for (int i = P.instr_off; i < (int)A.instrs.size(); ++i) {
      const DevInstr& in = A.instrs[i];
      if (in.kind == IK_CNOT || in.kind == IK_MAT4) P.flags |= PF_FULL;
      if (in.kind != IK_RY && in.kind != IK_RYM && in.kind != IK_RY_ADJ && in.kind != IK_RYM_ADJ &&
          in.kind != IK_DIAG && in.kind != IK_DIAG_ADJ && in.kind != IK_SPHASE)
        P.flags |= PF_LEAN;
      if (in.kind == IK_DIAG || in.kind == IK_GRADDIAG || in.kind == IK_DIAG_ADJ) {
        const DevDiag& dg = A.diags[P.diag_off + in.slot];
        if (dg.n_ent != 1) P.flags |= dg.sign_mode ? PF_FULL : PF_MULTI;
        if (dg.sign_mode) P.flags |= PF_LEAN;
      }
    }
    P.n_mats = (int)A.mats.size() - P.mat_off;
    P.n_diag = (int)A.diags.size() - P.diag_off;
    P.n_dent = (int)A.dents.size() - P.dent_off;
    P.table_size = table;
    P.table_off = sc.table_total;
    sc.table_total += table;
    P.n_gslots = (int)local_slot.size();
    sc.n_gslots += P.n_gslots;
    sc.n_stages += P.n_stages;
    if (adjoint && P.n_gslots > 0) {
      // mark each gradient slot's last instruction in execution order (stage
      // by stage): the kernel reduces the slot there, so its accumulator is
      // live over the slot's own gates only
      std::vector<int> last(P.n_gslots, -1);
      for (int si = 0; si < P.n_stages; ++si) {
        const DevStage& S = A.stages[P.stage_off + si];
        for (int q = 0; q < S.n_instr; ++q) {
          const int ii = P.instr_off + S.instr_off + q;
          const DevInstr& in = A.instrs[ii];
          if (in.kind != IK_CNOT && in.gslot >= 0 && in.gslot < P.n_gslots) last[in.gslot] = ii;
        }
      }
      for (int ii : last)
        if (ii >= 0) A.instrs[ii].jc = 1;
      P.flags |= PF_GFLUSH;
    }
    A.passes.push_back(P);
    remaining = deferred;
    first = false;
  }
  sc.n_passes = (int)A.passes.size() - sc.first_pass;
  sc.n_mats = (int)A.mats.size() - sc.first_mat;
  // the states after an adjoint sweep's last pass are not needed
  if (adjoint && sc.n_passes > 0) A.passes.back().flags |= PF_SKIP_PSI | PF_SKIP_LAM;
  return sc;
}

Schedule build_plain_schedule(const std::vector<HGate>& gates, int N, int rb, PlanArrays& A) {
  Schedule sc;
  sc.first_pass = (int)A.passes.size();
  sc.first_mat = (int)A.mats.size();
  sc.k = kMinQubits;
  auto absorb = [&](const Schedule& s) {
    // shift the sub-schedule's tables behind the ones already placed
    for (int p = s.first_pass; p < s.first_pass + s.n_passes; ++p) A.passes[p].table_off += sc.table_total;
    for (int m = s.first_mat; m < s.first_mat + s.n_mats; ++m) A.mats[m].dst += sc.table_total;
    sc.table_total += s.table_total;
    sc.n_stages += s.n_stages;
  };
  // a gate-free pass that writes the initial state, then one pass per gate
  absorb(build_schedule({}, N, kMinQubits, rb, false, true, A, 0));
  for (size_t i = 0; i < gates.size(); ++i) {
    std::vector<HGate> one{gates[i]};
    absorb(build_schedule(one, N, kMinQubits, rb, false, false, A, 0));
  }
  sc.n_passes = (int)A.passes.size() - sc.first_pass;
  sc.n_mats = (int)A.mats.size() - sc.first_mat;
  return sc;
}

bool build_hamiltonian(int n_user, int N, int k, const uint8_t* structures, const double* weights, int T,
                       HamPlan& H, std::string& err) {
  H = HamPlan{};
  H.k = k;
  const uint32_t io_low = (1u << kIOLowBits) - 1;  // positions every tile holds
  // ---- classify terms -----------------------------------------------------
  std::map<std::pair<double, uint32_t>, std::vector<uint32_t>> zz;  // (w, d) -> lower-position bits
  std::map<uint32_t, std::vector<DevHTerm>> flips;
  std::vector<DevHDiag> diag;
  for (int t = 0; t < T; ++t) {
    uint32_t mx = 0, my = 0, mz = 0;
    for (int q = 0; q < n_user; ++q) {
      const uint8_t c = structures[(size_t)t * n_user + q];
      if (c > 3) {
        err = "structure entry outside {0,1,2,3} in term " + std::to_string(t);
        return false;
      }
      const uint32_t b = 1u << (N - 1 - q);
      if (c == 1) mx |= b;
      if (c == 2) my |= b;
      if (c == 3) mz |= b;
    }
    const double w = weights[t];
    if (!std::isfinite(w)) {
      err = "weight not finite in term " + std::to_string(t);
      return false;
    }
    const uint32_t f = mx | my;
    if (f) {
      DevHTerm ht{};
      ht.sm = my | mz;
      ht.ny = popc(my) & 3;
      ht.w = w;
      flips[f].push_back(ht);
    } else if (popc(mz) == 2) {
      const int a = __builtin_ctz(mz), b = 31 - __builtin_clz(mz);
      zz[{w, (uint32_t)(b - a)}].push_back(1u << a);
    } else {
      DevHDiag d{};
      d.d = 0;
      d.mask = mz;
      d.cnt = -1;  // parity form
      d.w = w;
      diag.push_back(d);
    }
  }
  // ZZ terms of one weight at several distances: one 64-bit column word per
  // position instead (term k sets bit k at both of its positions), so that
  // the count of odd terms is one XOR walk and a popcount per amplitude
  std::map<double, std::vector<std::pair<uint32_t, uint32_t>>> by_w;  // w -> (d, lower-position bit)
  for (auto& kv : zz)
    for (uint32_t m : kv.second) by_w[kv.first.first].push_back({kv.first.second, m});
  for (auto& kv : by_w) {
    std::map<uint32_t, int> dists;
    for (auto& t : kv.second) dists[t.first]++;
    if (dists.size() < 3) continue;
    for (size_t c0 = 0; c0 < kv.second.size(); c0 += 64) {
      const size_t c1 = std::min(kv.second.size(), c0 + 64);
      std::vector<uint64_t> col(N, 0);
      for (size_t t = c0; t < c1; ++t) {
        const int a = __builtin_ctz(kv.second[t].second);
        col[a] |= 1ull << (t - c0);
        col[a + (int)kv.second[t].first] |= 1ull << (t - c0);
      }
      DevHDiag h{};
      h.cnt = (int32_t)(c1 - c0);
      h.pad = 1;  // packed header; the N column records follow
      h.w = kv.first;
      diag.push_back(h);
      for (int q = 0; q < N; ++q) {
        DevHDiag cr{};
        cr.d = (uint32_t)(col[q] & 0xffffffffu);
        cr.mask = (uint32_t)(col[q] >> 32);
        cr.pad = 2;
        diag.push_back(cr);
      }
      H.packed_groups++;
    }
    for (auto it = zz.begin(); it != zz.end();) it = it->first.first == kv.first ? zz.erase(it) : std::next(it);
  }
  for (auto& kv : zz) {
    std::vector<DevHDiag> ents;
    for (uint32_t m : kv.second) {
      bool placed = false;
      for (auto& e : ents)
        if (!(e.mask & m)) {
          e.mask |= m;
          e.cnt++;
          placed = true;
          break;
        }
      if (!placed) {
        DevHDiag e{};
        e.d = kv.first.second;
        e.mask = m;
        e.cnt = 1;
        e.w = kv.first.first;
        ents.push_back(e);
      }
    }
    for (auto& e : ents) diag.push_back(e);
  }
  // ---- passes ---------------------------------------------------------------
  // A group whose flip mask fits one tile together with the positions every
  // tile holds goes into an ordinary pass (its partners sit in the same tile).
  // A wider group goes into a paired pass: the tile takes as many of its flip
  // bits as fit, and the rest (f_out) pair each tile with tile ^ f_out.
  std::vector<std::pair<uint32_t, std::vector<DevHTerm>>> groups(flips.begin(), flips.end());
  std::vector<int> narrow, wide;
  for (size_t g = 0; g < groups.size(); ++g)
    (popc(io_low | groups[g].first) <= k ? narrow : wide).push_back((int)g);
  std::vector<bool> done(groups.size(), false);
  auto emit = [&](uint32_t tile, const std::vector<int>& mine, bool with_diag, bool lam_load, uint32_t fout) {
    DevPass P{};
    P.k = k;
    P.nfix = N - k;
    P.rb = kRBHam;
    int tbit[32];
    {
      int j = 0, f = 0;
      for (int p = 0; p < N; ++p) {
        if (tile & bit(p)) {
          P.pos[j] = (uint8_t)p;
          tbit[p] = j++;
        } else {
          if (fout & bit(p)) P.pair_fout_idx |= 1u << f;
          P.fixpos[f++] = (uint8_t)p;
        }
      }
    }
    fill_fix_runs(P);
    P.pair_fout = fout;
    P.pair_bit = fout ? 31 - __builtin_clz(P.pair_fout_idx) : 0;
    P.flags = lam_load ? (PF_LAM_LOAD | PF_LAM_STORE) : PF_LAM_STORE;
    if (with_diag) {
      P.hdiag_off = (int)H.hdiag.size();
      P.n_hdiag = (int)diag.size();
      for (auto& d : diag) H.hdiag.push_back(d);
    }
    P.hflip_off = (int)H.hflips.size();
    P.n_hflip = (int)mine.size();
    P.hterm_off = (int)H.hterms.size();
    for (int g : mine) {
      DevHFlip fl{};
      fl.f = groups[g].first;
      uint32_t ft = 0;
      for (int p = 0; p < N; ++p)
        if (fl.f & tile & bit(p)) ft |= 1u << tbit[p];
      fl.f_tile = ft;
      fl.term_off = (int)H.hterms.size();
      fl.n_terms = (int)groups[g].second.size();
      for (auto& t : groups[g].second) H.hterms.push_back(t);
      H.hflips.push_back(fl);
      done[g] = true;
    }
    P.n_hterm = (int)H.hterms.size() - P.hterm_off;
    P.epart_index = (int)H.passes.size();
    H.passes.push_back(P);
  };
  auto fill_tile = [&](uint32_t tile) {
    for (int p = 0; popc(tile) < k && p < N; ++p) tile |= bit(p);
    return tile;
  };
  // ordinary passes; the first one always exists (it starts lambda and holds
  // the diagonal terms)
  size_t n_left = narrow.size();
  bool first = true;
  while (first || n_left > 0) {
    uint32_t tile = io_low;
    std::vector<int> mine;
    // the pass stages its diagonal entries, groups and terms in shared memory
    size_t staged = first ? sizeof(DevHDiag) * diag.size() : 0;
    for (int g : narrow) {
      if (done[g]) continue;
      const size_t gb = sizeof(DevHFlip) + sizeof(DevHTerm) * groups[g].second.size();
      if (!mine.empty() && staged + gb > (size_t)kHamStageBytes) continue;
      if (popc(tile | groups[g].first) <= k) {
        tile |= groups[g].first;
        mine.push_back(g);
        staged += gb;
      }
    }
    if (!first && mine.empty()) {
      err = "internal: a tile-sized flip group did not fit an empty pass";
      return false;
    }
    for (int g : mine) done[g] = true;
    n_left -= mine.size();
    emit(fill_tile(tile), mine, first, !first, 0u);
    first = false;
  }
  // paired passes.  Groups g with the same f_g & ~tile share a pass, which
  // holds when the tile contains every bit where f_g differs from the first
  // open group's f0.  So the tile starts with the positions every tile holds
  // and takes, group by group, the differing bits while they fit; the rest of
  // the tile is filled from the lowest positions.  f_out = f0 & ~tile is not
  // empty: f0 does not fit one tile with the fixed positions.
  for (size_t wi = 0; wi < wide.size(); ++wi) {
    const int g0 = wide[wi];
    if (done[g0]) continue;
    const uint32_t f0 = groups[g0].first;
    uint32_t tile = io_low;
    std::vector<int> mine{g0};
    size_t staged = sizeof(DevHFlip) + sizeof(DevHTerm) * groups[g0].second.size();
    for (size_t wj = wi + 1; wj < wide.size(); ++wj) {
      const int g = wide[wj];
      if (done[g]) continue;
      const uint32_t d = (groups[g].first ^ f0) & ~tile;
      const size_t gb = sizeof(DevHFlip) + sizeof(DevHTerm) * groups[g].second.size();
      if (popc(tile | d) > k || staged + gb > (size_t)kHamStageBytes) continue;
      tile |= d;
      mine.push_back(g);
      staged += gb;
    }
    tile = fill_tile(tile);
    emit(tile, mine, false, true, f0 & ~tile);
  }
  return true;
}

}  // namespace tcb
