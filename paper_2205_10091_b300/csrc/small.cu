// Small circuits in one launch: state, gates and Pauli-sum expectations.
//
// A circuit of 5..10 qubits fits in the shared memory of one CTA, and the
// tile-pass engine runs it on one SM: its arithmetic (complex128 gates are
// FP64, which this GPU executes at a small fraction of its FP32 rate) then
// waits on that SM's four FP64 pipes, and the state, each Pauli sum and its
// reduction are separate launches.  Here one launch per batch row does all of
// it, with the state spread over a thread-block cluster: 2^L amplitudes per
// CTA (L = min(n, 7)), one amplitude per thread, 2^(n-L) CTAs (at most 8, the
// portable cluster size).  Bits 0..4 of the index are warp lanes, bits 5..L-1
// warps of the CTA, bits L..n-1 the CTA's rank in the cluster.
//
// Each gate reads its partner amplitudes (index ^ mask) by a warp shuffle
// (mask inside the lanes), through the CTA's shared memory (mask inside the
// CTA) or through the cluster's distributed shared memory (mask reaching the
// rank bits).  Exchanges through memory alternate between two buffers; the
// host plans which exchanges need a CTA barrier, a cluster barrier, and a
// cluster barrier before a buffer is reused after remote reads.  Consecutive
// one-qubit ops on a qubit with nothing else on it in between are fused into
// one 2x2 matrix (built per row in FP64 from theta at the start of the launch).
// The expectations <psi|P|psi> of the Pauli terms (Section "Pauli structures
// and weights") are summed per observable in FP64, within the CTA and then
// across the cluster into rank 0.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"

namespace cg = cooperative_groups;

namespace tcb {

enum : int8_t {
  SK_MAT2 = 0,  // 2x2 matrix slot `slot` on position p0
  SK_CNOT = 1,  // control position p1, target position p0
  SK_CZ = 2,    // positions p0, p1
  SK_RZZ = 3,   // phase slot `slot` (even, odd parity of positions p0, p1)
  SK_MAT4 = 4,  // 4x4 matrix slot `slot`; row bit 1 = position p0, row bit 0 = position p1
};
enum : uint8_t {
  SX_NONE = 0,     // diagonal: no partner
  SX_SHFL = 1,     // partners inside the warp
  SX_CTA = 2,      // partners inside the CTA: shared memory + CTA barrier
  SX_CLUSTER = 3,  // partners in other CTAs: distributed shared memory + cluster barrier
};

// The index a thread holds is physical: g = (rank << L) | thread.  CNOTs
// between two rank qubits are not executed: they relabel which CTA holds
// which logical rank, a linear map over GF(2) that the host tracks.  So a
// step names, per logical qubit it touches, the physical flip mask (its
// partner is g ^ f) and the physical selector mask (its bit is the parity of
// g & s); for qubits inside a CTA both are the position's own bit.
struct SmallStep {  // 24 bytes
  uint32_t f0, f1;  // flip masks: target (MAT2, CNOT) / row bit 1 and row bit 0 (MAT4)
  uint32_t s0, s1;  // selector masks: target (MAT2), p0 / p1 (CZ, RZZ, MAT4), control in s1 (CNOT)
  int8_t kind;
  uint8_t xch;      // SX_*
  uint8_t buf;      // exchange buffer (0 or 1)
  uint8_t guard;    // 1: cluster barrier before writing the buffer (remote readers of its last use)
  int16_t slot;     // matrix slot (host); first entry of its matrix in the table (device copy)
  int16_t pad;
};
static_assert(sizeof(SmallStep) == 24, "SmallStep layout");
struct SmallComp {  // one op multiplied into a matrix slot
  int32_t kind;     // tc_opkind
  int32_t param;
  double scale;
  int32_t pool;
  int32_t pad;
};
struct SmallSlot {
  int32_t comp_off, n_comp;
  int32_t dim;     // 2 (MAT2), 4 (MAT4) or 1 (RZZ phase pair)
  int32_t entry;   // first complex entry in the CTA's matrix table
};
struct SmallTerm {
  uint32_t f, sm;  // flip mask, sign mask (Z and Y positions)
  int32_t ny, obs;
  double w;
};

struct SmallPlan {
  int n = 0, L = 0, cb = 0;  // qubits, local qubits, log2 of the cluster size
  std::vector<SmallStep> steps;
  std::vector<SmallStep> dsteps;  // steps with matrix entries (uploaded)
  std::vector<SmallComp> comps;
  std::vector<SmallSlot> slots;
  int n_entries = 0;         // complex entries of the matrix table
  uint32_t arow[3] = {1, 2, 4};  // logical rank bit q = parity(physical rank & arow[q]) after the last step
  uint32_t acol[3] = {1, 2, 4};  // flipping logical rank bit q flips physical rank bits acol[q]
  int final_buf = 0, final_guard = 0;
  // device copies (owned)
  SmallStep* d_steps = nullptr;
  SmallComp* d_comps = nullptr;
  SmallSlot* d_slots = nullptr;
  // observables of the last call (device, cached by their bytes)
  std::vector<char> obs_key;
  SmallTerm* d_terms = nullptr;
  int n_terms = 0, K = 0;
};

void small_free(SmallPlan* p) {
  if (!p) return;
  dev_free(p->d_steps);
  dev_free(p->d_comps);
  dev_free(p->d_slots);
  dev_free(p->d_terms);
  delete p;
}

constexpr int kSmallMinQubits = 5;
constexpr int kSmallMaxQubits = 10;
constexpr int kSmallLocal = 7;
constexpr int kSmallMaxTerms = 256;
constexpr int kSmallMaxObs = 16;
constexpr size_t kSmallSmemCap = 48 * 1024;

// Plan of a circuit for the one-launch path, or nullptr with the reason.
SmallPlan* small_build(const tc_circuit* c, std::string& why) {
  const int n = c->n;
  if (n < kSmallMinQubits || n > kSmallMaxQubits) {
    why = "width outside 5..10 qubits";
    return nullptr;
  }
  if (c->n_noise > 0) {
    why = "noise events";
    return nullptr;
  }
  auto* P = new SmallPlan();
  P->n = n;
  P->L = std::min(n, kSmallLocal);
  P->cb = n - P->L;
  const uint32_t lane_mask = 31u, cta_mask = (1u << P->L) - 1u;
  std::vector<int> open(n, -1);  // per position: matrix slot still open to fusion
  auto new_slot = [&](int dim) {
    SmallSlot s{};
    s.comp_off = (int)P->comps.size();
    s.n_comp = 0;
    s.dim = dim;
    s.entry = P->n_entries;
    P->n_entries += dim == 1 ? 2 : dim * dim;
    P->slots.push_back(s);
    return (int)P->slots.size() - 1;
  };
  auto add_comp = [&](int slot, const tc_op& o) {
    // components of a slot are contiguous: a fused op is appended right after
    // the slot's last one, moving later slots' components up by one
    SmallSlot& s = P->slots[slot];
    const int at = s.comp_off + s.n_comp;
    SmallComp k{};
    k.kind = o.kind;
    k.param = o.param;
    k.scale = o.scale;
    k.pool = o.mat;
    P->comps.insert(P->comps.begin() + at, k);
    s.n_comp++;
    for (size_t j = 0; j < P->slots.size(); ++j)
      if ((int)j != slot && P->slots[j].comp_off >= at) P->slots[j].comp_off++;
  };
  auto xch_of = [&](uint32_t m) -> uint8_t {
    if (m == 0) return SX_NONE;
    if ((m & ~lane_mask) == 0) return SX_SHFL;
    if ((m & ~cta_mask) == 0) return SX_CTA;
    return SX_CLUSTER;
  };
  // physical masks of logical position p under the current rank map
  auto fmask = [&](int p) -> uint32_t { return p < P->L ? 1u << p : P->acol[p - P->L] << P->L; };
  auto smask = [&](int p) -> uint32_t { return p < P->L ? 1u << p : P->arow[p - P->L] << P->L; };
  for (const tc_op& o : c->ops_in) {
    const int p0 = n - 1 - o.q0;
    const int p1 = (o.kind == TC_OP_RZZ || o.kind == TC_OP_CNOT || o.kind == TC_OP_CZ || o.kind == TC_OP_U2)
                       ? n - 1 - o.q1 : -1;
    SmallStep st{};
    st.slot = -1;
    switch (o.kind) {
      case TC_OP_H:
      case TC_OP_X:
      case TC_OP_RX:
      case TC_OP_RY:
      case TC_OP_RZ:
      case TC_OP_U1:
        if (open[p0] >= 0) {
          add_comp(open[p0], o);
          continue;
        }
        st.kind = SK_MAT2;
        st.slot = (int16_t)new_slot(2);
        add_comp(st.slot, o);
        open[p0] = st.slot;
        st.f0 = fmask(p0);
        st.s0 = smask(p0);
        st.xch = xch_of(st.f0);
        break;
      case TC_OP_CNOT:
        // control q0 (position p0), target q1 (position p1)
        if (p0 >= P->L && p1 >= P->L) {
          // between two rank qubits: logical target bit t becomes t ^ u
          const int u = p0 - P->L, t = p1 - P->L;
          P->arow[t] ^= P->arow[u];
          P->acol[u] ^= P->acol[t];
          if (open[p0] >= 0) open[p0] = -1;
          if (open[p1] >= 0) open[p1] = -1;
          continue;
        }
        st.kind = SK_CNOT;
        st.f0 = fmask(p1);
        st.s1 = smask(p0);
        st.xch = xch_of(st.f0);
        break;
      case TC_OP_CZ:
        st.kind = SK_CZ;
        st.s0 = smask(p0);
        st.s1 = smask(p1);
        st.xch = SX_NONE;
        break;
      case TC_OP_RZZ:
        st.kind = SK_RZZ;
        st.slot = (int16_t)new_slot(1);
        add_comp(st.slot, o);
        st.s0 = smask(p0);
        st.s1 = smask(p1);
        st.xch = SX_NONE;
        break;
      case TC_OP_U2:
        st.kind = SK_MAT4;
        st.slot = (int16_t)new_slot(4);
        add_comp(st.slot, o);
        st.f0 = fmask(p0);
        st.f1 = fmask(p1);
        st.s0 = smask(p0);
        st.s1 = smask(p1);
        st.xch = xch_of(st.f0 | st.f1);
        break;
      default:
        why = "op kind without a one-launch form";
        delete P;
        return nullptr;
    }
    // a non-diagonal step or any two-qubit step ends fusion on its positions
    if (st.kind != SK_MAT2) {
      if (p0 >= 0) open[p0] = -1;
      if (p1 >= 0) open[p1] = -1;
    }
    P->steps.push_back(st);
  }
  // exchange buffers and barriers: buffered exchanges alternate between the
  // two buffers; a buffer whose last use was read by other CTAs may be
  // written again only after a cluster barrier that follows those reads
  int use = 0;                   // buffered exchanges so far
  uint8_t last_type[2] = {0, 0};  // type of each buffer's last use
  uint8_t prev_type = 0;          // type of the latest buffered exchange
  auto plan_buffer = [&](uint8_t type, uint8_t& buf, uint8_t& guard) {
    buf = (uint8_t)(use & 1);
    guard = (last_type[buf] == SX_CLUSTER && prev_type != SX_CLUSTER) ? 1 : 0;
    last_type[buf] = type;
    prev_type = type;
    ++use;
  };
  for (auto& st : P->steps)
    if (st.xch == SX_CTA || st.xch == SX_CLUSTER) plan_buffer(st.xch, st.buf, st.guard);
  // the kernel addresses matrices by table entry
  P->dsteps = P->steps;
  for (auto& st : P->dsteps)
    if (st.slot >= 0) st.slot = (int16_t)P->slots[st.slot].entry;

  // the observables read the final state from a buffer, across the cluster
  {
    uint8_t b = 0, g = 0;
    plan_buffer(P->cb > 0 ? SX_CLUSTER : SX_CTA, b, g);
    P->final_buf = b;
    P->final_guard = g;
  }
  return P;
}

namespace {

struct SmallArgs {
  const SmallStep* steps;
  const SmallComp* comps;
  const SmallSlot* slots;
  const SmallTerm* terms;
  const double* theta;
  const double* pool;
  void* states_out;    // [B][2^n] or nullptr
  double* values_out;  // [B][K] or nullptr
  int n, L, cb, n_steps, n_slots, n_comps, n_entries, n_params, init;
  int n_terms, K, final_buf, final_guard;
  uint32_t arow[3];  // logical rank bit q = parity(rank & arow[q]) at the end
  // shared-memory regions (byte offsets; laid out by the host, small_layout)
  uint32_t o_mt, o_cm, o_red, o_cpart, o_sst;
};

// r = a b for 2x2 complex row-major matrices of (re, im) pairs
__device__ __forceinline__ void cmatmul2(double (&r)[8], const double (&a)[8], const double (&b)[8]) {
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double re = 0, im = 0;
      for (int k = 0; k < 2; ++k) {
        const double ar = a[2 * (2 * i + k)], ai = a[2 * (2 * i + k) + 1];
        const double br = b[2 * (2 * k + j)], bi = b[2 * (2 * k + j) + 1];
        re += ar * br - ai * bi;
        im += ar * bi + ai * br;
      }
      r[2 * (2 * i + j)] = re;
      r[2 * (2 * i + j) + 1] = im;
    }
}

// 2x2 matrix of one op (row-major (re, im) pairs), angle = scale * theta[param]
__device__ void op_mat2(double (&m)[8], const SmallComp& k, const double* th, const double* pool) {
  const double a = (k.param >= 0 && th) ? k.scale * th[k.param] : 0.0;
  double s, c;
  sincos(0.5 * a, &s, &c);
  for (int e = 0; e < 8; ++e) m[e] = 0;
  switch (k.kind) {
    case TC_OP_H: {
      const double r = 0.70710678118654752440;
      m[0] = r, m[2] = r, m[4] = r, m[6] = -r;
    } break;
    case TC_OP_X:
      m[2] = 1, m[4] = 1;
      break;
    case TC_OP_RX:  // [[c, -is], [-is, c]]
      m[0] = c, m[3] = -s, m[5] = -s, m[6] = c;
      break;
    case TC_OP_RY:  // [[c, -s], [s, c]]
      m[0] = c, m[2] = -s, m[4] = s, m[6] = c;
      break;
    case TC_OP_RZ:  // diag(e^{-ia/2}, e^{ia/2})
      m[0] = c, m[1] = -s, m[6] = c, m[7] = s;
      break;
    default:  // TC_OP_U1
      for (int e = 0; e < 8; ++e) m[e] = pool[2 * k.pool + e];
      break;
  }
}

template <typename V>
__device__ __forceinline__ V cmadd(V u, V x, V acc) {
  acc.x = fma(u.x, x.x, fma(-u.y, x.y, acc.x));
  acc.y = fma(u.x, x.y, fma(u.y, x.x, acc.y));
  return acc;
}

template <typename T>
struct SmallV;
template <>
struct SmallV<float> {
  using V = float2;
};
template <>
struct SmallV<double> {
  using V = double2;
};

template <typename V>
__device__ __forceinline__ V shfl_x(V v, uint32_t m) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, (int)m);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, (int)m);
  return v;
}

// One batch row per cluster of 2^cb CTAs; one amplitude per thread.
template <typename T>
__global__ void __launch_bounds__(128) k_small(const __grid_constant__ SmallArgs a) {
  using V = typename SmallV<T>::V;
  extern __shared__ __align__(16) unsigned char smem[];
  const int nloc = 1 << a.L;
  V* const buf0 = (V*)smem;  // exchange buffers at offset 0
  V* const buf1 = buf0 + nloc;
  V* mt = (V*)(smem + a.o_mt);                 // matrix table
  double* cm = (double*)(smem + a.o_cm);       // [n_comps][8] each op's own 2x2 (FP64)
  double* red = (double*)(smem + a.o_red);     // [warps][K]
  double* cpart = (double*)(smem + a.o_cpart); // [2^cb][K] (rank 0)
  SmallStep* sst = (SmallStep*)(smem + a.o_sst);  // the step program
  cg::cluster_group cl = cg::this_cluster();
  const int rank = a.cb ? (int)cl.block_rank() : 0;
  const int row = (int)(blockIdx.x >> a.cb);
  const int tid = threadIdx.x;
  const uint32_t g = ((uint32_t)rank << a.L) | (uint32_t)tid;
  // ---- this row's matrices (FP64, later ops multiplied on the left) -------
  // the step program into shared memory (one 8-byte record per gate)
  for (int i = tid; i < a.n_steps; i += blockDim.x) sst[i] = a.steps[i];
  const double* th = a.theta ? a.theta + (size_t)row * a.n_params : nullptr;
  // every one-qubit op's own matrix, one per thread
  for (int i = tid; i < a.n_comps; i += blockDim.x) {
    const SmallComp k = a.comps[i];
    if (k.kind == TC_OP_RZZ || k.kind == TC_OP_U2) continue;
    double m[8];
    op_mat2(m, k, th, a.pool);
    for (int e = 0; e < 8; ++e) cm[8 * i + e] = m[e];
  }
  __syncthreads();
  // each slot: the product of its ops' matrices
  for (int s = tid; s < a.n_slots; s += blockDim.x) {
    const SmallSlot sl = a.slots[s];
    V* out = mt + sl.entry;
    if (sl.dim == 2) {
      double m[8], r[8];
      for (int e = 0; e < 8; ++e) m[e] = cm[8 * sl.comp_off + e];
      for (int k = 1; k < sl.n_comp; ++k) {
        double o[8];
        for (int e = 0; e < 8; ++e) o[e] = cm[8 * (sl.comp_off + k) + e];
        cmatmul2(r, o, m);
        for (int e = 0; e < 8; ++e) m[e] = r[e];
      }
      for (int e = 0; e < 4; ++e) out[e] = V{(T)m[2 * e], (T)m[2 * e + 1]};
    } else if (sl.dim == 4) {
      const int p = a.comps[sl.comp_off].pool;
      for (int e = 0; e < 16; ++e) out[e] = V{(T)a.pool[2 * (p + e)], (T)a.pool[2 * (p + e) + 1]};
    } else {
      const SmallComp k = a.comps[sl.comp_off];
      const double ang = (k.param >= 0 && th) ? k.scale * th[k.param] : 0.0;
      double s2, c2;
      sincos(0.5 * ang, &s2, &c2);
      out[0] = V{(T)c2, (T)-s2};  // even parity: e^{-ia/2}
      out[1] = V{(T)c2, (T)s2};   // odd parity: e^{+ia/2}
    }
  }
  V amp;
  if (a.init == TC_INIT_PLUS) {
    amp = V{(T)(1.0 / sqrt((double)(1u << a.n))), (T)0};
  } else {
    amp = V{(T)(g == 0 ? 1 : 0), (T)0};
  }
  __syncthreads();
  // ---- exchanges ----------------------------------------------------------
  auto publish = [&](int b, int guard, bool cluster) -> V* {
    if (guard) cl.sync();
    V* const bb = b ? buf1 : buf0;
    bb[tid] = amp;
    if (cluster) cl.sync();
    else __syncthreads();
    return bb;
  };
  auto partner = [&](V* b, uint32_t m) -> V {  // amplitude at g ^ m
    const uint32_t idx = g ^ m;
    const int r = (int)(idx >> a.L);
    const uint32_t li = idx & (uint32_t)(nloc - 1);
    if (r == rank) return b[li];
    const V* rb = cl.map_shared_rank(b, r);
    return rb[li];
  };
  // ---- gates --------------------------------------------------------------
  auto par = [&](uint32_t m) -> int { return __popc(g & m) & 1; };
  for (int si = 0; si < a.n_steps; ++si) {
    const SmallStep st = sst[si];
    switch (st.kind) {
      case SK_MAT2: {
        const int bit = par(st.s0);
        V p;
        if (st.xch == SX_SHFL) p = shfl_x(amp, st.f0);
        else p = partner(publish(st.buf, st.guard, st.xch == SX_CLUSTER), st.f0);
        const V* M = mt + st.slot;
        V r = V{(T)0, (T)0};
        r = cmadd(M[2 * bit + bit], amp, r);
        r = cmadd(M[2 * bit + (bit ^ 1)], p, r);
        amp = r;
      } break;
      case SK_CNOT: {
        V p;
        if (st.xch == SX_SHFL) p = shfl_x(amp, st.f0);
        else p = partner(publish(st.buf, st.guard, st.xch == SX_CLUSTER), st.f0);
        if (par(st.s1)) amp = p;
      } break;
      case SK_CZ:
        if (par(st.s0) & par(st.s1)) amp = V{-amp.x, -amp.y};
        break;
      case SK_RZZ: {
        const V ph = mt[st.slot + par(st.s0 ^ st.s1)];
        V r = V{(T)0, (T)0};
        amp = cmadd(ph, amp, r);
      } break;
      default: {  // SK_MAT4: row index 2 b(q0) + b(q1)
        const int rr = 2 * par(st.s0) + par(st.s1);
        V y[4];  // y[d] = amplitude with the row bits flipped by d
        y[0] = amp;
        if (st.xch == SX_SHFL) {
          y[1] = shfl_x(amp, st.f1);
          y[2] = shfl_x(amp, st.f0);
          y[3] = shfl_x(amp, st.f0 ^ st.f1);
        } else {
          V* b = publish(st.buf, st.guard, st.xch == SX_CLUSTER);
          y[1] = partner(b, st.f1);
          y[2] = partner(b, st.f0);
          y[3] = partner(b, st.f0 ^ st.f1);
        }
        const V* M = mt + st.slot;
        V r = V{(T)0, (T)0};
#pragma unroll
        for (int d = 0; d < 4; ++d) r = cmadd(M[4 * rr + (rr ^ d)], y[d], r);
        amp = r;
      } break;
    }
  }
  if (a.states_out) {
    uint32_t rl = 0;
    for (int q = 0; q < a.cb; ++q) rl |= (uint32_t)(__popc((uint32_t)rank & a.arow[q]) & 1) << q;
    ((V*)a.states_out)[((size_t)row << a.n) | (rl << a.L) | (uint32_t)tid] = amp;
  }
  // ---- Pauli-sum expectations: sum_g Re(conj(psi_{g^f}) i^ny (-1)^popc(g & sm) psi_g) w
  const int nw = blockDim.x >> 5, warp = tid >> 5, lane = tid & 31;
  if (a.K > 0) {
    V* b = publish(a.final_buf, a.final_guard, a.cb > 0);
    int t = 0;
    for (int k = 0; k < a.K; ++k) {
      double acc = 0;
      for (; t < a.n_terms && a.terms[t].obs == k; ++t) {
        const SmallTerm tm = a.terms[t];
        const V p = tm.f ? partner(b, tm.f) : amp;
        const double re = (double)p.x * (double)amp.x + (double)p.y * (double)amp.y;  // Re(conj(p) amp)
        const double im = (double)p.x * (double)amp.y - (double)p.y * (double)amp.x;  // Im(conj(p) amp)
        double v = (tm.ny & 1) ? ((tm.ny & 2) ? im : -im) : ((tm.ny & 2) ? -re : re);
        if (__popc(g & tm.sm) & 1) v = -v;
        acc = fma(tm.w, v, acc);
      }
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) red[warp * a.K + k] = acc;
    }
    __syncthreads();
    if (tid < a.K) {
      double s = 0;
      for (int w = 0; w < nw; ++w) s += red[w * a.K + tid];
      if (a.cb == 0) {
        if (a.values_out) a.values_out[(size_t)row * a.K + tid] = s;
      } else {
        double* p0 = cl.map_shared_rank(cpart, 0);
        p0[rank * a.K + tid] = s;
      }
    }
    if (a.cb > 0) {
      cl.sync();
      if (rank == 0 && tid < a.K) {
        double s = 0;
        for (int r = 0; r < (1 << a.cb); ++r) s += cpart[r * a.K + tid];
        if (a.values_out) a.values_out[(size_t)row * a.K + tid] = s;
      }
    }
  }
  // no CTA leaves while another may still read its shared memory
  if (a.cb > 0) cl.sync();
}

}  // namespace

// Observables as a sorted term list (device copy cached by the inputs' bytes).
static tc_status small_set_obs(SmallPlan* P, int K, const int* T, const uint8_t* st, const double* w) {
  int total = 0;
  for (int k = 0; k < K; ++k) total += T[k];
  std::vector<char> key(sizeof(int) * (K + 1) + (size_t)total * P->n + (size_t)total * 8);
  {
    char* q = key.data();
    memcpy(q, &K, sizeof(int));
    memcpy(q + sizeof(int), T, sizeof(int) * K);
    q += sizeof(int) * (K + 1);
    if (total) memcpy(q, st, (size_t)total * P->n);
    if (total) memcpy(q + (size_t)total * P->n, w, (size_t)total * 8);
  }
  if (key == P->obs_key && (total == 0 || P->d_terms)) return TC_OK;
  std::vector<SmallTerm> terms;
  int t = 0;
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < T[k]; ++j, ++t) {
      SmallTerm tm{};
      for (int q = 0; q < P->n; ++q) {
        const uint8_t code = st[(size_t)t * P->n + q];
        if (code > 3) return fail(TC_E_INVALID, "structure entry outside {0,1,2,3}");
        const uint32_t b = 1u << (P->n - 1 - q);
        if (code == 1 || code == 2) tm.f |= b;
        if (code == 2 || code == 3) tm.sm |= b;
        if (code == 2) tm.ny++;
      }
      tm.ny &= 3;
      // to physical masks under the final rank map
      const uint32_t loc = (1u << P->L) - 1u;
      uint32_t f = tm.f & loc, sm = tm.sm & loc;
      for (int q = 0; q < P->cb; ++q) {
        if ((tm.f >> (P->L + q)) & 1u) f ^= P->acol[q] << P->L;
        if ((tm.sm >> (P->L + q)) & 1u) sm ^= P->arow[q] << P->L;
      }
      tm.f = f;
      tm.sm = sm;
      tm.obs = k;
      tm.w = w[t];
      if (!std::isfinite(tm.w)) return fail(TC_E_INVALID, "weight not finite");
      terms.push_back(tm);
    }
  dev_free(P->d_terms);
  P->d_terms = nullptr;
  P->obs_key.clear();
  cudaError_t e = dev_upload(terms, &P->d_terms);
  if (e != cudaSuccess) return cuda_fail(e, "observable upload");
  P->n_terms = total;
  P->K = K;
  P->obs_key.swap(key);
  return TC_OK;
}

// Shared-memory layout of one CTA: exchange buffers, matrix table, op
// matrices, reduction scratch, step program (16-byte aligned regions).
struct SmallLayout {
  uint32_t o_mt, o_cm, o_red, o_cpart, o_sst, bytes;
};
static SmallLayout small_layout(const SmallPlan* P, bool dbl, int K) {
  auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
  const size_t v = dbl ? 16 : 8;
  const size_t nloc = (size_t)1 << P->L;
  SmallLayout l{};
  size_t o = al(2 * nloc * v);
  l.o_mt = (uint32_t)o;
  o = al(o + (size_t)P->n_entries * v);
  l.o_cm = (uint32_t)o;
  o = al(o + 64 * P->comps.size());
  l.o_red = (uint32_t)o;
  o = al(o + (nloc / 32) * (size_t)K * 8);
  l.o_cpart = (uint32_t)o;
  o = al(o + 8 * (size_t)K * 8);
  l.o_sst = (uint32_t)o;
  o = al(o + sizeof(SmallStep) * P->steps.size());
  l.bytes = (uint32_t)o;
  return l;
}
static size_t small_smem(const SmallPlan* P, bool dbl, int K) { return small_layout(P, dbl, K).bytes; }

// Built on first use; nullptr if the circuit has no one-launch form.
static SmallPlan* small_get(tc_circuit* c, std::string& why) {
  if (!c->small_tried) {
    c->small_tried = true;
    c->small = small_build(c, c->small_why);
  }
  why = c->small_why;
  return c->small;
}

static tc_status small_run(tc_circuit* c, SmallPlan* P, const double* d_params, int B, void* d_states,
                           double* d_values, cudaStream_t s) {
  cudaError_t e;
  if (!P->d_steps) {
    if ((e = dev_upload(P->dsteps, &P->d_steps)) != cudaSuccess || (e = dev_upload(P->comps, &P->d_comps)) != cudaSuccess ||
        (e = dev_upload(P->slots, &P->d_slots)) != cudaSuccess)
      return cuda_fail(e, "one-launch plan upload");
  }
  const bool dbl = c->dtype == TC_C128;
  SmallArgs a{};
  a.steps = P->d_steps;
  a.comps = P->d_comps;
  a.slots = P->d_slots;
  a.terms = P->d_terms;
  a.theta = d_params;
  a.pool = c->d_pool;
  a.states_out = d_states;
  a.values_out = d_values;
  a.n = P->n;
  a.L = P->L;
  a.cb = P->cb;
  a.n_steps = (int)P->steps.size();
  a.n_slots = (int)P->slots.size();
  a.n_comps = (int)P->comps.size();
  a.n_entries = P->n_entries;
  a.n_params = c->n_params;
  a.init = (int)c->init;
  a.n_terms = P->n_terms;
  a.K = P->K;
  a.final_buf = P->final_buf;
  a.final_guard = P->final_guard;
  for (int q = 0; q < 3; ++q) a.arow[q] = P->arow[q];
  const SmallLayout lay = small_layout(P, dbl, P->K);
  a.o_mt = lay.o_mt;
  a.o_cm = lay.o_cm;
  a.o_red = lay.o_red;
  a.o_cpart = lay.o_cpart;
  a.o_sst = lay.o_sst;
  const size_t smem = lay.bytes;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)B << P->cb);
  cfg.blockDim = dim3(1u << P->L);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1u << P->cb;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = P->cb > 0 ? 1 : 0;
  prof_before(PK_SMALL, (double)B * (double)(1ull << P->n) * (dbl ? 16.0 : 8.0), s);
  e = dbl ? cudaLaunchKernelEx(&cfg, k_small<double>, a) : cudaLaunchKernelEx(&cfg, k_small<float>, a);
  prof_after(s);
  if (e != cudaSuccess) return cuda_fail(e, "one-launch kernel");
  return TC_OK;
}

bool small_eligible(tc_circuit* c) {
  std::string why;
  return small_get(c, why) != nullptr;
}

}  // namespace tcb

using namespace tcb;

extern "C" {

tc_status tc_apply_expect(tc_circuit* c, const double* d_params, int B, int K, const int* T,
                          const uint8_t* structures, const double* weights, void* d_states_out,
                          double* d_values_out, void* stream) {
  if (!c) return fail(TC_E_INVALID, "NULL circuit");
  if (B < 0 || K < 0) return fail(TC_E_INVALID, "B < 0 or K < 0");
  if (K > 0 && (!T || (B != 0 && !d_values_out))) return fail(TC_E_INVALID, "T or d_values_out is NULL");
  if (c->n_params > 0 && !d_params && B > 0) return fail(TC_E_INVALID, "d_params is NULL");
  if (c->dm_n > 0) return fail(TC_E_UNSUPPORTED, "density-matrix circuits: use tc_dm_expect_pauli_sum");
  int total = 0;
  for (int k = 0; k < K; ++k) {
    if (T[k] < 0) return fail(TC_E_INVALID, "T[k] < 0");
    total += T[k];
  }
  if (total > 0 && (!structures || !weights)) return fail(TC_E_INVALID, "structures/weights NULL");
  if (B == 0) return TC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  std::string why;
  SmallPlan* P = small_get(c, why);
  const bool dbl = c->dtype == TC_C128;
  if (P && total <= kSmallMaxTerms && K <= kSmallMaxObs && small_smem(P, dbl, K) <= kSmallSmemCap) {
    tc_status st = small_set_obs(P, K, T, structures, weights);
    if (st == TC_OK) st = circuit_upload(c);  // the matrix pool lives with the circuit's plan
    if (st != TC_OK) return st;
    return small_run(c, P, d_params, B, d_states_out, d_values_out, s);
  }
  // the general path: states through the tile passes, then one Pauli-sum call per observable
  const size_t per = ((size_t)1 << c->n) * (dbl ? 16 : 8);
  void* states = d_states_out;
  void* own = nullptr;
  double* tmp = nullptr;
  cudaError_t e;
  if (!states) {
    if ((e = cudaMallocAsync(&own, per * B, s)) != cudaSuccess) return cuda_fail(e, "state scratch");
    states = own;
  }
  tc_status st = tc_apply_layers(c, d_params, B, nullptr, 0, nullptr, 0, states, stream);
  if (st == TC_OK && K > 0 && (e = cudaMallocAsync((void**)&tmp, 8 * (size_t)B, s)) != cudaSuccess)
    st = cuda_fail(e, "value scratch");
  for (int k = 0, t0 = 0; st == TC_OK && k < K; t0 += T[k], ++k) {
    st = tc_expect_pauli_sum(c, states, B, structures + (size_t)t0 * c->n, weights + t0, T[k], tmp, stream);
    if (st == TC_OK && (e = cudaMemcpy2DAsync(d_values_out + k, 8 * (size_t)K, tmp, 8, 8, B, cudaMemcpyDeviceToDevice,
                                              s)) != cudaSuccess)
      st = cuda_fail(e, "value copy");
  }
  if (tmp) cudaFreeAsync(tmp, s);
  if (own) cudaFreeAsync(own, s);
  return st;
}

}  // extern "C"
