// State-vector tile-pass kernels for sm_103a.
//
// One CTA owns one tile of 2^k amplitudes of one batch row (its k tile bits
// sit at the positions listed in the pass; the other bits are fixed by the
// CTA index).  Each thread keeps 2^RB amplitudes in registers.  A pass runs
// a list of register stages: the first stage loads straight from HBM with the
// warp's lanes on positions 0..4 (fully coalesced 256-byte rows), each later
// stage re-maps the register bits through a swizzled shared-memory transpose,
// and the last stage stores straight to HBM.  Gates run on registers; diagonal
// groups read one phase from a per-CTA table per amplitude.
//
// Modes
//   KM_FWD  apply gates to psi                      (Section "Circuits and gates")
//   KM_BWD  adjoint sweep: per gate, accumulate s*Im<lam|G|psi> and apply
//           U^dagger to psi and lam (reverse-mode gradient of Section
//           "Gradients, optimization and variational algorithms")
//   KM_HAM  lambda (+)= H psi and the energy partial sum_x Re conj(psi_x) (H psi)_x
//           with terms grouped by flip mask (Section "vmap over Pauli
//           structures"; Eq. H-pauli)
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <vector>

#include "sv_kernels.cuh"

namespace tcb {

template <typename T>
struct VT;
template <>
struct VT<float> {
  using V = float2;
};
template <>
struct VT<double> {
  using V = double2;
};

template <typename V, typename S>
__device__ __forceinline__ V mk(S x, S y) {
  V v;
  v.x = x;
  v.y = y;
  return v;
}

// m0*x0 + m1*x1 (complex)
template <typename V>
__device__ __forceinline__ V cmac2(V m0, V x0, V m1, V x1) {
  V r;
  r.x = fma(m0.x, x0.x, fma(-m0.y, x0.y, fma(m1.x, x1.x, -m1.y * x1.y)));
  r.y = fma(m0.x, x0.y, fma(m0.y, x0.x, fma(m1.x, x1.y, m1.y * x1.x)));
  return r;
}
// complex64: the same m0 x0 + m1 x1 as four packed FP32x2 operations,
// (re, im) * m.re + (-im, re) * m.im per term
template <>
__device__ __forceinline__ float2 cmac2(float2 m0, float2 x0, float2 m1, float2 x1) {
  float2 r = __fmul2_rn(make_float2(m0.x, m0.x), x0);
  r = __ffma2_rn(make_float2(-m0.y, m0.y), make_float2(x0.y, x0.x), r);
  r = __ffma2_rn(make_float2(m1.x, m1.x), x1, r);
  return __ffma2_rn(make_float2(-m1.y, m1.y), make_float2(x1.y, x1.x), r);
}
template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
  V r;
  r.x = fma(a.x, b.x, -a.y * b.y);
  r.y = fma(a.x, b.y, a.y * b.x);
  return r;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// uniform number of noise event e for batch row `row`
__device__ double noise_uniform(const KArgs& a, int row, int e) {
  if (a.status) return (double)a.status[(size_t)row * a.n_noise + e];
  const uint64_t traj = (uint64_t)(a.row_offset + row);
  const uint4 w = philox4x32_10(make_uint4((uint32_t)(e >> 2), (uint32_t)traj, (uint32_t)(traj >> 32), 0u),
                                make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32)));
  const uint32_t word = (e & 3) == 0 ? w.x : (e & 3) == 1 ? w.y : (e & 3) == 2 ? w.z : w.w;
  return (double)(word >> 8) * (1.0 / 16777216.0);
}

// ---------------------------------------------------------------------------
// Per-CTA matrix table (gate matrices for this row's angles)
// ---------------------------------------------------------------------------
template <typename V>
__device__ void build_mat(const DevMat& m, V* tab, const double* th, const double* pool, const KArgs& a,
                          int row) {
  using S = decltype(V::x);
  double ang = (m.param >= 0 && th) ? m.scale * th[m.param] : 0.0;
  if (m.adj) ang = -ang;  // rotations: U(a)^dagger = U(-a)
  V* t = tab + m.dst;
  switch (m.type) {
    case MT_H: {
      const double r = 0.70710678118654752440;
      t[0] = mk<V>((S)r, (S)0);
      t[1] = mk<V>((S)r, (S)0);
      t[2] = mk<V>((S)r, (S)0);
      t[3] = mk<V>((S)-r, (S)0);
    } break;
    case MT_X:
      t[0] = mk<V>((S)0, (S)0);
      t[1] = mk<V>((S)1, (S)0);
      t[2] = mk<V>((S)1, (S)0);
      t[3] = mk<V>((S)0, (S)0);
      break;
    case MT_RX:
    case MT_RY: {
      // (cos(a/2), sin(a/2)) of the effective angle; the kernel applies
      // RX = [[c, -is], [-is, c]] or RY = [[c, -s], [s, c]].  Complex64 RY
      // entries are (t, c) with t = s / c: the kernel applies c [[1, -t], [t, 1]]
      // with c carried by a running scale (|c| kept >= 2^-60; the rotation
      // error that clamp allows is below 1e-18)
      double s, c;
      sincos(0.5 * ang, &s, &c);
      if (m.type == MT_RY && sizeof(S) == 4) {
        // c is recomputed from the rounded t, so that c [[1, -t], [t, 1]] is
        // orthogonal; it is stored as hi + lo so the running scale sees it
        // to ~2^-48 (a rounded c, repeated over a layer of gates that share
        // an angle, would drift the norm systematically)
        if (fabs(c) < 0x1p-60) c = c < 0 ? -0x1p-60 : 0x1p-60;
        const float tf = (float)(s / c);
        const double ce = copysign(1.0 / sqrt(1.0 + (double)tf * (double)tf), c);
        const float hi = (float)ce;
        t[0] = mk<V>((S)tf, (S)hi);
        t[1] = mk<V>((S)(ce - (double)hi), (S)0);
      } else {
        t[0] = mk<V>((S)c, (S)s);
        if (m.type == MT_RY) t[1] = mk<V>((S)0, (S)0);
      }
    } break;
    case MT_U1: {
      // P_after M P_before with the row's outcomes of the folded noise events
      // (I, X, Y, Z; the same selection as MT_NOISE), then the adjoint if asked
      double re[4], im[4];
      for (int e = 0; e < 4; ++e) {
        re[e] = pool[2 * (m.pool + e)];
        im[e] = pool[2 * (m.pool + e) + 1];
      }
      auto pick = [&](int ev, double t1, double t2, double t3) {
        if (ev < 0) return 0;
        const double u = noise_uniform(a, row, ev);
        return u < t1 ? 0 : u < t2 ? 1 : u < t3 ? 2 : 3;
      };
      auto swap_e = [&](int x, int y) {
        const double r = re[x], i = im[x];
        re[x] = re[y];
        im[x] = im[y];
        re[y] = r;
        im[y] = i;
      };
      auto times_i = [&](int e, double sgn) {  // entry *= sgn * i
        const double r = re[e];
        re[e] = -sgn * im[e];
        im[e] = sgn * r;
      };
      const int wb = pick(m.T, m.t1, m.t2, m.t3), wa = pick(m.T2, m.u1, m.u2, m.u3);
      if (wb == 1 || wb == 2) {  // M X: swap columns; M Y = [[i b, -i a], [i d, -i c]]
        swap_e(0, 1);
        swap_e(2, 3);
        if (wb == 2) {
          times_i(0, 1.0);
          times_i(2, 1.0);
          times_i(1, -1.0);
          times_i(3, -1.0);
        }
      } else if (wb == 3) {  // M Z: negate column 1
        re[1] = -re[1], im[1] = -im[1], re[3] = -re[3], im[3] = -im[3];
      }
      if (wa == 1 || wa == 2) {  // X M: swap rows; Y M = [[-i c, -i d], [i a, i b]]
        swap_e(0, 2);
        swap_e(1, 3);
        if (wa == 2) {
          times_i(0, -1.0);
          times_i(1, -1.0);
          times_i(2, 1.0);
          times_i(3, 1.0);
        }
      } else if (wa == 3) {  // Z M: negate row 1
        re[2] = -re[2], im[2] = -im[2], re[3] = -re[3], im[3] = -im[3];
      }
      for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
          const int src = m.adj ? (c * 2 + r) : (r * 2 + c);
          t[r * 2 + c] = mk<V>((S)re[src], (S)(m.adj ? -im[src] : im[src]));
        }
    } break;
    case MT_U2: {
      const int d = 4;
      for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) {
          const int src = m.adj ? (c * d + r) : (r * d + c);
          const double re = pool[2 * (m.pool + src)], im = pool[2 * (m.pool + src) + 1];
          t[r * d + c] = mk<V>((S)re, (S)(m.adj ? -im : im));
        }
    } break;
    case MT_RSEL: {
      // the row's axis from its number for this event; U(a) = exp(-i a G / 2)
      // (the angle is already negated for an adjoint table)
      const double u = noise_uniform(a, row, m.T);
      const int ax = u < m.t1 ? 1 : u < m.t2 ? 2 : 3;  // X, Y, Z
      double s, c;
      sincos(0.5 * ang, &s, &c);
      if (ax == 1) {
        t[0] = mk<V>((S)c, (S)0);
        t[1] = mk<V>((S)0, (S)-s);
        t[2] = mk<V>((S)0, (S)-s);
        t[3] = mk<V>((S)c, (S)0);
      } else if (ax == 2) {
        t[0] = mk<V>((S)c, (S)0);
        t[1] = mk<V>((S)-s, (S)0);
        t[2] = mk<V>((S)s, (S)0);
        t[3] = mk<V>((S)c, (S)0);
      } else {
        t[0] = mk<V>((S)c, (S)-s);
        t[1] = mk<V>((S)0, (S)0);
        t[2] = mk<V>((S)0, (S)0);
        t[3] = mk<V>((S)c, (S)s);
      }
      t[4] = mk<V>((S)ax, (S)0);
    } break;
    case MT_CHAN: {
      // (a, b) on the (00, 11) block, (c, d) on the (01, 10) block of the 4x4
      auto re = [&](int r, int col) { return pool[2 * (m.pool + 4 * r + col)]; };
      t[0] = mk<V>((S)re(0, 0), (S)re(0, 3));
      t[1] = mk<V>((S)re(1, 1), (S)re(1, 2));
    } break;
    case MT_DIAGTAB: {
      // phase(m) = exp(-i (ang/2) (T - 2m))
      for (int j = 0; j <= m.T; ++j) {
        double s, c;
        sincos(-0.5 * ang * (double)(m.T - 2 * j), &s, &c);
        t[j] = mk<V>((S)c, (S)s);
      }
    } break;
    case MT_QUARTER: {
      // i^{q m}: S (q = +1) or S^dagger (q = -1) on each member qubit with bit 1
      const int q = (m.scale > 0 ? 1 : -1) * (m.adj ? -1 : 1);
      for (int j = 0; j <= m.T; ++j) {
        const int e = ((q * j) % 4 + 4) % 4;
        t[j] = mk<V>((S)(e == 0 ? 1 : e == 2 ? -1 : 0), (S)(e == 1 ? 1 : e == 3 ? -1 : 0));
      }
    } break;
    case MT_NOISE: {
      const double u = noise_uniform(a, row, m.T);
      const int w = u < m.t1 ? 0 : u < m.t2 ? 1 : u < m.t3 ? 2 : 3;  // I, X, Y, Z
      t[0] = mk<V>((S)w, (S)0);
    } break;
    default:
      break;
  }
}

// ---------------------------------------------------------------------------
// Thread <-> amplitude mapping for one stage
// ---------------------------------------------------------------------------
template <int RB>
struct Map {
  uint32_t g;         // global index of register 0 (within the state)
  uint32_t t;         // tile index of register 0
  uint32_t ro[RB];    // global offset of register bit r
  uint32_t rt[RB];    // tile offset of register bit r
};

template <int RB>
__device__ __forceinline__ Map<RB> make_map(const DevPass& P, const int8_t* S, uint32_t tid, uint32_t base) {
  Map<RB> m;
  m.g = base;
  m.t = 0;
  uint32_t smask = 0;
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    smask |= 1u << S[r];
    m.ro[r] = 1u << P.pos[S[r]];
    m.rt[r] = 1u << S[r];
  }
  int b = 0;
  for (int j = 0; j < P.k; ++j) {
    if ((smask >> j) & 1u) continue;
    if ((tid >> b) & 1u) {
      m.t |= 1u << j;
      m.g |= 1u << P.pos[j];
    }
    ++b;
  }
  return m;
}

// Map of a gate-pass stage from its precomputed runs (a few shifts per run).
template <int RB>
__device__ __forceinline__ Map<RB> stage_map(const DevStage& st, uint32_t tid, uint32_t base) {
  Map<RB> m;
  m.g = base;
  m.t = 0;
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    m.ro[r] = 1u << st.P[r];
    m.rt[r] = 1u << st.S[r];
  }
  const int n = st.n_runs;
  for (int q = 0; q < n; ++q) {
    const DevRun u = st.run[q];
    const uint32_t v = (tid >> u.b) & ((1u << u.len) - 1u);
    m.t |= v << u.j;
    m.g |= v << u.p;
  }
  return m;
}

// bit i set when register bit r of amplitude i is set (i < 32)
__constant__ uint32_t kRegBitPattern[5] = {0xaaaaaaaau, 0xccccccccu, 0xf0f0f0f0u, 0xff00ff00u, 0xffff0000u};

template <int RB>
__device__ __forceinline__ uint32_t offg(const Map<RB>& m, int i) {
  uint32_t o = 0;
#pragma unroll
  for (int r = 0; r < RB; ++r)
    if ((i >> r) & 1) o |= m.ro[r];
  return o;
}
template <int RB>
__device__ __forceinline__ uint32_t offt(const Map<RB>& m, int i) {
  uint32_t o = 0;
#pragma unroll
  for (int r = 0; r < RB; ++r)
    if ((i >> r) & 1) o |= m.rt[r];
  return o;
}

// XOR swizzle of the tile index in shared memory: the bank group of an
// amplitude is mixed with bits 4.. of its index so that both "lanes along
// bits 0..4" and "lanes along bits 4..8" access patterns are conflict-free.
template <typename V>
__device__ __forceinline__ uint32_t swz(uint32_t t) {
  return t ^ ((t >> 4) & (sizeof(V) == 8 ? 15u : 7u));
}

// Lowest set bit of a compile-time constant j > 0 (folds after unrolling).
__host__ __device__ constexpr int low_bit(int j) {
  return (j & 1) ? 0 : (j & 2) ? 1 : (j & 4) ? 2 : (j & 8) ? 3 : 4;
}

// Register i of a stage lives at index base ^ XOR_{r in i} off[r].  Walking
// i in reflected Gray-code order (j -> j ^ (j >> 1)) changes one register bit
// per step, so each address is one XOR from the previous one.
template <int RB, typename V>
__device__ __forceinline__ void load_regs(V (&A)[1 << RB], const V* st, const Map<RB>& m) {
  uint32_t idx = m.g;
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) {
    if (j) idx ^= m.ro[low_bit(j)];
    A[j ^ (j >> 1)] = st[idx];
  }
}
template <int RB, typename V>
__device__ __forceinline__ void store_regs(const V (&A)[1 << RB], V* st, const Map<RB>& m) {
  uint32_t idx = m.g;
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) {
    if (j) idx ^= m.ro[low_bit(j)];
    st[idx] = A[j ^ (j >> 1)];
  }
}
template <int RB, typename V>
__device__ __forceinline__ void smem_write(const V (&A)[1 << RB], V* sm, const Map<RB>& m) {
  // swz is linear over XOR and t, rt[r] have disjoint bits
  uint32_t idx = swz<V>(m.t);
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) {
    if (j) idx ^= swz<V>(m.rt[low_bit(j)]);
    sm[idx] = A[j ^ (j >> 1)];
  }
}
template <int RB, typename V>
__device__ __forceinline__ void smem_read(V (&A)[1 << RB], const V* sm, const Map<RB>& m) {
  uint32_t idx = swz<V>(m.t);
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) {
    if (j) idx ^= swz<V>(m.rt[low_bit(j)]);
    A[j ^ (j >> 1)] = sm[idx];
  }
}

// ---------------------------------------------------------------------------
// Register-tile gate primitives (J = register bit; compile-time indices)
// ---------------------------------------------------------------------------
template <int RB, int J, typename V>
__device__ __forceinline__ void g_mat2(V (&A)[1 << RB], const V* t) {
  const V m00 = t[0], m01 = t[1], m10 = t[2], m11 = t[3];
#pragma unroll
  for (int i = 0; i < (1 << RB); ++i) {
    if (i & (1 << J)) continue;
    const V x0 = A[i], x1 = A[i | (1 << J)];
    A[i] = cmac2(m00, x0, m01, x1);
    A[i | (1 << J)] = cmac2(m10, x0, m11, x1);
  }
}
// RX: a0' = c a0 - i s a1, a1' = c a1 - i s a0
template <int RB, int J, typename V>
__device__ __forceinline__ void g_rx(V (&A)[1 << RB], V cs) {
  const auto c = cs.x, s = cs.y;
#pragma unroll
  for (int i = 0; i < (1 << RB); ++i) {
    if (i & (1 << J)) continue;
    const V x0 = A[i], x1 = A[i | (1 << J)];
    A[i] = mk<V>(fma(c, x0.x, s * x1.y), fma(c, x0.y, -s * x1.x));
    A[i | (1 << J)] = mk<V>(fma(c, x1.x, s * x0.y), fma(c, x1.y, -s * x0.x));
  }
}
// Packed FP32x2 arithmetic (sm_100+ FFMA2/FMUL2 on a 64-bit register pair).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
// element-wise a * b on both components (packed for complex64)
__device__ __forceinline__ float2 cmul_re(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 cmul_re(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
// element-wise a * b + c on both components (packed for complex64)
__device__ __forceinline__ float2 cfma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 cfma2(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}

// RY: a0' = c a0 - s a1, a1' = s a0 + c a1.  Complex64 uses the tangent form
// a0' = a0 - t a1, a1' = a1 + t a0 (cs = (t, c); the factor c is left to the
// caller's running scale, see rot_scale): one packed FMA per output.
template <int RB, int J, typename V>
__device__ __forceinline__ void g_ry(V (&A)[1 << RB], V cs) {
  if constexpr (sizeof(V) == 8) {
    const float2 t2 = make_float2(cs.x, cs.x), n2 = make_float2(-cs.x, -cs.x);
#pragma unroll
    for (int i = 0; i < (1 << RB); ++i) {
      if (i & (1 << J)) continue;
      const float2 x0 = A[i], x1 = A[i | (1 << J)];
      A[i] = fma2(n2, x1, x0);
      A[i | (1 << J)] = fma2(t2, x0, x1);
    }
    return;
  }
  const auto c = cs.x, s = cs.y;
#pragma unroll
  for (int i = 0; i < (1 << RB); ++i) {
    if (i & (1 << J)) continue;
    const V x0 = A[i], x1 = A[i | (1 << J)];
    A[i] = mk<V>(fma(c, x0.x, -s * x1.x), fma(c, x0.y, -s * x1.y));
    A[i | (1 << J)] = mk<V>(fma(s, x0.x, c * x1.x), fma(s, x0.y, c * x1.y));
  }
}
template <int RB, int J, typename V>
__device__ __forceinline__ void g_h(V (&A)[1 << RB]) {
  using S = decltype(V::x);
  const S r = (S)0.70710678118654752440;
#pragma unroll
  for (int i = 0; i < (1 << RB); ++i) {
    if (i & (1 << J)) continue;
    const V x0 = A[i], x1 = A[i | (1 << J)];
    A[i] = mk<V>(r * (x0.x + x1.x), r * (x0.y + x1.y));
    A[i | (1 << J)] = mk<V>(r * (x0.x - x1.x), r * (x0.y - x1.y));
  }
}
// Pauli p = 1 (X), 2 (Y), 3 (Z); Y|0> = i|1>, Y|1> = -i|0>
template <int RB, int J, typename V>
__device__ __forceinline__ void g_pauli(V (&A)[1 << RB], int p) {
#pragma unroll
  for (int i = 0; i < (1 << RB); ++i) {
    if (i & (1 << J)) continue;
    const V x0 = A[i], x1 = A[i | (1 << J)];
    if (p == 1) {
      A[i] = x1;
      A[i | (1 << J)] = x0;
    } else if (p == 2) {
      A[i] = mk<V>(x1.y, -x1.x);
      A[i | (1 << J)] = mk<V>(-x0.y, x0.x);
    } else if (p == 3) {
      A[i | (1 << J)] = mk<V>(-x1.x, -x1.y);
    }
  }
}
template <int RB, int J, typename V>
__device__ __forceinline__ void g_cnot(V (&A)[1 << RB], int jc, uint32_t cbase) {
#pragma unroll
  for (int i = 0; i < (1 << RB); ++i) {
    if (i & (1 << J)) continue;
    const uint32_t c = cbase | (jc >= 0 ? ((uint32_t)i >> jc) & 1u : 0u);
    const V x0 = A[i], x1 = A[i | (1 << J)];
    A[i] = c ? x1 : x0;
    A[i | (1 << J)] = c ? x0 : x1;
  }
}
template <int RB, int J0, int J1, typename V>
__device__ __forceinline__ void g_mat4(V (&A)[1 << RB], const V* t) {
#pragma unroll
  for (int i = 0; i < (1 << RB); ++i) {
    if (i & ((1 << J0) | (1 << J1))) continue;
    // row/column index 2*b(q0) + b(q1); q0 on register bit J0, q1 on J1
    const int i00 = i, i01 = i | (1 << J1), i10 = i | (1 << J0), i11 = i | (1 << J0) | (1 << J1);
    const V v0 = A[i00], v1 = A[i01], v2 = A[i10], v3 = A[i11];
    V r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      V a = cmac2(t[4 * q], v0, t[4 * q + 1], v1), b = cmac2(t[4 * q + 2], v2, t[4 * q + 3], v3);
      r[q] = mk<V>(a.x + b.x, a.y + b.y);
    }
    A[i00] = r[0];
    A[i01] = r[1];
    A[i10] = r[2];
    A[i11] = r[3];
  }
}

// Two lowest register bits other than J (compile-time), used to spread a
// reduction over four independent accumulators.
template <int RB, int J>
struct AccBits {
  static constexpr int b0 = (J == 0) ? 1 : 0;
  static constexpr int b1 = (J <= 1) ? 2 : 1;
};

// Adjoint steps: return sum over pairs of Im<lam|G|psi> (G = X or Y) with the
// states as they are, then (if update) apply RX/RY(-a) to psi and lam.
template <int RB, int J, bool ISX, typename V>
__device__ __forceinline__ decltype(V::x) g_adj(V (&P)[1 << RB], V (&L)[1 << RB], V cs, bool update) {
  using S = decltype(V::x);
  if constexpr (!ISX && sizeof(V) == 8) {
    // (l1 . p0) - (l0 . p1) in two packed accumulators
    float2 ap = make_float2(0.f, 0.f), an = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < (1 << RB); ++i) {
      if (i & (1 << J)) continue;
      ap = fma2(L[i | (1 << J)], P[i], ap);
      an = fma2(L[i], P[i | (1 << J)], an);
    }
    if (update) {
      g_ry<RB, J>(P, cs);
      g_ry<RB, J>(L, cs);
    }
    return (ap.x + ap.y) - (an.x + an.y);
  }
  S acc[4] = {0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < (1 << RB); ++i) {
    if (i & (1 << J)) continue;
    const int k = ((i >> AccBits<RB, J>::b0) & 1) | (((i >> AccBits<RB, J>::b1) & 1) << 1);
    const V p0 = P[i], p1 = P[i | (1 << J)], l0 = L[i], l1 = L[i | (1 << J)];
    if (ISX) {
      acc[k] = fma(l0.x, p1.y, acc[k]);
      acc[k] = fma(-l0.y, p1.x, acc[k]);
      acc[k] = fma(l1.x, p0.y, acc[k]);
      acc[k] = fma(-l1.y, p0.x, acc[k]);
    } else {
      acc[k] = fma(-l0.x, p1.x, acc[k]);
      acc[k] = fma(-l0.y, p1.y, acc[k]);
      acc[k] = fma(l1.x, p0.x, acc[k]);
      acc[k] = fma(l1.y, p0.y, acc[k]);
    }
  }
  if (update) {
    if (ISX) {
      g_rx<RB, J>(P, cs);
      g_rx<RB, J>(L, cs);
    } else {
      g_ry<RB, J>(P, cs);
      g_ry<RB, J>(L, cs);
    }
  }
  return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// Sum over pairs of Im<lam|Z|psi> = Im(conj(l0) p0) - Im(conj(l1) p1) on register bit J.
template <int RB, int J, typename V>
__device__ __forceinline__ decltype(V::x) g_zgrad(const V (&P)[1 << RB], const V (&L)[1 << RB]) {
  using S = decltype(V::x);
  S a0 = 0, a1 = 0;
#pragma unroll
  for (int i = 0; i < (1 << RB); ++i) {
    if (i & (1 << J)) continue;
    const V p0 = P[i], p1 = P[i | (1 << J)], l0 = L[i], l1 = L[i | (1 << J)];
    a0 = fma(l0.x, p0.y, fma(-l0.y, p0.x, a0));
    a1 = fma(l1.x, p1.y, fma(-l1.y, p1.x, a1));
  }
  return a0 - a1;
}

// Running scale of complex64 tangent-form RY: every such gate multiplies the
// true state by c = cs.y on top of what the registers hold.  The scale is a
// compensated product sc + sl (the rounding error of each sc * c is carried in
// sl), so it adds no drift of its own.  Once |sc| falls below 2^-20 its
// power-of-two part moves into the registers, which is exact; the register
// values then stay within 2^21 / |c| of the true ones, far from FP32 overflow.
// TWO: the adjoint's psi and lambda share the scale.  A no-op for complex128.
template <int RB, bool TWO, typename V, typename T>
__device__ __forceinline__ void rot_scale(T& sc, T& sl, const V* e, V (&A)[1 << RB], V (&L)[1 << RB]) {
  if constexpr (sizeof(V) == 8) {
    const float c = e[0].y, clo = e[1].x;  // c = c + clo to ~2^-48
    const float p = sc * c;
    sl = fmaf(sl, c, fmaf(sc, clo, fmaf(sc, c, -p)));
    sc = p;
    if (fabsf(sc) < 0x1p-20f) {
      // m = 2^floor(log2 |sc|); |sc| >= 2^-80 here, a normal number
      const float m = __int_as_float(__float_as_int(sc) & 0x7f800000);
      const float inv = __int_as_float((254 << 23) - __float_as_int(m));  // 1 / m, exact
      const float2 m2 = make_float2(m, m);
#pragma unroll
      for (int i = 0; i < (1 << RB); ++i) {
        A[i] = mul2(m2, A[i]);
        if (TWO) L[i] = mul2(m2, L[i]);
      }
      sc *= inv;
      sl *= inv;
    }
  }
}

// Rotations on the register bits of a compile-time mask (entry of bit r at
// t[rank of r in the mask]); adj returns the summed gradient terms, each
// weighted by the running scale squared at its gate.
template <int RB, int MASK, bool ISX, int R0 = 0, int E = 0>
struct RotM {
  // TWO: rotate A and L alike (non-parametric rotations inside an adjoint pass)
  template <bool TWO, typename V, typename T>
  __device__ __forceinline__ static void run(V (&A)[1 << RB], V (&L)[1 << RB], const V* t, T& sc, T& sl) {
    if constexpr (R0 < RB) {
      if constexpr (((MASK >> R0) & 1) != 0) {
        if constexpr (ISX) {
          g_rx<RB, R0>(A, t[E]);
          if (TWO) g_rx<RB, R0>(L, t[E]);
        } else {
          g_ry<RB, R0>(A, t[kRYEntries * E]);
          if (TWO) g_ry<RB, R0>(L, t[kRYEntries * E]);
          rot_scale<RB, TWO>(sc, sl, t + kRYEntries * E, A, L);
        }
        RotM<RB, MASK, ISX, R0 + 1, E + 1>::template run<TWO>(A, L, t, sc, sl);
      } else {
        RotM<RB, MASK, ISX, R0 + 1, E>::template run<TWO>(A, L, t, sc, sl);
      }
    }
  }
  template <typename V, typename T>
  __device__ __forceinline__ static decltype(V::x) adj(V (&P)[1 << RB], V (&L)[1 << RB], const V* t, T& sc, T& sl) {
    if constexpr (R0 < RB) {
      if constexpr (((MASK >> R0) & 1) != 0) {
        decltype(V::x) a = g_adj<RB, R0, ISX>(P, L, t[ISX ? E : kRYEntries * E], true);
        if constexpr (!ISX) {
          const T se = sc + sl;
          a *= se * se;
          rot_scale<RB, true>(sc, sl, t + kRYEntries * E, P, L);
        }
        return a + RotM<RB, MASK, ISX, R0 + 1, E + 1>::adj(P, L, t, sc, sl);
      } else {
        return RotM<RB, MASK, ISX, R0 + 1, E>::adj(P, L, t, sc, sl);
      }
    } else {
      return 0;
    }
  }
};

// Jump-table dispatch of a runtime mask to its compile-time instantiation.
#define TC_MASK_CASES(X) \
  X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) \
  X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30) X(31)

template <int RB, bool ISX, bool TWO, typename V, typename T>
__device__ __forceinline__ void rot_mask(int mask, V (&A)[1 << RB], V (&L)[1 << RB], const V* t, T& sc, T& sl) {
  switch (mask) {
#define TC_ROT_CASE(M) \
  case M:              \
    if constexpr ((M) < (1 << RB)) RotM<RB, (M), ISX>::template run<TWO>(A, L, t, sc, sl); \
    break;
    TC_MASK_CASES(TC_ROT_CASE)
#undef TC_ROT_CASE
    default:
      break;
  }
}
template <int RB, bool ISX, typename V, typename T>
__device__ __forceinline__ decltype(V::x) rot_mask_adj(int mask, V (&P)[1 << RB], V (&L)[1 << RB], const V* t,
                                                       T& sc, T& sl) {
  decltype(V::x) acc = 0;
  switch (mask) {
#define TC_ADJ_CASE(M) \
  case M:              \
    if constexpr ((M) < (1 << RB)) acc = RotM<RB, (M), ISX>::adj(P, L, t, sc, sl); \
    break;
    TC_MASK_CASES(TC_ADJ_CASE)
#undef TC_ADJ_CASE
    default:
      break;
  }
  return acc;
}

// switch helpers: run F<J>() for the runtime register bit j
#define TC_DISPATCH_J(RB, j, CALL)         \
  switch (j) {                             \
    case 0: { constexpr int J = 0; CALL; } break; \
    case 1: { constexpr int J = 1; CALL; } break; \
    case 2: if constexpr (RB > 2) { constexpr int J = 2; CALL; } break; \
    case 3: if constexpr (RB > 3) { constexpr int J = 3; CALL; } break; \
    default: if constexpr (RB > 4) { constexpr int J = 4; CALL; } break; \
  }

template <int RB, typename V>
__device__ __forceinline__ void mat4_dispatch(V (&A)[1 << RB], int j0, int j1, const V* t) {
#define TC_M4(a, b) \
  case a * 8 + b: g_mat4<RB, a, (b < RB ? b : 0)>(A, t); break;
  if constexpr (RB == 2) {
    switch (j0 * 8 + j1) {
      TC_M4(0, 1) TC_M4(1, 0)
      default: break;
    }
  } else if constexpr (RB == 3) {
    switch (j0 * 8 + j1) {
      TC_M4(0, 1) TC_M4(0, 2) TC_M4(1, 0) TC_M4(1, 2) TC_M4(2, 0) TC_M4(2, 1)
      default: break;
    }
  } else if constexpr (RB == 4) {
    switch (j0 * 8 + j1) {
      TC_M4(0, 1) TC_M4(0, 2) TC_M4(0, 3) TC_M4(1, 0) TC_M4(1, 2) TC_M4(1, 3)
      TC_M4(2, 0) TC_M4(2, 1) TC_M4(2, 3) TC_M4(3, 0) TC_M4(3, 1) TC_M4(3, 2)
      default: break;
    }
  } else {
    switch (j0 * 8 + j1) {
      TC_M4(0, 1) TC_M4(0, 2) TC_M4(0, 3) TC_M4(0, 4) TC_M4(1, 0) TC_M4(1, 2) TC_M4(1, 3) TC_M4(1, 4)
      TC_M4(2, 0) TC_M4(2, 1) TC_M4(2, 3) TC_M4(2, 4) TC_M4(3, 0) TC_M4(3, 1) TC_M4(3, 2) TC_M4(3, 4)
      case 4 * 8 + 0: g_mat4<RB, (RB > 4 ? 4 : 1), 0>(A, t); break;
      case 4 * 8 + 1: g_mat4<RB, (RB > 4 ? 4 : 0), 1>(A, t); break;
      case 4 * 8 + 2: g_mat4<RB, (RB > 4 ? 4 : 0), 2>(A, t); break;
      case 4 * 8 + 3: g_mat4<RB, (RB > 4 ? 4 : 0), 3>(A, t); break;
      default: break;
    }
  }
#undef TC_M4
}

// Pauli-channel superoperator on register bits (J0, J1): with the index
// 2 b(J0) + b(J1), x00' = a x00 + b x11, x11' = b x00 + a x11,
// x01' = c x01 + d x10, x10' = d x01 + c x10 (t[0] = (a, b), t[1] = (c, d)).
template <int RB, int J0, int J1, typename V>
__device__ __forceinline__ void g_chan(V (&A)[1 << RB], const V* t) {
  const V a2 = mk<V>(t[0].x, t[0].x), b2 = mk<V>(t[0].y, t[0].y), c2 = mk<V>(t[1].x, t[1].x), d2 = mk<V>(t[1].y, t[1].y);
#pragma unroll
  for (int i = 0; i < (1 << RB); ++i) {
    if (i & ((1 << J0) | (1 << J1))) continue;
    const int i00 = i, i01 = i | (1 << J1), i10 = i | (1 << J0), i11 = i | (1 << J0) | (1 << J1);
    const V x00 = A[i00], x01 = A[i01], x10 = A[i10], x11 = A[i11];
    A[i00] = cfma2(a2, x00, cmul_re(b2, x11));
    A[i11] = cfma2(b2, x00, cmul_re(a2, x11));
    A[i01] = cfma2(c2, x01, cmul_re(d2, x10));
    A[i10] = cfma2(d2, x01, cmul_re(c2, x10));
  }
}

template <int RB, typename V>
__device__ __forceinline__ void chan_dispatch(V (&A)[1 << RB], int j0, int j1, const V* t) {
  // the superoperator is symmetric under exchanging its two qubits: order the bits
  const int lo = j0 < j1 ? j0 : j1, hi = j0 < j1 ? j1 : j0;
#define TC_CH(a, b) \
  case a * 8 + b:   \
    if constexpr (b < RB) g_chan<RB, a, b>(A, t); \
    break;
  switch (lo * 8 + hi) {
    TC_CH(0, 1) TC_CH(0, 2) TC_CH(0, 3) TC_CH(0, 4) TC_CH(1, 2) TC_CH(1, 3) TC_CH(1, 4) TC_CH(2, 3) TC_CH(2, 4)
    TC_CH(3, 4)
    default: break;
  }
#undef TC_CH
}

// Mean and standard error (sample std, ddof = 1, over sqrt(n)) of n doubles,
// FP64, fixed-order reduction (one block).
__global__ void __launch_bounds__(256) k_mean_stderr(const double* x, int n, double* out) {
  __shared__ double s1[256], s2[256];
  double a = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += x[i];
  s1[threadIdx.x] = a;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s1[threadIdx.x] += s1[threadIdx.x + w];
    __syncthreads();
  }
  const double mean = s1[0] / n;
  double b = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) b += (x[i] - mean) * (x[i] - mean);
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s2[threadIdx.x] += s2[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = mean;
    out[1] = n > 1 ? sqrt(s2[0] / (n - 1) / n) : 0.0;
  }
}

cudaError_t launch_mean_stderr(const double* x, int n, double* out, cudaStream_t s) {
  k_mean_stderr<<<1, 256, 0, s>>>(x, n, out);
  return cudaGetLastError();
}

// Squared norm of each state, FP64 accumulation: block (b, row) sums |psi_x|^2
// over its contiguous slice of the row (16-byte loads: two complex64 or one
// complex128 amplitude each) into part[row][b].
__global__ void __launch_bounds__(256) k_norm2(const void* __restrict__ psi, int dbl, int n_qubits, int nblk,
                                               double* __restrict__ part) {
  const int row = blockIdx.y;
  const size_t words = ((size_t)1 << n_qubits) >> (dbl ? 0 : 1);  // 16-byte words per row
  const size_t per = (words + nblk - 1) / nblk;
  const size_t lo = per * blockIdx.x, hi = lo + per < words ? lo + per : words;
  const float4* f4 = (const float4*)psi + (size_t)row * words;
  const double2* d2 = (const double2*)psi + (size_t)row * words;
  double acc = 0.0;
  for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    if (dbl) {
      const double2 v = d2[i];
      acc = fma(v.x, v.x, fma(v.y, v.y, acc));
    } else {
      const float4 v = f4[i];
      const double a = v.x, b = v.y, c = v.z, d = v.w;
      acc = fma(a, a, fma(b, b, fma(c, c, fma(d, d, acc))));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[(size_t)row * nblk + blockIdx.x] = t;
  }
}

cudaError_t launch_norm2(bool dbl, const void* psi, int n_qubits, int rows, int nblk, double* part, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  if (rows > 65535 || nblk < 1) return cudaErrorInvalidConfiguration;
  k_norm2<<<dim3((unsigned)nblk, (unsigned)rows), 256, 0, s>>>(psi, dbl ? 1 : 0, n_qubits, nblk, part);
  return cudaGetLastError();
}

// Warp reduction in the working precision, then FP64 (T -> double).
template <typename S>
__device__ __forceinline__ double warp_sum(S v) {
  double d = (double)v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  return d;
}

// op(x) & mask of one diagonal entry.  For XOR (ZZ/Z) entries op is linear
// over XOR; for AND (CZ) entries the register part is split with the
// thread part g: (g ^ o) & ((g ^ o) >> d) = (g & g>>d) ^ (g & o>>d) ^ (o & g>>d) ^ (o & o>>d),
// which is linear in o only when o is a single bit and o's partners are
// fixed by g, so AND entries take the general path below.
__device__ __forceinline__ uint32_t diag_op(uint32_t x, const DevDiagEnt& en, int sign_mode) {
  const uint32_t v = en.d == 0 ? x : (sign_mode ? (x & (x >> en.d)) : (x ^ (x >> en.d)));
  return v & en.mask;
}
__device__ __forceinline__ uint32_t diag_op_lin(uint32_t g, uint32_t o, const DevDiagEnt& en, int sign_mode) {
  (void)g;
  (void)sign_mode;
  return (en.d == 0 ? o : (o ^ (o >> en.d))) & en.mask;
}

// m(x) of an XOR-type diagonal group for every register amplitude: per entry
// the count is popc(v(g) ^ v(o_i)), walked in Gray-code order.
template <int RB>
__device__ __forceinline__ void diag_counts_lin(int (&cnt)[1 << RB], const Map<RB>& m, const DevDiag& dg,
                                                const DevDiagEnt* ents) {
#pragma unroll
  for (int i = 0; i < (1 << RB); ++i) cnt[i] = 0;
  for (int e = 0; e < dg.n_ent; ++e) {
    const DevDiagEnt en = ents[dg.ent_off + e];
    uint32_t v = diag_op(m.g, en, 0);
    uint32_t vr[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) vr[r] = diag_op_lin(m.g, m.ro[r], en, 0);
#pragma unroll
    for (int j = 0; j < (1 << RB); ++j) {
      if (j) v ^= vr[low_bit(j)];
      cnt[j ^ (j >> 1)] += __popc(v);
    }
  }
}

// m(x) of a diagonal group for one amplitude index
__device__ __forceinline__ int diag_count(uint32_t x, const DevDiag& dg, const DevDiagEnt* ents) {
  int c = 0;
  for (int e = 0; e < dg.n_ent; ++e) {
    const DevDiagEnt en = ents[dg.ent_off + e];
    const uint32_t v = en.d == 0 ? x : (dg.sign_mode ? (x & (x >> en.d)) : (x ^ (x >> en.d)));
    c += __popc(v & en.mask);
  }
  return c;
}

// VAR selects the instruction set compiled into an instantiation (smaller
// code and fewer live registers for simpler passes); bit flags over the
// rotation-layer core (RY, RY multi, their adjoint steps, single-entry
// ZZ/Z/S phase groups):
//   +1  lean: RX, H, X, noise outcomes, 2x2 matrices, CZ groups
//   +2  full: CNOT, 4x4 matrices
//   +4  multi-entry ZZ/Z phase groups (ZZ at several qubit distances)
template <typename T, int MODE, int RB, int VAR>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 ? (RB <= 3 ? 4 : 2) : (RB <= 3 ? 2 : 1)))
    k_pass(const __grid_constant__ KArgs a, const __grid_constant__ PassArgs pa) {
  constexpr bool FULL = (VAR & 2) != 0;
  constexpr bool LEAN = (VAR & 1) != 0;
  constexpr bool MULTI = (VAR & 4) != 0;
  using V = typename VT<T>::V;
  constexpr int R = 1 << RB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the pass descriptor and its first stage arrive as kernel parameters, so
  // the first state loads need no dependent global reads
  const DevPass& sp = pa.pass;

  const int k = sp.k;
  const uint32_t tid = threadIdx.x;
  const int nwarps = blockDim.x >> 5;
  const int warp = tid >> 5, lane = tid & 31;
  // a paired Pauli-sum pass runs one CTA per tile pair: the CTA index skips
  // tile-index bit pair_bit, which is 0 on the CTA's own tile
  const bool paired = MODE == KM_HAM && sp.pair_fout != 0u;
  const int cbits = sp.nfix - (paired ? 1 : 0);
  const int row = (int)(blockIdx.x >> cbits);
  uint32_t tile = blockIdx.x & ((1u << cbits) - 1u);
  if (paired) tile = ((tile >> sp.pair_bit) << (sp.pair_bit + 1)) | (tile & ((1u << sp.pair_bit) - 1u));
  uint32_t base = 0;
  for (int q = 0; q < sp.n_fixruns; ++q) {
    const DevRun u = sp.fixrun[q];
    base |= ((tile >> u.b) & ((1u << u.len) - 1u)) << u.p;
  }
  const size_t soff = (size_t)row << a.N;
  V* psi = (V*)a.psi + soff;
  V* lam = a.lam ? (V*)a.lam + soff : nullptr;

  // shared memory carve-up: tile(s) | table | instructions | diag groups | entries | reduction
  const int tsize = 1 << k;
  V* sm0 = (V*)smem_raw;
  V* sm1 = sm0 + tsize;
  V* tab = sm0 + ((MODE == KM_BWD || paired) ? 2 * tsize : tsize);
  DevInstr* ins = (DevInstr*)(tab + ((sp.table_size + 1) & ~1));
  DevStage* sst = (DevStage*)(ins + sp.n_instr);
  DevDiag* dgs = (DevDiag*)(sst + (MODE == KM_HAM ? 0 : sp.n_stages));
  DevDiagEnt* des = (DevDiagEnt*)(dgs + sp.n_diag);
  double* red = (double*)(des + ((sp.n_dent + 1) & ~1));

  V A[R];
  V L[R];

  if (MODE == KM_HAM) {
    // ---------------- lambda (+)= H psi, energy partial -------------------
    // Ordinary pass: one side, the CTA's tile, whose partners x ^ f lie in the
    // same tile.  Paired pass: side 0 is the CTA's tile t (in sm0), side 1 its
    // partner t ^ pair_fout (in sm1); each side reads its partners from the
    // other side's copy.
    int8_t S[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) S[r] = (int8_t)(k - RB + r);
    const Map<RB> m0 = make_map<RB>(sp, S, tid, base);
    if (paired) {
      const Map<RB> m1 = make_map<RB>(sp, S, tid, base ^ sp.pair_fout);
      load_regs<RB>(L, psi, m1);
      load_regs<RB>(A, psi, m0);
      smem_write<RB>(L, sm1, m1);
    } else {
      load_regs<RB>(A, psi, m0);
    }
    // energy-only calls split the pass's flip groups over gridDim.y blocks;
    // the diagonal terms go to the first of them
    const int nch = gridDim.y, ch = blockIdx.y;
    const int g_lo = (int)(((long long)sp.n_hflip * ch) / nch), g_hi = (int)(((long long)sp.n_hflip * (ch + 1)) / nch);
    // this block's diagonal entries, flip groups and their terms (contiguous),
    // staged in shared memory
    const int n_diag_here = ch == 0 ? sp.n_hdiag : 0;
    int term_lo = 0, term_hi = 0;
    if (g_hi > g_lo) {
      term_lo = a.hflips[sp.hflip_off + g_lo].term_off;
      const DevHFlip last = a.hflips[sp.hflip_off + g_hi - 1];
      term_hi = last.term_off + last.n_terms;
    }
    DevHDiag* hds = (DevHDiag*)(red + 2 * nwarps);
    DevHFlip* hfs = (DevHFlip*)(hds + n_diag_here);
    DevHTerm* hts = (DevHTerm*)(hfs + (g_hi - g_lo));
    {
      auto stage = [&](void* dst, const void* src, int bytes) {
        for (int i = tid; i < bytes / 4; i += blockDim.x) ((uint32_t*)dst)[i] = ((const uint32_t*)src)[i];
      };
      stage(hds, a.hdiag + sp.hdiag_off, n_diag_here * (int)sizeof(DevHDiag));
      stage(hfs, a.hflips + sp.hflip_off + g_lo, (g_hi - g_lo) * (int)sizeof(DevHFlip));
      stage(hts, a.hterms + term_lo, (term_hi - term_lo) * (int)sizeof(DevHTerm));
    }
    smem_write<RB>(A, sm0, m0);
    __syncthreads();
    // swizzled tile offsets of the register bits (the swizzle is XOR-linear)
    uint32_t srt[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) srt[r] = swz<V>(m0.rt[r]);
    const int nsides = paired ? 2 : 1;
    for (int side = 0; side < nsides; ++side) {
      const Map<RB> m = side ? make_map<RB>(sp, S, tid, base ^ sp.pair_fout) : m0;
      // the tile that holds this side's partners
      const V* smp = paired ? (side ? sm0 : sm1) : sm0;
      if (side) smem_read<RB>(A, sm1, m);
      if ((sp.flags & PF_LAM_LOAD) && lam) {
        load_regs<RB>(L, lam, m);
      } else {
  #pragma unroll
        for (int i = 0; i < R; ++i) L[i] = mk<V>((T)0, (T)0);
      }
      T eacc = 0;
      {
        // diagonal terms: the count (or parity) is XOR-linear in the index, so
        // it is walked in Gray-code order over the registers
        V e2 = mk<V>((T)0, (T)0);
        for (int e = 0; e < n_diag_here; ++e) {
          const DevHDiag hd = hds[e];
          const T w = (T)hd.w;
          const uint32_t dd = hd.cnt < 0 ? 0u : hd.d;
          auto op = [&](uint32_t x) { return (dd == 0 ? x : (x ^ (x >> dd))) & hd.mask; };
          uint32_t v = op(m.g);
          uint32_t vr[RB];
  #pragma unroll
          for (int r = 0; r < RB; ++r) vr[r] = op(m.ro[r]);
          if (hd.cnt < 0) {
  #pragma unroll
            for (int j = 0; j < R; ++j) {
              if (j) v ^= vr[low_bit(j)];
              const int i = j ^ (j >> 1);
              const T h = (__popc(v) & 1) ? -w : w;
              const V h2 = mk<V>(h, h);
              L[i] = cfma2(h2, A[i], L[i]);
              e2 = cfma2(cmul_re(h2, A[i]), A[i], e2);
            }
          } else {
  #pragma unroll
            for (int j = 0; j < R; ++j) {
              if (j) v ^= vr[low_bit(j)];
              const int i = j ^ (j >> 1);
              const T h = w * (T)(hd.cnt - 2 * __popc(v));
              const V h2 = mk<V>(h, h);
              L[i] = cfma2(h2, A[i], L[i]);
              e2 = cfma2(cmul_re(h2, A[i]), A[i], e2);
            }
          }
        }
        eacc = e2.x + e2.y;
      }
      for (int g = 0; g < g_hi - g_lo; ++g) {
        const DevHFlip fl = hfs[g];
        const DevHTerm* tt0 = hts + (fl.term_off - term_lo);
        if (fl.n_terms == 1) {
          const DevHTerm ht = tt0[0];
          const T w = (T)ht.w;
          if (ht.sm == 0 && ht.ny == 0) {
            // X string: (P psi)_x = w psi_{x ^ f}; partner index walked in Gray-code order
            uint32_t tt = swz<V>(m.t) ^ swz<V>(fl.f_tile);
            V e2 = mk<V>((T)0, (T)0);
            const V w2 = mk<V>(w, w);
  #pragma unroll
            for (int j = 0; j < R; ++j) {
              if (j) tt ^= srt[low_bit(j)];
              const int i = j ^ (j >> 1);
              const V pp = smp[tt];
              L[i] = cfma2(w2, pp, L[i]);
              e2 = cfma2(A[i], pp, e2);
            }
            eacc = fma(w, e2.x + e2.y, eacc);
            continue;
          }
  #pragma unroll
          for (int i = 0; i < R; ++i) {
            const uint32_t xp = (m.g | offg(m, i)) ^ fl.f;
            const V pp = smp[swz<V>((m.t | offt(m, i)) ^ fl.f_tile)];
            const T ws = (__popc(xp & ht.sm) & 1) ? -w : w;
            const T hr = (ht.ny == 0) ? ws : (ht.ny == 2) ? -ws : (T)0;
            const T hi = (ht.ny == 1) ? ws : (ht.ny == 3) ? -ws : (T)0;
            const T vr = hr * pp.x - hi * pp.y, vi = hr * pp.y + hi * pp.x;
            L[i].x += vr;
            L[i].y += vi;
            eacc = fma(A[i].x, vr, fma(A[i].y, vi, eacc));
          }
          continue;
        }
        if (fl.n_terms <= 4) {
          // up to four terms: each term's sign over this thread's amplitudes is
          // XOR-linear in the index, a base parity (the thread's fixed bits)
          // times a pattern over the register bits, built once per term
          const uint32_t gb = m.g ^ fl.f;
          uint32_t pat[4];
          T wre[4], wim[4];
  #pragma unroll
          for (int q = 0; q < 4; ++q) {
            pat[q] = 0u;
            wre[q] = (T)0;
            wim[q] = (T)0;
            if (q < fl.n_terms) {
              const DevHTerm ht = tt0[q];
              uint32_t pq = (__popc(gb & ht.sm) & 1) ? 0xffffffffu : 0u;
  #pragma unroll
              for (int r = 0; r < RB; ++r)
                if (__popc(m.ro[r] & ht.sm) & 1) pq ^= kRegBitPattern[r];
              pat[q] = pq;
              const T w = (T)ht.w;
              wre[q] = ht.ny == 0 ? w : (ht.ny == 2 ? -w : (T)0);
              wim[q] = ht.ny == 1 ? w : (ht.ny == 3 ? -w : (T)0);
            }
          }
  #pragma unroll
          for (int i = 0; i < R; ++i) {
            const V pp = smp[swz<V>((m.t | offt(m, i)) ^ fl.f_tile)];
            T hr = 0, hi = 0;
  #pragma unroll
            for (int q = 0; q < 4; ++q) {
              const bool neg = (pat[q] >> i) & 1u;
              hr += neg ? -wre[q] : wre[q];
              hi += neg ? -wim[q] : wim[q];
            }
            // (P psi)_x = h(x ^ f) psi_{x ^ f}
            const T vr = hr * pp.x - hi * pp.y, vi = hr * pp.y + hi * pp.x;
            L[i].x += vr;
            L[i].y += vi;
            eacc = fma(A[i].x, vr, fma(A[i].y, vi, eacc));
          }
          continue;
        }
        // more terms: the same in chunks of four
        const uint32_t gb = m.g ^ fl.f;
        for (int q0 = 0; q0 < fl.n_terms; q0 += 4) {
          uint32_t pat[4];
          T wre[4], wim[4];
  #pragma unroll
          for (int q = 0; q < 4; ++q) {
            pat[q] = 0u;
            wre[q] = (T)0;
            wim[q] = (T)0;
            if (q0 + q < fl.n_terms) {
              const DevHTerm ht = tt0[q0 + q];
              uint32_t pq = (__popc(gb & ht.sm) & 1) ? 0xffffffffu : 0u;
  #pragma unroll
              for (int r = 0; r < RB; ++r)
                if (__popc(m.ro[r] & ht.sm) & 1) pq ^= kRegBitPattern[r];
              pat[q] = pq;
              const T w = (T)ht.w;
              wre[q] = ht.ny == 0 ? w : (ht.ny == 2 ? -w : (T)0);
              wim[q] = ht.ny == 1 ? w : (ht.ny == 3 ? -w : (T)0);
            }
          }
  #pragma unroll
          for (int i = 0; i < R; ++i) {
            const V pp = smp[swz<V>((m.t | offt(m, i)) ^ fl.f_tile)];
            T hr = 0, hi = 0;
  #pragma unroll
            for (int q = 0; q < 4; ++q) {
              const bool neg = (pat[q] >> i) & 1u;
              hr += neg ? -wre[q] : wre[q];
              hi += neg ? -wim[q] : wim[q];
            }
            // (P psi)_x = h(x ^ f) psi_{x ^ f}
            const T vr = hr * pp.x - hi * pp.y, vi = hr * pp.y + hi * pp.x;
            L[i].x += vr;
            L[i].y += vi;
            eacc = fma(A[i].x, vr, fma(A[i].y, vi, eacc));
          }
        }
      }
      if ((sp.flags & PF_LAM_STORE) && lam && a.store_lambda && nch == 1) store_regs<RB>(L, lam, m);
      const double ws = warp_sum(eacc);
      if (lane == 0) red[side * nwarps + warp] = ws;
    }
    __syncthreads();
    if (tid < nsides) {
      double s = 0;
      for (int w = 0; w < nwarps; ++w) s += red[tid * nwarps + w];
      const uint32_t t = tid ? (tile ^ sp.pair_fout_idx) : tile;
      a.epart[(((size_t)row * a.n_hpasses + sp.epart_index) * nch + ch) * (1u << sp.nfix) + t] = s;
    }
    return;
  }

  // ---------------- gate passes (forward / adjoint) ------------------------
  {
    const V* trow = (const V*)a.tables + (size_t)row * a.table_stride + sp.table_off;
    for (int i = tid; i < sp.table_size; i += blockDim.x) tab[i] = trow[i];
    for (int i = tid; i < sp.n_instr; i += blockDim.x) ins[i] = a.instrs[sp.instr_off + i];
    {
      const uint32_t* src = (const uint32_t*)(a.stages + sp.stage_off);
      uint32_t* dst = (uint32_t*)sst;
      const int words = sp.n_stages * (int)(sizeof(DevStage) / 4);
      for (int i = tid; i < words; i += blockDim.x) dst[i] = src[i];
    }
    for (int i = tid; i < sp.n_diag; i += blockDim.x) dgs[i] = a.diags[sp.diag_off + i];
    for (int i = tid; i < sp.n_dent; i += blockDim.x) des[i] = a.dents[sp.dent_off + i];
    if (MODE == KM_BWD)
      for (int i = tid; i < sp.n_gslots * nwarps; i += blockDim.x) red[i] = 0.0;
  }
  // gradient partials: one per-thread accumulator per local slot (reduced
  // once at the end of the pass); slots beyond kLocalSlots reduce at once
  T gl[kLocalSlots];
  if (MODE == KM_BWD)
    for (int g = 0; g < sp.n_gslots && g < kLocalSlots; ++g) gl[g] = 0;
  // running scale sc + sl of tangent-form rotations (complex64; stays 1 for complex128)
  T sc = 1, sl = 0;
  auto sq = [](T x) { return x * x; };
  auto add_grad = [&](int slot, T v) {
    if (slot < kLocalSlots) {
      gl[slot] += v;
      return;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[slot * nwarps + warp] += (double)v;
  };
  // stage 0's map from the kernel parameters: the state loads are in flight
  // while the per-CTA tables are being staged
  Map<RB> m = stage_map<RB>(pa.st0, tid, base);
  if (MODE == KM_FWD && (sp.flags & PF_INIT) && a.synth_init) {
    if (a.init == 1) {
      const uint32_t anc = (1u << (a.N - a.n_user)) - 1u;
      const T amp = (T)exp2(-0.5 * (double)a.n_user);
#pragma unroll
      for (int i = 0; i < R; ++i) A[i] = mk<V>(((m.g | offg(m, i)) & anc) ? (T)0 : amp, (T)0);
    } else {
#pragma unroll
      for (int i = 0; i < R; ++i) A[i] = mk<V>((m.g | offg(m, i)) == 0 ? (T)1 : (T)0, (T)0);
    }
  } else {
    load_regs<RB>(A, psi, m);
    if (MODE == KM_BWD) load_regs<RB>(L, lam, m);
  }
  __syncthreads();  // table, instructions, stages and groups ready

  for (int s = 0; s < sp.n_stages; ++s) {
    const int n_instr = sst[s].n_instr, instr_off = sst[s].instr_off;
    if (s > 0) {
      smem_write<RB>(A, sm0, m);
      if (MODE == KM_BWD) smem_write<RB>(L, sm1, m);
      m = stage_map<RB>(sst[s], tid, base);
      __syncthreads();
      smem_read<RB>(A, sm0, m);
      if (MODE == KM_BWD) smem_read<RB>(L, sm1, m);
      __syncthreads();
    }
    for (int q = 0; q < n_instr; ++q) {
      const DevInstr in = ins[instr_off + q];
      switch (in.kind) {
        case IK_RX: {
          if (!LEAN) break;
          const V cs = tab[in.slot];
          TC_DISPATCH_J(RB, in.j0, (g_rx<RB, J>(A, cs)));
          if (MODE == KM_BWD) TC_DISPATCH_J(RB, in.j0, (g_rx<RB, J>(L, cs)));
        } break;
        case IK_RXM: {
          if (!LEAN) break;
          const uint32_t mask = (uint8_t)in.j0;
          int e = 0;
          for (int r = 0; r < RB; ++r) {
            if (!((mask >> r) & 1u)) continue;
            const V cs = tab[in.slot + e++];
            TC_DISPATCH_J(RB, r, (g_rx<RB, J>(A, cs)));
            if (MODE == KM_BWD) TC_DISPATCH_J(RB, r, (g_rx<RB, J>(L, cs)));
          }
        } break;
        case IK_RYM: {
          // adjoint passes carry fixed-angle RY as IK_RYM_ADJ without a gradient slot
          if (MODE != KM_FWD) break;
          rot_mask<RB, false, false>((uint8_t)in.j0, A, L, tab + in.slot, sc, sl);
        } break;
        case IK_H:
          if (!LEAN) break;
          TC_DISPATCH_J(RB, in.j0, (g_h<RB, J>(A)));
          if (MODE == KM_BWD) TC_DISPATCH_J(RB, in.j0, (g_h<RB, J>(L)));
          break;
        case IK_X:
          if (!LEAN) break;
          TC_DISPATCH_J(RB, in.j0, (g_pauli<RB, J>(A, 1)));
          if (MODE == KM_BWD) TC_DISPATCH_J(RB, in.j0, (g_pauli<RB, J>(L, 1)));
          break;
        case IK_PAULI: {
          if (!LEAN) break;
          const int p = (int)tab[in.slot].x;
          if (p) {
            TC_DISPATCH_J(RB, in.j0, (g_pauli<RB, J>(A, p)));
            if (MODE == KM_BWD) TC_DISPATCH_J(RB, in.j0, (g_pauli<RB, J>(L, p)));
          }
        } break;
        case IK_MAT2:
          if (!LEAN) break;
          TC_DISPATCH_J(RB, in.j0, (g_mat2<RB, J>(A, tab + in.slot)));
          if (MODE == KM_BWD) TC_DISPATCH_J(RB, in.j0, (g_mat2<RB, J>(L, tab + in.slot)));
          break;
        case IK_CNOT: {
          if (!FULL) break;
          const uint32_t cb = (m.g >> in.pos) & 1u;
          TC_DISPATCH_J(RB, in.j0, (g_cnot<RB, J>(A, in.jc, cb)));
          if (MODE == KM_BWD) TC_DISPATCH_J(RB, in.j0, (g_cnot<RB, J>(L, in.jc, cb)));
        } break;
        case IK_RSEL:
          if (!LEAN) break;
          TC_DISPATCH_J(RB, in.j0, (g_mat2<RB, J>(A, tab + in.slot)));
          if (MODE == KM_BWD) TC_DISPATCH_J(RB, in.j0, (g_mat2<RB, J>(L, tab + in.slot)));
          break;
        case IK_RSEL_ADJ: {
          if (MODE != KM_BWD || !LEAN) break;
          // gradient with the row's axis, then U^dagger (the adjoint table) on psi and lam
          const int ax = (int)tab[in.slot + 4].x;
          const V one = mk<V>((T)1, (T)0);
          T acc = 0;
          if (ax == 1) {
            TC_DISPATCH_J(RB, in.j0, (acc = g_adj<RB, J, true>(A, L, one, false)));
          } else if (ax == 2) {
            TC_DISPATCH_J(RB, in.j0, (acc = g_adj<RB, J, false>(A, L, one, false)));
          } else {
            TC_DISPATCH_J(RB, in.j0, (acc = g_zgrad<RB, J>(A, L)));
          }
          TC_DISPATCH_J(RB, in.j0, (g_mat2<RB, J>(A, tab + in.slot)));
          TC_DISPATCH_J(RB, in.j0, (g_mat2<RB, J>(L, tab + in.slot)));
          add_grad(in.gslot, acc * sq(sc + sl) * (T)in.gscale);
        } break;
        case IK_CHAN:
          if (!LEAN) break;
          chan_dispatch<RB>(A, in.j0, in.j1, tab + in.slot);
          if (MODE == KM_BWD) chan_dispatch<RB>(L, in.j0, in.j1, tab + in.slot);
          break;
        case IK_MAT4:
          if (!FULL) break;
          mat4_dispatch<RB>(A, in.j0, in.j1, tab + in.slot);
          if (MODE == KM_BWD) mat4_dispatch<RB>(L, in.j0, in.j1, tab + in.slot);
          break;
        case IK_DIAG: {
          const DevDiag dg = dgs[in.slot];
          if (dg.n_ent == 1 && !dg.sign_mode) {
            // v(x) = op(x) & mask is linear over XOR: v(g ^ o_i) = v(g) ^ v(o_i)
            const DevDiagEnt en = des[dg.ent_off];
            uint32_t v = diag_op(m.g, en, dg.sign_mode);
            uint32_t vr[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r) vr[r] = diag_op_lin(m.g, m.ro[r], en, dg.sign_mode);
#pragma unroll
            for (int j = 0; j < R; ++j) {
              if (j) v ^= vr[low_bit(j)];
              const int i = j ^ (j >> 1);
              const V ph = tab[dg.tab + __popc(v)];
              A[i] = cmul(ph, A[i]);
              if (MODE == KM_BWD) L[i] = cmul(ph, L[i]);
            }
            break;
          }
          if (MULTI && !dg.sign_mode) {
            // several entries: per entry, the count is XOR-linear in the register offset
            int cnt[R];
            diag_counts_lin<RB>(cnt, m, dg, des);
#pragma unroll
            for (int i = 0; i < R; ++i) {
              const V ph = tab[dg.tab + cnt[i]];
              A[i] = cmul(ph, A[i]);
              if (MODE == KM_BWD) L[i] = cmul(ph, L[i]);
            }
            break;
          }
          if (dg.n_ent == 1 && LEAN) {
            // CZ-type (AND) group: per-amplitude index in Gray-code order
            const DevDiagEnt en = des[dg.ent_off];
            uint32_t x = m.g;
#pragma unroll
            for (int j = 0; j < R; ++j) {
              if (j) x ^= m.ro[low_bit(j)];
              const int i = j ^ (j >> 1);
              if (__popc(x & (x >> en.d) & en.mask) & 1) {
                A[i] = mk<V>(-A[i].x, -A[i].y);
                if (MODE == KM_BWD) L[i] = mk<V>(-L[i].x, -L[i].y);
              }
            }
            break;
          }
          if (!FULL) break;
#pragma unroll
          for (int i = 0; i < R; ++i) {
            const int c = diag_count(m.g | offg(m, i), dg, des);
            if (dg.sign_mode) {
              if (c & 1) {
                A[i] = mk<V>(-A[i].x, -A[i].y);
                if (MODE == KM_BWD) L[i] = mk<V>(-L[i].x, -L[i].y);
              }
            } else {
              const V ph = tab[dg.tab + c];
              A[i] = cmul(ph, A[i]);
              if (MODE == KM_BWD) L[i] = cmul(ph, L[i]);
            }
          }
        } break;
        case IK_RYM_ADJ: {
          if (MODE != KM_BWD) break;
          const T acc = rot_mask_adj<RB, false>((uint8_t)in.j0, A, L, tab + in.slot, sc, sl);
          if (in.gslot >= 0) add_grad(in.gslot, acc * (T)in.gscale);
        } break;
        case IK_RXM_ADJ:
        case IK_GRADDIAG:
        case IK_RX_ADJ: {
          if (MODE != KM_BWD) break;
          T acc = 0;
          if (!LEAN) break;
          if (in.kind == IK_RXM_ADJ) {
            const uint32_t mask = (uint8_t)in.j0;
            int e = 0;
            for (int r = 0; r < RB; ++r) {
              if (!((mask >> r) & 1u)) continue;
              const V cs = tab[in.slot + e++];
              T part = 0;
              TC_DISPATCH_J(RB, r, (part = g_adj<RB, J, true>(A, L, cs, true)));
              acc += part;
            }
          } else if (in.kind == IK_GRADDIAG) {
            const DevDiag dg = dgs[in.slot];
            if (dg.n_ent == 1 && !dg.sign_mode) {
              const DevDiagEnt en = des[dg.ent_off];
              const uint32_t vg = diag_op(m.g, en, 0);
              uint32_t vr[RB];
#pragma unroll
              for (int r = 0; r < RB; ++r) vr[r] = diag_op_lin(m.g, m.ro[r], en, 0);
              T a2[2] = {0, 0};
#pragma unroll
              for (int i = 0; i < R; ++i) {
                uint32_t v = vg;
#pragma unroll
                for (int r = 0; r < RB; ++r)
                  if ((i >> r) & 1) v ^= vr[r];
                a2[i & 1] = fma((T)(dg.T - 2 * __popc(v)), fma(L[i].x, A[i].y, -L[i].y * A[i].x), a2[i & 1]);
              }
              acc = a2[0] + a2[1];
            } else if (FULL) {
#pragma unroll
              for (int i = 0; i < R; ++i) {
                const int c = diag_count(m.g | offg(m, i), dg, des);
                acc += (T)(dg.T - 2 * c) * (L[i].x * A[i].y - L[i].y * A[i].x);
              }
            }
          } else {
            const V cs = tab[in.slot];
            TC_DISPATCH_J(RB, in.j0, (acc = g_adj<RB, J, true>(A, L, cs, true)));
          }
          add_grad(in.gslot, acc * sq(sc + sl) * (T)in.gscale);
        } break;
        case IK_DIAG_ADJ: {
          if (MODE != KM_BWD) break;
          const DevDiag dg = dgs[in.slot];
          if (dg.n_ent == 1 && !dg.sign_mode) {
            // gradient and inverse phase from one index count per amplitude
            const DevDiagEnt en = des[dg.ent_off];
            uint32_t v = diag_op(m.g, en, 0);
            uint32_t vr[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r) vr[r] = diag_op_lin(m.g, m.ro[r], en, 0);
            T a2[2] = {0, 0};
#pragma unroll
            for (int j = 0; j < R; ++j) {
              if (j) v ^= vr[low_bit(j)];
              const int i = j ^ (j >> 1);
              const int c = __popc(v);
              a2[j & 1] = fma((T)(dg.T - 2 * c), fma(L[i].x, A[i].y, -L[i].y * A[i].x), a2[j & 1]);
              const V ph = tab[dg.tab + c];
              A[i] = cmul(ph, A[i]);
              L[i] = cmul(ph, L[i]);
            }
            add_grad(in.gslot, (a2[0] + a2[1]) * sq(sc + sl) * (T)in.gscale);
          } else if (MULTI && !dg.sign_mode) {
            int cnt[R];
            diag_counts_lin<RB>(cnt, m, dg, des);
            T a2[2] = {0, 0};
#pragma unroll
            for (int i = 0; i < R; ++i) {
              a2[i & 1] = fma((T)(dg.T - 2 * cnt[i]), fma(L[i].x, A[i].y, -L[i].y * A[i].x), a2[i & 1]);
              const V ph = tab[dg.tab + cnt[i]];
              A[i] = cmul(ph, A[i]);
              L[i] = cmul(ph, L[i]);
            }
            add_grad(in.gslot, (a2[0] + a2[1]) * sq(sc + sl) * (T)in.gscale);
          } else if (FULL) {
            T acc = 0;
#pragma unroll
            for (int i = 0; i < R; ++i) {
              const int c = diag_count(m.g | offg(m, i), dg, des);
              acc += (T)(dg.T - 2 * c) * (L[i].x * A[i].y - L[i].y * A[i].x);
              const V ph = tab[dg.tab + c];
              A[i] = cmul(ph, A[i]);
              L[i] = cmul(ph, L[i]);
            }
            add_grad(in.gslot, acc * sq(sc + sl) * (T)in.gscale);
          }
        } break;
        default:
          break;
      }
    }
  }
  if (sc != (T)1 || sl != (T)0) {
    const T se = sc + sl;
    const V s2 = mk<V>(se, se);
#pragma unroll
    for (int i = 0; i < R; ++i) {
      A[i] = cmul_re(s2, A[i]);
      if (MODE == KM_BWD) L[i] = cmul_re(s2, L[i]);
    }
  }
  store_regs<RB>(A, psi, m);
  if (MODE == KM_BWD) {
    store_regs<RB>(L, lam, m);
    for (int g = 0; g < sp.n_gslots && g < kLocalSlots; ++g) {
      T v = gl[g];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[g * nwarps + warp] += (double)v;
    }
    __syncthreads();
    for (int g = tid; g < sp.n_gslots; g += blockDim.x) {
      double s = 0;
      for (int w = 0; w < nwarps; ++w) s += red[g * nwarps + w];
      a.gpart[((size_t)row * a.gslots_total + sp.gslot_base + g) * (1u << sp.nfix) + tile] = s;
    }
  }
}

template <typename V>
__global__ void __launch_bounds__(128) k_tables(const __grid_constant__ KArgs a, int first_mat, int n_mats) {
  const int row = blockIdx.x;
  const double* th = a.theta ? a.theta + (size_t)row * a.n_params : nullptr;
  V* trow = (V*)a.tables + (size_t)row * a.table_stride;
  for (int i = threadIdx.x; i < n_mats; i += blockDim.x) build_mat<V>(a.mats[first_mat + i], trow, th, a.pool, a, row);
}

cudaError_t launch_tables(bool dbl, const KArgs& a, int first_mat, int n_mats, int rows, cudaStream_t s) {
  if (rows <= 0 || n_mats <= 0) return cudaSuccess;
  prof_before(PK_TABLES, (double)rows * a.table_stride * (dbl ? 16.0 : 8.0), s);
  if (dbl)
    k_tables<double2><<<rows, 128, 0, s>>>(a, first_mat, n_mats);
  else
    k_tables<float2><<<rows, 128, 0, s>>>(a, first_mat, n_mats);
  prof_after(s);
  return cudaGetLastError();
}

size_t pass_smem_bytes(int mode, bool dbl, const DevPass& p) {
  const size_t v = dbl ? 16 : 8;
  const size_t tsize = (size_t)1 << p.k;
  const int threads = (int)(tsize >> p.rb);
  const int nwarps = threads >= 32 ? threads / 32 : 1;
  size_t b = tsize * v * (mode == KM_BWD ? 2 : 1);
  b += (size_t)((p.table_size + 1) & ~1) * v;
  b += (size_t)p.n_instr * sizeof(DevInstr) + (size_t)p.n_diag * sizeof(DevDiag);
  if (mode != KM_HAM) b += (size_t)p.n_stages * sizeof(DevStage);
  b += (size_t)((p.n_dent + 1) & ~1) * sizeof(DevDiagEnt);
  if (mode == KM_BWD) b += (size_t)p.n_gslots * nwarps * 8;
  if (mode == KM_HAM)
    b += (p.pair_fout ? tsize * v : 0) + (size_t)nwarps * 16 + (size_t)p.n_hdiag * sizeof(DevHDiag) +
         (size_t)p.n_hflip * sizeof(DevHFlip) + (size_t)p.n_hterm * sizeof(DevHTerm);
  return b + 16;
}

template <typename T, int MODE, int RB, int VAR>
static cudaError_t launch_tf(const KArgs& a, const PassArgs& pa, int rows, cudaStream_t s, size_t smem) {
  const DevPass& hp = pa.pass;
  static int configured_max = -1;
  if (configured_max < 0) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_pass<T, MODE, RB, VAR>);
    if (e != cudaSuccess) return e;
    const int dyn = optin - (int)fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(k_pass<T, MODE, RB, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
    configured_max = dyn;
  }
  if ((int)smem > configured_max) return cudaErrorInvalidConfiguration;
  if (hp.rb != RB) return cudaErrorInvalidValue;
  const unsigned threads = 1u << (hp.k - RB);
  if (threads < 32 || threads > 256) return cudaErrorInvalidConfiguration;
  // a paired Pauli-sum pass runs one CTA per pair of tiles
  const size_t blocks = (size_t)rows << (hp.nfix - ((MODE == KM_HAM && hp.pair_fout) ? 1 : 0));
  if (blocks == 0) return cudaSuccess;
  if (blocks > 0x7fffffffull) return cudaErrorInvalidConfiguration;
  const unsigned chunks = (MODE == KM_HAM && a.hchunks > 1) ? (unsigned)a.hchunks : 1u;
  if (chunks > 65535u) return cudaErrorInvalidConfiguration;
  k_pass<T, MODE, RB, VAR><<<dim3((unsigned)blocks, chunks), threads, smem, s>>>(a, pa);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launch profiler: CUDA events on the launching stream around each launch
// ---------------------------------------------------------------------------
namespace {
struct ProfRec {
  int kind;
  double bytes;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;
thread_local int g_prof_kind = -1;
thread_local double g_prof_bytes = 0;
thread_local cudaEvent_t g_prof_a = nullptr;
}  // namespace

void prof_begin() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& r : g_prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_prof.clear();
  g_prof_on = true;
}
bool prof_enabled() { return g_prof_on; }
void prof_before(int kind, double bytes, cudaStream_t s) {
  if (!g_prof_on) return;
  g_prof_kind = kind;
  g_prof_bytes = bytes;
  cudaEventCreate(&g_prof_a);
  cudaEventRecord(g_prof_a, s);
}
void prof_after(cudaStream_t s) {
  if (!g_prof_on || !g_prof_a) return;
  cudaEvent_t b;
  cudaEventCreate(&b);
  cudaEventRecord(b, s);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof.push_back({g_prof_kind, g_prof_bytes, g_prof_a, b});
  g_prof_a = nullptr;
}
bool prof_end(int* launches, double* ms, double* bytes) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = false;
  for (int k = 0; k < PK_COUNT; ++k) {
    launches[k] = 0;
    ms[k] = 0;
    bytes[k] = 0;
  }
  bool ok = true;
  for (auto& r : g_prof) {
    float t = 0;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) ok = false;
    launches[r.kind]++;
    ms[r.kind] += t;
    bytes[r.kind] += r.bytes;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_prof.clear();
  return ok;
}

// Algorithmic HBM bytes of one pass launch: every amplitude of every state
// the pass reads or writes, once.
static double pass_bytes(int mode, bool dbl, const DevPass& hp, const KArgs& a, int rows) {
  const double amps = (double)rows * (double)(1ull << a.N) * (dbl ? 16.0 : 8.0);
  if (mode == KM_FWD) return amps * (((hp.flags & PF_INIT) && a.synth_init) ? 1.0 : 2.0);
  if (mode == KM_BWD) return amps * 4.0;
  double t = 1.0;  // psi read
  if ((hp.flags & PF_LAM_LOAD) && a.lam) t += 1.0;
  if ((hp.flags & PF_LAM_STORE) && a.lam && a.store_lambda) t += 1.0;
  return amps * t;
}

template <typename T, int MODE, int RB>
static cudaError_t launch_t(const KArgs& a, const PassArgs& pa, int rows, cudaStream_t s, size_t smem) {
  if constexpr (MODE == KM_HAM) {
    return launch_tf<T, MODE, RB, 0>(a, pa, rows, s, smem);
  } else {
    const DevPass& hp = pa.pass;
    const bool lean = hp.flags & PF_LEAN, full = hp.flags & PF_FULL, multi = hp.flags & PF_MULTI;
    if (full || (lean && multi)) return launch_tf<T, MODE, RB, 7>(a, pa, rows, s, smem);
    if (lean) return launch_tf<T, MODE, RB, 1>(a, pa, rows, s, smem);
    if (multi) return launch_tf<T, MODE, RB, 4>(a, pa, rows, s, smem);
    return launch_tf<T, MODE, RB, 0>(a, pa, rows, s, smem);
  }
}

cudaError_t launch_pass(int mode, bool dbl, const KArgs& a, const DevPass& hp, const DevStage* st0, int rows,
                        cudaStream_t s) {
  if (mode != KM_HAM && !st0) return cudaErrorInvalidValue;
  PassArgs pa;
  pa.pass = hp;
  if (st0) pa.st0 = *st0;
  else pa.st0 = DevStage{};
  const size_t smem = pass_smem_bytes(mode, dbl, hp);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  prof_before(mode == KM_FWD ? PK_FWD : mode == KM_BWD ? PK_BWD : PK_HAM, pass_bytes(mode, dbl, hp, a, rows), s);
  cudaError_t e;
  if (dbl) {
    if (mode == KM_FWD) e = launch_t<double, KM_FWD, kRBFwdC128>(a, pa, rows, s, smem);
    else if (mode == KM_BWD) e = launch_t<double, KM_BWD, kRBBwdC128>(a, pa, rows, s, smem);
    else e = launch_t<double, KM_HAM, kRBHam>(a, pa, rows, s, smem);
  } else {
    if (mode == KM_FWD) e = launch_t<float, KM_FWD, kRBFwd>(a, pa, rows, s, smem);
    else if (mode == KM_BWD) e = launch_t<float, KM_BWD, kRBBwd>(a, pa, rows, s, smem);
    else e = launch_t<float, KM_HAM, kRBHam>(a, pa, rows, s, smem);
  }
  prof_after(s);
  return e;
}

// ---------------------------------------------------------------------------
// Finalize: fixed-order sums (deterministic, independent of batch size)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_finalize(const double* epart, int ne, const double* gpart, int gslots,
                                                  int tiles_b, const int* csr_off, const int* csr_slots,
                                                  int n_params, double* e_out, double* g_out) {
  __shared__ double sh[256];
  const int row = blockIdx.x;
  const int tid = threadIdx.x;
  if (e_out) {
    double s = 0;
    for (int i = tid; i < ne; i += blockDim.x) s += epart[(size_t)row * ne + i];
    sh[tid] = s;
    __syncthreads();
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
      if (tid < w) sh[tid] += sh[tid + w];
      __syncthreads();
    }
    if (tid == 0) e_out[row] = sh[0];
  }
  if (g_out) {
    for (int p = tid; p < n_params; p += blockDim.x) {
      double g = 0;
      for (int c = csr_off[p]; c < csr_off[p + 1]; ++c) {
        const double* src = gpart + ((size_t)row * gslots + csr_slots[c]) * tiles_b;
        for (int t = 0; t < tiles_b; ++t) g += src[t];
      }
      g_out[(size_t)row * n_params + p] = g;
    }
  }
}

cudaError_t launch_finalize(const double* epart, int n_hpasses, int tiles_h, const double* gpart, int gslots,
                            int tiles_b, const int* csr_off, const int* csr_slots, int n_params, int rows,
                            double* e_out, double* g_out, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  prof_before(PK_FINALIZE, (double)rows * 8.0 * ((double)n_hpasses * tiles_h + (double)gslots * tiles_b), s);
  k_finalize<<<rows, 256, 0, s>>>(epart, n_hpasses * tiles_h, gpart, gslots, tiles_b, csr_off, csr_slots,
                                  n_params, e_out, g_out);
  prof_after(s);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Narrow circuits: user index x <-> internal index x << (N - n)
// ---------------------------------------------------------------------------
template <typename V>
__global__ void k_pad(const V* src, V* dst, int n_user, int N, int rows, int to_padded) {
  const int sh = N - n_user;
  const size_t per = (size_t)1 << (to_padded ? N : n_user);
  const size_t total = per * rows;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t r = i / per, y = i % per;
    if (to_padded) {
      V v;
      v.x = 0;
      v.y = 0;
      if ((y & ((1u << sh) - 1)) == 0) v = src[(r << n_user) + (y >> sh)];
      dst[i] = v;
    } else {
      dst[i] = src[(r << N) + (y << sh)];
    }
  }
}

cudaError_t launch_pad_states(bool dbl, const void* src, void* dst, int n_user, int N, int rows, bool to_padded,
                              cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  const int blocks = 592;
  prof_before(PK_PAD, (double)rows * (double)((1ull << N) + (1ull << n_user)) * (dbl ? 16.0 : 8.0), s);
  if (dbl)
    k_pad<double2><<<blocks, 256, 0, s>>>((const double2*)src, (double2*)dst, n_user, N, rows, to_padded);
  else
    k_pad<float2><<<blocks, 256, 0, s>>>((const float2*)src, (float2*)dst, n_user, N, rows, to_padded);
  prof_after(s);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Explicit-loop baseline term: one sweep per Pauli string
// ---------------------------------------------------------------------------
template <typename V>
__global__ void __launch_bounds__(256) k_plain_term(const V* psi, int N, uint32_t f, uint32_t sm, int ny, double w,
                                                    double* e_acc) {
  using S = decltype(V::x);
  __shared__ double sh[8];
  const int row = blockIdx.y;
  const V* st = psi + ((size_t)row << N);
  const uint32_t n = 1u << N;
  S acc = 0;
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    const V a = st[x];
    const V b = st[x ^ f];
    // conj(psi_{x^f}) * i^ny * (-1)^popc(x & sm) * psi_x
    S re = b.x * a.x + b.y * a.y, im = b.x * a.y - b.y * a.x;
    S r2 = ny == 0 ? re : ny == 1 ? -im : ny == 2 ? -re : im;
    if (__popc(x & sm) & 1) r2 = -r2;
    acc += r2;
  }
  const double ws = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = ws;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    atomicAdd(e_acc + row, w * s);
  }
}

cudaError_t launch_plain_term(bool dbl, const void* psi, int N, int rows, uint32_t f, uint32_t sm, int ny,
                              double w, double* e_acc, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  const unsigned bx = (unsigned)std::min<size_t>(((size_t)1 << N) / 256 > 0 ? ((size_t)1 << N) / 256 : 1, 1184);
  dim3 grid(bx, rows);
  prof_before(PK_PLAIN, (double)rows * (double)(1ull << N) * (dbl ? 16.0 : 8.0) * (f ? 2.0 : 1.0), s);
  if (dbl)
    k_plain_term<double2><<<grid, 256, 0, s>>>((const double2*)psi, N, f, sm, ny, w, e_acc);
  else
    k_plain_term<float2><<<grid, 256, 0, s>>>((const float2*)psi, N, f, sm, ny, w, e_acc);
  prof_after(s);
  return cudaGetLastError();
}

}  // namespace tcb
