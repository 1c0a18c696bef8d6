// Device core of the state-vector tile passes: amplitude maps, register-tile
// gate primitives, diagonal-group helpers and the gate-pass body.  Included
// by the library's kernels (sv_kernels.cu) and by the pass kernels generated
// per circuit at plan time (jit.cpp), which compile the same code with their
// program as compile-time constants.
#pragma once
#include "sv_args.h"

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
  // a static bound (a stage has at most 10 runs): with a compile-time stage
  // the loop unrolls and the record's fields fold
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    if (q >= st.n_runs) break;
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

// The same transposes addressed in bytes from the start of the dynamic shared
// memory: the thread's byte offset is XOR-walked (one XOR per access) and the
// buffer's offset `buf` (0 or a power of two above every tile offset) folds
// into the walk, so each access is a register plus the constant base.
template <int RB, typename V>
__device__ __forceinline__ void smem_write_x(const V (&A)[1 << RB], unsigned char* base, uint32_t buf,
                                             const Map<RB>& m) {
  uint32_t ro[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) ro[r] = swz<V>(m.rt[r]) * (uint32_t)sizeof(V);
  uint32_t off = buf ^ (swz<V>(m.t) * (uint32_t)sizeof(V));
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) {
    if (j) off ^= ro[low_bit(j)];
    *reinterpret_cast<V*>(base + off) = A[j ^ (j >> 1)];
  }
}
template <int RB, typename V>
__device__ __forceinline__ void smem_read_x(V (&A)[1 << RB], const unsigned char* base, uint32_t buf,
                                            const Map<RB>& m) {
  uint32_t ro[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) ro[r] = swz<V>(m.rt[r]) * (uint32_t)sizeof(V);
  uint32_t off = buf ^ (swz<V>(m.t) * (uint32_t)sizeof(V));
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) {
    if (j) off ^= ro[low_bit(j)];
    A[j ^ (j >> 1)] = *reinterpret_cast<const V*>(base + off);
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
// Quarter phase on register bit J: amplitudes with the bit set times i^s
// (s = +1: (x, y) -> (-y, x); s = -1: (x, y) -> (y, -x)).
template <int RB, int J, typename V, typename T>
__device__ __forceinline__ void g_sphase(V (&A)[1 << RB], T s) {
#pragma unroll
  for (int i = 0; i < (1 << RB); ++i)
    if (i & (1 << J)) A[i] = mk<V>(-s * A[i].y, s * A[i].x);
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
template <class Ents>
__device__ __forceinline__ uint64_t diag_col(const Ents& ents, const DevDiag& dg, int p) {
  const DevDiagEnt c = ents[dg.ent_off + p];
  return ((uint64_t)c.mask << 32) | c.d;
}
// term parities of index x for a packed group: XOR of the columns of x's set bits
template <class Ents>
__device__ __forceinline__ uint64_t diag_word(uint32_t x, const DevDiag& dg, const Ents& ents) {
  uint64_t w = 0;
  for (int p = 0; p < dg.n_ent; ++p)
    if ((x >> p) & 1u) w ^= diag_col(ents, dg, p);
  return w;
}

template <int RB, class Ents>
__device__ __forceinline__ void diag_counts_lin(int (&cnt)[1 << RB], const Map<RB>& m, const DevDiag& dg,
                                                const Ents& ents) {
  if (dg.packed) {
    // one word per amplitude, walked in Gray-code order over the register bits
    uint64_t w = diag_word(m.g, dg, ents);
    uint64_t wr[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) wr[r] = diag_col(ents, dg, __ffs((int)m.ro[r]) - 1);
#pragma unroll
    for (int j = 0; j < (1 << RB); ++j) {
      if (j) w ^= wr[low_bit(j)];
      cnt[j ^ (j >> 1)] = __popcll(w);
    }
    return;
  }
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
template <class Ents>
__device__ __forceinline__ int diag_count(uint32_t x, const DevDiag& dg, const Ents& ents) {
  if (dg.packed) return __popcll(diag_word(x, dg, ents));
  int c = 0;
  for (int e = 0; e < dg.n_ent; ++e) {
    const DevDiagEnt en = ents[dg.ent_off + e];
    const uint32_t v = en.d == 0 ? x : (dg.sign_mode ? (x & (x >> en.d)) : (x ^ (x >> en.d)));
    c += __popc(v & en.mask);
  }
  return c;
}


// ---------------------------------------------------------------------------
// Gate passes (forward / adjoint) over a pass program
// ---------------------------------------------------------------------------
// The program of a pass (its descriptor, register stages, instructions,
// diagonal groups and their entries) comes from a source:
//   RtSrc     the plan as the host planner wrote it, staged into shared memory
//             by the pass (the library's k_pass kernels);
//   CtSrc<P>  a generated program P whose members are compile-time constants
//             (pass kernels generated per circuit at plan time): every loop
//             over stages and instructions unrolls and every field folds.
// Both run this same function, so their arithmetic is the same.
template <int I>
struct IntC {
  static constexpr int value = I;
};
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(IntC<B>{});
    static_for<B + 1, E>(f);
  }
}

struct RtSrc {
  static constexpr bool kConst = false;
};
// FENCE: a compiler memory fence after every instruction, which keeps each
// instruction's table reads inside it (bounds register pressure the way the
// interpreter's instruction loop does)
template <class P, bool FENCE = false>
struct CtSrc {
  static constexpr bool kConst = true;
  static constexpr bool kFence = FENCE;
  using Prog = P;
};
// indexers over a generated program's constant arrays
template <class P>
struct CtStages {
  __device__ __forceinline__ constexpr DevStage operator[](int i) const { return P::stage(i); }
};
template <class P>
struct CtInstrs {
  __device__ __forceinline__ constexpr DevInstr operator[](int i) const { return P::instr(i); }
};
template <class P>
struct CtDiags {
  __device__ __forceinline__ constexpr DevDiag operator[](int i) const { return P::diag(i); }
};
template <class P>
struct CtDents {
  __device__ __forceinline__ constexpr DevDiagEnt operator[](int i) const { return P::dent(i); }
};

template <class Src>
struct SrcTypes {  // runtime plan: pointers into shared memory
  using Stages = const DevStage*;
  using Instrs = const DevInstr*;
  using Diags = const DevDiag*;
  using Dents = const DevDiagEnt*;
};
template <class P, bool F>
struct SrcTypes<CtSrc<P, F>> {
  using Stages = CtStages<P>;
  using Instrs = CtInstrs<P>;
  using Diags = CtDiags<P>;
  using Dents = CtDents<P>;
};

template <class Src>
__device__ __forceinline__ DevPass src_pass(const PassArgs& pa) {
  if constexpr (Src::kConst) return Src::Prog::pass();
  else return DevPass{};
}

// VAR selects the instruction set compiled into an instantiation of the
// library's kernels (smaller code and fewer live registers for simpler
// passes); bit flags over the rotation-layer core (RY, RY multi, their
// adjoint steps, single-entry ZZ/Z/S phase groups, quarter phases):
//   +1  lean: RX, H, X, noise outcomes, 2x2 matrices, CZ groups
//   +2  full: CNOT, 4x4 matrices
//   +4  multi-entry ZZ/Z phase groups (ZZ at several qubit distances)
template <typename T, int MODE, int RB, int VAR, class Src>
__device__ __forceinline__ void gate_pass(const KArgs& a, const PassArgs& pa) {
  constexpr bool FULL = (VAR & 2) != 0;
  constexpr bool LEAN = (VAR & 1) != 0;
  constexpr bool MULTI = (VAR & 4) != 0;
  using V = typename VT<T>::V;
  constexpr int R = 1 << RB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the pass descriptor: a kernel parameter (runtime plans; with its first
  // stage, so the first state loads need no dependent global reads) or a
  // compile-time constant
  const DevPass spc = src_pass<Src>(pa);
  const DevPass& sp = Src::kConst ? spc : pa.pass;

  const int k = sp.k;
  const uint32_t tid = threadIdx.x;
  const int nwarps = blockDim.x >> 5;
  const int warp = tid >> 5, lane = tid & 31;
  const int row = (int)(blockIdx.x >> sp.nfix);
  const uint32_t tile = blockIdx.x & ((1u << sp.nfix) - 1u);
  uint32_t base = 0;
#pragma unroll
  for (int q = 0; q < 32; ++q) {  // static bound: unrolls (and folds) for a compile-time pass
    if (q >= sp.n_fixruns) break;
    const DevRun u = sp.fixrun[q];
    base |= ((tile >> u.b) & ((1u << u.len) - 1u)) << u.p;
  }
  const size_t soff = (size_t)row << a.N;
  V* psi = (V*)a.psi + soff;
  V* lam = a.lam ? (V*)a.lam + soff : nullptr;

  // shared memory carve-up: tile(s) | table | (runtime plans: instructions |
  // stages | diag groups | entries) | reduction
  const int tsize = 1 << k;
  V* sm0 = (V*)smem_raw;
  V* tab = sm0 + (MODE == KM_BWD ? 2 * tsize : tsize);
  typename SrcTypes<Src>::Instrs ins{};
  typename SrcTypes<Src>::Stages sst{};
  typename SrcTypes<Src>::Diags dgs{};
  typename SrcTypes<Src>::Dents des{};
  double* red;
  if constexpr (Src::kConst) {
    red = (double*)(tab + ((sp.table_size + 1) & ~1));
  } else {
    DevInstr* ins_s = (DevInstr*)(tab + ((sp.table_size + 1) & ~1));
    DevStage* sst_s = (DevStage*)(ins_s + sp.n_instr);
    DevDiag* dgs_s = (DevDiag*)(sst_s + sp.n_stages);
    DevDiagEnt* des_s = (DevDiagEnt*)(dgs_s + sp.n_diag);
    red = (double*)(des_s + ((sp.n_dent + 1) & ~1));
    ins = ins_s;
    sst = sst_s;
    dgs = dgs_s;
    des = des_s;
  }

  V A[R];
  V L[R];

  {
    const V* trow = (const V*)a.tables + (size_t)row * a.table_stride + sp.table_off;
    for (int i = tid; i < sp.table_size; i += blockDim.x) tab[i] = trow[i];
    if constexpr (!Src::kConst) {
      for (int i = tid; i < sp.n_instr; i += blockDim.x) const_cast<DevInstr*>(ins)[i] = a.instrs[sp.instr_off + i];
      {
        const uint32_t* src = (const uint32_t*)(a.stages + sp.stage_off);
        uint32_t* dst = (uint32_t*)const_cast<DevStage*>(sst);
        const int words = sp.n_stages * (int)(sizeof(DevStage) / 4);
        for (int i = tid; i < words; i += blockDim.x) dst[i] = src[i];
      }
      for (int i = tid; i < sp.n_diag; i += blockDim.x) const_cast<DevDiag*>(dgs)[i] = a.diags[sp.diag_off + i];
      const DevDiagEnt* drow = a.dents + (size_t)row * a.dent_row_stride + sp.dent_off;
      for (int i = tid; i < sp.n_dent; i += blockDim.x) const_cast<DevDiagEnt*>(des)[i] = drow[i];
    }
    if (MODE == KM_BWD)
      for (int i = tid; i < sp.n_gslots * nwarps; i += blockDim.x) red[i] = 0.0;
  }
  // gradient partials: one per-thread accumulator per local slot (reduced
  // once at the end of the pass); slots beyond kLocalSlots reduce at once
  T gl[kLocalSlots];
  if (MODE == KM_BWD) {
#pragma unroll
    for (int g = 0; g < kLocalSlots; ++g) gl[g] = 0;
  }
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
  Map<RB> m = stage_map<RB>(Src::kConst ? sst[0] : pa.st0, tid, base);
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

  // one stage change: registers -> shared memory -> the next stage's registers
  auto transpose = [&](const DevStage& st) {
    const uint32_t lbuf = (uint32_t)tsize * (uint32_t)sizeof(V);  // sm1 - sm0 in bytes
    smem_write_x<RB>(A, smem_raw, 0u, m);
    if (MODE == KM_BWD) smem_write_x<RB>(L, smem_raw, lbuf, m);
    m = stage_map<RB>(st, tid, base);
    __syncthreads();
    smem_read_x<RB>(A, smem_raw, 0u, m);
    if (MODE == KM_BWD) smem_read_x<RB>(L, smem_raw, lbuf, m);
    __syncthreads();
  };
  // one instruction on the register tile
  auto exec = [&](const DevInstr in) {
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
        case IK_SPHASE: {
          const T sg = (T)in.gscale;
          const uint32_t rmask = (uint8_t)in.j0;
#pragma unroll
          for (int r = 0; r < RB; ++r) {
            if (!((rmask >> r) & 1u)) continue;
            TC_DISPATCH_J(RB, r, (g_sphase<RB, J>(A, sg)));
            if (MODE == KM_BWD) TC_DISPATCH_J(RB, r, (g_sphase<RB, J>(L, sg)));
          }
          // the thread's own bits: one phase i^e for all its amplitudes
          const int e = ((int)sg * __popc(m.g & (uint32_t)in.slot)) & 3;
          if (e) {
            const T cr = e == 2 ? (T)-1 : (T)0, ci = e == 1 ? (T)1 : (e == 3 ? (T)-1 : (T)0);
#pragma unroll
            for (int i = 0; i < R; ++i) {
              A[i] = mk<V>(cr * A[i].x - ci * A[i].y, cr * A[i].y + ci * A[i].x);
              if (MODE == KM_BWD) L[i] = mk<V>(cr * L[i].x - ci * L[i].y, cr * L[i].y + ci * L[i].x);
            }
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
      // the last instruction of its gradient slot in this pass: reduce the
      // slot now (the same sum as at the end of the pass, one reduction).  In
      // a compiled pass this ends the accumulator's register live range; the
      // interpreter keeps its accumulators in local memory and reduces at the end
      if (Src::kConst && MODE == KM_BWD && in.kind != IK_CNOT && in.jc == 1 && in.gslot >= 0 &&
          in.gslot < kLocalSlots) {
        T v = gl[in.gslot];
        gl[in.gslot] = 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[in.gslot * nwarps + warp] += (double)v;
      }
  };
  if constexpr (Src::kConst) {
    // a generated program: every stage and instruction a compile-time constant
    using Prog = typename Src::Prog;
    static_for<0, Prog::kStages>([&](auto S) {
      constexpr int s = decltype(S)::value;
      if constexpr (s > 0) transpose(Prog::stage(s));
      static_for<0, Prog::stage(s).n_instr>([&](auto Q) {
        constexpr int q = decltype(Q)::value;
        exec(Prog::instr(Prog::stage(s).instr_off + q));
        if constexpr (Src::kFence) asm volatile("" ::: "memory");
      });
    });
  } else {
#pragma unroll 1
    for (int s = 0; s < sp.n_stages; ++s) {
      const int n_instr = sst[s].n_instr, instr_off = sst[s].instr_off;
      if (s > 0) transpose(sst[s]);
#pragma unroll 1
      for (int q = 0; q < n_instr; ++q) exec(ins[instr_off + q]);
    }
  }
  const bool skip_psi = MODE == KM_BWD && (sp.flags & PF_SKIP_PSI);
  const bool skip_lam = MODE == KM_BWD && (sp.flags & PF_SKIP_LAM);
  if ((sc != (T)1 || sl != (T)0) && !(skip_psi && skip_lam)) {
    const T se = sc + sl;
    const V s2 = mk<V>(se, se);
#pragma unroll
    for (int i = 0; i < R; ++i) {
      A[i] = cmul_re(s2, A[i]);
      if (MODE == KM_BWD) L[i] = cmul_re(s2, L[i]);
    }
  }
  if (!skip_psi) store_regs<RB>(A, psi, m);
  if (MODE == KM_BWD) {
    if (!skip_lam) store_regs<RB>(L, lam, m);
#pragma unroll
    for (int g = 0; g < kLocalSlots; ++g) {
      if (g >= sp.n_gslots || (Src::kConst && (sp.flags & PF_GFLUSH))) break;
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

}  // namespace tcb
