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

#include "sv_core.cuh"
#include "sv_kernels.cuh"

namespace tcb {

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

// Mean and standard error (sample std, ddof = 1, over sqrt(n)) of n doubles,
// FP64, fixed-order reduction (one block); moments = 1: out = (n, mean, M2)
// with M2 the sum of squared deviations from the mean (one shard's share of a
// split estimate).
__global__ void __launch_bounds__(256) k_mean_stderr(const double* x, int n, double* out, int moments) {
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
    if (moments) {
      out[0] = n;
      out[1] = mean;
      out[2] = s2[0];
    } else {
      out[0] = mean;
      out[1] = n > 1 ? sqrt(s2[0] / (n - 1) / n) : 0.0;
    }
  }
}

cudaError_t launch_mean_stderr(const double* x, int n, double* out, cudaStream_t s, bool moments) {
  k_mean_stderr<<<1, 256, 0, s>>>(x, n, out, moments ? 1 : 0);
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

// The library's pass kernel: Pauli-sum passes here, gate passes through
// gate_pass over the runtime plan (sv_core.cuh).
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
      stage(hds, a.hdiag + (size_t)row * a.hdiag_row_stride + sp.hdiag_off, n_diag_here * (int)sizeof(DevHDiag));
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
        // it is walked in Gray-code order over the registers; the terms'
        // values h(x) are summed first and applied to the amplitude once
        T hsum[R];
  #pragma unroll
        for (int i = 0; i < R; ++i) hsum[i] = 0;
        for (int e = 0; e < n_diag_here; ++e) {
          const DevHDiag hd = hds[e];
          const T w = (T)hd.w;
          if (hd.pad == 1) {
            // packed ZZ terms: column words of the N positions follow
            const DevHDiag* cols = hds + e + 1;
            auto colw = [&](int p) { return ((uint64_t)cols[p].mask << 32) | cols[p].d; };
            uint64_t W = 0;
            for (int p = 0; p < a.N; ++p)
              if ((m.g >> p) & 1u) W ^= colw(p);
            uint64_t wr[RB];
  #pragma unroll
            for (int r = 0; r < RB; ++r) wr[r] = colw(__ffs((int)m.ro[r]) - 1);
  #pragma unroll
            for (int j = 0; j < R; ++j) {
              if (j) W ^= wr[low_bit(j)];
              const int i = j ^ (j >> 1);
              hsum[i] = fma(w, (T)(hd.cnt - 2 * __popcll(W)), hsum[i]);
            }
            e += a.N;
            continue;
          }
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
              hsum[i] += (__popc(v) & 1) ? -w : w;
            }
          } else {
  #pragma unroll
            for (int j = 0; j < R; ++j) {
              if (j) v ^= vr[low_bit(j)];
              const int i = j ^ (j >> 1);
              hsum[i] = fma(w, (T)(hd.cnt - 2 * __popc(v)), hsum[i]);
            }
          }
        }
        if (n_diag_here) {
          V e2 = mk<V>((T)0, (T)0);
  #pragma unroll
          for (int i = 0; i < R; ++i) {
            const V h2 = mk<V>(hsum[i], hsum[i]);
            L[i] = cfma2(h2, A[i], L[i]);
            e2 = cfma2(cmul_re(h2, A[i]), A[i], e2);
          }
          eacc = e2.x + e2.y;
        }
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
  if constexpr (MODE != KM_HAM) gate_pass<T, MODE, RB, VAR, RtSrc>(a, pa);
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
  if (mode == KM_BWD)
    return amps * (2.0 + ((hp.flags & PF_SKIP_PSI) ? 0.0 : 1.0) + ((hp.flags & PF_SKIP_LAM) ? 0.0 : 1.0));
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

cudaError_t launch_pass_specialised(cudaKernel_t kern, int mode, bool dbl, const KArgs& a, const DevPass& hp, int rows,
                                    cudaStream_t s) {
  const size_t v = dbl ? 16 : 8;
  const size_t tsize = (size_t)1 << hp.k;
  const unsigned threads = (unsigned)(tsize >> hp.rb);
  if (threads < 32 || threads > 256) return cudaErrorInvalidConfiguration;
  const size_t smem = tsize * v * (mode == KM_BWD ? 2 : 1) + (size_t)((hp.table_size + 1) & ~1) * v +
                      (mode == KM_BWD ? (size_t)hp.n_gslots * (threads / 32) * 8 : 0) + 16;
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const size_t blocks = (size_t)rows << hp.nfix;
  if (blocks == 0) return cudaSuccess;
  if (blocks > 0x7fffffffull) return cudaErrorInvalidConfiguration;
  PassArgs pa;
  pa.pass = hp;
  pa.st0 = DevStage{};
  void* args[] = {(void*)&a, (void*)&pa};
  prof_before(mode == KM_FWD ? PK_FWD : PK_BWD, pass_bytes(mode, dbl, hp, a, rows), s);
  e = cudaLaunchKernel((const void*)kern, dim3((unsigned)blocks), dim3(threads), args, smem, s);
  prof_after(s);
  return e;
}

// ---------------------------------------------------------------------------
// Finalize: fixed-order sums (deterministic, independent of batch size)
// ---------------------------------------------------------------------------
// One block per (row, output): output 0 is the row's energy (sum of the
// Pauli-sum passes' per-tile partials), output 1 + p the gradient of
// parameter p (sum over its slots' per-tile partials).  Every thread of the
// block sums a strided share; the order is fixed, so a row's result does not
// depend on the other rows.
__global__ void __launch_bounds__(512) k_finalize(const double* epart, int ne, const double* gpart, int gslots,
                                                  int tiles_b, const int* csr_off, const int* csr_slots,
                                                  int n_params, double* e_out, double* g_out, int accumulate) {
  __shared__ double sh[32];
  const int row = blockIdx.x;
  const int tid = threadIdx.x;
  for (int which = blockIdx.y; which <= n_params; which += gridDim.y) {
    double s = 0;
    if (which == 0) {
      if (!e_out) continue;
      for (int i = tid; i < ne; i += blockDim.x) s += epart[(size_t)row * ne + i];
    } else {
      if (!g_out) break;
      const int p = which - 1;
      // four independent partial sums keep several loads in flight per thread
      double s4[4] = {0, 0, 0, 0};
      for (int c = csr_off[p]; c < csr_off[p + 1]; ++c) {
        const double* src = gpart + ((size_t)row * gslots + csr_slots[c]) * tiles_b;
        int t = tid;
        for (; t + 3 * (int)blockDim.x < tiles_b; t += 4 * blockDim.x) {
#pragma unroll
          for (int u = 0; u < 4; ++u) s4[u] += src[t + u * blockDim.x];
        }
        for (; t < tiles_b; t += blockDim.x) s4[0] += src[t];
      }
      s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((tid & 31) == 0) sh[tid >> 5] = s;
    __syncthreads();
    if (tid < 32) {
      s = tid < (int)(blockDim.x >> 5) ? sh[tid] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (tid == 0) {
        if (which == 0) e_out[row] = s;
        else if (accumulate) g_out[(size_t)row * n_params + which - 1] += s;
        else g_out[(size_t)row * n_params + which - 1] = s;
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_finalize(const double* epart, int n_hpasses, int tiles_h, const double* gpart, int gslots,
                            int tiles_b, const int* csr_off, const int* csr_slots, int n_params, int rows,
                            double* e_out, double* g_out, cudaStream_t s, bool accumulate) {
  if (rows <= 0) return cudaSuccess;
  prof_before(PK_FINALIZE, (double)rows * 8.0 * ((double)n_hpasses * tiles_h + (double)gslots * tiles_b), s);
  const unsigned outs = (unsigned)std::min(1 + (g_out ? n_params : 0), 65535);
  k_finalize<<<dim3((unsigned)rows, outs), 512, 0, s>>>(epart, n_hpasses * tiles_h, gpart, gslots, tiles_b, csr_off,
                                                        csr_slots, n_params, e_out, g_out, accumulate ? 1 : 0);
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
