// Quantum geometric tensor of a parameterised circuit (Section "Quantum
// Fisher Information"):
//   G_ij = <d_i psi|d_j psi> - <d_i psi|psi><psi|d_j psi>,  QFI = 4 Re G.
//
// Every parameterised gate is exp(-i a G / 2) with G^2 = I, a = s theta_p, and
// d/da exp(-i a G / 2) = (-i/2) G exp(-i a G / 2) = (1/2) exp(-i (a + pi) G / 2).
// So d|psi>/d theta_p = sum over the occurrences k of p of c_k |psi_k>, with
// c_k = s_k / 2 and |psi_k> the circuit's state with occurrence k's angle
// advanced by pi, which is -i times the state with the Pauli generator G_k
// inserted right after the gate; the phase cancels in G, so the engine uses
// the insertion states chi_k.  An insertion moves right past every later gate
// that commutes with G_k (disjoint qubits; diagonal gates for Z-type G; RX
// after X, RY after Y; a CNOT's control for Z, its target for X), and the
// occurrences are grouped by a common insertion point (fewest points
// stabbing the intervals).  Per group: the segment of the circuit up to the
// point advances each row's prefix state phi, the group's states are G_k phi,
// and the suffix after the point runs on them, all with the circuit's own
// parameters (so diagonal gates sharing an angle stay grouped).  The last
// slot holds the unshifted state.  A Gram kernel forms M_kl = <chi_k|chi_l>,
// and a fold kernel sums G_ij = sum_{k in i, l in j} c_k c_l M_kl - u_i v_j,
// u_i = sum_k c_k M_{k,S-1}, v_j = sum_l c_l M_{S-1,l}.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "engine.h"
#include "tcgen05.cuh"

namespace tcb {

namespace {

constexpr int kGramTile = 64;    // states per tile side
constexpr int kGramX = 16;       // amplitudes per shared-memory stage
constexpr int kGramChunk = 2048; // amplitudes summed in the state's precision per chunk partial

template <typename R>
struct Cplx;
template <>
struct Cplx<float> {
  using T = float2;
};
template <>
struct Cplx<double> {
  using T = double2;
};

// out[(t R + r)][p] = theta[r][p] for t < count: the row's parameters for
// each of its states in a group
__global__ void k_qgt_rep(const double* __restrict__ theta, int P, int R, int count, double* __restrict__ out) {
  const int64_t total = (int64_t)count * R * P;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e % P);
    const int r = (int)((e / P) % R);
    out[e] = theta[(size_t)r * P + p];
  }
}

// out[(t R + r)][x] = (G_t phi_r)[x] for the group's slots t < count (the
// last slot of the last group takes phi itself: pauli entry = 0, 0, 0).
// G = (-i)^{#Y} (-1)^{popc(x & sign)} applied to phi[x ^ flip] (qubit q is
// bit n - 1 - q; X and Y flip, Z and Y give the sign).
template <typename C2>
__global__ void k_qgt_pauli(const C2* __restrict__ phi, int R, int64_t L, const uint32_t* __restrict__ pauli,
                            int count, C2* __restrict__ out) {
  const int64_t total = (int64_t)count * R * L;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = e % L;
    const int64_t tr = e / L;
    const int r = (int)(tr % R);
    const int t = (int)(tr / R);
    const uint32_t flip = pauli[3 * t], sign = pauli[3 * t + 1], ny = pauli[3 * t + 2];
    C2 v = phi[(size_t)r * L + (x ^ (int64_t)flip)];
    if (__popc((uint32_t)x & sign) & 1) {
      v.x = -v.x;
      v.y = -v.y;
    }
    switch (ny & 3) {  // multiply by (-i)^ny
      case 1: { const auto re = v.x; v.x = v.y; v.y = -re; } break;
      case 2: v.x = -v.x; v.y = -v.y; break;
      case 3: { const auto re = v.x; v.x = -v.y; v.y = re; } break;
      default: break;
    }
    out[e] = v;
  }
}

// M[r][k][l] += sum_x conj(psi_{r,k}[x]) psi_{r,l}[x] over one amplitude
// chunk, for the tile pair (kt <= lt) of blockIdx.x; 4 x 4 outputs a thread.
// The Gram partials of the amplitude chunks, summed in chunk order.
__global__ void __launch_bounds__(256) k_gram_sum(const double* __restrict__ Mp, int nchunk, size_t per,
                                                  double* __restrict__ M) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < per; i += (size_t)gridDim.x * blockDim.x) {
    double s = 0;
    for (int y = 0; y < nchunk; ++y) s += Mp[(size_t)y * per + i];
    M[i] = s;
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_gram(const typename Cplx<R>::T* __restrict__ states, int S, int64_t L,
                                              int64_t kstride, int ntile, double* __restrict__ M) {
  using C2 = typename Cplx<R>::T;
  __shared__ C2 As[kGramX][kGramTile + 1];
  __shared__ C2 Bs[kGramX][kGramTile + 1];
  // tile pair from the upper-triangle index
  int pair = blockIdx.x, kt = 0;
  while (pair >= ntile - kt) {
    pair -= ntile - kt;
    ++kt;
  }
  const int lt = kt + pair;
  const int r = blockIdx.z;
  const int64_t x0 = (int64_t)blockIdx.y * kGramChunk;
  const int64_t x1 = x0 + kGramChunk < L ? x0 + kGramChunk : L;
  const C2* base = states + (size_t)r * L;  // state slot k of row r at base + k kstride
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  R ar[4][4], ai[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) ar[i][j] = ai[i][j] = R(0);
  for (int64_t xs = x0; xs < x1; xs += kGramX) {
#pragma unroll
    for (int q = 0; q < kGramTile * kGramX / 256; ++q) {
      const int e = tid + 256 * q;
      const int xx = e % kGramX, kk = e / kGramX;
      const int64_t x = xs + xx;
      const int ka = kt * kGramTile + kk, kb = lt * kGramTile + kk;
      C2 z;
      z.x = R(0);
      z.y = R(0);
      As[xx][kk] = (ka < S && x < x1) ? base[(size_t)ka * kstride + x] : z;
      Bs[xx][kk] = (kb < S && x < x1) ? base[(size_t)kb * kstride + x] : z;
    }
    __syncthreads();
#pragma unroll 4
    for (int xx = 0; xx < kGramX; ++xx) {
      C2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[xx][ty * 4 + i];
        b[i] = Bs[xx][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {  // conj(a) b
          ar[i][j] = fma(a[i].x, b[j].x, fma(a[i].y, b[j].y, ar[i][j]));
          ai[i][j] = fma(a[i].x, b[j].y, fma(-a[i].y, b[j].x, ai[i][j]));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = kt * kGramTile + ty * 4 + i, l = lt * kGramTile + tx * 4 + j;
      if (k < S && l < S) {  // this chunk's partial (summed over chunks in fixed order later)
        double* m = M + ((((size_t)blockIdx.y * gridDim.z + r) * S + k) * S + l) * 2;
        m[0] = (double)ar[i][j];
        m[1] = (double)ai[i][j];
      }
    }
}

// ---------------------------------------------------------------------------
// Tensor-core Gram for complex64 states (tcgen05, kind::tf32, cta_group::1).
// With the state rows interleaved as real vectors a = (re_0, im_0, re_1, ...),
// Re <psi_k|psi_l> = a_k . a_l and Im <psi_k|psi_l> = a_k . b_l with
// b = (im_0, -re_0, im_1, -re_1, ...): two real GEMMs D = A B^T over K = 2L.
// Operands split x = hi + lo, hi = tf32(x): A B = A_hi B_hi + A_hi B_lo +
// A_lo B_hi.  The tensor core's FP32 accumulation is not round-to-nearest
// (its error grows with the chain length: measured 3e-3 on G over 4096
// amplitudes, 3e-5 over 64), so each stage's MMAs start a fresh TMEM
// accumulator and every thread adds its 64 accumulator values into FP32
// registers (round-to-nearest) after the stage; per-chunk FP64 partials combine the
// CTAs.  One CTA: 128 x 128 outputs (state rows k of tile kt by rows l of
// tile lt), Re and Im in TMEM columns [0, 128) and [128, 256), over kTcChunk
// amplitudes.  The raw amplitudes of stage s + 1 (16 per row of the 256 rows)
// are copied global -> shared with cp.async while stage s is converted and
// multiplied.  Per stage all threads convert the raw amplitudes into the
// operand tiles (hi and lo of A, B1 = a, B2 = b) in the K-major no-swizzle
// layout (8-row x 16-byte core matrices, K-adjacent core matrices kTcLBO
// bytes apart, 8-row groups kTcSBO bytes apart), one thread issues the 24
// MMAs and commits them to an mbarrier that every thread waits on (bounded).
constexpr int kTcThreads = 512;
constexpr int kTcTile = 128;                      // rows per side = TMEM lanes
constexpr int kTcKA = 16;                         // amplitudes per stage
constexpr int kTcK = 2 * kTcKA;                   // TF32 elements per stage
constexpr int kTcLBO = 128;                       // bytes between K-adjacent core matrices
constexpr int kTcSBO = (kTcK / 4) * 128;          // bytes between 8-row groups
constexpr int kTcTileBytes = kTcTile * kTcK * 4;  // one operand tile (16 KiB)
constexpr int kTcRawBytes = 2 * kTcTile * kTcKA * 8;  // one stage's raw amplitudes (32 KiB)
constexpr int kTcSetBytes = 6 * kTcTileBytes;            // one stage's operand tiles (96 KiB)
constexpr int kTcSmem = 2 * kTcSetBytes + kTcRawBytes;   // two tile sets + the raw stage (224 KiB)
constexpr int kTcChunk = 4096;                    // amplitudes per CTA
constexpr int kTcCols = 512;                      // TMEM: two accumulators of Re then Im columns
constexpr long long kTcSpin = 1ll << 20;          // bounded mbarrier waits

constexpr uint32_t kTcIdesc = tc_idesc(kTcFmtTF32, kTcTile, kTcTile);

__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr) { return tc_smem_desc(saddr, kTcLBO, kTcSBO); }
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  tc_mma_tf32(d, a, b, kTcIdesc, acc);
}
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) { return mbar_wait(bar, parity, kTcSpin); }

// skip_mma (tests only): issue no MMA and no commit, so the first completion
// wait has nothing to wait for and runs out: the bounded-wait path end to end.
__global__ void __launch_bounds__(kTcThreads, 1) k_gram_tc(const float2* __restrict__ states, int S, int64_t L,
                                                           int64_t kstride, int ntile, double* __restrict__ M,
                                                           int* __restrict__ err, int skip_mma) {
  extern __shared__ __align__(1024) uint8_t tc_smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  int pair = blockIdx.x, kt = 0;
  while (pair >= ntile - kt) {
    pair -= ntile - kt;
    ++kt;
  }
  const int lt = kt + pair;
  const int r = blockIdx.z;
  const int64_t x0 = (int64_t)blockIdx.y * kTcChunk;
  const int64_t x1 = x0 + kTcChunk < L ? x0 + kTcChunk : L;
  const int nst = (int)((x1 - x0 + kTcKA - 1) / kTcKA);
  const float2* base = states + (size_t)r * L;  // state slot k of row r at base + k kstride
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // accumulator share: TMEM lanes 32 (warp % 4).. (rows k), 64 columns
  // starting at 64 (warp / 4): Re columns [0, 128), then Im
  const int lg = warp & 3, part = warp >> 2;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(tc_smem);
  const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&mbar[0]);
  const uint32_t bar1 = (uint32_t)__cvta_generic_to_shared(&mbar[1]);
  if (warp == 0) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tacc = tmem_base;
  const uint32_t tmine = ((uint32_t)(32 * lg) << 16) + (uint32_t)(64 * part);
  float acc[64];
#pragma unroll
  for (int j = 0; j < 64; ++j) acc[j] = 0.f;
  uint32_t parity0 = 0, parity1 = 0;
  bool pending0 = false, pending1 = false;  // a commit not yet waited for
  bool ok = true;
  // raw stage layout: [operand][row][8 amplitude pairs], pair p of a row stored
  // at slot p ^ (row % 8) (so both the copy mapping below, row-major for
  // coalesced global reads, and the conversion mapping, rows fastest, hit
  // distinct shared-memory banks)
  const uint32_t raw0 = sbase + 2 * kTcSetBytes;
  auto prefetch = [&](int64_t xs) {
#pragma unroll
    for (int q = 0; q < 1024 / kTcThreads; ++q) {
      const int e = tid + kTcThreads * q;
      const int row = e >> 3, c4 = e & 7;
      const int64_t x = xs + 2 * c4;
      const int ka = kt * kTcTile + row, kb = lt * kTcTile + row;
      const uint32_t d = raw0 + (uint32_t)(row * (kTcKA * 8) + ((c4 ^ (row & 7)) * 16));
      const bool va = ka < S && x < x1, vb = kb < S && x < x1;
      cp_async16(d, va ? (const void*)(base + (size_t)ka * kstride + x) : (const void*)base, va);
      cp_async16(d + kTcRawBytes / 2, vb ? (const void*)(base + (size_t)kb * kstride + x) : (const void*)base, vb);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // add the accumulator of stage set `set` into the registers once its MMAs completed
  auto drain = [&](int set) -> bool {
    const bool done = set ? tc_wait(bar1, parity1) : tc_wait(bar0, parity0);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!done) return false;
    if (set) {
      parity1 ^= 1u;
      pending1 = false;
    } else {
      parity0 ^= 1u;
      pending0 = false;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t v[32];
      tmem_ld32(tacc + (uint32_t)(set * 2 * kTcTile) + tmine + 32 * h, v);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[32 * h + j] += __uint_as_float(v[j]);
    }
    return true;
  };
  prefetch(x0);
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  int issued = 0;  // stages whose MMAs were committed
  for (int st = 0; st < nst && ok; ++st) {
    const int set = st & 1;
    uint8_t* tiles = tc_smem + set * kTcSetBytes;
    // ---- convert the raw amplitudes into this stage's operand tiles (rows
    // fastest: a warp's 16-byte tile stores cover the 8 row slots of a core matrix)
#pragma unroll
    for (int q = 0; q < 1024 / kTcThreads; ++q) {
      const int e = tid + kTcThreads * q;  // 0..1023
      const int row = e & (kTcTile - 1), c4 = e >> 7;
      const uint32_t off = (uint32_t)((row >> 3) * kTcSBO + c4 * kTcLBO + (row & 7) * 16);
      const uint8_t* rp = tc_smem + 2 * kTcSetBytes + row * (kTcKA * 8) + ((c4 ^ (row & 7)) * 16);
      const float4 va = *reinterpret_cast<const float4*>(rp);
      const float4 vb = *reinterpret_cast<const float4*>(rp + kTcRawBytes / 2);
      const float4 ah = make_float4(tf32_rna(va.x), tf32_rna(va.y), tf32_rna(va.z), tf32_rna(va.w));
      const float4 al = make_float4(va.x - ah.x, va.y - ah.y, va.z - ah.z, va.w - ah.w);
      const float4 bh = make_float4(tf32_rna(vb.x), tf32_rna(vb.y), tf32_rna(vb.z), tf32_rna(vb.w));
      const float4 bl = make_float4(vb.x - bh.x, vb.y - bh.y, vb.z - bh.z, vb.w - bh.w);
      *reinterpret_cast<float4*>(tiles + 0 * kTcTileBytes + off) = ah;
      *reinterpret_cast<float4*>(tiles + 1 * kTcTileBytes + off) = al;
      *reinterpret_cast<float4*>(tiles + 2 * kTcTileBytes + off) = bh;
      *reinterpret_cast<float4*>(tiles + 3 * kTcTileBytes + off) = bl;
      // b = (im, -re) per amplitude; rounding to TF32 commutes with this
      *reinterpret_cast<float4*>(tiles + 4 * kTcTileBytes + off) = make_float4(bh.y, -bh.x, bh.w, -bh.z);
      *reinterpret_cast<float4*>(tiles + 5 * kTcTileBytes + off) = make_float4(bl.y, -bl.x, bl.w, -bl.z);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // tiles complete; the raw stage is free
    if (st + 1 < nst) prefetch(x0 + (int64_t)(st + 1) * kTcKA);
    if (tid == 0 && !skip_mma) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t tb = sbase + (uint32_t)(set * kTcSetBytes);
      const uint32_t dre = tacc + (uint32_t)(set * 2 * kTcTile), dim = dre + kTcTile;
#pragma unroll
      for (int ks = 0; ks < kTcK / 8; ++ks) {  // 8 TF32 = two core matrices along K per MMA
        const uint32_t o = (uint32_t)(ks * 2 * kTcLBO);
        const uint64_t ah = tc_sdesc(tb + 0 * kTcTileBytes + o), al = tc_sdesc(tb + 1 * kTcTileBytes + o);
        const uint64_t bh = tc_sdesc(tb + 2 * kTcTileBytes + o), bl = tc_sdesc(tb + 3 * kTcTileBytes + o);
        const uint64_t ch = tc_sdesc(tb + 4 * kTcTileBytes + o), cl = tc_sdesc(tb + 5 * kTcTileBytes + o);
        const uint32_t first = ks == 0 ? 0u : 1u;  // a fresh accumulator every stage
        tc_mma(dre, ah, bh, first);
        tc_mma(dre, ah, bl, 1u);
        tc_mma(dre, al, bh, 1u);
        tc_mma(dim, ah, ch, first);
        tc_mma(dim, ah, cl, 1u);
        tc_mma(dim, al, ch, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       set ? bar1 : bar0)
                   : "memory");
    }
    ++issued;
    if (set) pending1 = true; else pending0 = true;
    // the previous stage's accumulator (its MMAs overlapped this stage's conversion)
    if (st > 0) ok = drain(set ^ 1);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    // TMEM reads done before that accumulator is reused; next raw stage
    // visible.  A timeout seen by any thread stops the whole CTA.
    ok = __syncthreads_and(ok) != 0;
  }
  if (ok && issued > 0) ok = drain((issued - 1) & 1);
  ok = __syncthreads_and(ok) != 0;
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    // let any committed MMAs finish (bounded) before TMEM is freed
    if (pending0) tc_wait(bar0, parity0);
    if (pending1) tc_wait(bar1, parity1);
  } else {
    const int k = kt * kTcTile + 32 * lg + lane;
    const int comp = part >> 1, l0 = lt * kTcTile + 64 * (part & 1);
    if (k < S) {
#pragma unroll
      for (int j = 0; j < 64; ++j)
        if (l0 + j < S) M[((((size_t)blockIdx.y * gridDim.z + r) * S + k) * S + l0 + j) * 2 + comp] = (double)acc[j];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tacc), "r"(kTcCols));
}

// M(k, l) from the computed triangle of tiles (tile = rows per tile side):
// M(l, k) = conj(M(k, l))
__device__ __forceinline__ double2 gram_at(const double* Mr, int S, int tile, int k, int l) {
  if (k / tile <= l / tile) return make_double2(Mr[((size_t)k * S + l) * 2], Mr[((size_t)k * S + l) * 2 + 1]);
  return make_double2(Mr[((size_t)l * S + k) * 2], -Mr[((size_t)l * S + k) * 2 + 1]);
}

__global__ void k_qgt_fold(const double* __restrict__ M, int S, int tile, const int* __restrict__ off,
                           const int* __restrict__ occ, const double* __restrict__ occ_c, int P, int rows,
                           double* __restrict__ out) {
  const int64_t total = (int64_t)rows * P * P;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % P);
    const int i = (int)((e / P) % P);
    const int64_t r = e / ((int64_t)P * P);
    const double* Mr = M + (size_t)r * S * S * 2;
    const int last = S - 1;
    double gr = 0, gi = 0, ur = 0, ui = 0, vr = 0, vi = 0;
    for (int a = off[i]; a < off[i + 1]; ++a) {
      const int k = occ[a];
      const double ck = occ_c[k];
      const double2 mk = gram_at(Mr, S, tile, k, last);  // <psi_k|psi>
      ur += ck * mk.x;
      ui += ck * mk.y;
      for (int b = off[j]; b < off[j + 1]; ++b) {
        const int l = occ[b];
        const double2 m = gram_at(Mr, S, tile, k, l);
        gr += ck * occ_c[l] * m.x;
        gi += ck * occ_c[l] * m.y;
      }
    }
    for (int b = off[j]; b < off[j + 1]; ++b) {
      const int l = occ[b];
      const double2 m = gram_at(Mr, S, tile, last, l);  // <psi|psi_l>
      vr += occ_c[l] * m.x;
      vi += occ_c[l] * m.y;
    }
    out[e * 2] = gr - (ur * vr - ui * vi);
    out[e * 2 + 1] = gi - (ur * vi + ui * vr);
  }
}

// Natural gradient: x = (4 Re G + eps I)^-1 grad per row.  One CTA per row:
// the matrix in shared memory (FP64), Cholesky A = L L^T in place on the lower
// triangle (column by column: pivot, scale the column, update the trailing
// lower triangle), then L y = grad and L^T x = y by one warp with shuffle-
// reduced dot products.  A pivot that is not positive marks the row bad
// (status flag) and its output NaN.
constexpr int kNgMaxP = 128;
__global__ void __launch_bounds__(256) k_natgrad(const double* __restrict__ qgt, const double* __restrict__ grad,
                                                 int P, double eps, double* __restrict__ out) {
  extern __shared__ double ng[];
  double* A = ng;          // P x P, row-major
  double* y = ng + P * P;  // P
  __shared__ int bad;
  const int r = blockIdx.x, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  const double* Gr = qgt + (size_t)r * P * P * 2;
  for (int e = tid; e < P * P; e += nt) A[e] = 4.0 * Gr[2 * e] + ((e / P) == (e % P) ? eps : 0.0);
  for (int i = tid; i < P; i += nt) y[i] = grad[(size_t)r * P + i];
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < P; ++j) {
    if (tid == 0) {
      const double d = A[j * P + j];
      if (!(d > 0.0)) bad = 1;
      A[j * P + j] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double djj = A[j * P + j];
    for (int i = j + 1 + tid; i < P; i += nt) A[i * P + j] /= djj;
    __syncthreads();
    const int m = P - j - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int i = j + 1 + e / m, k = j + 1 + e % m;
      if (k <= i) A[i * P + k] -= A[i * P + j] * A[k * P + j];
    }
    __syncthreads();
  }
  if (tid < 32) {
    for (int i = 0; i < P; ++i) {  // L y = grad
      double sdot = 0.0;
      for (int k = lane; k < i; k += 32) sdot += A[i * P + k] * y[k];
      for (int o = 16; o > 0; o >>= 1) sdot += __shfl_xor_sync(0xffffffffu, sdot, o);
      if (lane == 0) y[i] = (y[i] - sdot) / A[i * P + i];
      __syncwarp();
    }
    for (int i = P - 1; i >= 0; --i) {  // L^T x = y
      double sdot = 0.0;
      for (int k = i + 1 + lane; k < P; k += 32) sdot += A[k * P + i] * y[k];
      for (int o = 16; o > 0; o >>= 1) sdot += __shfl_xor_sync(0xffffffffu, sdot, o);
      if (lane == 0) y[i] = (y[i] - sdot) / A[i * P + i];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = tid; i < P; i += nt) out[(size_t)r * P + i] = bad ? __longlong_as_double(0x7ff8000000000000ll) : y[i];
}

}  // namespace

}  // namespace tcb

using namespace tcb;

namespace {

bool diag_op(const tc_op& o, const std::vector<double>& pool) {
  if (o.kind == TC_OP_RZ || o.kind == TC_OP_RZZ || o.kind == TC_OP_CZ) return true;
  if (o.kind != TC_OP_U1 && o.kind != TC_OP_U2) return false;
  const int d = o.kind == TC_OP_U1 ? 2 : 4;
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c)
      if (r != c && (pool[2 * ((size_t)o.mat + r * d + c)] != 0.0 || pool[2 * ((size_t)o.mat + r * d + c) + 1] != 0.0))
        return false;
  return true;
}

bool two_qubit(const tc_op& o) {
  return o.kind == TC_OP_RZZ || o.kind == TC_OP_CNOT || o.kind == TC_OP_CZ || o.kind == TC_OP_U2;
}

// Does op o commute with the generator (Pauli code on qubits g0 and g1, g1 = -1 if none)?
bool commutes(const tc_op& o, int code, int g0, int g1, const std::vector<double>& pool) {
  const int a = o.q0, b = two_qubit(o) ? o.q1 : -1;
  auto on = [&](int q) { return q >= 0 && (q == g0 || q == g1); };
  if (!on(a) && !on(b)) return true;  // disjoint qubits
  if (code == 3 && diag_op(o, pool)) return true;
  if (g1 < 0) {  // one-qubit generator on g0
    if (code == 1 && b < 0 && (o.kind == TC_OP_RX || o.kind == TC_OP_X)) return true;
    if (code == 2 && b < 0 && o.kind == TC_OP_RY) return true;
    if (o.kind == TC_OP_CNOT && ((code == 3 && g0 == a) || (code == 1 && g0 == b))) return true;
  }
  return false;
}

tc_status qgt_prepare(tc_circuit* c) {
  if (c->qgt_ready) return TC_OK;
  const std::vector<tc_op>& ops = c->ops_in;
  const int n_ops = (int)ops.size();
  struct Occ {
    int op, param, lo, hi;  // insertion point interval [lo, hi]
    double chalf;
    uint32_t flip, sign, ny;
  };
  std::vector<Occ> occ;
  for (int i = 0; i < n_ops; ++i) {
    const tc_op& o = ops[i];
    if (o.kind == TC_OP_PAULI_NOISE || o.kind == TC_OP_RSEL)
      return fail(TC_E_UNSUPPORTED, "geometric tensor of circuits with noise or random-axis rotations");
    const bool rot = o.kind == TC_OP_RX || o.kind == TC_OP_RY || o.kind == TC_OP_RZ || o.kind == TC_OP_RZZ;
    if (o.param < 0 || !rot) continue;
    const int code = o.kind == TC_OP_RX ? 1 : o.kind == TC_OP_RY ? 2 : 3;
    const int g1 = o.kind == TC_OP_RZZ ? o.q1 : -1;
    int j = i + 1;
    while (j < n_ops && commutes(ops[j], code, o.q0, g1, c->pool)) ++j;
    Occ k{};
    k.op = i;
    k.param = o.param;
    k.lo = i + 1;
    k.hi = j;
    k.chalf = 0.5 * o.scale;
    const uint32_t m0 = 1u << (c->n - 1 - o.q0), m1 = g1 >= 0 ? 1u << (c->n - 1 - g1) : 0u;
    k.flip = code == 3 ? 0u : m0;
    k.sign = code == 1 ? 0u : (m0 | m1);
    k.ny = code == 2 ? 1u : 0u;
    occ.push_back(k);
  }
  // fewest insertion points: greedy by interval end
  std::vector<int> order(occ.size());
  for (size_t i = 0; i < occ.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return occ[x].hi < occ[y].hi; });
  std::vector<int> point_of(occ.size(), -1);
  std::vector<int> points;
  for (int k : order) {
    if (point_of[k] >= 0) continue;
    const int p = occ[k].hi;
    points.push_back(p);
    for (size_t m = 0; m < occ.size(); ++m)
      if (point_of[m] < 0 && occ[m].lo <= p && occ[m].hi >= p) point_of[m] = p;
  }
  std::sort(points.begin(), points.end());
  // slots in point order
  std::vector<int> slot_occ;
  std::vector<tc_circuit::QgtGroup> groups;
  int prev = 0;
  auto make = [&](int from, int to, tc_circuit** out) -> tc_status {
    *out = nullptr;
    if (to <= from) return TC_OK;
    return tc_circuit_create(c->n, c->dtype, c->init, ops.data() + from, to - from, c->n_params,
                             c->pool.empty() ? nullptr : c->pool.data(), (int)(c->pool.size() / 2), &c->opt, out);
  };
  tc_status st = TC_OK;
  for (int p : points) {
    tc_circuit::QgtGroup g;
    g.point = p;
    g.first = (int)slot_occ.size();
    for (size_t m = 0; m < occ.size(); ++m)
      if (point_of[m] == p) slot_occ.push_back((int)m);
    g.count = (int)slot_occ.size() - g.first;
    if ((st = make(prev, p, &g.seg)) != TC_OK || (st = make(p, n_ops, &g.suffix)) != TC_OK) {
      delete g.seg;
      delete g.suffix;
      break;
    }
    groups.push_back(g);
    prev = p;
  }
  if (st != TC_OK) {
    for (auto& g : groups) {
      delete g.seg;
      delete g.suffix;
    }
    return st;
  }
  const int Pp = (int)slot_occ.size();
  std::vector<int> occ_param(std::max(Pp, 1), 0), off(c->n_params + 1, 0), list(std::max(Pp, 1), 0);
  std::vector<double> occ_c(std::max(Pp, 1), 0.0);
  std::vector<uint32_t> pauli(3 * (size_t)(Pp + 1), 0u);  // + the unshifted slot (identity)
  for (int t = 0; t < Pp; ++t) {
    const Occ& k = occ[slot_occ[t]];
    occ_param[t] = k.param;
    occ_c[t] = k.chalf;
    pauli[3 * t] = k.flip;
    pauli[3 * t + 1] = k.sign;
    pauli[3 * t + 2] = k.ny;
    off[k.param + 1]++;
  }
  for (int p = 0; p < c->n_params; ++p) off[p + 1] += off[p];
  {
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (int t = 0; t < Pp; ++t) list[fill[occ_param[t]]++] = t;
  }
  cudaError_t e;
  if ((e = dev_upload(occ_param, &c->d_qgt_occ_param)) != cudaSuccess ||
      (e = dev_upload(occ_c, &c->d_qgt_occ_c)) != cudaSuccess || (e = dev_upload(off, &c->d_qgt_off)) != cudaSuccess ||
      (e = dev_upload(list, &c->d_qgt_occ)) != cudaSuccess || (e = dev_upload(pauli, &c->d_qgt_pauli)) != cudaSuccess) {
    for (auto& g : groups) {
      delete g.seg;
      delete g.suffix;
    }
    return cuda_fail(e, "geometric tensor tables");
  }
  c->qgt_groups = groups;
  c->qgt_occ = Pp;
  c->qgt_ready = true;
  return TC_OK;
}

int grid_for(int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 148 * 16)); }

}  // namespace

extern "C" {

tc_status tc_qgt(tc_circuit* c, const double* d_params, int B, double* d_out, void* stream) {
  if (!c || (B != 0 && !d_out)) return fail(TC_E_INVALID, "NULL circuit or output");
  if (B < 0) return fail(TC_E_INVALID, "B < 0");
  if (c->n_params > 0 && !d_params && B > 0) return fail(TC_E_INVALID, "d_params is NULL");
  if (c->dm_n > 0) return fail(TC_E_UNSUPPORTED, "geometric tensor of a density-matrix circuit");
  if (B == 0 || c->n_params == 0) return TC_OK;
  tc_status st = qgt_prepare(c);
  if (st != TC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int P = c->n_params, Pp = c->qgt_occ, S = Pp + 1;
  const int64_t L = (int64_t)1 << c->n;
  cudaError_t e;
  if (Pp == 0) {  // no parameter drives a gate
    if ((e = cudaMemsetAsync(d_out, 0, (size_t)B * P * P * 16, s)) != cudaSuccess) return cuda_fail(e, "memset");
    return TC_OK;
  }
  const bool dbl = c->dtype == TC_C128;
  const size_t amp = dbl ? 16 : 8;
  int maxc = 0;
  for (const auto& g : c->qgt_groups) maxc = std::max(maxc, g.count + 1);
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const bool tcg = !dbl;  // complex64: tensor-core Gram
  const int64_t nchunk = (L + (tcg ? kTcChunk : kGramChunk) - 1) / (tcg ? kTcChunk : kGramChunk);
  // per row: S states, the prefix state, replicated parameters, the Gram matrix
  // and its per-chunk partials (summed in a fixed order: reproducible bits)
  const size_t row_bytes = al((size_t)S * L * amp) + al((size_t)L * amp) + al((size_t)maxc * P * 8) +
                           al((size_t)S * S * 16) + al((size_t)nchunk * S * S * 16);
  int64_t cap = c->opt.mem_budget_bytes;
  if (cap <= 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    cap = (int64_t)((double)(fr + c->qgt_ws_bytes) * 0.5);
  }
  const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(std::min(B, 65535), cap / (int64_t)row_bytes));
  const size_t need = row_bytes * chunk + 1024;
  if (need > c->qgt_ws_bytes) {
    dev_free(c->qgt_ws);
    c->qgt_ws = nullptr;
    c->qgt_ws_bytes = 0;
    e = cudaMalloc(&c->qgt_ws, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(TC_E_NOMEM, "geometric tensor workspace (" + std::to_string(need >> 20) + " MiB)");
    }
    c->qgt_ws_bytes = need;
  }
  char* w = (char*)c->qgt_ws;
  char* states = w;                                              // [S][R][L], slot-major
  char* phi = states + al((size_t)S * L * amp) * chunk;         // [R][L]
  double* th = (double*)(phi + al((size_t)L * amp) * chunk);   // [count][R][P]
  double* M = (double*)((char*)th + al((size_t)maxc * P * 8) * chunk);
  double* Mp = (double*)((char*)M + al((size_t)S * S * 16) * chunk);  // [nchunk][R][S][S][2]
  int* d_err = (int*)(w + row_bytes * chunk);                  // in the workspace's slack
  // complex64: tensor-core Gram (128-row tiles); complex128: FP64 CUDA-core Gram
  const bool tc = !dbl;
  // tests only: TC_TEST_GRAM_SKIP_MMA=1 makes the tensor-core Gram issue no MMA,
  // so its bounded completion wait runs out and the call reports TC_E_TIMEOUT
  const char* skip_env = getenv("TC_TEST_GRAM_SKIP_MMA");
  const int skip_mma = (skip_env && skip_env[0] == '1') ? 1 : 0;
  const int tile = tc ? kTcTile : kGramTile;
  const int ntile = (S + tile - 1) / tile;
  if (nchunk > 65535) return fail(TC_E_UNSUPPORTED, "too many qubits for the Gram kernel");
  if (tc) {
    if ((e = cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem)) != cudaSuccess)
      return cuda_fail(e, "gram smem");
    if ((e = cudaMemsetAsync(d_err, 0, sizeof(int), s)) != cudaSuccess) return cuda_fail(e, "memset");
  }
  const int ng = (int)c->qgt_groups.size();
  for (int r0 = 0; r0 < B; r0 += chunk) {
    const int R = std::min(chunk, B - r0);
    const double* th_rows = d_params + (size_t)r0 * P;
    const int64_t slot_bytes = (int64_t)R * L * (int64_t)amp;  // one slot of every row
    for (int gi = 0; gi < ng; ++gi) {
      const auto& g = c->qgt_groups[gi];
      // advance the prefix state to this group's insertion point
      if (g.seg) {
        if ((st = tc_apply_layers(g.seg, th_rows, R, gi == 0 ? nullptr : phi, 0, nullptr, 0, phi, s)) != TC_OK)
          return st;
      } else if (gi == 0) {
        return fail(TC_E_INVALID, "geometric tensor plan: no prefix before the first insertion point");
      }
      // the group's states (plus the unshifted state after the last group)
      const int cnt = g.count + (gi == ng - 1 ? 1 : 0);
      char* dst = states + (int64_t)g.first * slot_bytes;
      const uint32_t* pz = c->d_qgt_pauli + 3 * (size_t)g.first;
      if (dbl)
        k_qgt_pauli<double2><<<grid_for((int64_t)cnt * R * L), 256, 0, s>>>((const double2*)phi, R, L, pz, cnt,
                                                                            (double2*)dst);
      else
        k_qgt_pauli<float2><<<grid_for((int64_t)cnt * R * L), 256, 0, s>>>((const float2*)phi, R, L, pz, cnt,
                                                                           (float2*)dst);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "geometric tensor states");
      if (g.suffix) {
        k_qgt_rep<<<grid_for((int64_t)cnt * R * P), 256, 0, s>>>(th_rows, P, R, cnt, th);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "geometric tensor parameters");
        if ((st = tc_apply_layers(g.suffix, th, cnt * R, dst, 0, nullptr, 0, dst, s)) != TC_OK) return st;
      }
    }
    const size_t per = (size_t)R * S * S * 2;  // doubles of one chunk's partial
    if ((e = cudaMemsetAsync(Mp, 0, (size_t)nchunk * per * 8, s)) != cudaSuccess) return cuda_fail(e, "memset");
    dim3 grid((unsigned)(ntile * (ntile + 1) / 2), (unsigned)nchunk, (unsigned)R);
    if (tc)
      k_gram_tc<<<grid, kTcThreads, kTcSmem, s>>>((const float2*)states, S, L, (int64_t)R * L, ntile, Mp, d_err,
                                                  skip_mma);
    else
      k_gram<double><<<grid, 256, 0, s>>>((const double2*)states, S, L, (int64_t)R * L, ntile, Mp);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gram");
    k_gram_sum<<<grid_for((int64_t)per), 256, 0, s>>>(Mp, (int)nchunk, per, M);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gram chunk sum");
    k_qgt_fold<<<grid_for((int64_t)R * P * P), 256, 0, s>>>(M, S, tile, c->d_qgt_off, c->d_qgt_occ, c->d_qgt_occ_c,
                                                             P, R, d_out + (size_t)r0 * P * P * 2);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "geometric tensor fold");
  }
  if (tc) {  // the tensor-core Gram's bounded waits report through a flag
    int h_err = 0;
    if ((e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_fail(e, "gram status");
    if (h_err) return fail(TC_E_TIMEOUT, "tensor-core Gram: an MMA completion wait timed out");
  }
  return TC_OK;
}

tc_status tc_natural_gradient(const double* d_qgt, const double* d_grad, int B, int P, double eps, double* d_out,
                              void* stream) {
  if (B != 0 && (!d_qgt || !d_grad || !d_out)) return fail(TC_E_INVALID, "NULL argument");
  if (B < 0 || P < 1) return fail(TC_E_INVALID, "B < 0 or P < 1");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(TC_E_INVALID, "eps must be positive and finite");
  if (P > kNgMaxP) return fail(TC_E_UNSUPPORTED, "natural gradient for more than 128 parameters");
  if (B == 0) return TC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int smem = (P * P + P) * 8;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_natgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
    return cuda_fail(e, "natural gradient smem");
  for (int r0 = 0; r0 < B; r0 += 65535) {
    const int rows = std::min(65535, B - r0);
    k_natgrad<<<rows, 256, smem, s>>>(d_qgt + (size_t)r0 * P * P * 2, d_grad + (size_t)r0 * P, P, eps,
                                      d_out + (size_t)r0 * P);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "natural gradient");
  }
  // status per call, from this call's own output: a row whose matrix is not
  // positive definite is all NaN, so its first element tells (one strided copy)
  std::vector<double> first(B);
  if ((e = cudaMemcpy2DAsync(first.data(), sizeof(double), d_out, (size_t)P * sizeof(double), sizeof(double), B,
                             cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(e, "natural gradient status");
  for (int r = 0; r < B; ++r)
    if (std::isnan(first[r]))
      return fail(TC_E_INVALID, "natural gradient: 4 Re G + eps I is not positive definite for row " +
                                    std::to_string(r) + " (or its inputs hold NaN); that row is NaN");
  return TC_OK;
}

}  // extern "C"
