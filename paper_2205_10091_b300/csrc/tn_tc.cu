// Tensor-core path step of a tensor-network contraction (tcgen05, cta_group::1).
//
// A path step is the complex GEMM C[i][j] = sum_k A[fa(i) + sa(k)] B[sb(k) + fb(j)]
// whose operands are gathered in place through the step's index tables (the
// index permutation of Section "Tensor network engine" folded into
// addresses).  Here it runs on the tensor cores:
//   - The larger of the two free sides is the MMA's M side ("P", 128 rows per
//     CTA); the other ("Q") gives 64 complex columns per CTA.  With
//     out(p, q) = sum_k P(p, k) Q(q, k), each P row is the real vector
//     (re, im) interleaved along k, and each Q row becomes two real rows,
//     (re, -im) and (im, re), so Re out and Im out are the real dot products
//     with them: one real GEMM with M = 128, N = 128 (64 Re then 64 Im).
//   - Precision (the operands are FP32): TF32X3 splits x = hi + lo with
//     hi = tf32(x) and sums P_hi Q_hi + P_hi Q_lo + P_lo Q_hi (kind::tf32);
//     BF16X6 splits x = h + m + l in bfloat16 and sums the six products
//     whose weight is above 2^-24 (hh, hm, mh, hl, lh, mm; kind::f16).
//   - The tensor core's FP32 accumulation does not round to nearest (it
//     truncates at the accumulator's magnitude), so each stage of 16 complex
//     k starts a fresh TMEM accumulator, the correction products enter it
//     before the full-size ones, and every thread adds its share of it into
//     FP32 registers (round to nearest).
//   - Per stage, all 256 threads gather the next stage's operands into
//     registers while the current stage's MMAs run (double-buffered operand
//     tiles and TMEM accumulators); one thread issues the MMAs and commits
//     them to an mbarrier.  Every wait is bounded; on a timeout the CTA sets
//     the error word, waits (bounded) for its own committed MMAs, frees its
//     TMEM and returns.
//   - The epilogue stages the 128 x 64 complex tile in shared memory and
//     writes C with consecutive threads on consecutive addresses.
#include "tcgen05.cuh"
#include "tn.h"

namespace tcb {

namespace {

constexpr int kTtThreads = 256;
constexpr int kTtP = 128;         // P rows per CTA (TMEM lanes)
constexpr int kTtQ = 64;          // Q complex columns per CTA (128 real MMA columns)
constexpr int kTtKC = 16;         // complex k per stage
constexpr int kTtCols = 256;      // TMEM: two accumulators of 128 columns
constexpr long long kTtSpin = 1ll << 20;

template <int PREC>
struct TtCfg;
template <>
struct TtCfg<TN_TF32X3> {  // 32 TF32 per row and stage: 8 core matrices along K
  static constexpr int kParts = 2;                     // hi, lo
  static constexpr uint32_t kLBO = 128, kSBO = 1024;   // bytes
  static constexpr int kTileBytes = kTtP * 2 * kTtKC * 4;  // 16 KiB (P tile; the Q tile has 128 real rows too)
  static constexpr uint32_t kIdesc = tc_idesc(kTcFmtTF32, 128, 128);
};
template <>
struct TtCfg<TN_BF16X6> {  // 32 BF16 per row and stage: 4 core matrices along K
  static constexpr int kParts = 3;                     // h, m, l
  static constexpr uint32_t kLBO = 128, kSBO = 512;
  static constexpr int kTileBytes = kTtP * 2 * kTtKC * 2;  // 8 KiB
  static constexpr uint32_t kIdesc = tc_idesc(kTcFmtBF16, 128, 128);
};

template <int PREC>
__host__ __device__ constexpr int tt_set_bytes() {
  return 2 * TtCfg<PREC>::kParts * TtCfg<PREC>::kTileBytes;  // P parts then Q parts
}
constexpr int kTtCStride = 2 * kTtQ + 1;  // floats per staged output row (odd: conflict-free column writes)

template <int PREC>
__host__ __device__ constexpr int tt_smem_bytes() {
  constexpr int sets = 2 * tt_set_bytes<PREC>();
  constexpr int cst = kTtP * kTtCStride * 4;
  return sets > cst ? sets : cst;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Split 4 FP32 values into the parts of the precision mode and store each
// part's 16 bytes (TF32: 4 values) or 8 bytes (BF16: 4 values) at `off` of
// every part tile (tiles `stride` bytes apart).
template <int PREC>
__device__ __forceinline__ void tt_store4(uint8_t* tiles, int stride, uint32_t off, float a, float b, float c,
                                          float d) {
  if constexpr (PREC == TN_TF32X3) {
    const float4 h = make_float4(tf32_rna(a), tf32_rna(b), tf32_rna(c), tf32_rna(d));
    *reinterpret_cast<float4*>(tiles + off) = h;
    *reinterpret_cast<float4*>(tiles + stride + off) = make_float4(a - h.x, b - h.y, c - h.z, d - h.w);
  } else {
    const float ha = __bfloat162float(__float2bfloat16_rn(a)), hb = __bfloat162float(__float2bfloat16_rn(b));
    const float hc = __bfloat162float(__float2bfloat16_rn(c)), hd = __bfloat162float(__float2bfloat16_rn(d));
    const float ra = a - ha, rb = b - hb, rc = c - hc, rd = d - hd;
    const float ma = __bfloat162float(__float2bfloat16_rn(ra)), mb = __bfloat162float(__float2bfloat16_rn(rb));
    const float mc = __bfloat162float(__float2bfloat16_rn(rc)), md = __bfloat162float(__float2bfloat16_rn(rd));
    *reinterpret_cast<uint2*>(tiles + off) = make_uint2(pack_bf16x2(ha, hb), pack_bf16x2(hc, hd));
    *reinterpret_cast<uint2*>(tiles + stride + off) = make_uint2(pack_bf16x2(ma, mb), pack_bf16x2(mc, md));
    *reinterpret_cast<uint2*>(tiles + 2 * stride + off) =
        make_uint2(pack_bf16x2(ra - ma, rb - mb), pack_bf16x2(rc - mc, rd - md));
  }
}

// Byte offset of (row, complex k pair kp) in a K-major no-swizzle tile: the
// pair's 4 reals are 16 bytes (TF32: one core-matrix row) or 8 bytes (BF16:
// half of one).
template <int PREC>
__device__ __forceinline__ uint32_t tt_off(int row, int kp) {
  if constexpr (PREC == TN_TF32X3)
    return (uint32_t)((row >> 3) * TtCfg<PREC>::kSBO + kp * TtCfg<PREC>::kLBO + (row & 7) * 16);
  else
    return (uint32_t)((row >> 3) * TtCfg<PREC>::kSBO + (kp >> 1) * TtCfg<PREC>::kLBO + (row & 7) * 16 + (kp & 1) * 8);
}

template <int PREC>
__global__ void __launch_bounds__(kTtThreads, 1) k_tn_tc(const int32_t* __restrict__ tables, TnStep st,
                                                         int64_t arena_total, float2* __restrict__ arena, int trans,
                                                         int* __restrict__ err) {
  using Cfg = TtCfg<PREC>;
  extern __shared__ __align__(1024) uint8_t tt_smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  const size_t inst = (size_t)blockIdx.z * arena_total;
  // P side (MMA rows) and Q side (columns): P(p, k) = Pm[prow(p) + pk(k)]
  const float2* Pm = arena + inst + (trans ? st.b_off : st.a_off);
  const float2* Qm = arena + inst + (trans ? st.a_off : st.b_off);
  const int32_t* prow = tables + (trans ? st.fb : st.fa);
  const int32_t* pk = tables + (trans ? st.sb : st.sa);
  const int32_t* qrow = tables + (trans ? st.fa : st.fb);
  const int32_t* qk = tables + (trans ? st.sa : st.sb);
  const int Pn = trans ? st.N : st.M, Qn = trans ? st.M : st.N, K = st.K;
  float2* C = arena + inst + st.c_off;
  const int p0 = blockIdx.y * kTtP, q0 = blockIdx.x * kTtQ;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lg = warp & 3, half = warp >> 2;  // TMEM lane quarter; Re (0) or Im (1) columns
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(tt_smem);
  const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&mbar[0]);
  const uint32_t bar1 = (uint32_t)__cvta_generic_to_shared(&mbar[1]);
  if (warp == 0) tmem_alloc((uint32_t)__cvta_generic_to_shared(&tmem_base), kTtCols);
  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tacc = tmem_base;

  // gather assignment.  TF32: a thread owns P row (tid & 127) at complex k
  // pairs (tid >> 7) + 2 u (u < 4), and Q row (tid & 63) at pairs
  // (tid >> 6) + 4 u (u < 2).  BF16: P row (tid & 127) at pair quads
  // (tid >> 7) + 2 u (u < 2), Q row (tid & 63) at quad (tid >> 6).
  constexpr int NP = 8;  // complex P elements per thread and stage
  constexpr int NQ = 4;
  const int pr = tid & (kTtP - 1), qr = tid & (kTtQ - 1);
  const int pbase = p0 + pr < Pn ? prow[p0 + pr] : -1;
  const int qbase = q0 + qr < Qn ? qrow[q0 + qr] : -1;
  auto pk_of = [&](int e) {  // complex k (within the stage) of P element e of this thread
    if constexpr (PREC == TN_TF32X3) return 2 * ((tid >> 7) + 2 * (e >> 1)) + (e & 1);
    else return 4 * ((tid >> 7) + 2 * (e >> 2)) + (e & 3);
  };
  auto qk_of = [&](int e) {
    if constexpr (PREC == TN_TF32X3) return 2 * ((tid >> 6) + 4 * (e >> 1)) + (e & 1);
    else return 4 * (tid >> 6) + e;
  };
  float2 pv[NP], qv[NQ];
  auto gather = [&](int k0) {
#pragma unroll
    for (int e = 0; e < NP; ++e) {
      const int k = k0 + pk_of(e);
      pv[e] = (pbase >= 0 && k < K) ? Pm[pbase + pk[k]] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int e = 0; e < NQ; ++e) {
      const int k = k0 + qk_of(e);
      qv[e] = (qbase >= 0 && k < K) ? Qm[qbase + qk[k]] : make_float2(0.f, 0.f);
    }
  };
  // operand tiles of one stage: P parts, then Q parts (128 real rows: the
  // (re, -im) rows of the 64 columns, then their (im, re) rows)
  auto convert = [&](int set) {
    uint8_t* tp = tt_smem + set * tt_set_bytes<PREC>();
    uint8_t* tq = tp + Cfg::kParts * Cfg::kTileBytes;
    if constexpr (PREC == TN_TF32X3) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float2 a = pv[2 * u], b = pv[2 * u + 1];
        tt_store4<PREC>(tp, Cfg::kTileBytes, tt_off<PREC>(pr, (tid >> 7) + 2 * u), a.x, a.y, b.x, b.y);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float2 a = qv[2 * u], b = qv[2 * u + 1];
        const int kp = (tid >> 6) + 4 * u;
        tt_store4<PREC>(tq, Cfg::kTileBytes, tt_off<PREC>(qr, kp), a.x, -a.y, b.x, -b.y);
        tt_store4<PREC>(tq, Cfg::kTileBytes, tt_off<PREC>(kTtQ + qr, kp), a.y, a.x, b.y, b.x);
      }
    } else {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int kq = (tid >> 7) + 2 * u;  // quad of complex k = pairs 2 kq, 2 kq + 1
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float2 a = pv[4 * u + 2 * h], b = pv[4 * u + 2 * h + 1];
          tt_store4<PREC>(tp, Cfg::kTileBytes, tt_off<PREC>(pr, 2 * kq + h), a.x, a.y, b.x, b.y);
        }
      }
      const int kq = tid >> 6;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float2 a = qv[2 * h], b = qv[2 * h + 1];
        tt_store4<PREC>(tq, Cfg::kTileBytes, tt_off<PREC>(qr, 2 * kq + h), a.x, -a.y, b.x, -b.y);
        tt_store4<PREC>(tq, Cfg::kTileBytes, tt_off<PREC>(kTtQ + qr, 2 * kq + h), a.y, a.x, b.y, b.x);
      }
    }
  };
  auto issue = [&](int set) {
    const uint32_t tp = sbase + (uint32_t)(set * tt_set_bytes<PREC>());
    const uint32_t tq = tp + (uint32_t)(Cfg::kParts * Cfg::kTileBytes);
    const uint32_t d = tacc + (uint32_t)(set * 128);
    auto desc = [&](uint32_t tile, int part, uint32_t o) {
      return tc_smem_desc(tile + (uint32_t)(part * Cfg::kTileBytes) + o, Cfg::kLBO, Cfg::kSBO);
    };
    // The accumulation truncates at the accumulator's magnitude on every MMA,
    // so the small correction products go first (while the sum is ~2^-8 of
    // its final size) and the full-size products last: one truncation at
    // full magnitude per K step instead of one per product.
    if constexpr (PREC == TN_TF32X3) {
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {  // K = 8 TF32 per MMA: two core matrices
        const uint32_t o = (uint32_t)(ks * 2 * Cfg::kLBO);
        tc_mma_tf32(d, desc(tp, 0, o), desc(tq, 1, o), Cfg::kIdesc, ks == 0 ? 0u : 1u);  // hi lo
        tc_mma_tf32(d, desc(tp, 1, o), desc(tq, 0, o), Cfg::kIdesc, 1u);                 // lo hi
      }
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint32_t o = (uint32_t)(ks * 2 * Cfg::kLBO);
        tc_mma_tf32(d, desc(tp, 0, o), desc(tq, 0, o), Cfg::kIdesc, 1u);  // hi hi
      }
    } else {
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {  // K = 16 BF16 per MMA: two core matrices
        const uint32_t o = (uint32_t)(ks * 2 * Cfg::kLBO);
        tc_mma_bf16(d, desc(tp, 1, o), desc(tq, 1, o), Cfg::kIdesc, ks == 0 ? 0u : 1u);  // m m
        tc_mma_bf16(d, desc(tp, 0, o), desc(tq, 2, o), Cfg::kIdesc, 1u);                 // h l
        tc_mma_bf16(d, desc(tp, 2, o), desc(tq, 0, o), Cfg::kIdesc, 1u);                 // l h
        tc_mma_bf16(d, desc(tp, 0, o), desc(tq, 1, o), Cfg::kIdesc, 1u);                 // h m
        tc_mma_bf16(d, desc(tp, 1, o), desc(tq, 0, o), Cfg::kIdesc, 1u);                 // m h
      }
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint32_t o = (uint32_t)(ks * 2 * Cfg::kLBO);
        tc_mma_bf16(d, desc(tp, 0, o), desc(tq, 0, o), Cfg::kIdesc, 1u);  // h h
      }
    }
    tc_commit(set ? bar1 : bar0);
  };
  float acc[64];
#pragma unroll
  for (int j = 0; j < 64; ++j) acc[j] = 0.f;
  uint32_t parity[2] = {0u, 0u};
  bool pending[2] = {false, false};
  bool ok = true;
  auto drain = [&](int set) -> bool {
    const bool done = mbar_wait(set ? bar1 : bar0, parity[set], kTtSpin);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!done) return false;
    parity[set] ^= 1u;
    pending[set] = false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t v[32];
      tmem_ld32(tacc + ((uint32_t)(32 * lg) << 16) + (uint32_t)(set * 128 + 64 * half + 32 * h), v);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[32 * h + j] += __uint_as_float(v[j]);
    }
    return true;
  };
  const int nst = (K + kTtKC - 1) / kTtKC;
  gather(0);
  for (int s = 0; s < nst && ok; ++s) {
    const int set = s & 1;
    convert(set);
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // this stage's tiles complete
    if (s + 1 < nst) gather((s + 1) * kTtKC);  // in flight while the MMAs run
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      issue(set);
    }
    pending[set] = true;
    if (s > 0) ok = drain(set ^ 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    // TMEM reads done before that accumulator and tile set are reused; a
    // timeout seen by any thread stops the whole CTA
    ok = __syncthreads_and(ok) != 0;
  }
  if (ok && nst > 0) ok = drain((nst - 1) & 1);
  ok = __syncthreads_and(ok) != 0;
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    if (pending[0]) mbar_wait(bar0, parity[0], kTtSpin);
    if (pending[1]) mbar_wait(bar1, parity[1], kTtSpin);
  } else {
    // stage the tile (every MMA has completed: the operand tiles are free)
    float* cs = reinterpret_cast<float*>(tt_smem);
    const int p = 32 * lg + lane;
#pragma unroll
    for (int j = 0; j < 64; ++j) cs[p * kTtCStride + 2 * j + half] = acc[j];
    __syncthreads();
    if (!trans) {  // C[(p0 + p) N + q0 + q]: q fastest
      for (int e = tid; e < kTtP * kTtQ; e += kTtThreads) {
        const int pp = e >> 6, qq = e & (kTtQ - 1);
        if (p0 + pp < Pn && q0 + qq < Qn)
          C[(size_t)(p0 + pp) * st.N + q0 + qq] =
              make_float2(cs[pp * kTtCStride + 2 * qq], cs[pp * kTtCStride + 2 * qq + 1]);
      }
    } else {  // C[(q0 + q) N + p0 + p]: p fastest
      for (int e = tid; e < kTtP * kTtQ; e += kTtThreads) {
        const int pp = e & (kTtP - 1), qq = e >> 7;
        if (p0 + pp < Pn && q0 + qq < Qn)
          C[(size_t)(q0 + qq) * st.N + p0 + pp] =
              make_float2(cs[pp * kTtCStride + 2 * qq], cs[pp * kTtCStride + 2 * qq + 1]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) tmem_dealloc(tacc, kTtCols);
}

template <int PREC>
cudaError_t launch_tc(const int32_t* tables, const TnStep& st, int B, int64_t arena_total, float2* arena, int* err,
                      cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_tn_tc<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tt_smem_bytes<PREC>());
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int trans = st.N > st.M ? 1 : 0;  // the larger free side on the MMA rows
  const int Pn = trans ? st.N : st.M, Qn = trans ? st.M : st.N;
  const dim3 grid((unsigned)((Qn + kTtQ - 1) / kTtQ), (unsigned)((Pn + kTtP - 1) / kTtP), (unsigned)B);
  if (grid.y > 65535u || B > 65535) return cudaErrorInvalidConfiguration;
  k_tn_tc<PREC><<<grid, kTtThreads, tt_smem_bytes<PREC>(), s>>>(tables, st, arena_total, arena, trans, err);
  return cudaGetLastError();
}

}  // namespace

bool tn_step_tc_eligible(const TnStep& st, double min_cmacs) {
  return st.K >= 2 && (double)st.M * st.N * st.K >= min_cmacs;
}

cudaError_t tn_launch_step_tc(const TnPlan& P, const TnStep& st, int B, float2* arena, int prec, int* d_err,
                              cudaStream_t s) {
  if (prec == TN_TF32X3) return launch_tc<TN_TF32X3>(P.d_tables, st, B, P.arena_total, arena, d_err, s);
  if (prec == TN_BF16X6) return launch_tc<TN_BF16X6>(P.d_tables, st, B, P.arena_total, arena, d_err, s);
  return cudaErrorInvalidValue;
}

}  // namespace tcb
