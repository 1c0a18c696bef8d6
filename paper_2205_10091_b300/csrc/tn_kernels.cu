// Device side of the light-cone contraction: input assembly, one gather-GEMM
// per path step, result conversion.  Every index of these networks has
// dimension 2, so a tensor of rank r is a 2^r array and a permutation of its
// indices is a permutation of address bits; the host precomputes, per step,
// the addresses of A's rows/columns and B's rows/columns (fa, sa, sb, fb) so
// the GEMM reads operands in place with no separate permute kernel.
#include <cooperative_groups.h>

#include "tn.h"

namespace cg = cooperative_groups;

namespace tcb {

__global__ void k_tn_assemble(const TnInput* inputs, int n_inputs, const float* gates, int n_gates, int64_t in_total,
                              int64_t arena_total, float2* arena) {
  const int t = blockIdx.x;
  const int b = blockIdx.y;
  const TnInput in = inputs[t];
  float2* dst = arena + (size_t)b * arena_total + in.off;
  const int n = 1 << in.rank;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    float2 v = make_float2(0.f, 0.f);
    if (in.kind == TS_KET || in.kind == TS_BRA) {
      const float* g = gates + ((size_t)b * n_gates + in.gate) * 32;
      v = make_float2(g[2 * e], in.kind == TS_BRA ? -g[2 * e + 1] : g[2 * e + 1]);
    } else if (in.kind == TS_ZERO) {
      v = make_float2(e == 0 ? 1.f : 0.f, 0.f);  // |0>
    } else {  // TS_Z, labels (bra, ket): Z[b][k] = delta(b, k) (-1)^k
      v = make_float2(e == 0 ? 1.f : (e == 3 ? -1.f : 0.f), 0.f);
    }
    dst[e] = v;
  }
}

// Entry e of a circuit-network input tensor (first label = most significant
// bit of e), evaluated from the instance's parameters.  Conventions: qubit 0
// is the most significant bit of a two-qubit matrix row (2 b(q0) + b(q1));
// RX, RY, RZ(a) = exp(-i a G / 2), RZZ(a) = exp(-i (a/2) Z Z); CNOT with q0 as
// control.
__device__ float2 tn_circuit_entry(const TnInput& in, int e, const TnOp* ops, const float* mats, const float* th) {
  const float r2 = 0.70710678118654752f;
  switch (in.kind) {
    case TS_ZERO: return make_float2(e == 0 ? 1.f : 0.f, 0.f);
    case TS_PLUS: return make_float2(r2, 0.f);
    case TS_PAULI: {  // labels (bra, ket): P[b][k]
      const int bb = e >> 1, kk = e & 1;
      if (in.gate == 1) return make_float2(bb != kk ? 1.f : 0.f, 0.f);
      if (in.gate == 2) return make_float2(0.f, bb == kk ? 0.f : (bb == 0 ? -1.f : 1.f));
      return make_float2(bb != kk ? 0.f : (kk ? -1.f : 1.f), 0.f);
    }
    default: break;
  }
  const TnOp o = ops[in.gate];
  const float a = o.param >= 0 ? o.scale * th[o.param] : 0.f;
  float s, c;
  sincosf(0.5f * a, &s, &c);
  if (in.kind == TS_OP1) {  // labels (out, in)
    const int r = e >> 1, col = e & 1;
    switch (o.kind) {
      case TC_OP_H: return make_float2((r & col) ? -r2 : r2, 0.f);
      case TC_OP_X: return make_float2(r != col ? 1.f : 0.f, 0.f);
      case TC_OP_RX: return r == col ? make_float2(c, 0.f) : make_float2(0.f, -s);
      case TC_OP_RY: return r == col ? make_float2(c, 0.f) : make_float2(r ? s : -s, 0.f);
      case TC_OP_RZ: return r != col ? make_float2(0.f, 0.f) : make_float2(c, r ? s : -s);
      default: return make_float2(mats[2 * (o.mat + e)], mats[2 * (o.mat + e) + 1]);  // TC_OP_U1
    }
  }
  if (in.kind == TS_OP2) {  // labels (o0, o1, i0, i1): U[2 o0 + o1][2 i0 + i1]
    const int r = e >> 2, col = e & 3;
    switch (o.kind) {
      case TC_OP_RZZ: {
        if (r != col) return make_float2(0.f, 0.f);
        const bool odd = (r == 1 || r == 2);  // Z Z = -1
        return make_float2(c, odd ? s : -s);
      }
      case TC_OP_CZ: return make_float2(r != col ? 0.f : (r == 3 ? -1.f : 1.f), 0.f);
      case TC_OP_CNOT: {
        const int t = r < 2 ? r : (r ^ 1);
        return make_float2(t == col ? 1.f : 0.f, 0.f);
      }
      default: return make_float2(mats[2 * (o.mat + e)], mats[2 * (o.mat + e) + 1]);  // TC_OP_U2
    }
  }
  // split halves, labels (out, in, k): gate = sum_k A_k (x) B_k
  const int r = e >> 2, col = (e >> 1) & 1, k = e & 1;
  if (in.kind == TS_SPA) {
    if (r != col) return make_float2(0.f, 0.f);
    if (o.kind == TC_OP_RZZ) return make_float2(k && r ? -1.f : 1.f, 0.f);  // A_0 = I, A_1 = Z
    return make_float2(r == k ? 1.f : 0.f, 0.f);                             // A_k = |k><k| (CZ, CNOT)
  }
  switch (o.kind) {  // TS_SPB
    case TC_OP_RZZ:  // B_0 = cos(a/2) I, B_1 = -i sin(a/2) Z
      if (r != col) return make_float2(0.f, 0.f);
      return k ? make_float2(0.f, r ? s : -s) : make_float2(c, 0.f);
    case TC_OP_CZ:  // B_0 = I, B_1 = Z
      return make_float2(r != col ? 0.f : (k && r ? -1.f : 1.f), 0.f);
    default:  // CNOT: B_0 = I, B_1 = X
      return make_float2((k ? r != col : r == col) ? 1.f : 0.f, 0.f);
  }
}

__global__ void k_tn_assemble_circuit(const TnInput* inputs, const TnOp* ops, const float* mats, const float* params,
                                      int n_params, int64_t arena_total, float2* arena) {
  const int t = blockIdx.x;
  const int b = blockIdx.y;
  const TnInput in = inputs[t];
  float2* dst = arena + (size_t)b * arena_total + in.off;
  const float* th = params + (size_t)b * n_params;
  const int n = 1 << in.rank;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    float2 v = tn_circuit_entry(in, e, ops, mats, th);
    if (in.conj) v.y = -v.y;
    dst[e] = v;
  }
}

// C[i][j] = sum_k A[fa[i] + sa[k]] * B[sb[k] + fb[j]]  (complex, FP32 accumulate)
constexpr int TM = kTnGemmTile, TN = kTnGemmTile, TK = 16;

// One TM x TN output tile (rows i0.., columns j0..) of step `st` of one
// instance (`inst` = that instance's arena); 256 threads.
__device__ __forceinline__ void tn_gemm_tile(const int32_t* tables, const TnStep& st, float2* inst, int i0, int j0) {
  __shared__ float2 As[TK][TM + 1];
  __shared__ float2 Bs[TK][TN + 1];
  const float2* A = inst + st.a_off;
  const float2* Bm = inst + st.b_off;
  float2* C = inst + st.c_off;
  const int32_t* fa = tables + st.fa;
  const int32_t* sa = tables + st.sa;
  const int32_t* sb = tables + st.sb;
  const int32_t* fb = tables + st.fb;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float2 acc[2][2] = {{{0.f, 0.f}, {0.f, 0.f}}, {{0.f, 0.f}, {0.f, 0.f}}};
  for (int k0 = 0; k0 < st.K; k0 += TK) {
    for (int e = threadIdx.x; e < TM * TK; e += 256) {
      const int ii = e % TM, kk = e / TM;
      const int i = i0 + ii, k = k0 + kk;
      As[kk][ii] = (i < st.M && k < st.K) ? A[fa[i] + sa[k]] : make_float2(0.f, 0.f);
    }
    for (int e = threadIdx.x; e < TN * TK; e += 256) {
      const int jj = e % TN, kk = e / TN;
      const int j = j0 + jj, k = k0 + kk;
      Bs[kk][jj] = (j < st.N && k < st.K) ? Bm[sb[k] + fb[j]] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      const float2 a0 = As[kk][2 * ty], a1 = As[kk][2 * ty + 1];
      const float2 b0 = Bs[kk][2 * tx], b1 = Bs[kk][2 * tx + 1];
      const float2 av[2] = {a0, a1}, bv[2] = {b0, b1};
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          acc[r][c].x = fmaf(av[r].x, bv[c].x, fmaf(-av[r].y, bv[c].y, acc[r][c].x));
          acc[r][c].y = fmaf(av[r].x, bv[c].y, fmaf(av[r].y, bv[c].x, acc[r][c].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int i = i0 + 2 * ty + r, j = j0 + 2 * tx + c;
      if (i < st.M && j < st.N) C[(size_t)i * st.N + j] = acc[r][c];
    }
}

__global__ void __launch_bounds__(256) k_tn_gemm(const int32_t* tables, TnStep st, int64_t arena_total, float2* arena) {
  tn_gemm_tile(tables, st, arena + (size_t)blockIdx.z * arena_total, blockIdx.y * TM, blockIdx.x * TN);
}

// Every step of one level of the contraction tree (independent of each
// other) in one launch: block x is output tile x of the level, counted over
// its steps in order (tile_start[s] = first tile of step s, n + 1 entries).
__global__ void __launch_bounds__(256) k_tn_gemm_level(const int32_t* tables, const TnStep* __restrict__ steps,
                                                       const int* __restrict__ tile_start, int n, int64_t arena_total,
                                                       float2* arena) {
  const int x = (int)blockIdx.x;
  int lo = 0, hi = n - 1;  // the last step whose first tile is <= x
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_start[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  const TnStep st = steps[lo];
  const int local = x - tile_start[lo], nj = (st.N + TN - 1) / TN;
  tn_gemm_tile(tables, st, arena + (size_t)blockIdx.z * arena_total, (local / nj) * TM, (local % nj) * TN);
}

__global__ void k_tn_result(const float2* arena, int64_t arena_total, int64_t off, int B, double* out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) {
    const float2 v = arena[(size_t)b * arena_total + off];
    out[2 * b] = (double)v.x;
    out[2 * b + 1] = (double)v.y;
  }
}

// Fused executor: one CTA per instance (grid-stride over instances) runs the
// assembly and the whole path with all live tensors in shared memory.  The
// path runs group by group (independent steps of one tree level, see tn.h),
// one barrier per group; a group's work items are spread over the CTA's warps,
// 32 items (one unit) per warp at a time.  A step computes
//   C[e] = sum_k A[fa(i) ^ sa(k)] B[sb(k) ^ fb(j)],  e = i N + j,
// where the tables hold swizzled entry offsets (tn_swz, tn.h) and C[e] is
// stored at tn_swz(e, rot_c); tpo items per output (a power of two <= 32:
// small results with long sums spread the sum over lanes and reduce by
// shuffles).  Group blocks fitting both shared slots are staged once, whole;
// a longer path's blocks stream through the two slots, the next block loaded
// into registers before the current group computes and stored after it.
// With few instances (CL) a thread-block cluster runs each instance: every
// CTA holds all live tensors, groups below split_min items run redundantly in
// every CTA (no exchange), and a larger group's units are dealt over the
// cluster's warps, each output written into every CTA's shared memory
// (distributed shared memory) between two cluster barriers: the first keeps
// those writes from landing in regions a slower CTA still reads, the second
// publishes them.  Each output is computed by the same code in either case, so
// results do not depend on CL.
constexpr int kFusedThreads = kTnFusedThreads;
constexpr int kFusedPf = (kTnBlobMax + kFusedThreads - 1) / kFusedThreads;

// an index set's swizzled entry offset (fused blob tables, see tn.h)
__device__ __forceinline__ int tn_tab(const int32_t* t, int lg, int v) {
  if (lg <= kTnFullTabBits) return t[v];
  const int lo = (lg + 1) >> 1;
  return t[v & ((1 << lo) - 1)] ^ t[(1 << lo) + (v >> lo)];
}

template <bool CIRCUIT, bool CL>
__global__ void __launch_bounds__(kFusedThreads) k_tn_fused(const TnInput* __restrict__ inputs,
                                                            const int32_t* __restrict__ in_soff, int n_inputs,
                                                            const int32_t* __restrict__ blob, int blob_ints,
                                                            int n_groups, const float* __restrict__ src, int n_src,
                                                            const TnOp* __restrict__ ops,
                                                            const float* __restrict__ mats, int result_soff, int B,
                                                            int split_min, double* __restrict__ out) {
  extern __shared__ float2 sm[];
  __shared__ __align__(16) int32_t tb[2][kTnBlobMax];
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  // instances and this CTA's rank: a cluster shares one instance
  int crank = 0, csize = 1;
  if constexpr (CL) {
    crank = (int)cg::this_cluster().block_rank();
    csize = (int)cg::this_cluster().num_blocks();
  }
  const int inst0 = (int)blockIdx.x / csize, istride = (int)gridDim.x / csize;
  // a path whose group blocks fit both slots is staged once, whole; a longer
  // one streams through the two slots, the next block loaded during a group
  const bool whole = blob_ints <= 2 * kTnBlobMax;
  int32_t* tbw = &tb[0][0];
  if (whole)
    for (int i = tid; i < blob_ints; i += kFusedThreads) tbw[i] = __ldg(blob + i);
  for (int b = inst0; b < B; b += istride) {
    // ---- group 0's block, and the inputs: one warp per tensor, a lane per entry
    if (!whole) {
      const int len0 = n_groups > 0 ? __ldg(blob + 2) : 0;
      for (int i = tid; i < len0; i += kFusedThreads) tb[0][i] = __ldg(blob + i);
    }
    for (int t = tid >> 5; t < n_inputs; t += kFusedThreads / 32) {
      const TnInput in = inputs[t];
      const int e = tid & 31;
      if (e < (1 << in.rank)) {
        float2 v;
        if (CIRCUIT) {
          v = tn_circuit_entry(in, e, ops, mats, src + (size_t)b * n_src);
          if (in.conj) v.y = -v.y;
        } else if (in.kind == TS_KET || in.kind == TS_BRA) {
          const float* g = src + ((size_t)b * n_src + in.gate) * 32;
          v = make_float2(g[2 * e], in.kind == TS_BRA ? -g[2 * e + 1] : g[2 * e + 1]);
        } else if (in.kind == TS_ZERO) {
          v = make_float2(e == 0 ? 1.f : 0.f, 0.f);
        } else {  // TS_Z
          v = make_float2(e == 0 ? 1.f : (e == 3 ? -1.f : 0.f), 0.f);
        }
        const int32_t so = in_soff[t];
        sm[(so & 0x0fffffff) + tn_swz(e, (so >> 28) & 3)] = v;
      }
    }
    __syncthreads();
    // ---- path, group by group ------------------------------------------------
    int off = 0;
    for (int gi = 0; gi < n_groups; ++gi) {
      const int32_t* g = whole ? tbw + off : tb[gi & 1];
      const int n_st = g[0], n_items = g[1], len = g[2];
      const int nlen = (!whole && gi + 1 < n_groups) ? g[3] : 0;
      int32_t pf[kFusedPf];
#pragma unroll
      for (int r = 0; r < kFusedPf; ++r) {
        const int i = tid + r * kFusedThreads;
        pf[r] = i < nlen ? __ldg(blob + off + len + i) : 0;
      }
      const int32_t* recs = g + kTnGHdr;
      // uniform over the cluster: every CTA reads the same group header
      const bool split = CL && csize > 1 && n_items >= split_min;
      if constexpr (CL) {
        if (split) cg::this_cluster().sync();
      }
      // a split group deals the two halves of a paired unit to different warps
      // (one output per lane), keeping the cluster's warps busy
      const int nunits = (n_items + 31) >> 5, nvirt = split ? 2 * nunits : nunits;
      const int ustride = split ? csize * (kFusedThreads / 32) : kFusedThreads / 32;
      for (int uv = (split ? crank * (kFusedThreads / 32) : 0) + warp; uv < nvirt; uv += ustride) {
        const int u = split ? uv >> 1 : uv, half = split ? uv & 1 : 0;
        const int w = (u << 5) + lane;
        int lo = 0, hi = n_st - 1;  // last step whose first item is <= w
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (recs[mid * kTnSRec] <= w) lo = mid; else hi = mid - 1;
        }
        const int4* rv = reinterpret_cast<const int4*>(recs + lo * kTnSRec);
        const int4 r0 = rv[0], r1 = rv[1], r2 = rv[2], r3 = rv[3];
        const int M = r0.y, K = r0.z, N = r0.w, lgM = r1.x, lgK = r1.y, lgN = r1.z, tpo = r1.w & 255;
        // outputs e and e + 32 (tpo 1, full tables): pmode 1 shares A's row, 2 B's column
        const int pmode = (r1.w >> 16) & 3;
        const bool pstep = pmode != 0;
        // a unit never mixes paired and other steps, so both flags are warp-uniform
        if (half && !pstep) continue;
        const bool paired = pstep && !split;
        const int local = w - r0.x;
        const int e = pstep ? (((local >> 5) << 6) | (local & 31)) + 32 * half : local >> (__ffs(tpo) - 1);
        const int part = pstep ? 0 : local & (tpo - 1);
        const int32_t* fa = g + r2.w;
        const int32_t* sa = g + r3.x;
        const int32_t* sb = g + r3.y;
        const int2* sab = reinterpret_cast<const int2*>(sa);  // full k tables: (sa[k], sb[k]) pairs
        const int32_t* fb = g + r3.z;
        float2 acc = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
        const bool valid = e < M * N;
        if (valid) {
          const float2* As = sm + r2.x;
          const float2* Bs = sm + r2.y;
          const int ai = tn_tab(fa, lgM, e >> lgN), bj = tn_tab(fb, lgN, e & (N - 1));
          auto mac = [&](int ka, int kb) {
            const float2 a = As[ai ^ ka];
            const float2 c = Bs[bj ^ kb];
            acc.x = fmaf(a.x, c.x, fmaf(-a.y, c.y, acc.x));
            acc.y = fmaf(a.x, c.y, fmaf(a.y, c.x, acc.y));
          };
          // the same sums in the same order; the loops differ in table form and stride only
          if (paired && pmode == 1) {
            const int bj1 = tn_tab(fb, lgN, (e + 32) & (N - 1));
#pragma unroll 4
            for (int k = 0; k < K; ++k) {
              const int2 kk = sab[k];
              const float2 a = As[ai ^ kk.x];
              const int kb = kk.y;
              const float2 c = Bs[bj ^ kb], c1 = Bs[bj1 ^ kb];
              acc.x = fmaf(a.x, c.x, fmaf(-a.y, c.y, acc.x));
              acc.y = fmaf(a.x, c.y, fmaf(a.y, c.x, acc.y));
              acc1.x = fmaf(a.x, c1.x, fmaf(-a.y, c1.y, acc1.x));
              acc1.y = fmaf(a.x, c1.y, fmaf(a.y, c1.x, acc1.y));
            }
          } else if (paired) {
            const int ai1 = tn_tab(fa, lgM, (e + 32) >> lgN);
#pragma unroll 4
            for (int k = 0; k < K; ++k) {
              const int2 kk = sab[k];
              const int ka = kk.x;
              const float2 a = As[ai ^ ka], a1 = As[ai1 ^ ka];
              const float2 c = Bs[bj ^ kk.y];
              acc.x = fmaf(a.x, c.x, fmaf(-a.y, c.y, acc.x));
              acc.y = fmaf(a.x, c.y, fmaf(a.y, c.x, acc.y));
              acc1.x = fmaf(a1.x, c.x, fmaf(-a1.y, c.y, acc1.x));
              acc1.y = fmaf(a1.x, c.y, fmaf(a1.y, c.x, acc1.y));
            }
          } else if (lgK <= kTnFullTabBits && tpo == 1) {
#pragma unroll 4
            for (int k = 0; k < K; ++k) {
              const int2 kk = sab[k];
              mac(kk.x, kk.y);
            }
          } else if (lgK <= kTnFullTabBits) {
#pragma unroll 4
            for (int k = part; k < K; k += tpo) {
              const int2 kk = sab[k];
              mac(kk.x, kk.y);
            }
          } else {
            for (int k = part; k < K; k += tpo) mac(tn_tab(sa, lgK, k), tn_tab(sb, lgK, k));
          }
        }
        // tpo is uniform over a warp: runs of equal tpo are padded to 32 items
        for (int o = tpo >> 1; o > 0; o >>= 1) {
          acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
          acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (valid && part == 0) {
          const int rot = (r1.w >> 8) & 3;
          const int ce = r2.z + tn_swz(e, rot), ce1 = r2.z + tn_swz(e + 32, rot);
          sm[ce] = acc;
          if (paired) sm[ce1] = acc1;
          if constexpr (CL) {
            if (split) {
              cg::cluster_group cl = cg::this_cluster();
              for (int q = 1; q < csize; ++q) {
                const int dst = crank + q < csize ? crank + q : crank + q - csize;
                *cl.map_shared_rank(sm + ce, dst) = acc;
                if (paired) *cl.map_shared_rank(sm + ce1, dst) = acc1;
              }
            }
          }
        }
      }
      // the other slot held the previous group's block, which no thread reads any more
      int32_t* nb = tb[(gi + 1) & 1];
#pragma unroll
      for (int r = 0; r < kFusedPf; ++r) {
        const int i = tid + r * kFusedThreads;
        if (i < nlen) nb[i] = pf[r];
      }
      off += len;
      if constexpr (CL) {
        if (split) {
          cg::this_cluster().sync();
          continue;
        }
      }
      __syncthreads();
    }
    if (tid == 0 && crank == 0) {
      const float2 v = sm[result_soff];
      out[2 * b] = (double)v.x;
      out[2 * b + 1] = (double)v.y;
    }
    __syncthreads();
  }
  // no CTA leaves while another may still write into its shared memory
  if constexpr (CL) cg::this_cluster().sync();
}

bool tn_fused_ok(const TnPlan& P) {
  return !P.steps.empty() && P.smem_entries > 0 && P.fblob_ok && !P.fblob.empty() &&
         P.smem_entries * 8 <= kTnFusedSmemMax;
}

namespace {
template <bool CIRCUIT, bool CL>
cudaError_t fused_attr(const TnPlan& P) {
  return cudaFuncSetAttribute(k_tn_fused<CIRCUIT, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(P.smem_entries * 8));
}
void fused_cfg(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, const TnPlan& P, int grid, int cl,
               cudaStream_t s) {
  cfg = cudaLaunchConfig_t{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kFusedThreads);
  cfg.dynamicSmemBytes = (size_t)(P.smem_entries * 8);
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = cl > 1 ? 1 : 0;
}
}  // namespace

int tn_fused_cluster(const TnPlan& P, int B) {
  int sms = 0, dev = 0;
  if (P.max_cluster < 2 || B < 1) return 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  int cl = 1;
  while (cl * 2 <= P.max_cluster && cl * 2 <= kTnMaxCluster) cl *= 2;
  if ((long long)B * cl > sms) return 1;
  // the cluster must be schedulable with this shared-memory size
  if ((P.circuit ? fused_attr<true, true>(P) : fused_attr<false, true>(P)) != cudaSuccess) return 1;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fused_cfg(cfg, attr, P, B * cl, cl, nullptr);
  int n = 0;
  const cudaError_t e = P.circuit ? cudaOccupancyMaxActiveClusters(&n, k_tn_fused<true, true>, &cfg)
                                  : cudaOccupancyMaxActiveClusters(&n, k_tn_fused<false, true>, &cfg);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return 1;
  }
  return n >= 1 ? cl : 1;
}

int tn_fused_grid(const TnPlan& P, int B, int cl) {
  if (cl > 1) return B * cl;
  const int smem = (int)(P.smem_entries * 8);
  int per_sm = 0, sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  auto kern = P.circuit ? k_tn_fused<true, false> : k_tn_fused<false, false>;
  if ((P.circuit ? fused_attr<true, false>(P) : fused_attr<false, false>(P)) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFusedThreads, smem) != cudaSuccess) return 0;
  if (per_sm < 1) return 0;
  return B < per_sm * sms ? B : per_sm * sms;
}

cudaError_t tn_launch_fused(const TnPlan& P, int B, const float* d_src, double* d_out, int grid, int cl,
                            cudaStream_t s) {
  if (!tn_fused_ok(P) || grid < 1 || cl < 1 || cl > kTnMaxCluster) return cudaErrorInvalidConfiguration;
  if (cl > 1 && grid != B * cl) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fused_cfg(cfg, attr, P, grid, cl, s);
  const int n_in = (int)P.inputs.size(), n_src = P.circuit ? P.n_params : P.n_gates;
  const int n_blob = (int)P.fblob.size();
  const TnInput* inp = P.d_inputs;
  const int32_t* soff = P.d_in_soff;
  const int32_t* fb = P.d_fblob;
  const TnOp* ops = P.d_ops;
  const float* mats = P.d_mats;
  const int rs = (int)P.result_soff, sm = P.split_min;
  if (cl > 1)
    return P.circuit ? cudaLaunchKernelEx(&cfg, k_tn_fused<true, true>, inp, soff, n_in, fb, n_blob, P.n_groups, d_src,
                                          n_src, ops, mats, rs, B, sm, d_out)
                     : cudaLaunchKernelEx(&cfg, k_tn_fused<false, true>, inp, soff, n_in, fb, n_blob, P.n_groups, d_src,
                                          n_src, ops, mats, rs, B, sm, d_out);
  auto kern = P.circuit ? k_tn_fused<true, false> : k_tn_fused<false, false>;
  kern<<<grid, kFusedThreads, cfg.dynamicSmemBytes, s>>>(inp, soff, n_in, fb, n_blob, P.n_groups, d_src, n_src, ops,
                                                          mats, rs, B, sm, d_out);
  return cudaGetLastError();
}

cudaError_t tn_launch_assemble(const TnPlan& P, int B, const float* d_src, float2* arena, cudaStream_t s) {
  if (P.inputs.empty()) return cudaSuccess;
  dim3 grid((unsigned)P.inputs.size(), (unsigned)B);
  if (P.circuit)
    k_tn_assemble_circuit<<<grid, 32, 0, s>>>(P.d_inputs, P.d_ops, P.d_mats, d_src, P.n_params, P.arena_total, arena);
  else
    k_tn_assemble<<<grid, 32, 0, s>>>(P.d_inputs, (int)P.inputs.size(), d_src, P.n_gates, P.in_total, P.arena_total,
                                      arena);
  return cudaGetLastError();
}

cudaError_t tn_launch_level(const TnPlan& P, const TnStep* d_steps, const int* d_tile_start, int n, int tiles, int B,
                            float2* arena, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_tn_gemm_level<<<dim3((unsigned)tiles, 1, (unsigned)B), 256, 0, s>>>(P.d_tables, d_steps, d_tile_start, n,
                                                                        P.arena_total, arena);
  return cudaGetLastError();
}

cudaError_t tn_launch_step(const TnPlan& P, const TnStep& st, int B, float2* arena, cudaStream_t s) {
  dim3 grid((unsigned)((st.N + TN - 1) / TN), (unsigned)((st.M + TM - 1) / TM), (unsigned)B);
  k_tn_gemm<<<grid, 256, 0, s>>>(P.d_tables, st, P.arena_total, arena);
  return cudaGetLastError();
}

cudaError_t tn_launch_result(const TnPlan& P, int B, const float2* arena, double* d_out, cudaStream_t s) {
  k_tn_result<<<(B + 127) / 128, 128, 0, s>>>(arena, P.arena_total, P.result_off, B, d_out);
  return cudaGetLastError();
}

}  // namespace tcb
