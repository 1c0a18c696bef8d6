// Device side of the light-cone contraction: input assembly, one gather-GEMM
// per path step, result conversion.  Every index of these networks has
// dimension 2, so a tensor of rank r is a 2^r array and a permutation of its
// indices is a permutation of address bits; the host precomputes, per step,
// the addresses of A's rows/columns and B's rows/columns (fa, sa, sb, fb) so
// the GEMM reads operands in place with no separate permute kernel.
#include "tn.h"

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
constexpr int TM = 32, TN = 32, TK = 16;

__global__ void __launch_bounds__(256) k_tn_gemm(const int32_t* tables, TnStep st, int64_t arena_total, float2* arena) {
  __shared__ float2 As[TK][TM + 1];
  __shared__ float2 Bs[TK][TN + 1];
  const size_t inst = (size_t)blockIdx.z * arena_total;
  const float2* A = arena + inst + st.a_off;
  const float2* Bm = arena + inst + st.b_off;
  float2* C = arena + inst + st.c_off;
  const int32_t* fa = tables + st.fa;
  const int32_t* sa = tables + st.sa;
  const int32_t* sb = tables + st.sb;
  const int32_t* fb = tables + st.fb;
  const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
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

__global__ void k_tn_result(const float2* arena, int64_t arena_total, int64_t off, int B, double* out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) {
    const float2 v = arena[(size_t)b * arena_total + off];
    out[2 * b] = (double)v.x;
    out[2 * b + 1] = (double)v.y;
  }
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
