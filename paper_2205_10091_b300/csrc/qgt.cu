// Quantum geometric tensor of a parameterised circuit (Section "Quantum
// Fisher Information"):
//   G_ij = <d_i psi|d_j psi> - <d_i psi|psi><psi|d_j psi>,  QFI = 4 Re G.
//
// Every parameterised gate is exp(-i a G / 2) with G^2 = I, a = s theta_p, and
// d/da exp(-i a G / 2) = (-i/2) G exp(-i a G / 2) = (1/2) exp(-i (a + pi) G / 2).
// So d|psi>/d theta_p = sum over the occurrences k of p of c_k |psi_k>, with
// c_k = s_k / 2 and |psi_k> the circuit's state with occurrence k's angle
// advanced by pi.  Per batch row the engine runs the occurrences' S - 1
// shifted states and the unshifted state as S rows of a companion circuit
// that gives every occurrence its own parameter (the forward tile passes),
// a Gram kernel forms M_kl = <psi_k|psi_l>, and a fold kernel sums
// G_ij = sum_{k in i, l in j} c_k c_l M_kl - u_i conj(u_j), u_i = sum_k c_k M_{k,S-1}.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "engine.h"

namespace tcb {

namespace {

constexpr int kGramTile = 64;    // states per tile side
constexpr int kGramX = 16;       // amplitudes per shared-memory stage
constexpr int kGramChunk = 2048; // amplitudes summed in the state's precision before the FP64 atomics

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

// theta'[(r S + t)][k] = s_k theta[r][p_k] + (t == k ? pi : 0), t = S - 1 unshifted
__global__ void k_qgt_params(const double* __restrict__ theta, int P, const int* __restrict__ occ_param,
                             const double* __restrict__ occ_c, int Pp, int rows, double* __restrict__ out) {
  const int S = Pp + 1;
  const int64_t total = (int64_t)rows * S * Pp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % Pp);
    const int64_t rt = e / Pp;
    const int t = (int)(rt % S);
    const int64_t r = rt / S;
    double v = 2.0 * occ_c[k] * theta[r * P + occ_param[k]];
    if (t == k) v += 3.14159265358979323846;
    out[e] = v;
  }
}

// M[r][k][l] += sum_x conj(psi_{r,k}[x]) psi_{r,l}[x] over one amplitude
// chunk, for the tile pair (kt <= lt) of blockIdx.x; 4 x 4 outputs a thread.
template <typename R>
__global__ void __launch_bounds__(256) k_gram(const typename Cplx<R>::T* __restrict__ states, int S, int64_t L,
                                              int ntile, double* __restrict__ M) {
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
  const C2* base = states + (size_t)r * S * L;
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
      As[xx][kk] = (ka < S && x < x1) ? base[(size_t)ka * L + x] : z;
      Bs[xx][kk] = (kb < S && x < x1) ? base[(size_t)kb * L + x] : z;
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
      if (k < S && l < S) {
        double* m = M + (((size_t)r * S + k) * S + l) * 2;
        atomicAdd(m, (double)ar[i][j]);
        atomicAdd(m + 1, (double)ai[i][j]);
      }
    }
}

// M(k, l) from the computed triangle of tiles: M(l, k) = conj(M(k, l))
__device__ __forceinline__ double2 gram_at(const double* Mr, int S, int k, int l) {
  if (k / kGramTile <= l / kGramTile) return make_double2(Mr[((size_t)k * S + l) * 2], Mr[((size_t)k * S + l) * 2 + 1]);
  return make_double2(Mr[((size_t)l * S + k) * 2], -Mr[((size_t)l * S + k) * 2 + 1]);
}

__global__ void k_qgt_fold(const double* __restrict__ M, int S, const int* __restrict__ off,
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
      const double2 mk = gram_at(Mr, S, k, last);  // <psi_k|psi>
      ur += ck * mk.x;
      ui += ck * mk.y;
      for (int b = off[j]; b < off[j + 1]; ++b) {
        const int l = occ[b];
        const double2 m = gram_at(Mr, S, k, l);
        gr += ck * occ_c[l] * m.x;
        gi += ck * occ_c[l] * m.y;
      }
    }
    for (int b = off[j]; b < off[j + 1]; ++b) {
      const int l = occ[b];
      const double2 m = gram_at(Mr, S, last, l);  // <psi|psi_l>
      vr += occ_c[l] * m.x;
      vi += occ_c[l] * m.y;
    }
    out[e * 2] = gr - (ur * vr - ui * vi);
    out[e * 2 + 1] = gi - (ur * vi + ui * vr);
  }
}

}  // namespace

}  // namespace tcb

using namespace tcb;

namespace {

tc_status qgt_prepare(tc_circuit* c) {
  if (c->qgt_sub) return TC_OK;
  std::vector<tc_op> ops = c->ops_in;
  std::vector<int> occ_param;
  std::vector<double> occ_c;
  for (auto& o : ops) {
    if (o.kind == TC_OP_PAULI_NOISE || o.kind == TC_OP_RSEL)
      return fail(TC_E_UNSUPPORTED, "geometric tensor of circuits with noise or random-axis rotations");
    const bool rot = o.kind == TC_OP_RX || o.kind == TC_OP_RY || o.kind == TC_OP_RZ || o.kind == TC_OP_RZZ;
    if (o.param < 0 || !rot) continue;
    occ_param.push_back(o.param);
    occ_c.push_back(0.5 * o.scale);
    o.param = (int32_t)occ_param.size() - 1;
    o.scale = 1.0;
  }
  const int Pp = (int)occ_param.size();
  std::vector<double> pool = c->pool;
  tc_circuit* sub = nullptr;
  tc_status st = tc_circuit_create(c->n, c->dtype, c->init, ops.data(), (int)ops.size(), Pp,
                                   pool.empty() ? nullptr : pool.data(), (int)(pool.size() / 2), &c->opt, &sub);
  if (st != TC_OK) return st;
  // parameter -> occurrences (CSR)
  std::vector<int> off(c->n_params + 1, 0), occ(Pp);
  for (int k = 0; k < Pp; ++k) off[occ_param[k] + 1]++;
  for (int p = 0; p < c->n_params; ++p) off[p + 1] += off[p];
  {
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (int k = 0; k < Pp; ++k) occ[fill[occ_param[k]]++] = k;
  }
  if (occ.empty()) occ.push_back(0);
  if (occ_param.empty()) {
    occ_param.push_back(0);
    occ_c.push_back(0.0);
  }
  cudaError_t e;
  if ((e = dev_upload(occ_param, &c->d_qgt_occ_param)) != cudaSuccess ||
      (e = dev_upload(occ_c, &c->d_qgt_occ_c)) != cudaSuccess || (e = dev_upload(off, &c->d_qgt_off)) != cudaSuccess ||
      (e = dev_upload(occ, &c->d_qgt_occ)) != cudaSuccess) {
    delete sub;
    return cuda_fail(e, "geometric tensor tables");
  }
  c->qgt_sub = sub;
  c->qgt_occ = Pp;
  return TC_OK;
}

}  // namespace

extern "C" {

tc_status tc_qgt(tc_circuit* c, const double* d_params, int B, double* d_out, void* stream) {
  if (!c || !d_out) return fail(TC_E_INVALID, "NULL circuit or output");
  if (B < 0) return fail(TC_E_INVALID, "B < 0");
  if (c->n_params > 0 && !d_params && B > 0) return fail(TC_E_INVALID, "d_params is NULL");
  if (c->dm_n > 0) return fail(TC_E_UNSUPPORTED, "geometric tensor of a density-matrix circuit");
  if (B == 0 || c->n_params == 0) return TC_OK;
  tc_status st = qgt_prepare(c);
  if (st != TC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int P = c->n_params, Pp = c->qgt_occ, S = Pp + 1;
  const int64_t L = (int64_t)1 << c->n;
  const size_t amp = c->dtype == TC_C128 ? 16 : 8;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  // per row: S states, S x P' shifted parameters, S x S Gram matrix
  const size_t row_bytes = al((size_t)S * L * amp) + al((size_t)S * Pp * 8) + al((size_t)S * S * 16);
  int64_t cap = c->opt.mem_budget_bytes;
  if (cap <= 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    cap = (int64_t)((double)(fr + c->qgt_ws_bytes) * 0.5);
  }
  const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(B, cap / (int64_t)row_bytes));
  const size_t need = row_bytes * chunk + 1024;
  if (need > c->qgt_ws_bytes) {
    dev_free(c->qgt_ws);
    c->qgt_ws = nullptr;
    c->qgt_ws_bytes = 0;
    cudaError_t e = cudaMalloc(&c->qgt_ws, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(TC_E_NOMEM, "geometric tensor workspace (" + std::to_string(need >> 20) + " MiB)");
    }
    c->qgt_ws_bytes = need;
  }
  char* w = (char*)c->qgt_ws;
  void* states = w;
  double* th = (double*)(w + al((size_t)S * L * amp) * chunk);
  double* M = (double*)((char*)th + al((size_t)S * Pp * 8) * chunk);
  const int ntile = (S + kGramTile - 1) / kGramTile;
  const int64_t nchunk = (L + kGramChunk - 1) / kGramChunk;
  if (nchunk > 65535) return fail(TC_E_UNSUPPORTED, "too many qubits for the Gram kernel");
  cudaError_t e;
  for (int r0 = 0; r0 < B; r0 += chunk) {
    const int rows = std::min(chunk, B - r0);
    if (Pp > 0) {
      const int64_t tot = (int64_t)rows * S * Pp;
      const int g = (int)std::min<int64_t>((tot + 255) / 256, 148 * 16);
      k_qgt_params<<<g, 256, 0, s>>>(d_params + (size_t)r0 * P, P, c->d_qgt_occ_param, c->d_qgt_occ_c, Pp, rows, th);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "geometric tensor parameters");
    }
    if ((st = tc_apply_layers(c->qgt_sub, Pp > 0 ? th : nullptr, rows * S, nullptr, 0, nullptr, 0, states, s)) !=
        TC_OK)
      return st;
    if ((e = cudaMemsetAsync(M, 0, (size_t)rows * S * S * 16, s)) != cudaSuccess) return cuda_fail(e, "memset");
    for (int r = 0; r < rows; r += 65535) {
      const int rr = std::min(65535, rows - r);
      dim3 grid((unsigned)(ntile * (ntile + 1) / 2), (unsigned)nchunk, (unsigned)rr);
      if (c->dtype == TC_C128)
        k_gram<double><<<grid, 256, 0, s>>>((const double2*)states + (size_t)r * S * L, S, L, ntile,
                                            M + (size_t)r * S * S * 2);
      else
        k_gram<float><<<grid, 256, 0, s>>>((const float2*)states + (size_t)r * S * L, S, L, ntile,
                                           M + (size_t)r * S * S * 2);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gram");
    }
    const int64_t tot = (int64_t)rows * P * P;
    const int g = (int)std::min<int64_t>((tot + 255) / 256, 148 * 16);
    k_qgt_fold<<<g, 256, 0, s>>>(M, S, c->d_qgt_off, c->d_qgt_occ, c->d_qgt_occ_c, P, rows,
                                 d_out + (size_t)r0 * P * P * 2);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "geometric tensor fold");
  }
  return TC_OK;
}

}  // extern "C"
