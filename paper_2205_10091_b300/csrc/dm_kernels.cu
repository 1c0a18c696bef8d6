// tr(rho P) on a vectorised density matrix: with P|y> = i^{ny} (-1)^{popc(y & sm)} |y ^ f>,
// tr(rho P) = sum_y rho_{y, y^f} i^{ny} (-1)^{popc(y & sm)}   (Section "Density matrix simulator").
#include "dm.h"

namespace tcb {

template <typename V>
__global__ void __launch_bounds__(256) k_dm_trace(const V* rho, int n, const DmTerm* terms, int T, double* partial) {
  __shared__ double sh[256];
  const int b = blockIdx.y;
  const uint32_t dim = 1u << n;
  const V* r = rho + ((size_t)b << (2 * n));
  double acc = 0;
  for (uint32_t y = blockIdx.x * blockDim.x + threadIdx.x; y < dim; y += gridDim.x * blockDim.x) {
    const size_t row = (size_t)y << n;
    for (int t = 0; t < T; ++t) {
      const DmTerm d = terms[t];
      const V v = r[row + (y ^ d.f)];
      // i^ny: 0 -> Re, 1 -> -Im, 2 -> -Re, 3 -> Im
      double x = (d.ny == 0) ? (double)v.x : (d.ny == 1) ? -(double)v.y : (d.ny == 2) ? -(double)v.x : (double)v.y;
      if (__popc(y & d.sm) & 1) x = -x;
      acc += d.w * x;
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(size_t)b * gridDim.x + blockIdx.x] = sh[0];
}

cudaError_t launch_dm_trace(bool dbl, const void* rho, int n, int B, const DmTerm* d_terms, int T, double* partial,
                            int nblk, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  if (B > 65535 || nblk < 1) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)nblk, (unsigned)B);
  if (dbl) k_dm_trace<double2><<<grid, 256, 0, s>>>((const double2*)rho, n, d_terms, T, partial);
  else k_dm_trace<float2><<<grid, 256, 0, s>>>((const float2*)rho, n, d_terms, T, partial);
  return cudaGetLastError();
}

}  // namespace tcb
