// Density-matrix circuits: the doubled op list and the trace kernel.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tc.h"

namespace tcb {

// A Pauli string of tr(rho P): flip mask f (X or Y), sign mask sm (Y or Z),
// number of Y mod 4, weight.
struct DmTerm {
  uint32_t f, sm;
  int32_t ny, pad;
  double w;
};

// ops on n qubits -> ops on 2n qubits acting on |rho>> (pool extended with the
// conjugate matrices and the channels' superoperators).
bool build_dm_ops(int n, const tc_op* ops, int n_ops, const double* pool, int n_pool, std::vector<tc_op>& out,
                  std::vector<double>& out_pool, std::string& err);
bool build_dm_terms(int n, const uint8_t* structures, const double* weights, int T, std::vector<DmTerm>& out,
                    std::string& err);

// partial[b][blk] = sum over the block's share of y of sum_t w_t Re(rho_{y, y^f_t} P_t(y^f_t, y))
cudaError_t launch_dm_trace(bool dbl, const void* rho, int n, int B, const DmTerm* d_terms, int T, double* partial,
                            int nblk, cudaStream_t s);

}  // namespace tcb
