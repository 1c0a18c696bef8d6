// Launch interface of the state-vector kernels (sv_kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "plan.h"
#include "sv_args.h"

namespace tcb {

// Launch one pass for `rows` batch rows (st0: the pass's first stage; NULL for
// a Pauli-sum pass).
cudaError_t launch_pass(int mode, bool dbl, const KArgs& a, const DevPass& host_pass, const DevStage* st0,
                        int rows, cudaStream_t s);
size_t pass_smem_bytes(int mode, bool dbl, const DevPass& p);
// Launch a pass kernel specialised at plan time for `rows` rows (its program
// is compiled in: only the tiles, the row's table and the reduction buffer
// take shared memory).
cudaError_t launch_pass_specialised(cudaKernel_t kern, int mode, bool dbl, const KArgs& a, const DevPass& hp, int rows,
                                    cudaStream_t s);

// Build the gate tables (rotation cos/sin pairs, phase tables, 2x2/4x4
// matrices, noise outcomes) of DevMat records [first_mat, first_mat+n_mats)
// for `rows` batch rows into a.tables (row stride a.table_stride entries).
cudaError_t launch_tables(bool dbl, const KArgs& a, int first_mat, int n_mats, int rows, cudaStream_t s);

// E[b] = sum of energy partials; grad[b][p] = sum over slots of p and tiles.
// accumulate: the gradients are added to g_out instead of written
cudaError_t launch_finalize(const double* epart, int n_hpasses, int tiles_h, const double* gpart, int gslots,
                            int tiles_b, const int* csr_off, const int* csr_slots, int n_params, int rows,
                            double* e_out, double* g_out, cudaStream_t s, bool accumulate = false);

// Copy a narrow (n < 9) state batch in or out of the padded internal layout.
cudaError_t launch_pad_states(bool dbl, const void* src, void* dst, int n_user, int N, int rows, bool to_padded,
                              cudaStream_t s);

// Explicit-loop baseline: E_b += w * <psi_b|P|psi_b> for one Pauli term, one
// full sweep of the state per term.
cudaError_t launch_plain_term(bool dbl, const void* psi, int N, int rows, uint32_t f, uint32_t sm, int ny,
                              double w, double* e_acc, cudaStream_t s);

// Partial squared norms of `rows` states of 2^n_qubits amplitudes (user
// layout): part[row][0..nblk) in FP64; the finalize reduction sums them.
cudaError_t launch_norm2(bool dbl, const void* psi, int n_qubits, int rows, int nblk, double* part, cudaStream_t s);

// Mean and standard error of n doubles into out[0], out[1].
cudaError_t launch_mean_stderr(const double* x, int n, double* out, cudaStream_t s, bool moments = false);

// Optional event timing of every launch (enabled by tc_profile_begin).
enum ProfKind : int { PK_FWD = 0, PK_BWD = 1, PK_HAM = 2, PK_FINALIZE = 3, PK_PAD = 4, PK_PLAIN = 5, PK_TABLES = 6, PK_SMALL = 7, PK_COUNT = 8 };
void prof_begin();
bool prof_enabled();
void prof_before(int kind, double algo_bytes, cudaStream_t s);
void prof_after(cudaStream_t s);
// fills launches/ms/bytes per kind; returns false on a CUDA error
bool prof_end(int* launches, double* ms, double* bytes);

}  // namespace tcb
