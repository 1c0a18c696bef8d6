/*
 * tc.h — C-ABI of libtc_b300.so, a B300 (sm_103a) engine for the batched
 * circuit-expectation hot path of arXiv 2205.10091 ("TensorCircuit").
 *
 * What is computed (the paper's definitions; readings stated where the paper
 * is silent):
 *   |psi(theta)> = U_G ... U_1 |psi_0>          (Section "Circuits and gates")
 *   E(theta)     = sum_j w_j <psi|P_j|psi>       (Eq. H-pauli; Section "Pauli
 *                                                 structures and weights")
 *   dE/dtheta_k  for every parameter, per batch row (Section "vmap and
 *                vectorized_value_and_grad": argnums == vectorized_argnums)
 *
 * Conventions
 *   - Qubit 0 is the most significant bit of the amplitude index (Section
 *     "Preliminaries"); a state of n qubits is 2^n interleaved complex
 *     numbers (re, im), complex64 (TC_C64) or complex128 (TC_C128).
 *   - Rotations are exp(-i a G / 2) with a = scale * theta[param] and
 *     G = X, Y, Z or Z(x)Z.  The paper's exp1 form exp(i t G) is scale = -2.
 *   - CNOT(q0, q1): q0 is the control (Section "Basic circuits and outputs").
 *   - A Pauli structure is n bytes over {0,1,2,3} = {I,X,Y,Z}; weights are
 *     real doubles (Section "Pauli structures and weights").
 *   - Batches: parameters are a row-major [B][n_params] array of doubles on
 *     the device; states are [B][2^n] complex on the device.
 *
 * Ownership: the caller owns every device buffer it passes and every stream.
 * The library owns only the opaque objects it returns (plans, networks,
 * servers) and their internal scratch, which it allocates on the device
 * within the memory budget of tc_options and frees in the destroy call.
 * Host arrays passed to a create call are copied before it returns.
 *
 * Errors: every entry point returns a tc_status.  Argument errors are found
 * on the host before any launch and leave device memory untouched.  B = 0 (no
 * rows or instances) is a valid call on every batched entry point: after the
 * checks of its other arguments it returns TC_OK without a launch, and its
 * device buffer pointers may then be NULL.  A CUDA
 * launch or runtime error returns TC_E_CUDA.  tc_last_error() returns a
 * thread-local message for the last non-TC_OK status.  No exception crosses
 * the ABI and no device code traps.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 * default stream).  Calls are asynchronous with respect to the host unless
 * stated otherwise; results are valid after the stream is synchronised.
 *
 * Host threads: an object returned by a create call (a circuit plan, a
 * network, a Hamiltonian) builds device copies, captured graphs, launch
 * shapes and scratch lazily on first use and keeps them; calls on one object
 * must not overlap in time (the caller serialises them).  Distinct objects
 * may be used from different threads at once.  A server is the exception:
 * tc_submit and tc_poll may be called from any thread while it runs.
 */
#ifndef TC_B300_H
#define TC_B300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TC_API __attribute__((visibility("default")))
#else
#define TC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TC_OK = 0,
  TC_E_INVALID = 1,     /* bad argument (message in tc_last_error) */
  TC_E_NOMEM = 2,       /* device allocation failed or budget exceeded */
  TC_E_CUDA = 3,        /* CUDA runtime error */
  TC_E_TIMEOUT = 4,     /* a bounded wait ran out */
  TC_E_UNSUPPORTED = 5, /* valid request outside what the engine implements */
  TC_E_BUSY = 6,        /* the server is full; retry later */
  TC_E_CANCELLED = 7    /* the request was cancelled */
} tc_status;

typedef enum { TC_C64 = 0, TC_C128 = 1 } tc_dtype;
typedef enum { TC_INIT_ZERO = 0, TC_INIT_PLUS = 1 } tc_init;

/* Gate kinds.  Matrices (qubit 0 of a two-qubit matrix = row bit 1):
 *   H, X                      standard
 *   RX, RY, RZ (a)            exp(-i a X/2), exp(-i a Y/2), exp(-i a Z/2)
 *   RZZ (a) on (q0, q1)       exp(-i a Z(x)Z / 2)
 *   CNOT (q0 control, q1 target), CZ = diag(1, 1, 1, -1)
 *   U1                        2x2 matrix from the pool (row-major)
 *   U2                        4x4 matrix from the pool (row-major,
 *                             row index 2*b(q0) + b(q1)) (Section "Arbitrary
 *                             unitaries")
 *   PAULI_NOISE (px,py,pz)    one Monte Carlo event of the Pauli channel
 *                             with Kraus weights (1-px-py-pz, px, py, pz) in
 *                             the order [I, X, Y, Z] (Section "Monte Carlo
 *                             simulation with tc.Circuit"): the uniform
 *                             number u of the event selects the outcome whose
 *                             left-closed interval contains u (Section
 *                             "Externalizing the randomness").
 */
typedef enum {
  TC_OP_H = 0,
  TC_OP_X = 1,
  TC_OP_RX = 2,
  TC_OP_RY = 3,
  TC_OP_RZ = 4,
  TC_OP_RZZ = 5,
  TC_OP_CNOT = 6,
  TC_OP_CZ = 7,
  TC_OP_U1 = 8,
  TC_OP_U2 = 9,
  TC_OP_PAULI_NOISE = 10,
  TC_OP_RSEL = 11  /* RX, RY or RZ(scale * theta[param]) on q0, chosen per row with
                      probabilities (px, py, pz) by the row's number for this event
                      (unitary_kraus over rotations, Section "Demonstration of
                      barren plateaus"); events are numbered with the noise events */
} tc_opkind;

/* One gate.  56 bytes, naturally aligned (the Python binding mirrors it). */
typedef struct {
  int32_t kind;  /* tc_opkind */
  int32_t q0;    /* first qubit */
  int32_t q1;    /* second qubit of a two-qubit gate, else -1 */
  int32_t param; /* parameter index for RX/RY/RZ/RZZ, -1 = none (angle 0) */
  double scale;  /* angle = scale * theta[param] */
  int32_t mat;   /* U1/U2: offset (complex entries) into the matrix pool */
  int32_t pad;
  double px, py, pz; /* PAULI_NOISE probabilities; RSEL: probabilities of RX, RY, RZ (sum 1) */
} tc_op;

typedef struct {
  int32_t tile_qubits_fwd;  /* qubits per shared-memory tile, forward (0 = default) */
  int32_t tile_qubits_bwd;  /* same for adjoint passes (0 = default) */
  int64_t mem_budget_bytes; /* scratch cap for tc_expect_grad (0 = 60% of free memory) */
  int32_t max_gates_per_pass; /* cap on non-diagonal gates fused into one pass (0 = default, <0 = none) */
  int32_t specialize;       /* 1 = compile the circuit's forward and adjoint passes into kernels of
                               their own at tc_circuit_create (NVRTC, sm_103a; seconds per circuit):
                               every plan constant is compiled in, the arithmetic is the same as the
                               default plan-interpreting kernels; 0 = no */
  int32_t reserved[6];
} tc_options;

/* Plan statistics, filled by tc_circuit_info. */
typedef struct {
  int32_t n_qubits;
  int32_t n_qubits_internal; /* >= 9: narrower circuits run with idle low qubits */
  int32_t n_ops;
  int32_t n_params;
  int32_t n_noise;
  int32_t fwd_passes;  /* HBM sweeps of the forward plan */
  int32_t bwd_passes;  /* HBM sweeps of the adjoint plan */
  int32_t fwd_stages;  /* register stages summed over forward passes */
  int32_t bwd_stages;
  int32_t tile_qubits_fwd;
  int32_t tile_qubits_bwd;
  int32_t fwd_instrs;  /* gate instructions over forward passes (diagonal groups count once) */
  int32_t bwd_instrs;
  int32_t specialized_passes; /* passes compiled into kernels of their own (tc_options.specialize) */
  int32_t packed_diag_groups; /* phase groups of several ZZ distances evaluated as one 64-bit
                                 linear map per amplitude (at most 64 terms a group), both plans */
  int32_t reserved[1];
} tc_plan_info;

typedef struct tc_circuit tc_circuit;

/*
 * tc_circuit_create — compile an op list into a fused-pass plan.
 *   n_qubits  1..30
 *   ops       host array of n_ops gates (copied)
 *   n_params  columns of the parameter matrix; every op.param < n_params
 *   pool      host array of 2*n_pool doubles (interleaved re, im) holding the
 *             U1/U2 matrices (copied; may be NULL when n_pool == 0)
 *   opt       NULL for defaults
 * Plan compilation (host): consecutive commuting gates are grouped into
 * passes whose non-diagonal gates act on at most `tile` qubits; diagonal
 * gates (RZ, RZZ, CZ) sharing a parameter fuse into one phase-table lookup
 * (the paper's "preprocessing" absorbs gates into neighbours, Section
 * "Custom contraction settings").  Returns TC_E_INVALID for out-of-range
 * qubits, parameters or matrix offsets.
 */
TC_API tc_status tc_circuit_create(int n_qubits, tc_dtype dtype, tc_init init, const tc_op* ops, int n_ops,
                            int n_params, const double* pool, int n_pool, const tc_options* opt,
                            tc_circuit** out);
TC_API void tc_circuit_destroy(tc_circuit* c);
TC_API tc_status tc_circuit_info(const tc_circuit* c, tc_plan_info* out);

/*
 * tc_pauli_sum_info — host-only plan of a Pauli sum (structures and weights
 * as in tc_expect_pauli_sum) for this circuit's width: the number of
 * Pauli-sum passes (sweeps over the state), how many of them are paired
 * passes (flip masks wider than a tile), the flip-mask groups and the
 * diagonal entries.  Touches no device.
 */
typedef struct {
  int32_t passes;
  int32_t paired_passes;
  int32_t flip_groups;
  int32_t diag_entries;       /* diagonal records (a packed group counts 1 + n_qubits_internal) */
  int32_t tile_qubits;
  int32_t packed_diag_groups; /* ZZ terms of one weight at three or more distances, up to 64 a group,
                                 evaluated as one 64-bit linear map and a popcount per amplitude */
  int32_t reserved[2];
} tc_pauli_sum_plan_info;
TC_API tc_status tc_pauli_sum_info(const tc_circuit* c, const uint8_t* structures, const double* weights, int T,
                                   tc_pauli_sum_plan_info* out);

/*
 * tc_apply_layers — |psi_b> = U(theta_b)|psi_0> for every batch row b
 * (Section "Basic circuits and outputs", batched as in Section "Batched
 * circuits").
 *   d_params      device [B][n_params] doubles (may be NULL if n_params == 0)
 *   d_init        NULL = the circuit's tc_init state, else device [B][2^n]
 *                 complex of the circuit's dtype (a batch of input states,
 *                 Section "Batched input states")
 *   seed          Philox4x32-10 key for noise events when d_status is NULL:
 *                 event e of trajectory t = row_offset + b uses counter
 *                 (e/4, t mod 2^32, t / 2^32, 0),
 *                 key (seed mod 2^32, seed / 2^32), output word e % 4, and
 *                 u = (word >> 8) * 2^-24
 *   d_status      NULL, or device [B][n_noise] floats in [0, 1): the uniform
 *                 numbers of the noise events in op order (the paper's
 *                 externalised `status`)
 *   row_offset    global index of row 0 (trajectory numbering for Philox)
 *   d_states_out  device [B][2^n] complex of the circuit's dtype (written)
 * Scratch: none beyond d_states_out.
 */
TC_API tc_status tc_apply_layers(const tc_circuit* c, const double* d_params, int B, const void* d_init,
                          uint64_t seed, const float* d_status, int64_t row_offset, void* d_states_out,
                          void* stream);

/*
 * tc_apply_expect — the state of every row and K Pauli-sum expectations of it
 * in one call: the "Plain method" of Section "Basic circuits and outputs"
 * (state, then c.expectation_ps per observable), equal to tc_apply_layers
 * (circuit's tc_init state, no noise) followed by K tc_expect_pauli_sum calls.
 *   T             host [K]: terms of observable k
 *   structures    host [sum T][n] bytes 0..3 (I, X, Y, Z), observables in order
 *   weights       host [sum T] doubles
 *   d_states_out  device [B][2^n] complex of the circuit's dtype, or NULL
 *   d_values_out  device [B][K] doubles (written; may be NULL if K == 0)
 * Circuits of 5..10 qubits without noise events run as one launch per call:
 * one thread-block cluster per row (up to 8 CTAs of 128 amplitudes) holds
 * the state in shared memory; gates exchange partner amplitudes by warp
 * shuffles, shared memory or distributed shared memory; consecutive one-qubit
 * ops on a qubit are fused; each observable is reduced in FP64.  Up to 16
 * observables and 256 terms take that path; other circuits run the tile
 * passes and one Pauli-sum call per observable (scratch from the stream's
 * memory pool when d_states_out is NULL).  Errors: TC_E_INVALID for bad
 * sizes or structure entries, TC_E_UNSUPPORTED for density-matrix circuits.
 */
TC_API tc_status tc_apply_expect(tc_circuit* c, const double* d_params, int B, int K, const int* T,
                                 const uint8_t* structures, const double* weights, void* d_states_out,
                                 double* d_values_out, void* stream);

/*
 * tc_expect_pauli_sum — E_b = sum_j w_j Re<psi_b|P_j|psi_b> for every row
 * (Eq. H-pauli; the "vmap over Pauli structures" evaluation of Section
 * "vmap over Pauli structures", fused: terms are grouped by their X/Y flip
 * mask m and each group is one pass over amplitude pairs (x, x^m)).
 *   d_states      device [B][2^n] complex of the circuit's dtype (read only)
 *   structures    host [T][n] bytes in {0,1,2,3} (copied)
 *   weights       host [T] doubles (copied)
 *   d_energy_out  device [B] doubles (written)
 * Any Pauli structure is accepted.  A group whose flip mask fits one
 * shared-memory tile (with the three lowest index bits every tile holds) is
 * evaluated inside that tile; a wider group runs in a paired pass, in which
 * one CTA holds tile t and tile t ^ f_out (f_out: the group's flip bits
 * outside the tile) and evaluates both; groups with the same f_out share a
 * paired pass.  Each pass reads every amplitude once.
 * Scratch: one double per (row, pass, shared-memory tile) inside the
 * circuit's workspace.  Reductions: FP32/FP64 partial sums per tile, FP64
 * across tiles.
 */
TC_API tc_status tc_expect_pauli_sum(tc_circuit* c, const void* d_states, int B, const uint8_t* structures,
                              const double* weights, int T, double* d_energy_out, void* stream);

/*
 * Gradient memory modes.
 *   TC_GRAD_UNCOMPUTE:  two states per row; the adjoint sweep un-applies
 *                       every gate from psi (no stored states).
 *   TC_GRAD_CHECKPOINT: the op list is cut into segments of checkpoint_ops
 *                       ops (0 = four segments), each planned as a circuit
 *                       of its own; the forward sweep keeps the state after
 *                       every segment (segments + 1 states per row), and the
 *                       adjoint sweep of each segment starts from its stored
 *                       state, so psi is un-applied across one segment at
 *                       most.  Circuits with noise events: TC_E_UNSUPPORTED.
 */
typedef enum { TC_GRAD_UNCOMPUTE = 0, TC_GRAD_CHECKPOINT = 1 } tc_grad_mode;

typedef struct {
  int32_t mode;           /* tc_grad_mode */
  int32_t max_rows;       /* rows per device chunk (0 = as many as the budget allows) */
  int32_t checkpoint_ops; /* TC_GRAD_CHECKPOINT: ops per segment (0 = a quarter of the circuit) */
  int32_t reserved[5];
} tc_grad_options;

/*
 * tc_expect_grad — energy and full gradient for every row (Section "Batched
 * VQE": vectorized_value_and_grad with argnums == vectorized_argnums).
 * Method: one forward sweep, lambda = H|psi>, then one adjoint sweep over
 * the gates in reverse that accumulates
 *   dE/dtheta_k += s * Im <lambda|G|psi>   for each gate exp(-i s theta_k G/2)
 * and un-applies the gate from psi and lambda (U^dagger).  The gradient is
 * per row; the paper's summed vvag variant is the sum over rows.
 *   d_params     device [B][n_params] doubles
 *   d_energy_out device [B] doubles (written)
 *   d_grad_out   device [B][n_params] doubles (written)
 *   opt          NULL for defaults
 * Noise events, if any, use `seed` as in tc_apply_layers (the gradient of
 * each fixed trajectory).
 * Scratch: two states per row in flight plus per-tile partial sums, from the
 * circuit's workspace, capped by tc_options.mem_budget_bytes; larger batches
 * run in chunks of rows.  TC_E_NOMEM if even one row does not fit.
 */
TC_API tc_status tc_expect_grad(tc_circuit* c, const double* d_params, int B, const uint8_t* structures,
                         const double* weights, int T, uint64_t seed, double* d_energy_out,
                         double* d_grad_out, const tc_grad_options* opt, void* stream);

/*
 * tc_expect_plain — the unfused per-circuit baseline: every gate is its own
 * HBM sweep and every Pauli term its own reduction (the explicit-loop
 * evaluation of Section "Explicit loop with c.expectation_ps").  Forward and
 * energy only.  Same arguments and outputs as tc_apply_layers followed by
 * tc_expect_pauli_sum; d_states_work is a caller buffer of [B][2^n].
 */
TC_API tc_status tc_expect_plain(tc_circuit* c, const double* d_params, int B, const uint8_t* structures,
                          const double* weights, int T, void* d_states_work, double* d_energy_out,
                          void* stream);

/*
 * tc_dm_circuit_create — a density-matrix circuit (Section "Density matrix
 * simulator"): the same op list acts on rho by U rho U^dagger and by exact
 * Pauli channels rho -> (1-px-py-pz) rho + px X rho X + py Y rho Y + pz Z rho Z
 * (the Kraus form of Section "Noisy circuits"; nothing is sampled).  rho is
 * held vectorised as a 2n-qubit state |rho>> = sum_xy rho_xy |x>|y> (row index
 * x on the first n qubits): each gate U becomes U on qubit q and conj(U) on
 * qubit n + q, and each channel a 4x4 superoperator on (q, n + q).
 *   n_qubits  1..15 (the state holds 4^n amplitudes)
 *   other arguments as tc_circuit_create; init |0..0> gives rho = |0..0><0..0|,
 *   TC_INIT_PLUS gives |+..+><+..+|
 * The returned circuit works with tc_apply_layers (d_states_out: [B][4^n]
 * entries of the dtype, rho_xy at x * 2^n + y; d_init, seed and d_status are
 * ignored for channels) and tc_dm_expect_pauli_sum; tc_circuit_info reports
 * the 2n-qubit plan.  Errors as tc_circuit_create.
 */
TC_API tc_status tc_dm_circuit_create(int n_qubits, tc_dtype dtype, tc_init init, const tc_op* ops, int n_ops,
                                      int n_params, const double* pool, int n_pool, const tc_options* opt,
                                      tc_circuit** out);

/*
 * tc_dm_expect_pauli_sum — d_out[b] = tr(rho_b H), H = sum_t w_t P_t over the
 * circuit's n qubits (structures as tc_expect_pauli_sum), for B vectorised
 * density matrices d_rho ([B][4^n], the circuit's dtype, device).  FP64
 * accumulation.  TC_E_INVALID if c was not made by tc_dm_circuit_create.
 */
TC_API tc_status tc_dm_expect_pauli_sum(tc_circuit* c, const void* d_rho, int B, const uint8_t* structures,
                                        const double* weights, int T, double* d_out, void* stream);

/*
 * tc_state_norms — d_norm2_out[b] = sum_x |psi_b(x)|^2 for B states of the
 * circuit's width and dtype (d_states: device [B][2^n] interleaved complex,
 * 16-byte aligned; d_norm2_out: device [B] doubles).  Squares and sums in FP64
 * with a fixed-order reduction (the same result for a row alone or in a
 * batch): the norm-preservation check of a simulated state (unitary gates keep
 * ||psi|| = 1), the one place besides the energy reduction where the
 * complex64 path uses FP64.  Uses the circuit's workspace (one double per row
 * and block); calls on one circuit must not overlap.
 */
TC_API tc_status tc_state_norms(tc_circuit* c, const void* d_states, int B, double* d_norm2_out, void* stream);

/*
 * tc_mean_stderr — d_out[0] = mean of d_x[0..n), d_out[1] = its standard
 * error (sample standard deviation with ddof = 1, over sqrt(n)), in FP64 with
 * a fixed-order reduction: the Monte Carlo estimate over trajectories
 * (Section "Batched Monte Carlo trajectory noise simulation").
 */
TC_API tc_status tc_mean_stderr(const double* d_x, int n, double* d_out, void* stream);

/*
 * Trajectories split over ranks (one process per GPU, each with its own
 * trajectory rows).  tc_shard_moments writes a shard's (count, mean, M2 =
 * sum of squared deviations from the mean) of d_x[0..n) to device d_out[0..2]
 * in FP64 (fixed-order reduction).  tc_merge_moments (host only) combines R
 * shards' triples, parts [R][3] in rank order, by the pairwise update of
 * sample variances (Chan, Golub and LeVeque) into out[0] = mean and out[1] =
 * standard error (ddof = 1): the same triples in the same order give the same
 * bits on every rank.  The exchange of the triples (an all-gather of 3 doubles
 * per rank) is the caller's.  TC_E_INVALID for NULL arguments, n < 1, negative
 * counts or M2, or no samples at all.
 */
TC_API tc_status tc_shard_moments(const double* d_x, int n, double* d_out, void* stream);
TC_API tc_status tc_merge_moments(const double* parts, int R, double* out);

/*
 * tc_expect_pauli_sum_noalloc — the energies of tc_expect_pauli_sum, for
 * callers that cannot allocate device memory at the call site (a fixed
 * memory reservation, an allocator callback, a latency-critical loop where
 * cudaMalloc's implicit synchronisation is not acceptable).  The paper has no
 * counterpart; this is a property of this library's interface.
 *   Arguments, layout and results are those of tc_expect_pauli_sum, except:
 *   - n_qubits of the circuit must be >= 10 (TC_E_UNSUPPORTED otherwise);
 *   - scratch is one 8 MiB array in the library's device memory (held by
 *     every GPU that loads the library until exit): the compiled Pauli sum
 *     plus one double per (row, Pauli-sum pass, tile).  A call that needs
 *     more returns TC_E_INVALID before touching the GPU; call with fewer rows.
 *   - It calls no cudaMalloc, cudaFree or other allocating routine.  The
 *     plan is copied in with cudaMemcpyAsync from pageable host memory; the
 *     CUDA runtime may stage such a copy before the call returns, so the call
 *     can wait on the host for the copy engine (it does not wait for the
 *     stream's earlier work).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress).  That lookup loads the library's module with
 *     the array on the device, which may allocate device memory; make one
 *     warm-up call (B = 0 is enough, with valid pointers) per device before
 *     any fixed reservation or allocator callback, and before any stream
 *     capture.  The address is cached per device index: do not use the
 *     library on a device after a cudaDeviceReset there.
 *   - Not under stream capture: the plan copy reads host memory that is
 *     freed when the call returns, so a call on a capturing stream returns
 *     TC_E_UNSUPPORTED (a B = 0 call is still accepted).
 *   - Every call shares the array and overwrites what it uses; calls that
 *     overlap on the GPU (other streams, other host threads) race.
 */
TC_API tc_status tc_expect_pauli_sum_noalloc(const tc_circuit* c, const void* d_states, int B,
                                             const uint8_t* structures, const double* weights, int T,
                                             double* d_energy_out, void* stream);

/*
 * Launch profiling: between tc_profile_begin and tc_profile_end every kernel
 * the library launches (from any thread) is bracketed by CUDA events recorded
 * on its own launch stream.  tc_profile_end synchronises those events and
 * reports, per kernel kind, the launch count, the summed device time and the
 * summed algorithmic HBM bytes (each amplitude a launch must read or write,
 * counted once).  Kinds: 0 forward tile pass, 1 adjoint tile pass,
 * 2 Pauli-sum pass, 3 finalize reduction, 4 narrow-state padding,
 * 5 unfused per-term reduction, 6 per-row gate-table build, 7 one-launch
 * small-circuit kernel (tc_apply_expect).  `out` may be
 * NULL to count kinds only.
 */
typedef struct {
  int32_t kind;
  int32_t launches;
  double total_ms;
  double algo_bytes;
} tc_kernel_stat;
TC_API tc_status tc_profile_begin(void);
TC_API tc_status tc_profile_end(tc_kernel_stat* out, int max_out, int* n_out);

/*
 * tc_qgt — quantum geometric tensor of each row's state (Section "Quantum
 * Fisher Information"):
 *   G_ij = <d_i psi|d_j psi> - <d_i psi|psi><psi|d_j psi>
 * with d_i = d / d theta_i; the quantum Fisher information is 4 Re G and the
 * natural gradient solves (4 Re G) x = grad.
 *   d_params  device [B][n_params] doubles
 *   d_out     device [B][n_params][n_params][2] doubles (Re, Im of G; Hermitian)
 * Every RX/RY/RZ/RZZ occurrence k (angle s_k theta_p) contributes
 * (-i s_k / 2) |chi_k> to d_p|psi>, chi_k being the state with the gate's
 * Pauli generator inserted right after it.  An insertion moves past later
 * gates that commute with it, occurrences sharing an insertion point form a
 * group, and per group the library runs the circuit's own ops after the
 * point on the generator-multiplied prefix states (forward tile passes);
 * the S = occurrences + 1 states of a row (the last unshifted) then go
 * through a Gram kernel <chi_k|chi_l> (complex64: tcgen05 tensor cores,
 * TF32 operands split hi + lo, FP32 sums per 16 amplitudes, FP64 across;
 * complex128: FP64 CUDA cores) and a fold onto parameters.  Scratch: S + 1
 * states and S x S complex doubles per row, rows chunked by the circuit's
 * memory budget (default half the free memory); TC_E_NOMEM if one row does
 * not fit, TC_E_TIMEOUT if a tensor-core completion wait ran out (bounded
 * waits; the call then synchronises its stream).  Circuits with noise or random-axis
 * rotations and density-matrix circuits: TC_E_UNSUPPORTED.
 */
TC_API tc_status tc_qgt(tc_circuit* c, const double* d_params, int B, double* d_out, void* stream);

/*
 * tc_natural_gradient — x = (4 Re G + eps I)^-1 grad per row (Section "Quantum
 * Fisher Information": the natural gradient solves the QFI system).
 *   d_qgt   device [B][P][P][2] doubles: tc_qgt's output
 *   d_grad  device [B][P] doubles (e.g. tc_expect_grad's gradients)
 *   eps     Tikhonov shift, > 0 (the QFI is only positive semidefinite)
 *   d_out   device [B][P] doubles
 * One CTA per row: Cholesky factorisation in shared memory (FP64) of the
 * symmetric matrix given by the lower triangle (i >= j) of 4 Re G + eps I,
 * and two triangular solves.  P <= 128 (else TC_E_UNSUPPORTED).  A row whose matrix
 * is not positive definite gets NaN and the call returns TC_E_INVALID; the
 * call synchronises its stream and reads the first element of every output
 * row to find out (the status lives in this call's own output, so calls on
 * other streams or threads do not interfere).
 */
TC_API tc_status tc_natural_gradient(const double* d_qgt, const double* d_grad, int B, int P, double eps,
                                     double* d_out, void* stream);

/*
 * Light-cone tensor-network contraction (Section "Tensor network engine",
 * Section "Custom contraction settings", Table "contractor").
 *
 * tc_tn_lightcone_create — plan <0|U^dagger Z_{z_0} ... Z_{z_m} U|0> for a
 * circuit of two-qubit gates on n_qubits.
 *   gate_qubits  host [n_gates][2] qubit pairs in circuit order (copied); gate
 *                matrices are supplied at contraction time (row index
 *                2*b(q0) + b(q1), like TC_OP_U2)
 *   z_qubits     host [n_z] qubits of the Z observable (copied)
 *   rank_cap     largest rank an intermediate tensor may have (every index
 *                has dimension 2)
 *   greedy_trials  without a path: 0 or 1 = the deterministic greedy path;
 *                k > 1 = the best of it and k - 1 randomised greedy runs
 *                (seeded Gumbel noise on the pair costs): plans whose live
 *                tensors fit the one-launch fused executor first, then fewer
 *                FLOPs, then less WRITE (deterministic for a given k)
 *   path         NULL = greedy path found on the host; else an
 *                opt_einsum-style list of n_path_steps position pairs over
 *                the plan's input tensors (operands removed, result appended)
 * Only gates in the backward causal cone of the observable enter the network
 * (the rest cancel against their conjugates).  The network holds the cone's
 * gates, their conjugates, |0> vectors and Z.  Greedy rule: contract the
 * connected pair minimising size(out) - size(a) - size(b), ties to the
 * smallest tensor ids, skipping pairs above rank_cap.  Host only.
 *
 * tc_contract_path — contract B instances of the planned network (same
 * structure, different gate values) along the plan's path.
 *   d_gates  device [B][n_gates][16] complex64 (interleaved floats): the
 *            4x4 gate matrices of every gate of the circuit (cone gates used)
 *   d_out    device [B][2] doubles: the complex scalar of each instance
 *   precision  tc_tn_precision (below): FP32 CUDA cores, or split TF32 /
 *            BF16 tensor cores for the steps above the plan's threshold
 * Each path step is one complex GEMM whose operand index permutation is
 * folded into precomputed gather tables; the whole sequence is captured once
 * (per batch size, buffers and precision) as a CUDA graph and replayed.
 * Scratch (inputs and all intermediates of B instances) is owned by the plan.
 * A tensor-core step whose bounded wait ran out sets the plan's error word;
 * the library reads it back after the call and the next call on the plan
 * returns TC_E_TIMEOUT.
 */
typedef struct tc_tn tc_tn;
typedef struct {
  double flops;   /* real FLOPs of the path's complex multiply-adds (8 per MAC) */
  double cmacs;   /* complex multiply-adds */
  double write;   /* elements written over all intermediates (the paper's WRITE) */
  double size;    /* elements of the largest intermediate (the paper's SIZE) */
  int32_t n_steps;
  int32_t max_rank;
  int32_t n_cone_gates;
  int32_t cone_lo, cone_hi; /* qubit span of the light cone */
  int32_t n_inputs;         /* input tensors of the doubled network */
  int32_t n_active;         /* qubits with ket/bra chains in the network */
  int32_t fused;            /* executor: 1 = one launch for the whole contraction, live tensors in
                               shared memory (when smem_bytes <= 200 KiB); 0 = one GEMM launch per
                               step, replayed as a CUDA graph */
  int32_t smem_bytes;       /* bytes of live tensors per instance under the liveness layout */
  int32_t fused_groups;     /* barriers of the fused launch: groups of independent steps */
  int32_t tc_steps;         /* steps the split-precision modes run on tensor cores (current threshold) */
  double tc_cmacs;          /* complex multiply-adds of those steps per instance */
  int32_t max_cluster;      /* fused launch with few instances: CTAs (a thread-block cluster) per instance */
  int32_t split_min_items;  /* groups of at least this many work items are split over the cluster */
  int32_t split_groups;     /* groups of the fused launch that are split */
  int32_t blob_ints;        /* fused launch: step records and tables (ints); up to 6144 are staged in shared
                               memory once, whole, a longer path streams group by group */
} tc_path_info;

/*
 * Precision of a contraction's dense steps (Section "Tensor network engine":
 * the pairwise contractions are matrix products):
 *   TC_TN_FP32    every step on CUDA cores, FP32 products and sums;
 *   TC_TN_TF32X3  steps of at least the plan's threshold of complex
 *                 multiply-adds (tc_tn_set_tc_threshold; default 32768) on the
 *                 tensor cores: operands split x = hi + lo, hi = tf32(x),
 *                 products hi hi + hi lo + lo hi (tcgen05 kind::tf32), FP32
 *                 accumulation rounded to nearest every 16 complex k;
 *   TC_TN_BF16X6  the same steps with x = h + m + l in bfloat16 and the six
 *                 products above 2^-24 relative weight (kind::f16).
 * Smaller steps run on CUDA cores in every mode.  A plan whose steps all fall
 * below the threshold runs as in TC_TN_FP32 (fused launch when it fits).
 */
typedef enum { TC_TN_FP32 = 0, TC_TN_TF32X3 = 1, TC_TN_BF16X6 = 2 } tc_tn_precision;
TC_API tc_status tc_tn_lightcone_create(int n_qubits, const int32_t* gate_qubits, int n_gates,
                                        const int32_t* z_qubits, int n_z, int rank_cap, int greedy_trials,
                                        const int32_t* path, int n_path_steps, tc_tn** out);
TC_API tc_status tc_tn_info(const tc_tn* t, tc_path_info* out);
TC_API tc_status tc_contract_path(tc_tn* t, int B, const float* d_gates, tc_tn_precision precision, double* d_out,
                                  void* stream);
/*
 * tc_tn_set_tc_threshold — complex multiply-adds per instance from which a
 * step runs on the tensor cores in TC_TN_TF32X3 / TC_TN_BF16X6 (>= 0; 0 puts
 * every step with K >= 2 there).  Host only.
 */
TC_API tc_status tc_tn_set_tc_threshold(tc_tn* t, double min_cmacs);
/*
 * tc_tn_set_cluster — the fused executor with few instances.  While B
 * clusters of max_cluster CTAs fit on the GPU at once (B x max_cluster <= the
 * SM count) and the cluster is schedulable, each instance runs on a
 * thread-block cluster: every CTA holds all live tensors, groups of fewer
 * than split_min_items work items run in every CTA, and larger groups are
 * split over the cluster with outputs written into every CTA's shared memory
 * (distributed shared memory).  Each output is computed by the same code
 * either way, so results are bitwise those of the one-CTA launch.
 * max_cluster: 1 (off), 2, 4 or 8 (default 8); split_min_items >= 1 (default
 * 2048).  TC_E_INVALID otherwise.  Host-only; takes effect at the next call.
 */
TC_API tc_status tc_tn_set_cluster(tc_tn* t, int max_cluster, int split_min_items);
TC_API void tc_tn_destroy(tc_tn* t);

/*
 * tc_tn_circuit_create — plan <init| U^dagger P U |init> of a parameterised
 * circuit as one closed tensor network (Section "Custom contraction
 * settings": the expectation of one Pauli string contracted as a single
 * network, two-qubit gates split in two tensors, the default greedy path).
 *   n_qubits, init, ops, n_ops, n_params, const_mats, n_mats
 *                as tc_circuit_create (host, copied); ops of kind H, X, RX,
 *                RY, RZ, RZZ, CNOT, CZ, U1, U2 (others: TC_E_UNSUPPORTED)
 *   pauli        host [n_qubits] codes 0..3 = I, X, Y, Z (copied; at least
 *                one non-identity)
 *   prune        0 = every op and qubit enters the network; 1 = the ops in
 *                the backward causal cone of the string; 2 = the same with
 *                diagonal gates (RZ, RZZ, CZ, diagonal U1/U2) dropped where
 *                they commute with the Heisenberg-evolved string (exact)
 *   split        1 = RZZ, CZ and CNOT enter as two rank-3 tensors joined by
 *                a dimension-2 bond (their operator-Schmidt decomposition);
 *                0 = as one rank-4 tensor
 *   rank_cap, path, n_path_steps   as tc_tn_lightcone_create
 *   greedy_trials  as tc_tn_lightcone_create
 * The network holds ket and bra (complex-conjugated) copies of the kept
 * ops, the initial vectors and the string's Pauli matrices; qubits carrying
 * the identity join their ket and bra legs.  Host only.
 *
 * tc_tn_circuit_expect — contract B instances (one parameter row each).
 *   d_params  device [B][n_params] float32
 *   d_out     device [B][2] doubles: Re and Im of <P> per row
 * Tensor entries are evaluated on the device from each row's angles (FP32),
 * then contracted along the path in the given precision (as
 * tc_contract_path).  Plans from tc_tn_lightcone_create are refused (TC_E_INVALID) and
 * vice versa.
 */
TC_API tc_status tc_tn_circuit_create(int n_qubits, tc_init init, const tc_op* ops, int n_ops, int n_params,
                                      const double* const_mats, int n_mats, const uint8_t* pauli, int prune,
                                      int split, int rank_cap, int greedy_trials, const int32_t* path,
                                      int n_path_steps, tc_tn** out);
TC_API tc_status tc_tn_circuit_expect(tc_tn* t, int B, const float* d_params, tc_tn_precision precision,
                                      double* d_out, void* stream);

/*
 * Serving loop (continuous batching of circuit-evaluation requests).
 *
 * A request is one energy + gradient evaluation: an op list, its parameters
 * and a Pauli sum (the arguments of tc_expect_grad with B = 1; complex64).
 * tc_submit queues it and returns at once; planner threads compile its plan
 * and Pauli sum on the host meanwhile.  A scheduler thread admits queued
 * requests in arrival order whenever a stream slot and enough of the memory
 * budget are free.  Queued requests of at most 20 qubits whose plans differ
 * only in the values of their diagonal-group entries and Pauli-sum diagonal
 * records (QAOA instances of one width and depth on different graphs, say)
 * are admitted together, up to max_group_rows of them, as the rows of one
 * evaluation: one launch per pass for the group.  Each admitted group takes
 * one stream-ordered block from the server's own memory pool (plan, per-row
 * diagonal entries, Pauli sum, parameters, two states per row, outputs) and
 * runs on its own CUDA stream, so groups that arrive while others run
 * overlap with them on the device.  The block returns to the pool when the
 * group completes and the next request is admitted.  A row's arithmetic is
 * exactly tc_expect_grad's on that request alone: a result does not depend
 * on what it was grouped or overlapped with.  The paper has no serving
 * layer; this realises the batched evaluation of Section "Batched VQE" for
 * a stream of independent circuits.
 *
 * Errors: a malformed request is refused by tc_submit (TC_E_INVALID); a full
 * queue returns TC_E_BUSY; a request larger than the whole budget completes
 * with TC_E_NOMEM; one that waited longer than timeout_ms before admission
 * completes with TC_E_TIMEOUT; tc_cancel removes a request not yet admitted
 * (TC_E_CANCELLED).  tc_poll returns TC_E_BUSY while a request is pending or
 * running, and TC_OK with its result (whose `status` may be an error) once it
 * is done; the id is then released.
 */
typedef struct tc_server tc_server;
typedef struct {
  int64_t mem_budget_bytes; /* device memory for in-flight requests (0 = 8 GiB) */
  int32_t max_inflight;     /* concurrent requests = CUDA streams (0 = 16, at most 256) */
  int32_t max_queue;        /* queued requests before tc_submit returns TC_E_BUSY (0 = unbounded) */
  int32_t timeout_ms;       /* queued longer than this -> TC_E_TIMEOUT (0 = never) */
  int32_t start_paused;     /* 1 = admit nothing (and touch no GPU) until tc_server_resume; requests are
                               still planned on the host */
  int32_t max_group_rows;   /* requests one admission may group as rows (0 = 32, 1 = no grouping) */
  int32_t planner_threads;  /* host threads compiling request plans (0 = 2) */
  int32_t reserved[4];
} tc_server_options;
typedef struct {
  int32_t n_qubits;
  int32_t init;     /* tc_init */
  int32_t n_ops;
  int32_t n_params; /* at most 256 */
  int32_t n_pool;
  int32_t T;        /* Pauli terms */
  const tc_op* ops;               /* host, copied */
  const double* pool;             /* host [2*n_pool], copied (may be NULL) */
  const double* theta;            /* host [n_params], copied */
  const uint8_t* structures;      /* host [T][n_qubits], copied */
  const double* weights;          /* host [T], copied */
} tc_request;
typedef struct {
  uint64_t id;
  int32_t status;   /* tc_status of the evaluation */
  int32_t n_params;
  double energy;
  double t_submit, t_start, t_done; /* seconds on the host steady clock */
} tc_result;
typedef struct {
  int64_t submitted, completed, cancelled, timed_out, failed, rejected;
  int32_t pending;        /* queued, not admitted */
  int32_t inflight;       /* admitted requests (rows) on the device */
  int32_t peak_inflight;
  int32_t planned;        /* queued requests whose plan is ready */
  int64_t bytes_in_use, peak_bytes;
  int64_t groups;           /* admissions (launch sequences) so far */
  int64_t grouped_requests; /* requests that ran as a row of a group of two or more */
} tc_server_stats;
TC_API tc_status tc_server_create(const tc_server_options* opt, tc_server** out);
TC_API tc_status tc_submit(tc_server* s, const tc_request* req, uint64_t* id_out);
TC_API tc_status tc_poll(tc_server* s, uint64_t id, tc_result* out, double* grad_out, int max_params);
TC_API tc_status tc_cancel(tc_server* s, uint64_t id);
TC_API tc_status tc_server_resume(tc_server* s);
TC_API tc_status tc_server_get_stats(tc_server* s, tc_server_stats* out);
TC_API tc_status tc_server_destroy(tc_server* s);

/* Thread-local message describing the last non-TC_OK status. */
TC_API const char* tc_last_error(void);

/* Library version string. */
TC_API const char* tc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TC_B300_H */
