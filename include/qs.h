/*
 * qs.h -- C ABI of a single-GPU (GB300, sm_103a) full-state quantum simulator
 * for statevectors and density matrices, after "Distributed Simulation of
 * Statevectors and Density Matrices" (arXiv 2311.01512).  Only the paper's
 * local (single-node) operations are provided; its distributed exchange
 * algorithms have no counterpart here.
 *
 * Conventions (paper, Sec. "Notation"):
 *   - qubit 0 is the least significant bit of a basis index;
 *   - a statevector of N qubits is 2^N complex amplitudes, interleaved
 *     (re, im), complex128 (QS_C128) or complex64 (QS_C64);
 *   - bit q of a gate-matrix row/column index belongs to target targs[q]
 *     (Sec. "Many-target gate": the order of targets is the order of the
 *     matrix's index bits);
 *   - a density matrix rho = sum_kl alpha_kl |k><l| of N qubits is stored as
 *     its Choi vector of 2N qubits, beta_i = alpha_{i mod 2^N, i / 2^N}
 *     (Sec. "State representation"): row index in the low N bits, column
 *     index in the high N bits;
 *   - Pauli codes: 0 = I, 1 = X, 2 = Y, 3 = Z (the order of the matrices in
 *     the paper's pauliTensorElem, Sec. "Pauli string expectation value").
 *
 * Memory and ownership:
 *   - amplitude storage is DEVICE memory owned by the caller (for example a
 *     torch tensor).  A state handle wraps it and never frees it; the caller
 *     keeps it alive until qs_destroy.  The pointer must be 256-byte aligned.
 *   - each handle owns a little library memory: a device scratch area for
 *     reductions and a pinned staging ring for gate matrices.  It is allocated
 *     by qs_create_* and freed by qs_destroy.
 *   - host arrays passed to any call are read before the call returns; the
 *     caller may reuse them at once.
 *
 * Streams: every call is ordered on the CUDA stream given at creation (NULL =
 * the legacy default stream).  Calls that apply operations return as soon as
 * the work is queued.  Calls that return a value to the host
 * (qs_expec_pauli_sum, qs_calc_norm_or_trace, qs_get_amps) synchronise that
 * stream.
 *
 * Errors: no call aborts or throws.  Each returns a qs_status; arguments are
 * validated on the host before anything is queued, so a call that returns an
 * argument error has changed nothing.  QS_ERR_CUDA reports a CUDA runtime
 * error from a launch or copy.  The gate matrices, Kraus operators and
 * probabilities are not checked for unitarity or complete positivity: the
 * paper's algorithms do not need either (Sec. "Many-target gate",
 * Sec. "Kraus map").
 */
#ifndef QS_H
#define QS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qs_state qs_state;

typedef enum {
  QS_OK = 0,
  QS_ERR_ARG = 1,              /* null pointer, bad size, bad enum, probability outside [0, 1] */
  QS_ERR_QUBIT_RANGE = 2,      /* a qubit index outside [0, N) */
  QS_ERR_DUP_QUBIT = 3,        /* a qubit repeated within targets or within controls */
  QS_ERR_TARGET_IS_CTRL = 4,   /* a qubit both target and control */
  QS_ERR_TOO_MANY_TARGETS = 5, /* more targets than the operation allows */
  QS_ERR_NOT_DENSMATR = 6,     /* a density-matrix-only call on a statevector */
  QS_ERR_OOM = 7,              /* the library's own scratch allocation failed */
  QS_ERR_CUDA = 8,             /* a CUDA runtime error */
  QS_ERR_TIMEOUT = 9,          /* a bounded device wait ran out */
  QS_ERR_ALIGN = 10            /* a device pointer that is not 256-byte aligned */
} qs_status;

typedef enum { QS_C64 = 0, QS_C128 = 1 } qs_prec;

/* Arithmetic of complex128 kernels.  GB300 executes FP64 FMA about 70 times
 * slower than FP32 FMA, so a plain FP64 gate is bound by the FP64 pipe, not by
 * memory.  Amplitudes are always stored as IEEE complex128.
 *
 * QS_ARITH_FX (default): at least the 53 bits of IEEE double.
 *   - One-target gates, diagonals, Pauli and phase gadgets, and the channels
 *     that mix amplitudes (depolarising, damping, Pauli channel) use block
 *     fixed point.  The doubles that one output combines share an exponent and
 *     become 60-bit integers.  Products and sums are exact, on 32-bit integer
 *     multiply-adds, and each output is rounded once.  Error of an output
 *     y = sum_k x_k m_k: at most 2^-53 |y| + 2^-55 max|x_k| max|m_k|.
 *     Inputs must be finite; subnormals count as zero.
 *   - Two-target gates use the same block fixed point (eight terms per
 *     output, summed in two 64-bit accumulators of four terms): at most
 *     2^-53 |y| + 2^-54 max|x_k| max|m_k|.  So does a one-qubit unitary or
 *     Kraus map on a density matrix, applied as one two-target pass of
 *     conj(U) (x) U or of its superoperator on (t, t + N).
 *   - Dense gates with 3..5 targets (and two-target fused blocks) run on the
 *     bf16 tensor cores with eight
 *     exact 7-bit integer slices of 56-bit operands (rows and columns scaled
 *     by their largest exponent), exact FP32 level sums, one rounding.
 *   - Everything else (6-target dense gates, dephasing, superoperators,
 *     norm, trace, expectation values, partial traces) is native FP64.
 * QS_ARITH_DF: double-float.  Amplitudes are split into float pairs (47-bit
 *   significands) and combined with error-free FP32 transformations; dense
 *   gates use seven 7-bit slices (49 bits).  Relative error per operation: a
 *   few units of 2^-46 for moduli in [2^-80, 2^128).  Somewhat faster than FX
 *   on dense gates, but narrower than IEEE double.
 * QS_ARITH_F64: native FP64 throughout (FP64-pipe bound on GB300).
 * complex64 states ignore the setting. */
typedef enum { QS_ARITH_DF = 0, QS_ARITH_F64 = 1, QS_ARITH_FX = 2 } qs_arith;

/* Largest number of storage qubits (N for a statevector, 2N for a density
 * matrix): 2^34 complex64 amplitudes are 128 GiB. */
#define QS_MAX_STORAGE_QUBITS 34
/* Largest number of targets of a dense gate (the matrix is at most 64 x 64). */
#define QS_MAX_DENSE_TARGETS 6

/* Text of a status code (static storage). */
const char* qs_status_str(qs_status status);

/* Wrap caller-owned device memory d_amps (2^num_qubits amplitudes of the given
 * precision) as a statevector (Sec. "Local statevector algorithms").  The
 * contents are left as they are.  cuda_stream is a cudaStream_t or NULL. */
qs_status qs_create_statevector(int num_qubits, qs_prec prec, void* d_amps, void* cuda_stream,
                                qs_state** out);

/* Wrap caller-owned device memory d_amps (2^(2 num_qubits) amplitudes) as the
 * Choi vector of a num_qubits-qubit density matrix (Sec. "State
 * representation"). */
qs_status qs_create_densmatr(int num_qubits, qs_prec prec, void* d_amps, void* cuda_stream,
                             qs_state** out);

/* Release the handle and its library memory (waits for its queued work).  The
 * wrapped amplitude storage is not freed. */
qs_status qs_destroy(qs_state* state);

/* num_qubits: N; storage_qubits: N (statevector) or 2N (density matrix). */
qs_status qs_get_info(const qs_state* state, int* num_qubits, int* storage_qubits, int* is_density,
                      int* prec);

/* Select the complex128 arithmetic of this handle (default QS_ARITH_FX).
 * f64_share_16ths (0..16): with QS_ARITH_DF, the share of one-target-gate
 * work, in sixteenths, done in native FP64 at the same time (the FP64 pipe is
 * otherwise idle); 0 = none. */
qs_status qs_set_arithmetic(qs_state* state, qs_arith arith, int f64_share_16ths);

/* complex64 dense gates with 3..5 targets run on the tensor cores (tcgen05,
 * 3xTF32 with FP32 accumulation: FP32-level accuracy) unless disabled here
 * (enable = 0: CUDA-core FP32 kernels).  complex128 states ignore it. */
qs_status qs_set_tensor_cores(qs_state* state, int enable);

/* Device address of the wrapped amplitudes. */
qs_status qs_device_ptr(const qs_state* state, void** d_amps);

/* Copy count amplitudes from host memory (interleaved re, im in the state's
 * precision) into storage indices [first, first + count).  Queued on the
 * state's stream.  From page-locked host memory (pinned allocations or
 * registered ranges) a copy of at least 1 MiB whose host and device
 * addresses and size are multiples of 16 bytes is made by a kernel that
 * reads the buffer through its mapped device pointer; any other copy goes
 * through cudaMemcpyAsync (synchronous staging for pageable memory).  The
 * host buffer must stay valid and unchanged until the stream reaches the
 * copy.  QS_ERR_CUDA if the launch or copy fails. */
qs_status qs_set_amps(qs_state* state, const void* host_amps, size_t first, size_t count);

/* Copy storage indices [first, first + count) to host memory; synchronises. */
qs_status qs_get_amps(const qs_state* state, void* host_amps, size_t first, size_t count);

/* |0><0| or |0>: amplitude 0 set to 1, every other amplitude to 0. */
qs_status qs_init_zero(qs_state* state);

/* Pure-state initialisation of a density matrix (Sec. "State
 * representation"): beta_{j + k 2^N} = weight psi_j psi_k^*, written
 * (accumulate = 0) or added (accumulate = 1), so that a mixture
 * sum_m w_m |psi_m><psi_m| is built by repeated calls.  psi must be a
 * statevector handle of the same N and precision, on the same stream. */
qs_status qs_init_pure_densmatr(qs_state* rho, const qs_state* psi, double weight, int accumulate);

/* Many-control many-target dense gate (Sec. "Many-control one-target gate",
 * Sec. "Many-target gate", Eq. (local many-target amplitude update)):
 * alpha_{kj} -> sum_l m_{jl} alpha_{kl} on the amplitudes whose control bits
 * are all 1.  mat: 2^ntarg x 2^ntarg complex128, row-major, interleaved
 * (re, im) doubles.  1 <= ntarg <= QS_MAX_DENSE_TARGETS, nctrl >= 0; ctrls
 * may be NULL when nctrl = 0.  On a density matrix this applies
 * U rho U^dagger: U on (ctrls, targs), then U^* on the same qubits shifted by
 * N (Sec. "Unitary gates", Eq. (unitary on a vectorised density matrix));
 * without controls, one or two targets (one: in block fixed point; two: on
 * the tensor-core path) take one pass of conj(U) (x) U instead. */
qs_status qs_apply_ctrl_multi_target(qs_state* state, const int* ctrls, int nctrl, const int* targs,
                                     int ntarg, const double* mat);

/* SWAP of qubits t1 != t2 (Sec. "Swap gate"): alpha_i -> alpha_{i with bits
 * t1 and t2 flipped} where bits t1 and t2 of i differ; the rest unchanged.
 * Exact (amplitudes are moved, not computed).  Density matrix: SWAP on
 * (t1, t2), then on (t1 + N, t2 + N). */
qs_status qs_apply_swap(qs_state* state, int t1, int t2);

/* Diagonal operator on ntarg <= QS_MAX_DENSE_TARGETS targets:
 * alpha_i -> diag[j] alpha_i with j the value of the target bits of i (bit q
 * of j on targs[q]); diag: 2^ntarg complex128 (re, im).  The diagonal case of
 * Eq. (local many-target amplitude update); the phase gadget of Sec. "Phase
 * gadget" is one such.  Density matrix: D on targs, then D^* on targs + N. */
qs_status qs_apply_diagonal(qs_state* state, const int* targs, int ntarg, const double* diag);

/* Pauli gadget exp(-i theta P / 2), P = (x)_q paulis[q] on targs[q]
 * (Sec. "Pauli gadget": the paper's exp(i phi P) with phi = -theta/2).
 * n >= 0 targets, paulis[q] in 0..3.  With only Z (and I) factors it is the
 * phase gadget of Sec. "Phase gadget".  Density matrix: the gadget on targs,
 * then on targs + N with angle (-1)^(#Y + 1) theta (Algorithm "specific
 * unitaries on density matrices"). */
qs_status qs_apply_pauli_gadget(qs_state* state, const int* targs, const int* paulis, int n,
                                double theta);

/* Kraus map rho -> sum_m K_m rho K_m^dagger on n targets, 1 <= n <= 3
 * (Sec. "Kraus map"): the superoperator S = sum_m conj(K_m) (x) K_m is built
 * on the device and applied as a dense 2n-target gate on targs u targs + N
 * (for n = 1 in block fixed point its 16 entries are formed on the host with
 * the pass's fixed-point constants).
 * kraus: num_ops matrices of 2^n x 2^n complex128, each row-major (re, im).
 * Density matrices only. */
qs_status qs_apply_kraus(qs_state* state, const int* targs, int n, const double* kraus, int num_ops);

/* One-qubit dephasing (Sec. "Dephasing channel"): beta_i *= 1 - 2p where
 * bit t and bit t + N of i differ.  Density matrices only; p in [0, 1]. */
qs_status qs_apply_dephasing(qs_state* state, int t, double p);

/* Two-qubit dephasing (Sec. "Dephasing channel", two-qubit update rule):
 * beta_i *= 1 - 4p/3 where bit t1 != bit t1 + N or bit t2 != bit t2 + N. */
qs_status qs_apply_two_qubit_dephasing(qs_state* state, int t1, int t2, double p);

/* One-qubit depolarising (Sec. "Depolarising channel", Eq. (one-qubit
 * depolarising amplitude update)). */
qs_status qs_apply_depolarising(qs_state* state, int t, double p);

/* Two-qubit depolarising (Sec. "Depolarising channel", Eq. (two-qubit
 * depolarising Choi amplitude update)).  The equation is implemented; the
 * coefficients of the paper's listing for this channel disagree with it. */
qs_status qs_apply_two_qubit_depolarising(qs_state* state, int t1, int t2, double p);

/* Amplitude damping (Sec. "Damping channel", Eq. (damping amplitude
 * update)). */
qs_status qs_apply_damping(qs_state* state, int t, double p);

/* One-qubit Pauli channel, rho -> (1 - px - py - pz) rho + px X rho X
 * + py Y rho Y + pz Z rho Z on qubit t: the general form of the depolarising
 * channel (Sec. "Depolarising channel"; the paper notes the extension), and
 * dephasing at (0, 0, p).  On the Choi vector, where bits t and t + N agree,
 * beta_i -> (1 - px - py) beta_i + (px + py) beta_{i flip t, t+N}; where they
 * differ, beta_i -> (1 - px - py - 2 pz) beta_i + (px - py) beta_{i flip t, t+N}.
 * Density matrices only; each probability in [0, 1] (their sum is not
 * checked, as the paper checks no CPTP condition). */
qs_status qs_apply_pauli_channel(qs_state* state, int t, double px, double py, double pz);

/* Partial trace over n targets, 1 <= n < N (Sec. "Partial trace", Eqs.
 * (reduced amplitude definition) and (index function)):
 * beta'_i = sum_v beta_{g(i, v)}.  The input is not modified.  The result is a
 * NEW density-matrix handle of N - n qubits wrapping caller-owned device
 * memory d_out_amps (2^(2(N - n)) amplitudes, same precision, 256-byte
 * aligned), on the input's stream; the kept qubits keep their order. */
qs_status qs_partial_trace(const qs_state* in, const int* targs, int n, void* d_out_amps,
                           qs_state** out);

/* Expectation value of H = sum_n coeffs[n] P_n, paulis: num_terms x N codes,
 * row n for term n, entry q for qubit q (Sec. "Pauli string expectation
 * value").  Density matrix: Tr(H rho) = sum_i H_i beta_i, summed over the
 * entries where H_i is non-zero (column k, row k xor x_n of each term).
 * Statevector: <psi|H|psi>.  out[0] = real part (the expectation value),
 * out[1] = imaginary part (zero up to rounding for Hermitian rho).  The sum is
 * in FP64.  Synchronises. */
qs_status qs_expec_pauli_sum(const qs_state* state, const int* paulis, const double* coeffs,
                             int num_terms, double* out);

/* ------------------------------------------------------------------------
 * Circuits and gate fusion.  A circuit records unitary operations (the gates
 * above); a plan cuts it into blocks of consecutive gates that together touch
 * at most max_block_qubits (<= QS_MAX_DENSE_TARGETS) qubits.  Each block of
 * two or more gates is composed on the device into one dense matrix in FP64
 * and applied as a single dense gate (tensor cores for complex64 blocks of
 * 3..5 qubits, the handle's complex128 arithmetic otherwise); a one-gate block
 * runs that gate's own kernel.  Not in the paper: this groups the paper's
 * many-target gate updates (Sec. "Many-target gate") so that each pass over
 * the state does more work.  The applied operation is the same up to rounding.
 * ------------------------------------------------------------------------ */
typedef struct qs_circuit qs_circuit;

typedef enum {
  QS_PLAN_NONE = 0,    /* every gate its own block */
  QS_PLAN_GREEDY = 1,  /* extend each block while its qubits fit */
  QS_PLAN_COST = 2     /* minimum predicted time under a cost model (qs_circuit_plan_cost) */
} qs_plan_kind;

qs_status qs_circuit_create(int num_qubits, qs_circuit** out);
qs_status qs_circuit_destroy(qs_circuit* circuit);
/* Record a gate; the arguments are those of the qs_apply_* call of the same
 * operation (copied; validated now). */
qs_status qs_circuit_add_unitary(qs_circuit* circuit, const int* ctrls, int nctrl, const int* targs, int ntarg,
                                 const double* mat);
qs_status qs_circuit_add_diagonal(qs_circuit* circuit, const int* targs, int ntarg, const double* diag);
qs_status qs_circuit_add_pauli_gadget(qs_circuit* circuit, const int* targs, const int* paulis, int n,
                                      double theta);
/* Plan (QS_PLAN_NONE or QS_PLAN_GREEDY) and compose the fused blocks on the
 * current device; synchronous.  Recording more gates discards the plan. */
qs_status qs_circuit_plan(qs_circuit* circuit, int kind, int max_block_qubits);
qs_status qs_circuit_get_plan(const qs_circuit* circuit, int* num_gates, int* num_blocks, int* num_fused);
/* Apply the planned circuit to a state of the same number of qubits
 * (statevector, or density matrix: each block B then B^* on the shifted
 * qubits).  An unplanned circuit is applied gate by gate.  Queued on the
 * state's stream. */
qs_status qs_circuit_apply(qs_circuit* circuit, qs_state* state);

/* Apply a dense matrix on targs through the fused-block kernels (the path a
 * planned block takes), whatever the number of targets; used to time blocks
 * for the cost model.  Same arguments and semantics as
 * qs_apply_ctrl_multi_target without controls. */
qs_status qs_apply_dense_block(qs_state* state, const int* targs, int ntarg, const double* mat);

/* ------------------------------------------------------------------------
 * Learned cost model for fusion planning (not in the paper).  A perceptron
 * with two hidden layers of 64 units predicts log(milliseconds) of one kernel
 * launch from QS_COST_FEATURES features (qs_costmodel_encode).  It is trained
 * on the GPU by this library's forward, backward and Adam kernels, on timings
 * the simulator measures itself.  Plans only regroup gates, so the model never
 * changes a result.
 * ------------------------------------------------------------------------ */
typedef struct qs_costmodel qs_costmodel;
#define QS_COST_FEATURES 64
#define QS_COST_PARAMS 8385   /* W1 64x64, b1 64, W2 64x64, b2 64, W3 64, b3 */

typedef enum {
  QS_COST_FUSED_DENSE = 0,  /* a fused block (qs_apply_dense_block) of `width` qubits */
  QS_COST_GATE1 = 1,        /* a one-target gate with nctrl controls */
  QS_COST_DENSE = 2,        /* a dense gate of `width` targets with nctrl controls */
  QS_COST_DIAGONAL = 3,     /* a diagonal on `width` targets */
  QS_COST_GADGET = 4,       /* a Pauli gadget with X or Y factors, `weight` factors */
  QS_COST_PHASE = 5         /* a phase gadget (Z factors only) */
} qs_cost_kind;

/* New model with He-uniform random weights (splitmix64 stream of seed). */
qs_status qs_costmodel_create(unsigned long long seed, qs_costmodel** out);
qs_status qs_costmodel_destroy(qs_costmodel* model);
/* Flat float parameters, layout as in QS_COST_PARAMS; n must equal it. */
qs_status qs_costmodel_get_params(const qs_costmodel* model, float* host_params, int n);
qs_status qs_costmodel_set_params(qs_costmodel* model, const float* host_params, int n);
/* Features of one launch on `state` (its size, precision and settings). */
qs_status qs_costmodel_encode(int kind, int width, unsigned long long qmask, int nctrl, int weight,
                              const qs_state* state, float* out_features);
/* Predictions (log ms) for n feature rows (host arrays). */
qs_status qs_costmodel_predict(qs_costmodel* model, const float* features, int n, float* out);
/* Mean-squared-error loss and its gradient over n rows (one batch). */
qs_status qs_costmodel_gradient(qs_costmodel* model, const float* features, const float* targets, int n,
                                float* out_grad, float* out_loss);
/* Adam training on n rows (minibatches of `batch`, reshuffled every epoch by
 * a splitmix64 stream of seed); final_loss = MSE over all rows. */
qs_status qs_costmodel_train(qs_costmodel* model, const float* features, const float* targets, int n, int epochs,
                             int batch, float lr, unsigned long long seed, float* final_loss);
/* Plan a circuit for `state` by minimum predicted time: dynamic programming
 * over cut points, each candidate block (at most max_block_qubits qubits,
 * at most `window` gates) against running its gates unfused.  Composes the
 * chosen blocks like qs_circuit_plan. */
qs_status qs_circuit_plan_cost(qs_circuit* circuit, qs_costmodel* model, const qs_state* state,
                               int max_block_qubits, int window);

/* Lazy qubit relabelling of a planned circuit on statevectors (Sec. "Swap
 * gate", and the paper's reason for moving targets before a many-target
 * gate, here on one GPU).  The tensor-core kernels tile rows on the lowest
 * free qubits, so a block with qubits among the `low_qubits` lowest physical
 * positions gathers strided rows.  Walking the blocks in order, a block whose
 * qubits lie there has one of them swapped with the high position whose
 * qubit the tensor-core blocks need last, whenever the cost model predicts
 * the block's saving to exceed the price of a SWAP pass, swap_passes times
 * the predicted time of a one-target pass (a SWAP moves half the state, but
 * on a low qubit touches every sector: about 1.2).  qs_circuit_apply then applies
 * those SWAPs (qs_apply_swap) and the blocks on the moved positions, and ends
 * with the SWAPs back to the identity layout: the result is the same up to
 * rounding.  low_qubits = 0 clears the relabelling; density matrices ignore
 * it.  Replanning clears it. */
qs_status qs_circuit_plan_relabel(qs_circuit* circuit, qs_costmodel* model, const qs_state* state, int low_qubits,
                                  double swap_passes);
/* SWAP passes the relabelling adds (0 when none). */
qs_status qs_circuit_get_relabel(const qs_circuit* circuit, int* num_swaps);

/* ------------------------------------------------------------------------
 * Batched engine (not in the paper): many independent states of at most 24
 * storage qubits (statevectors, or density matrices of at most 12 qubits as
 * Choi vectors), each with its own circuit of dense gates (1 or 2 targets,
 * up to 5 controls), diagonals (up to 3 targets), Pauli gadgets and, on
 * density matrices, Kraus maps and the decoherence channels, run by ONE
 * persistent kernel launch recorded in a CUDA graph.  CTAs take states from
 * a work counter, largest first; a state that fits in shared memory is
 * processed there, a larger one tile by tile.  complex64 in FP32, complex128
 * in double-float arithmetic (see qs_arith).  The semantics are those of the
 * single-state calls of the same names (qs_apply_ctrl_multi_target, ...,
 * qs_apply_damping); on a density matrix a unitary, diagonal or gadget is
 * applied as U on t and U* on t + N, a Kraus map or channel as one pass of
 * its superoperator on (t, t + N) or (t1, t2, t1 + N, t2 + N).
 * ------------------------------------------------------------------------ */
typedef struct qs_batch qs_batch;

/* Statevectors only: num_qubits[s] in 1..24 for every state s; all states
 * share `prec` and the stream. */
qs_status qs_batch_create(int num_states, const int* num_qubits, qs_prec prec, void* cuda_stream, qs_batch** out);
/* is_density[s] != 0: state s is an num_qubits[s]-qubit density matrix held
 * as a 2 num_qubits[s]-qubit Choi vector (is_density NULL: all
 * statevectors).  Storage qubits at most 24. */
qs_status qs_batch_create_mixed(int num_states, const int* num_qubits, const int* is_density, qs_prec prec,
                                void* cuda_stream, qs_batch** out);
qs_status qs_batch_destroy(qs_batch* batch);
/* Amplitudes the caller's device pool must hold, and where state s starts
 * (each state starts on a 256-byte boundary). */
qs_status qs_batch_pool_amps(const qs_batch* batch, size_t* num_amps);
qs_status qs_batch_state_offset(const qs_batch* batch, int state, size_t* offset_amps);
/* Caller-owned device memory (256-byte aligned) holding every state. */
qs_status qs_batch_bind_pool(qs_batch* batch, void* d_pool);
qs_status qs_batch_add_unitary(qs_batch* batch, int state, const int* ctrls, int nctrl, const int* targs, int ntarg,
                               const double* mat);
qs_status qs_batch_add_diagonal(qs_batch* batch, int state, const int* targs, int ntarg, const double* diag);
qs_status qs_batch_add_pauli_gadget(qs_batch* batch, int state, const int* targs, const int* paulis, int n,
                                    double theta);
/* Density-matrix states only (QS_ERR_NOT_DENSMATR otherwise): a Kraus map of
 * num_ops operators on n = 1 or 2 targets (as qs_apply_kraus), and the
 * channels of qs_apply_dephasing, qs_apply_two_qubit_dephasing,
 * qs_apply_depolarising, qs_apply_two_qubit_depolarising, qs_apply_damping
 * and qs_apply_pauli_channel (probabilities in [0, 1]). */
qs_status qs_batch_add_kraus(qs_batch* batch, int state, const int* targs, int n, const double* kraus, int num_ops);
qs_status qs_batch_add_dephasing(qs_batch* batch, int state, int t, double p);
qs_status qs_batch_add_two_qubit_dephasing(qs_batch* batch, int state, int t1, int t2, double p);
qs_status qs_batch_add_depolarising(qs_batch* batch, int state, int t, double p);
qs_status qs_batch_add_two_qubit_depolarising(qs_batch* batch, int state, int t1, int t2, double p);
qs_status qs_batch_add_damping(qs_batch* batch, int state, int t, double p);
qs_status qs_batch_add_pauli_channel(qs_batch* batch, int state, int t, double px, double py, double pz);
/* Upload the programs and record the launch in a CUDA graph.  With
 * autotune != 0 every candidate launch shape is timed by running the whole
 * batch once on the bound pool: the pool's contents are unspecified
 * afterwards, so write the initial states after compiling.  Synchronous. */
qs_status qs_batch_compile(qs_batch* batch, int autotune);
/* Replay the recorded launch on the batch's stream (asynchronous). */
qs_status qs_batch_run(qs_batch* batch);
qs_status qs_batch_info(const qs_batch* batch, int* threads, int* ctas, int* smem_qubits, long* total_ops);

/* ---------------------------------------------------------------------------
 * Test hooks (not in the paper).  Failures are made on the host, never on
 * the GPU.
 * ------------------------------------------------------------------------ */

/* Make library allocations fail: after this call the next `skip` device or
 * pinned-host allocations the library makes for itself (handle scratch and
 * staging ring, recorded-program arenas, circuit matrices, batch tables)
 * succeed and the `count` after them fail as if out of memory, without
 * calling CUDA.  The caller then returns QS_ERR_OOM having freed what it had
 * taken.  count = 0 turns the injection off.  Process-wide; QS_ERR_ARG for
 * negative arguments. */
qs_status qs_test_fail_allocations(int skip, int count);

/* Set the handle's device error word, as a tensor-core kernel does when one
 * of its bounded waits runs out, so that the next qs_synchronize reports
 * QS_ERR_TIMEOUT (once) and clears it.  Synchronises the stream. */
qs_status qs_test_set_error_word(qs_state* state);

/* Run the bounded-wait path on the GPU: one thread waits on a barrier that
 * nothing arrives at, gives up after `polls` polls (at most 2^20), and sets
 * the handle's error word as a tensor-core kernel does when its wait runs
 * out.  Queued on the handle's stream; the next qs_synchronize reports
 * QS_ERR_TIMEOUT once.  Nothing faults or hangs. */
qs_status qs_test_bounded_wait(qs_state* state, unsigned polls);

/* Largest number of terms qs_expec_pauli_sum_noalloc accepts. */
#define QS_NOALLOC_MAX_TERMS 256

/* The expectation value of qs_expec_pauli_sum, for callers that cannot
 * allocate GPU memory: it takes a raw device pointer instead of a handle
 * (creating a handle allocates scratch and a pinned ring) and allocates
 * nothing, not even the scratch its reduction needs.  The paper has no
 * counterpart; this is a deployment variant of the same computation.
 *
 * d_amps: 2^num_qubits amplitudes (statevector) or 2^(2 num_qubits) (Choi
 * vector, is_density = 1) of precision prec, 256-byte aligned, read only.
 * paulis, coeffs, out: as for qs_expec_pauli_sum; out is host memory.
 * num_terms must be 1..QS_NOALLOC_MAX_TERMS; more returns QS_ERR_ARG.
 *
 * Scratch: a fixed array of about 28 KB in the library's device image (term
 * list, one partial sum per reduction block, the result), held by every GPU
 * that loads the library until the process exits.  The first call on a device
 * looks up that array's device address, so make the first call on each device
 * before capturing any stream.  All calls share the array: calls that overlap
 * on the GPU (other streams, other host threads) race and must be serialised
 * by the caller.  complex128 products and sums are native FP64, as with the
 * default arithmetic of a handle.  Synchronises cuda_stream. */
qs_status qs_expec_pauli_sum_noalloc(const void* d_amps, int num_qubits, int is_density, qs_prec prec,
                                     const int* paulis, const double* coeffs, int num_terms,
                                     void* cuda_stream, double* out);

/* Statevector: out[0] = sum_i |alpha_i|^2, out[1] = 0.  Density matrix:
 * out = Tr rho = sum_j beta_{j (2^N + 1)} (re, im).  FP64 sum.  Synchronises. */
qs_status qs_calc_norm_or_trace(const qs_state* state, double* out);

/* Wait for all work queued on the state's stream.  Returns QS_ERR_TIMEOUT
 * (once) if a kernel's bounded wait ran out since the last check; the state's
 * amplitudes are then unspecified. */
qs_status qs_synchronize(const qs_state* state);

/* ---------------------------------------------------------------------------
 * Recorded programs (not in the paper): the operations applied to one state
 * between qs_record_begin and qs_record_end are captured as a CUDA graph on the
 * state's stream and replayed with one launch by qs_program_run, which removes
 * the per-call host work (validation, staging, one launch per kernel) that
 * bounds small states.
 * - While recording, operation calls (gates, diagonals, gadgets, SWAP, Kraus
 *   maps, channels, dense blocks, planned circuits) validate their arguments as
 *   usual but launch nothing; their matrices and Kraus operators are copied to
 *   device memory owned by the program.  Calls that read results or
 *   synchronise (amplitude copies, norms, expectation values, partial traces,
 *   qs_synchronize, qs_destroy) return QS_ERR_ARG while recording.
 * - The state must use a stream other than the legacy default stream
 *   (QS_ERR_ARG otherwise).  One recording per state at a time.
 * - qs_program_run queues one replay on the state's stream (asynchronous); a
 *   replay applies the recorded operations to the state's current amplitudes.
 * - The program must be destroyed before its state, and before any planned
 *   circuit whose qs_circuit_apply it recorded (the fused blocks' matrices stay
 *   in the circuit's device memory); qs_program_destroy waits for the state's
 *   stream.
 * ------------------------------------------------------------------------- */
typedef struct qs_program qs_program;
qs_status qs_record_begin(qs_state* state);
/* Ends the recording; *out receives the program (NULL on error). */
qs_status qs_record_end(qs_state* state, qs_program** out);
qs_status qs_program_run(qs_program* program);
qs_status qs_program_destroy(qs_program* program);

#ifdef __cplusplus
}
#endif

#endif /* QS_H */
