/*
 * tqs.h - C ABI of the GB300 (sm_103a) unitary-matrix quantum circuit
 * simulator.
 *
 * Model (TornadoQSim, arXiv 2305.14398):
 *   - a circuit of n qubits records operations through gate calls; steps are
 *     created as operations are added (Sec. 5.2, circuit model);
 *   - each step's 2^n x 2^n unitary is the Kronecker product of the step's
 *     gate matrices, identity on idle qubits (Algorithm 2, eq. 9s1), with a
 *     controlled gate written as the projector sum
 *     |0><0|_c (x) I_t + |1><1|_c (x) U_t (eq. 7);
 *   - the state evolves as psi <- S_k psi (eq. 11); the circuit unitary is
 *     the chain U <- S_k U (Algorithm 1);
 *   - simulateFullState returns the state; probabilities |psi_i|^2 give the
 *     measurement statistics (Sec. 5.2, Simulator interface).
 *
 * Conventions shared by every call:
 *   - Qubit q is bit q of an amplitude index (little-endian).  A state is
 *     2^n interleaved complex64 values (tqs_c64) in index order.
 *   - Controlled gates take qubits {control, target}.
 *   - Pointers named d_* are DEVICE pointers (cudaMalloc'd or from a CUDA
 *     caching allocator) owned by the caller; pointers named h_* are host
 *     pointers owned by the caller.  The library never frees caller memory.
 *   - Device buffers passed in must be 16-byte aligned (any cudaMalloc or
 *     torch allocation is); a misaligned pointer returns TQS_ERR_ARG.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued on it and the call returns without
 *     synchronising unless stated.  Library-internal scratch (programs,
 *     step tables, operand planes, partial sums) is allocated with
 *     cudaMalloc by the first call that needs it, cached on its handle (or,
 *     for calls without a handle, per host thread), and freed by the
 *     handle's destroy call (cudaFree waits for the device).  Make that
 *     first call outside any stream capture.
 *   - Every call returns a tqs_status; no exception crosses the ABI.  On
 *     error, tqs_last_error() returns a message for the calling thread.
 *     Argument errors are detected before any device work is enqueued.
 *     Asynchronous CUDA errors surface as TQS_ERR_CUDA from a later call.
 */
#ifndef TQS_ABI_H_
#define TQS_ABI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { float re, im; } tqs_c64;

typedef struct tqs_circuit tqs_circuit;
typedef struct tqs_batch tqs_batch;

typedef enum {
  TQS_OK = 0,
  TQS_ERR_ARG = 1,              /* NULL pointer, bad count, bad gate id, bad params */
  TQS_ERR_QUBIT_RANGE = 2,      /* qubit index outside [0, n) */
  TQS_ERR_QUBIT_DUP = 3,        /* the same qubit twice in one gate */
  TQS_ERR_TOO_MANY_QUBITS = 4,  /* n above the call's limit */
  TQS_ERR_NOMEM = 5,            /* host or device allocation failed */
  TQS_ERR_BUDGET = 6,           /* request does not fit the given memory budget */
  TQS_ERR_CUDA = 7,             /* a CUDA runtime call failed */
  TQS_ERR_TIMEOUT = 8,          /* a bounded device wait ran out */
  TQS_ERR_STATE = 9,            /* object used in the wrong state */
  TQS_ERR_UNSUPPORTED = 10      /* valid request this build does not implement */
} tqs_status;

/* Gate kinds.  Table 1 (Sec. 2.3): H, X, Y, Z, R (phase shift R_phi,
 * params {phi}).  Sec. 5.2 names S and T (S = R_{pi/2}, T = R_{pi/4}).
 * RX, RY, RZ (params {theta}) and U3 (params {theta, phi, lambda}) use the
 * textbook definitions.  Controlled gates (eq. 7, qubits {control, target}):
 * CNOT (eq. 8), CZ, CP (params {phi}) and CU (params: 8 doubles, re/im of
 * u00, u01, u10, u11; must be unitary to 1e-9).  SWAP (qubits {a, b})
 * appears in the QFT circuit of Sec. 2.5.
 * Instructions (Sec. 5.2, operation interface; one qubit, no params):
 * TQS_MEASURE measures the qubit (projective, the state renormalised);
 * TQS_RESET measures it and, on outcome 1, flips it back to |0>.  Each takes
 * one caller-supplied uniform u in [0, 1): with S_0 the probability mass of the
 * indices whose bit is 0 and T the total, the outcome is 0 iff u * T < S_0 (FP64,
 * summed in a fixed order).  An instruction is a barrier: it forms a step of its
 * own, after every earlier operation and before every later one.  Circuits with
 * instructions run through tqs_simulate_measured / tqs_batch_run_measured; the
 * unitary forms (tqs_simulate, tqs_simulate_plain, tqs_circuit_unitary, the
 * server) return TQS_ERR_UNSUPPORTED for them. */
typedef enum {
  TQS_H = 0, TQS_X = 1, TQS_Y = 2, TQS_Z = 3, TQS_S = 4, TQS_T = 5, TQS_R = 6,
  TQS_RX = 7, TQS_RY = 8, TQS_RZ = 9, TQS_U3 = 10,
  TQS_CNOT = 11, TQS_CZ = 12, TQS_CP = 13, TQS_CU = 14, TQS_SWAP = 15,
  TQS_MEASURE = 16, TQS_RESET = 17,
  TQS_GATE_COUNT = 18
} tqs_gate;

/* Arithmetic of the circuit-unitary chain (Algorithm 1). */
typedef enum {
  TQS_PREC_FP32_SIMT = 0,   /* FP32 CUDA-core complex GEMM (4 real products) */
  TQS_PREC_TC_BF16X3 = 1,   /* tcgen05 tensor cores, 3M complex product, each real
                               product as BF16 hi*hi + hi*lo + lo*hi, FP32 accumulate */
  TQS_PREC_TC_TF32X3 = 2    /* as above with TF32 hi/lo splits (kind::tf32) */
} tqs_prec;

#define TQS_MAX_QUBITS 16          /* fused state-vector calls, batches, server */
#define TQS_MAX_FSV_QUBITS 34      /* circuits; tqs_simulate_fsv (2^34 x 8 B = 128 GiB) */
#define TQS_MAX_DENSE_QUBITS 14    /* calls that hold a 2^n x 2^n matrix */

/* ------------------------------------------------------------------ circuit
 * Sec. 5.2 (circuit model): create a circuit of n qubits, add operations
 * through gate calls, which check each operation's preconditions; steps
 * are created as operations are added ("as soon as possible": an operation
 * joins the step after the last step that touches one of its qubits). */

/* Create an empty circuit of 1 <= n_qubits <= TQS_MAX_FSV_QUBITS qubits.
 * *out receives the handle (owned by the caller until tqs_circuit_destroy).
 * Calls other than tqs_simulate_fsv need n <= TQS_MAX_QUBITS (the dense-matrix
 * forms n <= TQS_MAX_DENSE_QUBITS) and return TQS_ERR_TOO_MANY_QUBITS above. */
tqs_status tqs_circuit_create(int n_qubits, tqs_circuit** out);

/* Destroy a circuit and any device memory it caches.  NULL is accepted. */
tqs_status tqs_circuit_destroy(tqs_circuit* c);

/* Append one gate.  qubits: nq = 1 (single-qubit gates) or 2 (controlled
 * gates: {control, target}; SWAP: {a, b}).  params: np doubles as listed
 * under tqs_gate (np may exceed the need; extra values are ignored; params
 * may be NULL when the gate takes none).  Errors: TQS_ERR_ARG,
 * TQS_ERR_QUBIT_RANGE, TQS_ERR_QUBIT_DUP.  On error the circuit is unchanged. */
tqs_status tqs_add_gate(tqs_circuit* c, int gate, const int* qubits, int nq,
                        const double* params, int np);

/* Custom unitaries (Sec. 5.2, operation interface: the data of a custom
 * function is registered with the operation data provider under a unique
 * name, then applied to qubits; insertion checks that data of the right
 * format and size was registered).
 * tqs_register_unitary: m holds the 2^k x 2^k matrix row-major as interleaved
 * (re, im) doubles (2 * 4^k of them), 1 <= k <= 5; it must be unitary to 1e-9
 * (every entry of M^dagger M - I).  The registry is process-wide and
 * thread-safe; registering a name again replaces its data for circuits built
 * afterwards (circuits keep the data they were built with).  The matrix is
 * copied.  Errors: TQS_ERR_ARG. */
tqs_status tqs_register_unitary(const char* name, int k, const double* m);

/* Append the registered unitary `name` on qubits[0..k): bit t of the matrix's
 * local row / column index is the bit of qubit qubits[t] (little-endian, as
 * for the state).  k must equal the registered size.  Like every operation
 * it joins the step after the last step touching one of its qubits.  Errors:
 * TQS_ERR_ARG (no such name, k mismatch), TQS_ERR_QUBIT_RANGE,
 * TQS_ERR_QUBIT_DUP.  Circuits with custom unitaries run in every form
 * (fused, plain, circuit unitary, batches built from handles); the packed
 * batch and server formats have no custom kind. */
tqs_status tqs_add_custom(tqs_circuit* c, const char* name, const int* qubits, int k);

/* Sizes of the circuit: qubits, gates, and steps of the step table. */
tqs_status tqs_circuit_info(const tqs_circuit* c, int* n_qubits, int* n_gates, int* n_steps);

/* Step table (Sec. 5.3 stages 1-3): h_step_of_gate[g] receives the step index
 * of gate g (n_gates ints, host memory). */
tqs_status tqs_circuit_steps(const tqs_circuit* c, int* h_step_of_gate);

/* Inspection of the fused step program that tqs_simulate runs (for tests
 * of the host compiler and for tools).  The circuit's steps are compiled
 * into passes; a pass names 4 "local" physical qubit bits, and each of its
 * ops applies one step factor to the amplitudes in registers.
 *   *n_passes, *n_ops : receive the sizes (may be NULL).
 *   h_passes : NULL or n_passes records of 16 bytes:
 *              {uint8 L[4]; uint32 op_begin; uint32 op_count; float scale}
 *              (scale: exact power of two applied at the end of the pass)
 *   h_ops    : NULL or n_ops records of 80 bytes:
 *              {uint8 code, t, c, tbit, d0one, fbit; uint16 act;
 *               uint32 pad[2]; float m[8] (4 complex entries); float lo[8]
 *               (their FP32 rounding residues, dense ops)}.  code: 0-3
 *               Hadamard without its 2^-1/2, 4-7 X, 8-11 X under a far
 *               control, 12-27 X under a local control (12 + 4 t + c), 28-31
 *               anti-diagonal, 32-35 dense, 36-39 controlled dense, each + the
 *               local target position t; diagonal: 40-43 local target, 44-47
 *               local target + far control, 48-51 far target + local control
 *               c, 52 far target, 53 both local (fields t, c).  fbit: far
 *               control bit (255 none); tbit: far target bit; act: active-pair
 *               mask over the 16 local indices; d0one: d0 == 1 exactly.
 *   h_map    : NULL or 17 uint16, the output map: logical index y of the
 *              result is the program's physical index h_map[16] ^ (XOR of
 *              h_map[q] over the set bits q of y), an affine map over GF(2)
 *              (SWAP factors relabel qubits; the trailing permutation gates
 *              X, CNOT, SWAP with no later other gate on their qubits are
 *              folded into it instead of being applied).
 *   h_out_scale : NULL or 1 float, the factor applied to the output state.
 *   h_gen_index : NULL or 1 int, the basis state the program starts from
 *              (leading X gates on untouched qubits are folded into it; the
 *              program for a given input state folds nothing).
 * Host memory only; no device work. */
tqs_status tqs_circuit_program(tqs_circuit* c, int* n_passes, int* n_ops, void* h_passes,
                               void* h_ops, uint16_t* h_map, float* h_out_scale,
                               int* h_gen_index);

/* ---------------------------------------------------------------- simulate
 * simulateFullState (Sec. 5.2): the final state psi = S_m ... S_1 psi_0.
 * Each step is applied by the fused step kernel, which generates the step
 * unitary from its Kronecker factors in registers instead of reading a
 * materialised matrix.
 *   d_init  : 2^n tqs_c64 initial state, or NULL for |0...0>.
 *   d_out   : 2^n tqs_c64, receives the final state (must not alias d_init).
 *   d_probs : 2^n doubles, receives |psi_i|^2 (FP32 arithmetic, or exact
 *             in FP64 under TQS_OPT_EXACT_PROBS), or NULL.
 *   d_norm  : 1 double, receives sum_i |psi_i|^2 (FP64), or NULL.
 * n <= TQS_MAX_QUBITS.  Arithmetic: FP32 amplitudes, probabilities stored as
 * FP64, FP64 norm.  The circuit's device program is uploaded on the first
 * call and kept until the circuit or the d_init pointer changes; a 15-16
 * qubit circuit runs on several cooperating CTAs
 * (TQS_OPT_MULTI_CTAS).  A circuit handle is used by one stream at a time. */
tqs_status tqs_simulate(tqs_circuit* c, const tqs_c64* d_init, tqs_c64* d_out,
                        double* d_probs, double* d_norm, void* stream);

/* The same result by the plain materialised form (Sec. 5.3 stages 4 and 6,
 * applied per step): for each step, S_k is written to device scratch as a
 * dense 2^n x 2^n complex64 matrix (Algorithm 2) and psi <- S_k psi is a
 * dense matrix-vector product.  n <= TQS_MAX_DENSE_QUBITS.  Scratch:
 * 8 * 4^n + 16 * 2^n bytes, cached on the circuit. */
tqs_status tqs_simulate_plain(tqs_circuit* c, const tqs_c64* d_init, tqs_c64* d_out,
                              void* stream);

/* Algorithm 2 alone: write step `step` (0-based) of the circuit as a dense
 * row-major matrix, d_S[r * 2^n + c] = <r|S|c>.  n <= TQS_MAX_DENSE_QUBITS. */
tqs_status tqs_materialize_step(tqs_circuit* c, int step, tqs_c64* d_S, void* stream);

/* ----------------------------------------------------------------- unitary
 * Algorithm 1: the circuit unitary U = S_m ... S_1 as a chain of complex
 * matrix products U <- S_k U (the product with the initial identity is
 * skipped), in the arithmetic `prec` (tqs_prec).
 *   d_U : 2^n x 2^n tqs_c64, row-major, d_U[r * 2^n + c] = <r|U|c>.
 * n <= TQS_MAX_DENSE_QUBITS; tensor-core precisions need n >= 7.
 * Scratch (cached on the circuit): 36 * 4^n bytes for TQS_PREC_TC_BF16X3
 * (three matrices of six BF16 planes), 72 * 4^n for TQS_PREC_TC_TF32X3 (FP32
 * words), 24 * 4^n for TQS_PREC_FP32_SIMT.
 * The tensor-core form synchronises `stream` before returning and returns
 * TQS_ERR_TIMEOUT if one of its bounded device waits ran out. */
tqs_status tqs_circuit_unitary(tqs_circuit* c, int prec, tqs_c64* d_U, void* stream);

/* A block of columns of the circuit unitary, U[:, col0 : col0 + ncols], by the
 * same chain (Algorithm 1).  Column j of U is the circuit applied to |j>, and
 * U <- S_k U acts on each column alone, so a column block needs only its own
 * columns and the step unitaries, which every caller generates from the step
 * table: blocks on different GPUs need no communication (the column-sharded
 * chain), and blocks computed separately are bitwise the columns of the whole
 * tqs_circuit_unitary result in the same precision.
 *   d_U : 2^n rows of ncols tqs_c64, d_U[r * ldu + j] = <r|U|col0 + j>,
 *         ldu >= ncols (ldu = 2^n with d_U pointing at column col0 of a full
 *         row-major U fills that block of it).
 * Limits as tqs_circuit_unitary; for n >= 7, col0 and ncols must be multiples
 * of 128 (the tensor-core tile), else TQS_ERR_ARG; a block outside the 2^n
 * columns is TQS_ERR_ARG.  Scratch (cached on the circuit): the step matrix's
 * operands plus two ncols x 2^n chain matrices (BF16x3: 12 * 4^n +
 * 24 * ncols * 2^n bytes; TF32x3 twice that; FP32 SIMT: 8 * 4^n +
 * 16 * ncols * 2^n). */
tqs_status tqs_circuit_unitary_cols(tqs_circuit* c, int prec, int col0, int ncols, tqs_c64* d_U,
                                    int64_t ldu, void* stream);

/* ----------------------------------------------------- full state vector
 * The per-gate state-vector update of Appendix A (eq. 12; the paper's future
 * work) for states held in HBM, up to TQS_MAX_FSV_QUBITS qubits: d_state
 * (2^n tqs_c64, in place, 16-byte aligned; the caller initialises it) goes
 * through the circuit's gates in the order they were added.  Gates are
 * grouped into passes; each pass is one launch that streams the state
 * through shared memory in tiles of 2^13 amplitudes from 24 qubits on, 2^12
 * below (the 5 lowest qubits plus up to 8, or 7, more that the pass's gates
 * act on non-diagonally; controls and diagonal gates may sit on any qubit),
 * so the state crosses HBM twice per pass.  Custom unitaries are supported; measure/reset instructions return
 * TQS_ERR_UNSUPPORTED.  Scratch (cached on the circuit): the pass program.
 * FP32 amplitudes, FP32 hi + lo coefficients. */
tqs_status tqs_simulate_fsv(tqs_circuit* c, tqs_c64* d_state, void* stream);

/* Pass count and tile bits of the circuit's full-state-vector program (host
 * only; either output may be NULL). */
tqs_status tqs_fsv_passes(tqs_circuit* c, int* n_passes, int* tile_bits);

/* ---------------------------------------------------------- probabilities
 * p_i = |psi_i|^2 in FP64 (the products of the FP32 parts are exact in
 * FP64) and their FP64 sum, summed in a fixed order (deterministic).
 *   d_state : 2^n tqs_c64;  d_probs : 2^n doubles or NULL;
 *   d_sum   : 1 double or NULL.  1 <= n <= 30.
 * Scratch: one double per reduction block. */
tqs_status tqs_probabilities(const tqs_c64* d_state, int n, double* d_probs,
                             double* d_sum, void* stream);

/* Allocation-free form of tqs_probabilities, for callers that cannot call
 * cudaMalloc: for example a host framework that hands out all device memory
 * from its own pre-sized pool and forbids any other allocation, or a
 * latency-critical loop that cannot afford cudaMalloc/cudaFree, which may
 * synchronise the device.  The paper has no counterpart; it is a deployment
 * convenience.  Same arguments, results and determinism as tqs_probabilities.
 *   - Scratch: the per-block partial sums live in one fixed device array of
 *     1024 doubles (8 KiB) that every GPU loading the library holds until the
 *     process exits; it holds the partial sums of every allowed n.
 *     1 <= n <= 30, as for tqs_probabilities; other n return
 *     TQS_ERR_TOO_MANY_QUBITS.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and caches it; make
 *     that first call before any stream capture.  The cached address is that
 *     of the device's primary context (the CUDA runtime's): do not call after
 *     cudaDeviceReset, or with another context of the same device current.
 *     No call allocates or frees device memory.
 *   - Every call on a GPU shares that GPU's copy of the array.  Each call
 *     overwrites all the partial sums it reads, so nothing carries over
 *     between calls, but calls that overlap on the same GPU (for example on
 *     two streams) race on it: serialise them. */
tqs_status tqs_probabilities_noalloc(const tqs_c64* d_state, int n, double* d_probs,
                                     double* d_sum, void* stream);

/* Marginal probability that every qubit set in `mask` reads 0:
 * sum of |psi_i|^2 over i with (i & mask) == 0, FP64, deterministic
 * (Deutsch-Jozsa input register, Sec. 2.5).  d_out: 1 double. */
tqs_status tqs_marginal_zero(const tqs_c64* d_state, int n, uint64_t mask,
                             double* d_out, void* stream);

/* Simulate a circuit that may hold TQS_MEASURE / TQS_RESET instructions
 * (fused form; arguments as tqs_simulate, plus):
 *   d_u        : one uniform in [0, 1) per instruction, in the order the
 *                instructions were added (may be NULL if there are none);
 *   d_outcomes : one int32 outcome (0 or 1) per instruction, same order
 *                (may be NULL).
 * With no instruction this is tqs_simulate. */
tqs_status tqs_simulate_measured(tqs_circuit* c, const tqs_c64* d_init, tqs_c64* d_out,
                                 double* d_probs, double* d_norm, const double* d_u,
                                 int32_t* d_outcomes, void* stream);

/* ---------------------------------------------------------------- collapse
 * simulateAndCollapse (Sec. 5.2): the state collapses to one basis state
 * drawn with the probabilities p_i = |psi_i|^2 (Sec. 2.1, eq. 2).  Random
 * numbers are inputs: each shot takes one uniform u in [0, 1) from the caller.
 * A shot picks, by inverse CDF, the first index i with p_i > 0 and
 * u * T < C_i, where C_i = p_0 + ... + p_i and T = C_{2^n - 1}, summed in FP64
 * in the library's fixed order (blocks of 256 entries, chunks of 8 entries
 * added in index order, an exclusive warp scan over the 32 chunks of a block,
 * then an exclusive prefix over the blocks); if rounding leaves no such index,
 * the last index before that point with p_i > 0; -1 when every p_i is 0.
 * Results are deterministic; an index whose p_i is 0 is never
 * returned.  The probabilities need not sum to 1. */

/* `shots` samples from one probability vector:
 *   d_probs : 2^n doubles (for example from tqs_probabilities);
 *   d_u     : `shots` doubles in [0, 1);  d_out : `shots` int64 indices.
 * 1 <= n <= 30, shots >= 0.  Scratch (per host thread, cached): 34 doubles
 * per 256 probabilities plus a few hundred bytes. */
tqs_status tqs_sample(const double* d_probs, int n, int64_t shots, const double* d_u,
                      int64_t* d_out, void* stream);

/* simulateAndCollapse for one circuit: simulate it from |0...0> (fused form),
 * draw one outcome with d_u[0], write its index to d_index[0] (int64) and,
 * if d_state is not NULL, the collapsed state |index> (2^n tqs_c64) there.
 * Scratch (cached on the circuit): the state and its probabilities. */
tqs_status tqs_simulate_and_collapse(tqs_circuit* c, const double* d_u, int64_t* d_index,
                                     tqs_c64* d_state, void* stream);

/* ------------------------------------------------------------------- batch
 * Many circuits of uneven size and depth simulated by one graph launch of
 * the persistent fused step kernels.  The batch copies what it needs from
 * the circuits at creation; they may be destroyed afterwards.
 * Output layout: circuit i's state occupies amplitudes
 * [offsets[i], offsets[i+1]) of d_states (and the same range of d_probs);
 * d_norms[i] receives its probability sum. */

/* Create a batch from `count` circuit handles (each n <= TQS_MAX_QUBITS). */
tqs_status tqs_batch_create(tqs_circuit* const* cs, int count, tqs_batch** out);

/* Create a batch straight from host gate arrays (no circuit handles):
 *   h_nq[count]         qubit count of each circuit
 *   h_gate_off[count+1] gate range of circuit i: [h_gate_off[i], h_gate_off[i+1])
 *   h_kind[G]           tqs_gate of each gate
 *   h_qubits[2*G]       qubits of each gate (second ignored for 1-qubit gates)
 *   h_params[8*G]       parameters of each gate, 8 slots per gate
 * Preconditions are checked as in tqs_add_gate. */
tqs_status tqs_batch_create_packed(int count, const int32_t* h_nq, const int64_t* h_gate_off,
                                   const int32_t* h_kind, const int32_t* h_qubits,
                                   const double* h_params, tqs_batch** out);

/* Sizes of a batch (each output may be NULL): number of circuits, total
 * amplitudes, total steps of the step tables (ASAP packing), bytes of the
 * device program the kernels read, and h_offsets (count+1 int64) the
 * amplitude offsets of the circuits. */
tqs_status tqs_batch_info(const tqs_batch* b, int* count, int64_t* total_amps,
                          int64_t* total_steps, int64_t* program_bytes, int64_t* h_offsets);

/* Run the batch on `stream`: d_states (total_amps tqs_c64), d_probs
 * (total_amps doubles or NULL), d_norms (count doubles or NULL).  The first
 * run uploads the batch program (cached) and, with use_graph != 0, captures
 * the launches into a CUDA graph that later runs with the same pointers
 * replay. */
tqs_status tqs_batch_run(tqs_batch* b, tqs_c64* d_states, double* d_probs, double* d_norms,
                         int use_graph, void* stream);

/* `shots` samples per circuit of a batch from its probabilities (the
 * d_probs a tqs_batch_run wrote, same layout):  d_u : count * shots uniforms,
 * circuit i's shot k at i * shots + k;  d_out : count * shots int64 indices
 * within circuit i's state, same layout.  Same rule as tqs_sample.  Scratch
 * (cached on the batch): 34 doubles per 256 amplitudes of the circuits with
 * n > 13 plus 32 bytes per circuit. */
tqs_status tqs_batch_sample(tqs_batch* b, const double* d_probs, int shots, const double* d_u,
                            int64_t* d_out, void* stream);

/* Instruction offsets of a batch: h_off (count+1 int64); circuit i's
 * instructions take uniforms / write outcomes [h_off[i], h_off[i+1]) in
 * their order in the circuit.  h_off[count] = all instructions. */
tqs_status tqs_batch_instructions(const tqs_batch* b, int64_t* h_off);

/* Launch shape of a batch's persistent kernel for one size class (0: circuits
 * of n <= 11, run by one or two warps each; 1: n = 12..14, one CTA each with
 * the state in shared memory; 2: n = 15..16, one CTA each on global scratch),
 * as the last tqs_batch_run chose it from the options in force then (a
 * scheduling fact: results do not depend on it).  Outputs (each may be
 * NULL): jobs = circuits of that class, grid = CTAs, threads = threads per
 * CTA, teams = circuits that run at once (the persistent teams; each takes
 * about jobs / teams circuits from the job counter).  All are 0 for a class
 * the batch does not hold.  TQS_ERR_STATE before the batch's first run. */
tqs_status tqs_batch_launch_info(const tqs_batch* b, int size_class, int* jobs, int* grid,
                                 int* threads, int* teams);

/* tqs_batch_run for batches that hold instructions: d_u (h_off[count]
 * doubles) and d_outcomes (h_off[count] int32, may be NULL) in the layout of
 * tqs_batch_instructions.  tqs_batch_run and tqs_batch_run_host return
 * TQS_ERR_UNSUPPORTED for such batches. */
tqs_status tqs_batch_run_measured(tqs_batch* b, tqs_c64* d_states, double* d_probs,
                                  double* d_norms, const double* d_u, int32_t* d_outcomes,
                                  int use_graph, void* stream);

/* Host-buffer form of tqs_batch_run: uploads the program, runs, and delivers
 * the results into h_states / h_probs / h_norms (host memory, NULL to skip),
 * then synchronises `stream`.  A buffer that is page-locked and mapped into
 * the device's address space (cudaHostAlloc / cudaHostRegister, torch's
 * pin_memory) is written by the kernel directly (over NVLink-C2C on
 * Grace-Blackwell); any other buffer receives a copy from device memory. */
tqs_status tqs_batch_run_host(tqs_batch* b, tqs_c64* h_states, double* h_probs,
                              double* h_norms, void* stream);

/* Destroy the batch and its device memory.  NULL is accepted. */
tqs_status tqs_batch_destroy(tqs_batch* b);

/* ------------------------------------------------------------------ server
 * Continuous batching of simulate requests (simulateFullState of Sec. 5.2
 * served to many callers; the serving loop itself has no counterpart in the
 * paper).  The server owns no thread: the caller submits requests as they
 * arrive and calls tqs_server_poll often.  Each poll
 *   1. reaps batches whose device work has finished (CUDA events), moves
 *      their results to host memory and releases their device bytes from
 *      the budget, reporting the finished tags;
 *   2. admits queued requests in arrival order while their device bytes
 *      (program, state, norm, and for n >= 15 a 512 KiB work slot) fit the
 *      budget, and launches each admitted group as one batch of the
 *      persistent fused step kernels on a free stream, so that requests that
 *      arrive while others run start as soon as a stream and memory are free,
 *      and up to max_inflight batches overlap on the device.
 * A request's result is bitwise the one tqs_simulate gives for the same
 * circuit: batching never changes the arithmetic. */

typedef struct tqs_server tqs_server;

/* hbm_budget_bytes: device bytes that in-flight batches may hold at once;
 * max_inflight: concurrent batches (streams), 1..64; max_batch: requests per
 * batch.  Device memory is taken stream-ordered (cudaMallocAsync) per batch
 * and returned when the batch's work is done. */
tqs_status tqs_server_create(size_t hbm_budget_bytes, int max_inflight, int max_batch,
                             tqs_server** out);

/* Queue one request: a circuit of n_qubits given by host gate arrays in the
 * layout of tqs_batch_create_packed (kind[n_gates], qubits[2*n_gates],
 * params[8*n_gates]).  `tag` names the result (must not name an untaken
 * result).  Preconditions are checked as in tqs_add_gate; a request that
 * alone exceeds the budget returns TQS_ERR_BUDGET. */
tqs_status tqs_server_submit_packed(tqs_server* s, int64_t tag, int n_qubits, int n_gates,
                                    const int32_t* h_kind, const int32_t* h_qubits,
                                    const double* h_params);

/* Reap finished batches, admit and launch queued requests (non-blocking).
 * h_done_tags[max_done] receives the tags finished since the last poll and
 * *n_done their number; a finished batch with more requests than the free
 * room is reported by a later poll. */
tqs_status tqs_server_poll(tqs_server* s, int64_t* h_done_tags, int max_done, int* n_done);

/* Copy a finished request's state (2^n tqs_c64, host, or NULL) and FP64 norm
 * (host, or NULL) and forget it.  TQS_ERR_STATE if `tag` is not finished. */
tqs_status tqs_server_take(tqs_server* s, int64_t tag, tqs_c64* h_state, double* h_norm);

/* Cancel a request that is still queued (not yet launched): it is dropped
 * and produces no result.  TQS_ERR_STATE if it is running or finished,
 * TQS_ERR_ARG if the server has no request with that tag. */
tqs_status tqs_server_cancel(tqs_server* s, int64_t tag);

/* Counters (each may be NULL): queued requests, requests in flight, requests
 * finished so far, device bytes held now and at most so far. */
tqs_status tqs_server_stats(const tqs_server* s, int64_t* queued, int64_t* inflight,
                            int64_t* done, int64_t* bytes_in_use, int64_t* peak_bytes);

/* Wait for in-flight work, then free everything.  NULL is accepted. */
tqs_status tqs_server_destroy(tqs_server* s);

/* --------------------------------------------------------------- allocator
 * Device scratch (programs, step tables, operand planes, partial sums, batch
 * and server buffers) comes from cudaMalloc / cudaMallocAsync unless the
 * caller installs its own allocator (for example a framework's caching
 * allocator), process-wide:
 *   alloc(bytes, stream, ctx) -> device pointer (16-byte aligned) or NULL;
 *   free(ptr, stream, ctx).
 * `stream` is the stream the buffer is used on (NULL for buffers cached on a
 * handle).  A free with a stream is stream-ordered: work already queued on
 * that stream may still use the buffer, so the allocator must not give it to
 * other streams before that work completes (as a per-stream caching
 * allocator or cudaFreeAsync behaves).  A free with a NULL stream follows a
 * device synchronisation.  Every buffer is returned to the allocator that
 * made it.  An allocation that returns NULL fails the call with
 * TQS_ERR_NOMEM.  tqs_set_allocator(NULL, NULL, NULL) restores the default.
 * The callbacks may be called from any host thread that calls the library. */
typedef void* (*tqs_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*tqs_free_fn)(void* ptr, void* stream, void* ctx);
tqs_status tqs_set_allocator(tqs_alloc_fn alloc, tqs_free_fn free, void* ctx);

/* Bounds-checked build (compiled with -DTQS_CHECKED; a debugging aid with no
 * counterpart in the paper): the fused, batch, instruction, custom-unitary
 * and full-state-vector kernels test every state, tile and output index; an
 * out-of-range index is counted and the access redirected to element 0
 * instead of faulting.  *count receives the number of such accesses since
 * the last reset (reset != 0 clears it); always 0 in the normal build.
 * Synchronises the device. */
tqs_status tqs_check_violations(uint32_t* count, int reset);

/* ----------------------------------------------------------------- options
 * Launch options read when a batch (or a single simulate) plans its launches.
 * TQS_OPT_WARPS_PER_CTA, key = log2 of the amplitudes of a circuit's shared
 * memory slice (4..11), value = warps per CTA of the warp-class kernel (1..16;
 * default 4; capped so that a CTA's slices fit 200 KiB).  It changes launch
 * shapes only, never a result bit.
 * TQS_OPT_TEAM_WARPS, same key, value = warps per circuit of the warp class
 * (1 or 2; default 1).  Two warps share one slice (twice the warps per byte of
 * shared memory).  States and probabilities are bitwise the same for 1 and 2;
 * the FP64 norm and the reductions of measure/reset instructions are summed
 * in a partition that depends on it, so they may differ in the last bits
 * between the two settings (every entry point uses the current setting, so
 * batch, server and single-circuit results agree).
 * TQS_OPT_FSV_MAX_GATES, key = 0, value = gates per pass of the
 * full-state-vector backend at most (0, the default: as many as fit a tile).
 * 1 gives the per-gate form of eq. 12 (Appendix A): one pass over the state
 * in HBM per gate.  Read by tqs_simulate_fsv and tqs_fsv_passes (a circuit's
 * cached passes are rebuilt when it changed).
 * TQS_OPT_MULTI_CTAS, key = 0, value = CTAs at most for one circuit of 15 or
 * 16 qubits in tqs_simulate, and for each such request of a server batch that
 * holds few of them (together at most the SMs divided by the server's batches
 * in flight) (0 or 1: one CTA; default 8; at most 64).  The
 * CTAs (a cooperative launch) share the circuit's passes, one thread per
 * amplitude group, and meet at a grid barrier after each pass; CTA 0 writes
 * the outputs exactly as one CTA would, so states, probabilities and the norm
 * are bitwise the same for every value.  Circuits with measure / reset
 * instructions or custom unitaries always take one CTA.  A grid barrier that
 * waits longer than about a second (it cannot while the launch is
 * cooperative) stops waiting and leaves NaN in the norm and in amplitude 0. */
#define TQS_OPT_WARPS_PER_CTA 1
#define TQS_OPT_TEAM_WARPS 2
#define TQS_OPT_FSV_MAX_GATES 3
#define TQS_OPT_MULTI_CTAS 4
/* TQS_OPT_HOST_WRITES, key = 0: 1 (default) lets tqs_batch_run_host's kernels
 * write outputs that live in page-locked host memory directly (over
 * NVLink-C2C on Grace-Blackwell); 0 writes them to device memory first and
 * copies them with the DMA engines.  Results are bitwise the same. */
#define TQS_OPT_HOST_WRITES 5
/* TQS_OPT_EXACT_PROBS, key = 0: how the fused kernels (tqs_simulate, batches)
 * form the probabilities they write.  0 (default): |psi_i|^2 = x^2 + y^2 in
 * FP32 arithmetic from the FP32 parts, stored as FP64 (relative error below
 * 2^-23); 1: the exact squares, rounded once to FP64 (bit-identical to
 * (double)x*x + (double)y*y).  The states and the FP64 norm do not depend on
 * it; tqs_probabilities always gives the exact form. */
#define TQS_OPT_EXACT_PROBS 6
/* Launch-shape options for the autotuner (results never depend on them
 * beyond the order of floating-point reductions noted):
 * TQS_OPT_CTA_THREADS, key = 0: threads of the one-CTA team that runs a
 *   circuit of 12..14 qubits, 256 or 512 (default 512).  States and
 *   probabilities are bitwise the same; the FP64 norm's reduction order
 *   follows the team size.  A batch reads it (with the warp-class options)
 *   when it is first run on the device, and keeps that launch plan.
 * TQS_OPT_FSV_TILE_Q, key = 0: tile bits of tqs_simulate_fsv's passes, 0
 *   (default: 13 from 24 qubits on, else 12) or 10..13.  Fewer tile bits mean
 *   more passes over HBM but more tiles to spread over the SMs.
 * TQS_OPT_CHAIN_GROUP, key = 0: output-tile rows per raster band of the
 *   tensor-core chain's GEMM grid, 1..64 (default 16); consecutive CTAs walk
 *   down a band, so CTAs resident at once share operand panels in L2.
 *   Results are bitwise the same. */
#define TQS_OPT_CTA_THREADS 7
#define TQS_OPT_FSV_TILE_Q 8
#define TQS_OPT_CHAIN_GROUP 9
/* TQS_OPT_CHAIN_KCHUNK, key = 0: K (columns of S_k summed over) per
 * accumulation chunk of the tensor-core chain's GEMMs, 0 or a multiple of 64
 * up to 2^20.  The tensor cores accumulate in FP32 with truncation, which
 * shrinks a sum of K products by a relative amount that grows with the number
 * of accumulation steps; the GEMMs restart the TMEM accumulators every chunk
 * and add the chunks' complex results in FP32 with rounding to nearest, which
 * bounds that shrink by the chunk length.  0 (default): 512 for
 * TQS_PREC_TC_BF16X3 and 256 for TQS_PREC_TC_TF32X3 (32 MMA accumulation
 * steps either way); a value >= 2^n: all of K in one chunk (a shrink of about
 * 2e-5 per product at K = 16384 in BF16x3).  Results depend on it only
 * through rounding. */
#define TQS_OPT_CHAIN_KCHUNK 10
/* TQS_OPT_CHAIN_PAIR, key = 0: 1 runs the tensor-core chain's GEMMs as
 * clusters of two CTAs on adjacent tile rows that load half of each shared B
 * tile and multicast it to both (half the B traffic from L2), where the number
 * of 128-row tiles is even; 0 (default): one CTA per tile (measured 1-2 %
 * faster at n = 12..14: a stage is released only when both CTAs have consumed
 * it).  Results are bitwise the same. */
#define TQS_OPT_CHAIN_PAIR 11

tqs_status tqs_set_option(int option, int key, int64_t value);
tqs_status tqs_get_option(int option, int key, int64_t* value);

/* Self-test of the bounded device waits (no counterpart in the paper): one
 * thread waits on an mbarrier that nothing completes, gives up after
 * `wait_cycles` SM cycles (1 .. 2^31), records the time-out in a device status
 * word and returns.  Returns TQS_ERR_TIMEOUT when the wait ran out (the
 * expected result), synchronising `stream`; the context stays usable. */
tqs_status tqs_selftest_wait_timeout(int64_t wait_cycles, void* stream);

/* ------------------------------------------------------------------ misc */

/* Thread-local message of the last failed call ("" if none). */
const char* tqs_last_error(void);

/* Static name of a status code. */
const char* tqs_status_string(int status);

/* Number of this library's kernel launches enqueued so far by this process
 * (a graph replay counts its kernel nodes). */
int64_t tqs_launch_count(void);

/* ------------------------------------------------------------- measurement
 * The device's FP32 FMA rate, measured: one launch in which every thread of
 * 8 blocks of 256 per SM runs 8 independent chains of 16 * iters fused
 * multiply-adds (2 flops each), timed with CUDA events on `stream` after one
 * warm-up launch (synchronises the stream).  *h_tflops = flops / time;
 * *h_ms (may be NULL) = the timed launch.  The denominator of the FP32-bound
 * roofline fractions (the paper has no counterpart: its evaluation reports
 * speedups only).  iters >= 1; 20000 takes about 10 ms on a GB300. */
tqs_status tqs_measure_fp32_peak(int iters, double* h_tflops, double* h_ms, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TQS_ABI_H_ */
