/*
 * tcng.h -- C ABI of the B300 (sm_103a) state-vector simulator.
 *
 * The library simulates the paper's circuit/observable statement (TensorCircuit-NG,
 * Sec. I.B "Primitives" and "Paradigms"):  build a circuit on n qubits from
 * parameterised 1- and 2-qubit gates (rx, ry, rz, rzz, h, cx, su4, ...),
 * evaluate Pauli-string expectations (expectation_ps) such as the TFIM energy
 * H = -sum Z_i Z_j - g sum X_i, and return the value and gradient of the energy
 * for a batch of parameter sets (value_and_grad under vmap).  It computes these
 * by in-place state-vector updates on one GPU, not by the paper's tensor-network
 * contraction.
 *
 * Conventions
 *   - qubit q is bit q of the amplitude index (little-endian);
 *   - R_P(t) = exp(-i t P / 2) for RX, RY, RZ, RZZ and RP; CP(phi) = diag(1,1,1,e^{i phi});
 *   - a gate's angle is angle0 + scale * params[item][param] (param < 0: angle0);
 *   - the local index of a k-qubit gate matrix is sum_j bit(q[j]) << (k-1-j);
 *   - complex64 states are interleaved float2, complex128 states double2;
 *   - a Pauli string is (xmask, zmask); Y where both bits are set.
 *
 * Errors: every call returns a tcng_status; no C++ exception crosses the ABI.
 * tcng_last_error() returns a thread-local message for the last failing call.
 * Host arrays are copied (or hashed and cached) during the call; device
 * pointers are borrowed and used in stream order on the stream passed in
 * (a cudaStream_t passed as void*; NULL = the legacy default stream).
 * The library keeps per-structure device scratch (matrix tables, partial sums):
 * calls that overlap on different streams and share a structure race on it.
 * No call synchronises the device except the first call of a new structure
 * (uploading its plan), scratch growth, tcng_autotune and tcng_sync_status.
 * With TCNG_OPT_USE_GRAPHS on, the second call of a structure (same device
 * pointers) also instantiates a CUDA graph (host work only).
 */
#ifndef TCNG_PUBLIC_API_H_
#define TCNG_PUBLIC_API_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TCNG_OK = 0,
    TCNG_EINVAL = 1,        /* bad argument (qubit out of range, null pointer, ...) */
    TCNG_ENOMEM = 2,        /* device or host allocation failed, or buffer too small */
    TCNG_ECUDA = 3,         /* a CUDA runtime call failed (message has the CUDA error) */
    TCNG_EUNSUPPORTED = 4,  /* valid request this library does not implement */
    TCNG_ETIMEOUT = 5       /* a bounded device-side wait expired (reported by tcng_sync_status) */
} tcng_status;

typedef enum { TCNG_C64 = 0, TCNG_C128 = 1 } tcng_dtype;

typedef enum {
    TCNG_I = 0, TCNG_X, TCNG_Y, TCNG_Z, TCNG_H, TCNG_S, TCNG_T,
    TCNG_RX, TCNG_RY, TCNG_RZ, TCNG_CX, TCNG_CZ, TCNG_CP, TCNG_SWAP, TCNG_RZZ,
    TCNG_U1, TCNG_U2, TCNG_UK,
    TCNG_RP     /* exp(-i t P / 2) for a Pauli word P on nq = 1..5 qubits: factor j on q[j]
                   is digit j of mat_off (bits 2j, 2j+1; 0 I, 1 X, 2 Y, 3 Z) */
} tcng_op;

/* One gate of the flat gate-list IR (56 bytes).  U1/U2/UK read a row-major
 * complex128 matrix at mat_off (in complex entries) of the matrix pool. */
typedef struct {
    uint16_t op;        /* tcng_op */
    uint8_t nq;         /* number of qubits (must match op; UK: 1..5) */
    uint8_t pad;
    int32_t q[5];       /* qubits; q[0] is the most significant local bit */
    int32_t param;      /* index into params (per item), -1 = none */
    double scale;       /* angle = angle0 + scale * params[param] */
    double angle0;
    int64_t mat_off;    /* complex offset into mat_pool, -1 = none */
} tcng_gate;

/* One Pauli string: X on xmask&~zmask, Z on zmask&~xmask, Y on xmask&zmask. */
typedef struct {
    uint64_t xmask;
    uint64_t zmask;
    double coeff;
} tcng_pauli;

typedef struct tcng_state tcng_state;   /* opaque batch of state vectors */

/* Maximum qubits per state vector and maximum fused block width. */
#define TCNG_MAX_QUBITS 34
#define TCNG_MAX_FUSE 5

/*
 * tcng_state_init -- create `batch` state vectors |0...0> (paper Sec. I.B:
 * tc.Circuit(n) starts from the all-zero product state).
 *   dt        element type of every amplitude;
 *   n_qubits  host array [batch]; item b holds 2^n_qubits[b] amplitudes
 *             (ragged batches allowed, each n in 1..TCNG_MAX_QUBITS);
 *   dev_buf   NULL: the library allocates device memory and owns it;
 *             else a caller-owned, 256-byte aligned device buffer of buf_bytes
 *             bytes (e.g. a torch tensor) that must outlive the state;
 *   stream    cudaStream_t for the initialising kernel.
 * Items are stored back to back, each starting on a 256-byte boundary.
 * Errors: EINVAL (bad sizes, null out), ENOMEM (allocation or buf_bytes too
 * small), ECUDA.
 */
tcng_status tcng_state_init(tcng_state** out, tcng_dtype dt, int batch, const int* n_qubits,
                            void* dev_buf, size_t buf_bytes, void* stream);

/* Bytes a caller-owned buffer needs for tcng_state_init with these sizes. */
tcng_status tcng_state_bytes(tcng_dtype dt, int batch, const int* n_qubits, size_t* bytes);

/* Free the handle (and the device memory if the library allocated it).
 * Waits for no work: the caller must not free while kernels using it run. */
tcng_status tcng_state_free(tcng_state* st);

/* Device pointer and byte size of item `item` (a view; no copy). */
tcng_status tcng_state_ptr(const tcng_state* st, int item, void** dev_amp, size_t* bytes);

/* Reset every item to |0...0> (stream-ordered). */
tcng_status tcng_state_reset(tcng_state* st, void* stream);

/*
 * tcng_apply_circuit -- apply the gate list to every item in place
 * (paper Sec. I.B: gates added to tc.Circuit act in order on the state).
 *   ops, n_ops        host gate list (validated and copied; the fused plan is
 *                     cached by a hash of the structure, so repeated calls with
 *                     the same structure and new parameters rebuild nothing);
 *   mat_pool, n_mat   host complex128 matrix pool as (re, im) doubles,
 *                     n_mat complex entries (may be NULL if n_mat == 0);
 *   params_dev        device double [batch][P] (may be NULL if P == 0);
 *   P                 parameters per item.
 * Every qubit must be < n of every item.  Gates are fused into blocks of at
 * most the configured width and grouped into shared-memory tile passes
 * (tcng_set_option).  Errors: EINVAL, ENOMEM, ECUDA.
 */
tcng_status tcng_apply_circuit(tcng_state* st, const tcng_gate* ops, size_t n_ops,
                               const double* mat_pool, size_t n_mat,
                               const void* params_dev, int P, void* stream);

/*
 * tcng_apply_circuit_pooled -- tcng_apply_circuit where every item has its own
 * explicit gate matrices: the trajectories of the paper's MIPT study draw an
 * independent Haar SU(4) for every gate of every trajectory (Sec. VII.C).
 *   mat_pool, n_mat   host complex128 pool with the same layout as every item's
 *                     (the planner reads it to classify each matrix as diagonal
 *                     or dense and as unitary or not; every item's matrices must
 *                     share those properties with it);
 *   item_pool_dev     device complex128 (re, im) [batch][pool_stride], 16-byte
 *                     aligned: gate g of item b uses the matrix at
 *                     item_pool_dev[b][g.mat_off ...];
 *   pool_stride       complex entries per item (>= n_mat).
 * All items must have the same n.  Errors: as tcng_apply_circuit, plus
 * EUNSUPPORTED (ragged state).
 */
tcng_status tcng_apply_circuit_pooled(tcng_state* st, const tcng_gate* ops, size_t n_ops,
                                      const double* mat_pool, size_t n_mat, const void* item_pool_dev,
                                      size_t pool_stride, const void* params_dev, int P, void* stream);

/*
 * tcng_expect_pauli -- out_dev[b][t] = <psi_b|P_t|psi_b> (real; the paper's
 * expectation_ps, Sec. I.B; coefficients are NOT applied).
 *   terms     host array [n_terms <= 4096] of Pauli strings (masks < 2^n of
 *             every item's n);
 *   out_dev   device double [batch][n_terms].
 * Terms are grouped into tile passes (one read of the state per pass); a term
 * with more X/Y factors above qubit 0 than a tile gathers (tile_bits - 1: 12
 * for complex64, 11 for complex128 at the default tile bits), e.g. the parity
 * X...X, gets a pass of its own that reads the amplitude pairs (x, x ^ m) from
 * global memory.  A ragged batch is evaluated one size class at a time.  Sums
 * accumulate in FP64 in a fixed order (bitwise reproducible).  Errors: EINVAL,
 * ENOMEM, ECUDA.
 */
tcng_status tcng_expect_pauli(const tcng_state* st, const tcng_pauli* terms, size_t n_terms,
                              double* out_dev, void* stream);

/*
 * tcng_expect_pauli_noalloc -- out_dev[t] = <psi|P_t|psi> for one state vector,
 * like tcng_expect_pauli, but without allocating any device memory.  The paper
 * has no counterpart; this is for callers that cannot let a library allocate:
 * an application whose own allocator already holds the GPU's free memory, or a
 * serving loop where cudaMalloc/cudaFree (and the synchronisation cudaFree
 * implies) are banned from the hot path.
 *   psi_dev   device state, 2^n amplitudes of type dt, 256-byte aligned;
 *   terms     host array of n_terms Pauli strings (masks < 2^n);
 *   out_dev   device double [n_terms].
 * Scratch: the per-CTA partial sums live in a fixed array of 65536 doubles
 * (512 KiB) in the library's own device memory; every GPU that loads the
 * library keeps it until the process exits.  Requests that need more than
 * 65536 partial sums (n_terms x CTAs, at most one CTA per SM) fail with
 * TCNG_EINVAL and a message giving the size.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  All calls share the array: calls that overlap
 * on the GPU (different streams, or different host threads) race on it and
 * must be serialised by the caller.  Each call writes every slot it reads, so
 * no state carries over between calls.  The call takes the library's host lock
 * like every other entry point.  No device-side error word is kept for this
 * call: a bounded device-side wait that times out ends the pass early and the
 * affected values of out_dev are NaN.  Terms wider than a tile (see
 * tcng_expect_pauli) are rejected with EINVAL here.
 */
tcng_status tcng_expect_pauli_noalloc(const void* psi_dev, int n, tcng_dtype dt,
                                      const tcng_pauli* terms, size_t n_terms, double* out_dev,
                                      void* stream);

/*
 * tcng_expect_energy -- both of the above from one plan: out_dev[b][t] =
 * <psi_b|P_t|psi_b> for every term and energy_dev[b] = sum_t c[b][t] out_dev[b][t]
 * (coefficients as in tcng_energy; give a term coefficient 0 to report it without
 * weighting it).  Planning all terms together packs them into fewer passes over
 * the state than separate calls.  Errors: as tcng_expect_pauli.
 */
tcng_status tcng_expect_energy(const tcng_state* st, const tcng_pauli* terms, size_t n_terms,
                               const double* coeffs_dev, double* out_dev, double* energy_dev,
                               void* stream);

/*
 * tcng_energy -- energy_dev[b] = sum_t c[b][t] <psi_b|P_t|psi_b>, the TFIM (or
 * any Pauli-sum) energy of Sec. I.B.  coeffs_dev: device double [batch][n_terms],
 * or NULL to use terms[t].coeff for every item.  Errors: as tcng_expect_pauli.
 */
tcng_status tcng_energy(const tcng_state* st, const tcng_pauli* terms, size_t n_terms,
                        const double* coeffs_dev, double* energy_dev, void* stream);

/*
 * tcng_hamiltonian_apply -- lambda_b = H_b psi_b for every item (the co-state
 * that starts the adjoint sweep); out must be a state with the same shape and
 * dtype as st.  H_b = sum_t c[b][t] P_t with coeffs_dev as in tcng_energy.  A
 * ragged batch is applied one size class at a time.
 */
tcng_status tcng_hamiltonian_apply(const tcng_state* st, const tcng_pauli* terms, size_t n_terms,
                                   const double* coeffs_dev, tcng_state* out, void* stream);

/*
 * tcng_energy_grad -- for every item b: run U(theta_b)|0..0>, then
 * E_b = <psi|H_b|psi> and dE_b/dtheta_b by an adjoint reverse sweep
 * (replaces the paper's reverse-mode AD through the tensor network, Sec. I.B
 * "Paradigms: AD"; cost independent of the number of parameters, O(1) states).
 *   st          batch of states (all items the same n); used as scratch for psi;
 *   ops/mat     gate list as in tcng_apply_circuit; parameterised gates may be
 *               RX, RY, RZ, RZZ, CP or RP (RP, states of at least
 *               TCNG_OPT_STATE_ADJOINT_N qubits and small batches under
 *               TCNG_OPT_STATE_ADJOINT_SMALL take the state-pass adjoint:
 *               items one after another, a parameterised RP on at most 2
 *               qubits; a scratch copy of one item's state is allocated);
 *   params_dev  device double [batch][P];
 *   H, n_terms  Pauli strings; coeffs_dev device double [batch][n_terms] or NULL;
 *   energy_dev  device double [batch];
 *   grad_dev    device double [batch][P] (dE/dtheta; params read by no gate get 0).
 * One persistent launch covers the whole batch.  Errors: EINVAL, ENOMEM, ECUDA.
 */
tcng_status tcng_energy_grad(tcng_state* st, const tcng_gate* ops, size_t n_ops,
                             const double* mat_pool, size_t n_mat,
                             const void* params_dev, int P,
                             const tcng_pauli* H, size_t n_terms, const double* coeffs_dev,
                             double* energy_dev, double* grad_dev, void* stream);

/* One circuit structure of a ragged batch (all arrays on the host). */
typedef struct {
    int n;                       /* qubits */
    const tcng_gate* ops;
    size_t n_ops;
    const double* mat_pool;      /* complex128 (re, im) pairs */
    size_t n_mat;
    int P;                       /* parameters per item of this structure */
    const tcng_pauli* H;
    size_t n_terms;
} tcng_problem;

/*
 * tcng_energy_grad_ragged -- one persistent launch over items of different
 * structures and qubit counts (the paper's vmap over "thousands of instances",
 * Sec. I.B, with ragged n).
 *   problems, n_problems   host structures;
 *   item_problem           host int [batch]: structure of item b;
 *   params_dev             device double, items packed back to back
 *                          (item b starts at sum_{b'<b} P of its structure);
 *   coeffs_dev             device double packed the same way over n_terms, or
 *                          NULL for the structures' own coefficients;
 *   energy_dev             device double [batch];
 *   grad_dev               device double packed like params_dev.
 * No state handle: the library keeps per-CTA scratch for the largest n.
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
tcng_status tcng_energy_grad_ragged(const tcng_problem* problems, int n_problems,
                                    const int* item_problem, int batch,
                                    const double* params_dev, const double* coeffs_dev,
                                    double* energy_dev, double* grad_dev, void* stream);

/*
 * tcng_marginal_probs -- out_dev[b][k] = sum of |psi_b(x)|^2 over the x whose
 * bits at qubits[0..nk-1] spell k, with k = sum_j bit(x, qubits[j]) << (nk-1-j)
 * (qubits[0] is the most significant bit of k): the diagonal of the reduced
 * density matrix of those qubits, which the paper's QML pipeline reads out as
 * class probabilities (Sec. VII.B, reduced_density_matrix over the first 7
 * qubits), i.e. the Born probabilities of measuring them.
 *   qubits    host int [nk], distinct, each < n; nk in 1..10;
 *   out_dev   device double [batch][2^nk].
 * All items must have the same n.  Sums accumulate per thread in the state's
 * precision (folded into FP64 every 256 amplitudes) and then in FP64 in a
 * fixed order (bitwise reproducible).  Errors: EINVAL, EUNSUPPORTED (ragged),
 * ENOMEM, ECUDA.
 */
tcng_status tcng_marginal_probs(const tcng_state* st, const int* qubits, int nk, double* out_dev,
                                void* stream);

/*
 * tcng_measure -- projective computational-basis (Z) measurement of the qubits
 * in mask_dev[b] of every item b (the per-qubit measurements of the paper's MIPT
 * trajectories, Sec. VII.C, and the bitstrings of its shadow snapshots,
 * Sec. VII.A).  Qubits are measured in increasing order; the outcome of qubit q
 * is 0 iff u_dev[b][q] < P(0 | the item's earlier outcomes of this call) (Born
 * rule); the state is projected onto the outcomes and rescaled to unit norm.
 *   mask_dev     device uint64 [batch]: bit q set = measure qubit q (0: the
 *                item is left unchanged);
 *   u_dev        device double [batch][n], uniforms in [0, 1) (only the
 *                entries of measured qubits are read);
 *   outcome_dev  device int8 [batch][n]: 0 or 1 written for each measured
 *                qubit, other entries untouched;
 *   logp_dev     device double [batch]: the natural log of the probability of
 *                this call's outcomes is ADDED (a trajectory's log-probability
 *                accumulates over calls); NULL to skip.
 * Outcomes are sampled in rounds of up to 10 qubits from the joint Born
 * probabilities of the round's qubits (summed in FP64, fixed order).  All
 * items must have the same n.  Errors: EINVAL, EUNSUPPORTED (ragged), ENOMEM,
 * ECUDA.
 */
tcng_status tcng_measure(tcng_state* st, const uint64_t* mask_dev, const double* u_dev, int8_t* outcome_dev,
                         double* logp_dev, void* stream);

/*
 * tcng_apply_shared_unitary -- apply one k-qubit unitary U (host complex128,
 * row-major, local index as in the gate list with qubits q[0..k-1]) to every
 * item of a complex64 batch: a complex GEMM [2^k x 2^k] x [2^k x batch*2^(n-k)],
 * run as a one-gate circuit without parameters, so one W set serves every tile
 * of every item on the tensor cores (FP16 hi/lo operands; items of fewer than
 * 13 qubits packed several to a tile).  The batched layer of the paper's QML
 * demonstration (Sec. VII.B), where every input state sees the same circuit.
 * k in 1..5; qubits distinct and < n.  Errors: EINVAL, EUNSUPPORTED (complex128
 * states), ECUDA.
 */
tcng_status tcng_apply_shared_unitary(tcng_state* st, const int* qubits, int k,
                                      const double* U, void* stream);

/*
 * tcng_adam_step -- device Adam update over n values (Kingma & Ba; the
 * optimiser of the paper's training listings):
 *   m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
 *   theta <- theta - lr * (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps),
 * with t = *step_dev + 1 read on the device; the kernel's last block writes the
 * new step back (so the call can be replayed from a CUDA graph).  All arrays
 * are device double.
 */
tcng_status tcng_adam_step(double* theta, double* m, double* v, const double* grad, size_t n,
                           double lr, double b1, double b2, double eps, int* step_dev,
                           void* stream);

/*
 * Warm-start MLP (no counterpart in the paper): y = W3 relu(W2 relu(W1 x + b1) + b2) + b3
 * with BF16 operands and FP32 accumulation.  Weights are FP32 master copies;
 * each GEMM reads BF16-rounded copies of its two operands.
 *   x        device float [N][F];
 *   w1,b1    [F][H], [H];  w2,b2 [H][H], [H];  w3,b3 [H][O], [O]  (device float)
 *   act      device float scratch [2][N][H] (pre-activations z1, z2), written;
 *   y        device float [N][O], written.
 */
tcng_status tcng_mlp_forward(const float* x, int N, int F, int H, int O,
                             const float* w1, const float* b1, const float* w2, const float* b2,
                             const float* w3, const float* b3, float* act, float* y,
                             void* stream);

/*
 * Loss and backward pass of the warm-start MLP.  Loss (periodic in the angle):
 *   L = sum_{n,o} mask[n][o] * 2 (1 - cos(y[n][o] - target[n][o])) / sum mask.
 *   mask, target  device float [N][O];
 *   act           the pre-activations tcng_mlp_forward wrote;
 *   grads         device float, the 6 gradients packed as w1,b1,w2,b2,w3,b3;
 *   loss_dev      device double [1].
 */
tcng_status tcng_mlp_backward(const float* x, int N, int F, int H, int O,
                              const float* w1, const float* w2, const float* w3,
                              const float* act, const float* y, const float* target,
                              const float* mask, float* grads, double* loss_dev, void* stream);

/* Adam over FP32 master weights (device float), same formula as tcng_adam_step. */
tcng_status tcng_adam_step_f32(float* theta, float* m, float* v, const float* grad, size_t n,
                               float lr, float b1, float b2, float eps, int* step_dev,
                               void* stream);

/* Options (process-wide). */
typedef enum {
    TCNG_OPT_FUSE_WIDTH = 0,   /* max qubits of a fused block, 1..5 (default 2) */
    TCNG_OPT_TILE_BITS = 1,    /* log2 amplitudes per shared-memory tile, 5..13 (default 13) */
    TCNG_OPT_CHUNK_BITS = 2,   /* log2 contiguous amplitudes per copied chunk (default 7;
                                  expectation passes use at most 3) */
    TCNG_OPT_USE_GRAPHS = 3,   /* 1 (default): tcng_apply_circuit, tcng_energy_grad and
                                  tcng_energy_grad_ragged replay one CUDA graph per key
                                  (structure, options, device pointers): the first call
                                  of a key runs eagerly, the second records its launches
                                  on a private stream and launches the graph, later
                                  calls only launch it.  Parameters, coefficients and
                                  states are read from device memory when the graph
                                  runs, so new values need no new recording.  Calls on
                                  a stream the caller is capturing, and calls while
                                  tcng_profile_enable is on, run eagerly.  0: always
                                  eager. */
    TCNG_OPT_UNFUSED = 4,      /* 1: one pair/quartet kernel launch per gate (default 0) */
    TCNG_OPT_TENSOR_CORES = 5  /* complex64 register stages as 16x16 GEMMs on the tensor cores
                                  (TF32 hi/lo split, ~1e-6 relative error per circuit):
                                  0 off, 1 on, 2 auto (default): on when all items share one
                                  parameter set and the state spans at least one 2^13-amplitude
                                  tile per SM, or spans 32 tiles per SM */,
    TCNG_OPT_STATE_ADJOINT_N = 6  /* tcng_energy_grad runs the state-pass adjoint (one pass over
                                  psi and lambda per run of consecutive blocks of <= 2 qubits
                                  that fits a shared-memory tile, all of a block's
                                  parameters from one cross-density matrix) for states of at
                                  least this many qubits (default 21; 1..35), and always for
                                  circuits with RP parameters; smaller states use the
                                  per-item persistent kernel */,
    TCNG_OPT_TC_FP16 = 7          /* 1 (default): tensor-core passes of unitary plans whose
                                  tiles share one parameter set split both GEMM operands
                                  into FP16 hi + lo (each tile scaled by a power of two
                                  first, FP32 accumulation; passes whose stages touch every
                                  tile bit keep two tiles in flight per CTA); 0: the TF32
                                  hi/lo split everywhere */,
    TCNG_OPT_STATE_ADJOINT_SMALL = 8  /* 1 (default): below TCNG_OPT_STATE_ADJOINT_N qubits, a
                                  batch too small to occupy the GPU with the per-item
                                  kernel (one CTA per item) takes the state-pass adjoint
                                  when a cost model measured on a B300 says it is faster:
                                  batch < ceil(batch / SMs) x r(n), r = 1.8 x 1.95^(n - 14)
                                  for complex64 (one item from 14 qubits, up to 99 items
                                  at 20), min(99, 4.8 x 2^(n - 14)) for complex128;
                                  0: only the qubit threshold decides */
} tcng_option;

tcng_status tcng_set_option(tcng_option opt, int value);
tcng_status tcng_get_option(tcng_option opt, int* value);

/*
 * tcng_autotune -- choose the options of the fused apply path by timing every
 * candidate (fusion width 1..5; tensor-core stages off/on for complex64; tile
 * bits tmax-1 and tmax; chunk bits 5 and 7) with CUDA events on a synthetic
 * SU(4)-like brickwork of n qubits applied to `batch` states of type dt (one
 * untimed call per candidate builds its plan, two are timed).  The fastest
 * becomes the current option set and is appended to cache_path (NULL: no file)
 * as "n dt batch fuse_width tile_bits chunk_bits tensor_cores ms"; a cached
 * line for (n, dt, batch) is loaded without timing.  Synchronises the device.
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
tcng_status tcng_autotune(int n, tcng_dtype dt, int batch, const char* cache_path);

/*
 * tcng_autotune_circuit -- the same search on the caller's own circuit and
 * state (the state's amplitudes are overwritten: it serves as scratch); the
 * cache key is the circuit's structure hash (with dt and the batch size).
 *   best_ms   host double, the best candidate's time per call (may be NULL;
 *             untouched when the choice comes from the cache).
 * Errors: EINVAL, EUNSUPPORTED (ragged state), ENOMEM, ECUDA.
 */
tcng_status tcng_autotune_circuit(tcng_state* st, const tcng_gate* ops, size_t n_ops,
                                  const double* mat_pool, size_t n_mat, const void* params_dev, int P,
                                  const char* cache_path, double* best_ms);

/* The last autotune run as text: one line "fuse_width tile_bits chunk_bits
 * tensor_cores ms" per candidate (ms < 0: the candidate failed), or "cached
 * <cache line>" when the choice was loaded.  NUL-terminated, truncated to len. */
tcng_status tcng_autotune_report(char* buf, size_t len);

/*
 * tcng_fma_peak -- measured FMA throughput of this GPU in TFLOP/s (2 flops per
 * FMA), FP32 (fp64 = 0) or FP64: every thread of 8 CTAs x 256 threads per SM
 * runs eight independent FMA chains; one timed launch after a warm-up.  The
 * denominator of the roofline of the SIMT kernels (the adjoint sweep).  Not
 * part of any computation of the paper; synchronises the device.
 */
tcng_status tcng_fma_peak(int fp64, double* tflops);

/* Synchronise the device and report a device-side error word (ETIMEOUT) if set. */
tcng_status tcng_sync_status(void);

/* Human-readable summary of the plan a gate list compiles to (thread-local string):
 * the plan of a one-item complex64 tcng_apply_circuit under the current options,
 * or with adjoint != 0 the plan of the adjoint kernel. */
const char* tcng_describe_plan(int n, const tcng_gate* ops, size_t n_ops, const double* mat_pool,
                               size_t n_mat, int P, int adjoint);

/*
 * Human-readable summary of the state-pass adjoint's plan for a gate list and a
 * Pauli sum (host only, no device call; thread-local string): the reverse
 * sweep's steps, last block first, as "seg tmask=<tile qubits> blocks=<block>:
 * <qubit mask>,..." (runs of blocks of <= 2 qubits sharing one pass over psi
 * and lambda) and "lone" lines (blocks of 3..5 qubits), then the passes of
 * lambda = H psi as "ham tmask=<tile qubits> terms=<indices>" (hampasses=-1 when
 * a term's X mask does not fit in a tile: the gather kernel runs instead).
 * dt selects the tile size (2^12 amplitudes for complex64, 2^11 for complex128).
 * Returns "error: ..." for an invalid gate list.
 */
const char* tcng_describe_state_adjoint(int n, const tcng_gate* ops, size_t n_ops, const double* mat_pool,
                                        size_t n_mat, int P, const tcng_pauli* H, size_t n_terms,
                                        tcng_dtype dt);

/*
 * Shared-memory layouts of one lock-step FP16 tile pass (host only, no device
 * call).  rbit: nst x 4 register tile bits of the pass's stages, each stage's four
 * ascending and in 0..12.  out (nst x 8 bytes, caller-owned): per stage the
 * positions of its four register bits in the layout it reads, then in the layout
 * it writes.  Every stage rewrites the whole tile, so it may move its register
 * bits (the other bits keep their order); stage 0 reads and the last stage writes
 * the tile map's layout.  The positions are chosen so that a warp's accesses reach
 * every shared-memory bank slot of the 128-byte swizzle; *relocated = 0 when the
 * tile map's layout is kept throughout (nothing to gain, or no way back to it).
 * TCNG_EINVAL on null pointers, nst outside 1..64 or bad register bits.
 */
tcng_status tcng_plan_lock_layouts(const unsigned char* rbit, int nst, unsigned char* out, int* relocated);

/*
 * Kernel timing with CUDA events recorded on the launch stream around every
 * kernel this library launches (off by default; a few microseconds per launch
 * when on).  tcng_profile_read synchronises the device and writes
 * "name count total_ms\n" lines, one per kernel kind, into buf (NUL-terminated,
 * truncated to len); reset clears the records.
 */
tcng_status tcng_profile_enable(int on);
tcng_status tcng_profile_read(char* buf, size_t len, int reset);

/* Kernels this library launched since load (for accounting). */
uint64_t tcng_launch_count(void);

/* Thread-local message for the last failing call ("" if none). */
const char* tcng_last_error(void);

/* Library version string. */
const char* tcng_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TCNG_PUBLIC_API_H_ */
