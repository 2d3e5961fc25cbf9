/*
 * sv.h - C ABI of the GB300 state-vector library (libsv.so).
 *
 * The library implements the Schroedinger approach to circuit simulation
 * described in Sec. 2 of "An open-source modular framework for quantum
 * computing" (Qibo 0.1.7): a state of n qubits is 2^n complex amplitudes,
 * a gate on n_tar targets is a 2^n_tar x 2^n_tar complex matrix G, and a
 * gate is applied by Eq. (1),
 *     psi'(tau, q) = sum_tau' G(tau, tau') psi(tau', q),
 * in place, for every gate of a circuit in order.  Everything runs in
 * hand-written CUDA kernels for sm_103a on the state's stream.
 *
 * Conventions (the paper leaves them open; one reading, used everywhere):
 *   - qubit q is bit p = n-1-q of the amplitude index (qubit 0 = MSB);
 *   - for targets t_0..t_{k-1}, G's row/column index is
 *     tau = sum_j b(t_j) 2^(k-1-j)  (t_0 is the MSB of tau), G row-major;
 *   - a controlled gate acts where every control qubit is 1 and leaves the
 *     rest of the state unchanged (Sec. 2: controlled and multi-target
 *     gates by modified index generation);
 *   - state layout: 2^n interleaved (re, im) pairs, float32 for SV_C64 and
 *     float64 for SV_C128, contiguous, 256-byte aligned;
 *   - Pauli masks use amplitude-index bits: bit p of xmask/zmask refers to
 *     qubit n-1-p.  A term is X where only x is set, Z where only z is set,
 *     Y where both are set.
 *
 * Ownership: a state handle either owns its device buffer (sv_alloc) or
 * borrows one (sv_wrap); the library also owns small per-handle work buffers
 * (reduction partials, adjoint work states, checkpoints), freed by sv_free.
 * Matrices, circuits, parameters and Pauli sums are read from host memory
 * during the call and not retained.
 *
 * Errors: every call validates all arguments before launching anything and
 * returns SV_ERR_INVALID with the state untouched if any is bad; CUDA
 * failures return SV_ERR_CUDA; nothing aborts.  sv_last_error() returns a
 * message for the calling thread's last failure.
 *
 * Asynchrony: calls are asynchronous on the handle's stream unless they
 * return a host value (sv_expval, sv_norm, sv_grad, sv_adjoint with host
 * outputs, sv_download, sv_sync), which synchronise that stream.
 */
#ifndef SV_H
#define SV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { SV_C64 = 0, SV_C128 = 1 } sv_dtype;

typedef enum {
  SV_OK = 0,
  SV_ERR_INVALID = 1,     /* bad argument; nothing was launched */
  SV_ERR_OOM = 2,         /* device allocation failed */
  SV_ERR_CUDA = 3,        /* a CUDA call failed; see sv_last_error() */
  SV_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
  SV_ERR_UNSUPPORTED = 5  /* valid request this build does not implement */
} sv_status;

/* Gate kinds of a circuit record.  Controlled forms are the same kinds with
 * controls: CZ = Z with one control, CNOT = X with one control,
 * CU1(l) = U1(l) with one control, Toffoli = X with two controls.
 * Matrices (c = cos(a/2), s = sin(a/2)):
 *   H = [[1,1],[1,-1]]/sqrt2, X, Y, Z the Pauli matrices,
 *   RX(a) = [[c,-is],[-is,c]], RY(a) = [[c,-s],[s,c]],
 *   RZ(a) = diag(e^{-ia/2}, e^{ia/2}), U1(a) = diag(1, e^{ia}),
 *   SWAP exchanges |01> and |10> of its two targets,
 *   MATRIX reads 4^n_tar complex128 entries from the circuit's pool,
 *   PAULI(a) = exp(-i a P / 2) = c I - i s P for the Pauli string
 *     P = sigma_{L_0} (x) ... (x) sigma_{L_{k-1}} on targets t_0..t_{k-1}
 *     (letter L_j in bits 2j..2j+1 of `paulis`: 1 X, 2 Y, 3 Z), 1..5
 *     targets and no controls: the rotations exp(-i gamma Z_i Z_j / 2) and
 *     exp(-i beta X_j / 2) of QAOA (Sec. 3: QAOA, MaxCut) and the
 *     exponentials of Pauli terms of Trotter products.  Differentiable:
 *     dE/da = Im<lambda|P|psi> as for RX, RY, RZ. */
enum {
  SV_GATE_H = 0, SV_GATE_X = 1, SV_GATE_Y = 2, SV_GATE_Z = 3,
  SV_GATE_RX = 4, SV_GATE_RY = 5, SV_GATE_RZ = 6, SV_GATE_U1 = 7,
  SV_GATE_SWAP = 8, SV_GATE_MATRIX = 9, SV_GATE_PAULI = 10
};

#define SV_MAX_QUBITS 34
#define SV_MAX_TARGETS 5
#define SV_MAX_CONTROLS 33  /* n - 1 at the largest state */
#define SV_MAX_PAULI_TERMS 4096

typedef struct sv_state_s* sv_state;   /* opaque handle */

/* One gate of a circuit (Sec. 3: circuits of one-, two- and three-qubit
 * gates; here any 1..5 targets plus up to SV_MAX_CONTROLS controls). */
typedef struct {
  int32_t kind;                        /* SV_GATE_* */
  int32_t n_tar;                       /* 1 (2 for SWAP, 1..5 for MATRIX) */
  int32_t n_ctrl;                      /* 0..SV_MAX_CONTROLS */
  int32_t param;                       /* index into theta[], or -1 */
  int32_t targets[SV_MAX_TARGETS];     /* qubit numbers */
  int32_t controls[SV_MAX_CONTROLS];   /* qubit numbers */
  double angle;                        /* angle when param == -1 */
  int64_t mat_off;                     /* MATRIX: offset (in complex entries) into mat_pool */
  int32_t paulis;                      /* PAULI: letter of targets[j] in bits 2j..2j+1 */
  int32_t reserved;                    /* 0 */
} sv_gate;

typedef struct {
  int32_t n_qubits;
  int32_t n_gates;
  int32_t n_params;                    /* length of theta[] */
  const sv_gate* gates;                /* host, n_gates records */
  const double* mat_pool;              /* host complex128 (re, im) pairs, or NULL */
} sv_circuit;

/* H = sum_k coeff[k] P_k, P_k a Pauli string given by (xmask[k], zmask[k])
 * (Sec. 3: Hamiltonians such as the transverse-field Ising model). */
typedef struct {
  int32_t n_terms;                     /* 0..SV_MAX_PAULI_TERMS */
  const uint64_t* xmask;               /* host */
  const uint64_t* zmask;               /* host */
  const double* coeff;                 /* host, real coefficients */
} sv_pauli_sum;

/* ---- state handles ---------------------------------------------------- */

/* Allocate a 2^n_qubits state (library-owned, contents undefined) on the
 * current device, bound to `cuda_stream` (a cudaStream_t, NULL = legacy
 * default stream).  Sec. 2: the state is 2^n complex numbers.
 * Errors: SV_ERR_INVALID (n_qubits outside 1..SV_MAX_QUBITS, bad dtype,
 * out NULL), SV_ERR_OOM. */
sv_status sv_alloc(int n_qubits, sv_dtype dtype, void* cuda_stream, sv_state* out);

/* Wrap caller-owned device memory `dev_ptr` (2^n_qubits amplitudes of
 * `dtype`, 16-byte aligned) without copying; the caller keeps ownership and
 * must keep it alive until sv_free.  Errors as sv_alloc, plus
 * SV_ERR_INVALID for a NULL or misaligned pointer. */
sv_status sv_wrap(void* dev_ptr, int n_qubits, sv_dtype dtype, void* cuda_stream,
                  sv_state* out);

/* Release the handle, its work buffers, and the state buffer if owned. */
sv_status sv_free(sv_state s);

/* Rebind the handle to another stream (e.g. a stream being captured into a
 * CUDA graph).  Later calls launch there. */
sv_status sv_set_stream(sv_state s, void* cuda_stream);

/* Rounding of complex64 gate arithmetic (Sec. 2, Eq. 1 evaluated in fp32).
 * Every mode rounds inexact matrices to fp32 with error feedback: the state
 * keeps the squared-norm factor that its rounded matrices have applied and
 * scales the next one against it, so the fp32 rounding of 1/sqrt2 in H
 * (2 h^2 = 1 - 3.4e-8) does not accumulate over many gates.
 *   SV_ROUNDING_DEFAULT: the one-kernel-per-gate 1-qubit kernels round each
 *     output with dither (a pseudo-random term below one fp32 step added
 *     before the final rounding, keyed by amplitude and launch), so equal
 *     amplitudes do not repeat one rounding error gate after gate; the
 *     fused qubit-block passes round to nearest (their 1-qubit products as
 *     scaled real rotations between diagonals).
 *   SV_ROUNDING_DITHERED: the fused passes keep dense 2x2 products and
 *     dither them too (about twice their arithmetic); for circuits whose
 *     states repeat, such as Grover's search (many equal amplitudes) or a
 *     Clifford brick applied thousands of times, where round-to-nearest
 *     repeats its errors period after period and the norm drifts linearly
 *     with the repetition count.
 * Results are reproducible: the dither restarts with sv_init / sv_upload.
 * complex128 states ignore the mode.  SV_ERR_INVALID for another value. */
typedef enum { SV_ROUNDING_DEFAULT = 0, SV_ROUNDING_DITHERED = 1 } sv_rounding;
sv_status sv_set_rounding(sv_state s, int mode);

/* Device pointer, qubit count and dtype of the state. */
sv_status sv_info(sv_state s, void** dev_ptr, int* n_qubits, sv_dtype* dtype);

/* Set the state to the basis state |basis_index> (Sec. 2: amplitudes in the
 * computational basis).  Asynchronous.  SV_ERR_INVALID if basis_index >= 2^n. */
sv_status sv_init(sv_state s, uint64_t basis_index);

/* Copy 2^n amplitudes between host memory (pinned or pageable, same dtype
 * layout) and the state.  sv_upload is asynchronous for pinned memory;
 * sv_download synchronises the stream. */
sv_status sv_upload(sv_state s, const void* host);
sv_status sv_download(sv_state s, void* host);

/* Page-locked host buffers for sv_upload / sv_download, allocated through
 * the same CUDA runtime as the library (so the copies see them as pinned
 * and run at the host link's bandwidth).  sv_host_alloc writes the buffer
 * to *out; SV_ERR_OOM if the host cannot pin `bytes`, SV_ERR_INVALID for a
 * null out or zero bytes.  sv_host_free releases a buffer from
 * sv_host_alloc (NULL is a no-op). */
sv_status sv_host_alloc(size_t bytes, void** out);
sv_status sv_host_free(void* p);

/* Copy the amplitudes of `src` into `dst` (same n and dtype). Asynchronous. */
sv_status sv_copy(sv_state dst, sv_state src);

/* ---- gate application (Sec. 2, Eq. 1) ---------------------------------- */

/* Apply G (host complex128, 2^n_tar x 2^n_tar, row-major (re, im) pairs) to
 * targets[0..n_tar-1] where every qubit in controls[0..n_ctrl-1] is 1,
 * in place.  1 <= n_tar <= 5, 0 <= n_ctrl <= SV_MAX_CONTROLS, all qubits distinct and
 * < n.  G is rounded once to the state's precision.  Asynchronous.
 * Errors: SV_ERR_INVALID for any bad argument (state untouched). */
sv_status sv_apply_gate(sv_state s, const int* targets, int n_tar,
                        const int* controls, int n_ctrl, const double* matrix);

/* Apply every gate of `c` in order (Sec. 2: Eq. 1 per gate; Sec. 1: cost
 * linear in the gate count).  theta: host, c->n_params angles (may be NULL
 * when n_params == 0).  Gate matrices are built in fp64 on the host from
 * the angles.  fuse_k = 0 launches one kernel per gate; fuse_k >= 2 lets
 * the planner group gates into passes over shared-memory qubit blocks of
 * which each gate group acts on at most fuse_k qubits (fuse_k <= 5).
 * Asynchronous.  Errors: SV_ERR_INVALID (validated before any launch). */
sv_status sv_apply_circuit(sv_state s, const sv_circuit* c, const double* theta,
                           int fuse_k);

/* Host-only dry run of the fusion planner used by sv_apply_circuit with
 * fuse_k >= 2 (no GPU call).  order[0..n_gates) receives the circuit gate
 * indices in the order they will be applied, pass_of[k] the pass that
 * applies order[k] (-1: applied alone by the unfused kernels), *n_passes
 * the number of passes; if staged_bits is not NULL, staged_bits[2p] and
 * [2p+1] receive the low and high 32 bits of pass p's staged amplitude-index
 * bit mask.  Arrays are caller-owned with n_gates (staged_bits: 2 n_gates)
 * entries.  Errors: SV_ERR_INVALID. */
sv_status sv_fusion_plan(const sv_circuit* c, const double* theta, sv_dtype dtype, int fuse_k,
                         int32_t* order, int32_t* pass_of, int32_t* n_passes,
                         int32_t* staged_bits);

/* Host-only dry run of the reverse-sweep planner used by sv_grad_fused for
 * the gates [lo, hi) of c (no GPU call).  The sweep un-applies the gates in
 * reverse and takes each parameterised gate's gradient Im<lambda|P|psi>
 * before its un-apply (Sec. 3 gradients; the adjoint form); uncontrolled
 * 1-qubit adjoints on a qubit are multiplied until another gate touches
 * it, and gradients on one qubit with nothing else touching it in between
 * share one evaluation.  events receives, in execution order, 4 ints per
 * event: kind (0 un-apply of a gate, 1 gradient of a gate), the circuit gate
 * index, the pass (-1: applied alone by the unfused kernels) and, for
 * gradients, the evaluation id (gradients sharing one evaluation share it;
 * -1 for un-applies).  Caller-owned, 8 (hi - lo) ints.  *n_events: events
 * written; *n_passes: passes planned.  Errors: SV_ERR_INVALID. */
sv_status sv_fusion_plan_reverse(const sv_circuit* c, const double* theta, sv_dtype dtype,
                                 int fuse_k, int lo, int hi, int32_t* events,
                                 int32_t* n_events, int32_t* n_passes);

/* ---- reductions (fp64 accumulation, fixed reduction order) ------------ */

/* <psi|psi>.  Synchronises.  Result bit-identical across calls. */
sv_status sv_norm(sv_state s, double* out);

/* <psi|H|psi> for a Pauli sum (Sec. 3: Hamiltonians, VQE energies).
 * Products in the state's precision, accumulation in fp64, fixed tree.
 * sv_expval writes the host double `out` and synchronises; sv_expval_async
 * writes the device double `dev_out` and does not synchronise (usable
 * under stream capture).  SV_ERR_INVALID for masks with bits >= n. */
sv_status sv_expval(sv_state s, const sv_pauli_sum* H, double* out);
sv_status sv_expval_async(sv_state s, const sv_pauli_sum* H, double* dev_out);

/* <psi|H|psi> like sv_expval_async, for callers that cannot allocate device
 * memory at the time of the call: a process whose device memory is all
 * handed to a caching allocator or a fixed arena, or code that has no way
 * to recover from a failed allocation.  The paper has no counterpart; this
 * is a deployment variant of sv_expval_async.
 *
 * It allocates nothing and needs no handle: dev_state is the caller's
 * device state (2^n_qubits amplitudes of `dtype`, 16-byte aligned),
 * dev_out the caller's device double that receives the result, and the
 * kernels run on `cuda_stream` (NULL: the legacy default stream; otherwise a
 * stream of the current device, else SV_ERR_INVALID) without
 * synchronising.  The reduction's
 * block partials live in one fixed array of SV_NOALLOC_MAX_TERMS / 64 *
 * 1216 doubles (152 KiB) compiled into the library, which every GPU that
 * loads the library keeps until the process exits.
 *   - More than SV_NOALLOC_MAX_TERMS terms: SV_ERR_INVALID with a message.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream
 *     capture begins.
 *   - All calls share the array and each overwrites it (nothing in it has to
 *     start at zero), so calls that overlap on the GPU race: serialise them
 *     on one stream.
 * Errors: SV_ERR_INVALID (bad pointers, sizes or masks, nothing launched),
 * SV_ERR_CUDA. */
#define SV_NOALLOC_MAX_TERMS 1024
sv_status sv_expval_noalloc(const void* dev_state, int n_qubits, sv_dtype dtype,
                            const sv_pauli_sum* H, double* dev_out, void* cuda_stream);

/* out = H psi_in (a full state; Sec. 3 Hamiltonian applied to a state).
 * in and out must be distinct handles of equal n and dtype. Asynchronous. */
sv_status sv_apply_pauli_sum(sv_state out, sv_state in, const sv_pauli_sum* H);

/* ---- Pauli rotations and time evolution (Sec. 3: Hamiltonians, Trotter) - */

/* psi <- exp(-i theta P) psi for the Pauli string P = (xmask, zmask) (mask
 * convention as in sv_pauli_sum); exp(-i theta P) = cos(theta) I -
 * i sin(theta) P.  One HBM pass.  Asynchronous.  SV_ERR_INVALID for mask
 * bits beyond n or a non-finite angle. */
sv_status sv_pauli_rotation(sv_state s, uint64_t xmask, uint64_t zmask, double theta);

/* psi <- (Trotter product for exp(-i t H)) psi, H = sum_k c_k P_k, with
 * `steps` steps of dt = t / steps.  order 1: exp(-i c_k dt P_k) for
 * k = 0..K-1 per step; order 2: exp(-i c_k dt/2 P_k) for k = 0..K-1 and
 * then k = K-1..0 per step.  Runs of consecutive diagonal (Z-only) terms
 * commute and are applied in one pass.  Asynchronous. */
sv_status sv_trotter(sv_state s, const sv_pauli_sum* H, double t, int steps, int order);

/* ---- measurement (Sec. 3: sampling of measurements) -------------------- */

/* Measuring qubits[0..n_meas-1] in the computational basis gives outcome
 * r = sum_j b(qubits[j]) 2^(n_meas-1-j) (qubits[0] the most significant
 * bit) with P(r) = sum of |psi_x|^2 over the x whose measured bits spell r.
 *
 * sv_probabilities writes P(0..2^n_meas-1) to the host array `out` (fp64
 * sums in a fixed order; n_meas <= SV_MAX_MEASURE_PROBS); synchronises.
 *
 * sv_sample draws n_shots outcomes by the inverse CDF
 * c(x) = sum_{y <= x} |psi_y|^2: shot s is the first x with
 * c(x) > uniforms[s] * c(2^n - 1), projected onto the measured qubits.
 * uniforms (host, in [0, 1)) are the caller's random numbers; out (host,
 * n_shots) receives the outcomes; synchronises.  The state is not
 * collapsed.  Errors: SV_ERR_INVALID (bad qubits, counts, uniforms). */
#define SV_MAX_MEASURE_PROBS 24
#define SV_MAX_SHOTS (1LL << 26)
sv_status sv_probabilities(sv_state s, const int* qubits, int n_meas, double* out);
sv_status sv_sample(sv_state s, const int* qubits, int n_meas, int64_t n_shots,
                    const double* uniforms, uint64_t* out);

/* ---- gradients --------------------------------------------------------- */

/* Adjoint gradient of E(theta) = <psi_N|H|psi_N>, psi_N = U(theta) psi_0
 * (Sec. 2: automatic gradients of variational circuits, here by the adjoint
 * method).  On entry `s` holds psi_N as left by sv_apply_circuit(s, c,
 * theta, *) on psi_0; it is not modified.  The reverse sweep keeps two work
 * states (lambda = H psi and the un-applied psi) owned by the handle.
 * Parameterised gates must be RX/RY/RZ (with or without controls) or PAULI
 * (without controls); energy (host) and grad (host,
 * c->n_params doubles, gradients of gates sharing a parameter are summed)
 * are written and the stream is synchronised.  Gradients accumulate in
 * fp64. */
sv_status sv_adjoint(sv_state s, const sv_circuit* c, const double* theta,
                     const sv_pauli_sum* H, double* energy, double* grad);

/* Forward pass plus adjoint gradient with forward-state checkpoints.  On
 * entry `s` holds psi_0; on return it holds psi_N.  checkpoint_gates lists
 * n_checkpoints increasing gate indices g: the forward state before gate g
 * is stored, and the reverse sweep replaces its un-applied psi by that
 * stored state when it reaches g (this bounds the rounding drift of
 * un-applying in complex64).  n_checkpoints = 0 gives the plain sweep.
 * Outputs as sv_adjoint. */
sv_status sv_grad(sv_state s, const sv_circuit* c, const double* theta,
                  const sv_pauli_sum* H, const int32_t* checkpoint_gates,
                  int n_checkpoints, double* energy, double* grad);

/* sv_grad with the forward circuit and the reverse sweep run as fused
 * qubit-block passes.  fuse_k as in sv_apply_circuit (0: exactly sv_grad;
 * 2..5).  Checkpoints split the circuit into segments that are fused
 * separately, so no gate moves across a checkpoint.  A reverse pass stages
 * psi and lambda together (one staged bit fewer than a forward pass,
 * register groups of at most 4 qubits for complex64 and 3 for complex128);
 * before un-applying each parameterised gate it accumulates that gate's
 * Im<lambda|P|psi> (gradients on one qubit with nothing else touching it in
 * between share one evaluation), per warp in compensated fp32 and per block
 * in fp64, and a fixed-order finish adds the block sums.  States of fewer
 * than 10 qubits, or passes without a bulk-copy geometry, take the unfused
 * sweep.  Outputs, checkpoints and errors as sv_grad. */
sv_status sv_grad_fused(sv_state s, const sv_circuit* c, const double* theta,
                        const sv_pauli_sum* H, const int32_t* checkpoint_gates,
                        int n_checkpoints, int fuse_k, double* energy, double* grad);

/* ---- batched energies and gradients (one persistent launch) ------------ */

/* Many small variational circuits at once (Sec. 3: variational layers and
 * VQE; Sec. 2 gradients): item i runs circuits[item_circuit[i]] from
 * |0...0> in complex64, evaluates E_i = <psi|H|psi> with
 * hamiltonians[item_circuit[i]] and the adjoint gradient dE_i/dtheta.  All
 * items run in one persistent kernel whose thread blocks pull items from an
 * atomic queue (longest first); each block keeps its item's two states in a
 * workspace slot that stays in L1/L2, or (a variant the autotuner may pick)
 * psi of up to 14 qubits and lambda of up to 13 in shared memory.  Energies
 * and gradients accumulate per warp in compensated fp32 and across warps in
 * fp64, in a fixed order.  A batch whose gates are all real (H X Z RY, with
 * controls) and whose terms are all real matrices (an even number of Y
 * factors) keeps real states: a variant the autotuner may pick carries psi
 * and lambda as fp32 real vectors (psi of up to 15 qubits and lambda of up to
 * 14 in shared memory), with the same results up to rounding.
 *
 * Limits: <= SV_BATCH_MAX_QUBITS qubits, <= 480 gates and <= 256
 * parameters per circuit, <= 64 Pauli terms per Hamiltonian; gates are the
 * 1-qubit kinds H X Y Z RX RY RZ U1 with up to 3 controls (CZ = Z with a
 * control), parameters on RX/RY/RZ only.  Violations: SV_ERR_INVALID.
 *
 * Parameters are packed per item in item order: item i's n_params angles
 * start at the sum of the parameter counts of items 0..i-1 (sv_batch_info
 * gives the total).  Gradients use the same packing.
 *
 * sv_batch_create uploads the descriptors and allocates the workspace.
 * tune = 0: single blocks of 256 threads, 2 per SM, register groups of k = 4
 * qubits, states in a global workspace slot per block.  tune = 1: the
 * autotuner times every (register-group width k in {2,3,4}, kernel: those
 * single blocks with 128/256/512 threads and 1/2/4/8 blocks per SM, single
 * blocks of 512 threads keeping psi (and lambda up to 13 qubits) in shared
 * memory up to 14 qubits, or two-block clusters of 512 threads that split each item's psi and lambda by
 * their top bit over the pair and keep them in shared memory up to 14 qubits,
 * k <= 3) on the batch and keeps the fastest (this synchronises the device).
 * For a real batch the autotuner also times the real-amplitude kernel
 * (single blocks of 512 threads, k in {3,4,5}).
 * tune = 2: the cluster kernel with k = 3 (the tune = 0 tile if a gate has 3
 * controls); tune = 3: single blocks of 512 threads with states in shared
 * memory, k = 4; tune = 4: the real-amplitude kernel, k = 4 (SV_ERR_INVALID
 * for a batch that is not real).  Other values: SV_ERR_INVALID.  The handle is
 * library-owned; sv_batch_free releases it. */
#define SV_BATCH_MAX_QUBITS 18
typedef struct sv_batch_s* sv_batch;

sv_status sv_batch_create(const sv_circuit* circuits, const sv_pauli_sum* hamiltonians,
                          int n_circuits, const int32_t* item_circuit, int n_items, int tune,
                          sv_batch* out);

/* Host-only dry run of the batch planner (no GPU call): validates the
 * circuits and Hamiltonians as sv_batch_create does and writes, per
 * circuit, the number of register groups of width k (max(2, widest gate)
 * <= k <= 5; 5 is the real-amplitude kernel's widest) its gates are
 * scheduled into.  Errors: SV_ERR_INVALID. */
sv_status sv_batch_plan(const sv_circuit* circuits, const sv_pauli_sum* hamiltonians,
                        int n_circuits, int k, int32_t* groups_per_circuit);

/* Chosen tile (k, threads per block, blocks) and total parameter count. */
sv_status sv_batch_info(sv_batch b, int* k, int* threads, int* blocks, int* total_params);

/* The chosen kernel: cluster_size 2 for the two-block cluster kernel (each
 * item's psi and lambda split by their top bit over the pair), else 1;
 * smem_states 1 if the kernel keeps small items' states in shared memory;
 * real_states 1 for the real-amplitude kernel.  SV_ERR_INVALID for a null
 * handle or output. */
sv_status sv_batch_kernel(sv_batch b, int* cluster_size, int* smem_states, int* real_states);

/* One persistent launch (a queue reset plus the kernel) on cuda_stream;
 * dev_theta, dev_energy (n_items) and dev_grad (total_params) are device
 * arrays.  Asynchronous; usable under stream capture. */
sv_status sv_batch_run(sv_batch b, const double* dev_theta, double* dev_energy, double* dev_grad,
                       void* cuda_stream);

/* The same launch through a CUDA graph the handle captures on first use
 * for these pointers and this stream and replays afterwards. */
sv_status sv_batch_run_graph(sv_batch b, const double* dev_theta, double* dev_energy,
                             double* dev_grad, void* cuda_stream);

/* One-shot host convenience: create (no tuning), copy theta from the host,
 * run, copy energies and gradients back to the host, free.  Synchronises. */
sv_status sv_batch_grad(const sv_circuit* circuits, const sv_pauli_sum* hamiltonians,
                        int n_circuits, const int32_t* item_circuit, int n_items,
                        const double* theta, void* cuda_stream, double* energies, double* grads);

sv_status sv_batch_free(sv_batch b);

/* ---- status ------------------------------------------------------------ */

/* Synchronise the stream and surface any asynchronous error; SV_ERR_TIMEOUT
 * if a bulk-copy pass gave up waiting for its copies (each such wait is
 * bounded by 1 s of GPU time, after which the pass's blocks record the
 * timeout and return without storing; the status is cleared when read). */
sv_status sv_sync(sv_state s);

/* States from sv_alloc, and the work states of the adjoint sweeps, are
 * allocated between two 4 KiB guard regions filled with a fixed byte.
 * sv_check_guards synchronises the stream and checks every guard of the
 * handle: SV_ERR_CUDA (with the region and offset in sv_last_error) if a
 * kernel wrote outside its state; SV_OK otherwise (a state from sv_wrap has
 * no guards of its own).  A substitute for a memory checker in tests. */
sv_status sv_check_guards(sv_state s);

/* Self-test of that bounded wait: queues one bulk-copy pass over the state
 * that applies no gate and whose barrier expects more bytes than it copies,
 * so its waits run out (about 1 s); the following sv_sync returns
 * SV_ERR_TIMEOUT and the state is unchanged.  No GPU fault is involved and
 * the context stays usable.  States of at least 10 qubits; SV_ERR_INVALID
 * otherwise.  Asynchronous.  (A test aid: the paper has no counterpart.) */
sv_status sv_selftest_wait(sv_state s);

/* Message describing the calling thread's last failure ("" if none). */
const char* sv_last_error(void);

/* Tracing: between sv_profile_start() and sv_profile_stop() every kernel
 * launch of the library is bracketed by two CUDA events on its stream.
 * sv_profile_stop synchronises on the last event and writes one line per
 * kernel name, "name launches total_ms\n", into buf (NUL-terminated);
 * SV_ERR_INVALID if buf is NULL or too small.  Not for use while a stream is
 * being captured into a CUDA graph. */
sv_status sv_profile_start(void);
sv_status sv_profile_stop(char* buf, size_t len);

/* Number of kernels this process has launched through the library. */
uint64_t sv_launch_count(void);

/* ABI version (major * 100 + minor). */
int sv_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SV_H */
