// Internal declarations of libsv: the state handle, error plumbing, the
// kernel launchers shared by the C-ABI translation unit and the kernel
// translation units.  Bit conventions: kernels speak in amplitude-index bit
// positions p (qubit q <-> p = n-1-q).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "sv.h"

namespace sv {

// ---- errors ----------------------------------------------------------------
void set_error(const char* fmt, ...);
extern std::atomic<uint64_t> g_launches;

#define SV_CUDA_TRY(expr)                                                   \
  do {                                                                      \
    cudaError_t e_ = (expr);                                                \
    if (e_ != cudaSuccess) {                                                \
      ::sv::set_error("%s failed: %s", #expr, cudaGetErrorString(e_));      \
      return e_ == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA;    \
    }                                                                       \
  } while (0)

// Check the most recent launch on this thread.
sv_status check_launch(const char* what);

// Per-launch CUDA-event timing while sv_profile_start() is active: the
// scope records an event before and after the launch it encloses, tagged
// with the kernel's name.  Inactive scopes cost one atomic load.
struct ProfScope {
  ProfScope(cudaStream_t st, const char* name);
  ~ProfScope();
  cudaStream_t st;
  int slot;
};

// ---- complex gate matrices on the host (fp64) ------------------------------
struct cd {
  double re, im;
};

// Up to 32 x 32 row-major.
struct HostMatrix {
  int k = 1;  // number of targets
  cd m[32 * 32];
  cd at(int r, int c) const { return m[r * (1 << k) + c]; }
};

// Builds the fp64 matrix of a circuit record (kinds of sv.h).  Returns false
// for an unknown kind or a wrong target count.
bool gate_matrix(const sv_gate& g, const double* theta, const double* pool, HostMatrix* out);

// ---- complex64 coefficients: rounding with error feedback --------------------
// Rounding a unitary to fp32 leaves it slightly non-unitary.  Applied without
// controls, the rounded matrix fl(G) scales the squared norm of the state by
// ||fl(G)||_F^2 / 2^k averaged over states - exactly, on every state, for
// H and for Pauli rotations, whose rounded forms are multiples of unitaries.
// For H that factor is 2 fl(1/sqrt2)^2 = 1 - 3.4e-8, so N Hadamards lose
// N * 3.4e-8 of ||psi||^2: a bias that grows with the gate count.  A state
// therefore carries `drift`, the log of the factor its roundings have applied
// so far, and each inexact matrix is scaled by exp(-drift / 2) before it is
// rounded: once the accumulated factor is off by more than half an fp32 step,
// the entries round the other way, and the factor stays within about 1e-7 of
// 1 however many gates run.  Matrices whose entries are fp32 numbers (X, Z,
// CZ, SWAP, ...) are left untouched.
//
// feedback_round scales the d x d row-major matrix m in place (when drift is
// not null and some entry is not an fp32 number) and adds the log of the
// rounded matrix's mean squared column norm to *drift.  feedback_round_diag
// does the same for a diagonal of d entries whose exact mean squared modulus
// is mean_sq (1 for a unitary diagonal; a scaled one, as in the rotation
// form of the fused layer programs, states its own).  feedback_round_pair
// treats a Pauli rotation c I + k P (P^2 = I, Hermitian) with factor
// |c|^2 + |k|^2.
void feedback_round(cd* m, int d, double* drift);
void feedback_round_diag(cd* dg, int d, double* drift, double mean_sq = 1.0);
void feedback_round_pair(double* c, cd* k, double* drift);

// A state's complex64 rounding context: the feedback factor above and the
// launch sequence that seeds the kernels' dithered rounding (mix32 of it;
// restarting with the state keeps results reproducible).  Null: plain
// rounding, no dither.
struct RoundCtx {
  double drift = 0.0;
  uint32_t seq = 0;
  int mode = SV_ROUNDING_DEFAULT;  // sv_set_rounding; kept across resets
  void reset() {
    drift = 0.0;
    seq = 0;
  }
  uint32_t next_seed() { return ((++seq) * 0x9E3779B9u) | 1u; }
};

// ---- reduction geometry -----------------------------------------------------
constexpr int kRedThreads = 256;
constexpr int kRedMaxBlocks = 1216;  // 152 SMs x 8
int red_blocks(uint64_t units);

}  // namespace sv

// ---- the state handle --------------------------------------------------------
struct sv_state_s {
  void* data = nullptr;
  void* base = nullptr;  // allocation of an owned state: guard, data, guard
  int n = 0;
  sv_dtype dt = SV_C64;
  cudaStream_t stream = nullptr;
  bool owned = false;
  int device = 0;
  // complex64 rounding context since the state was last set (see RoundCtx)
  sv::RoundCtx rc;
  // fp64 reduction scratch: partials and device results
  double* partials = nullptr;
  size_t partials_cap = 0;  // doubles
  double* dres = nullptr;   // 64 doubles of device results
  double* hres = nullptr;   // pinned host mirror of dres
  // adjoint work states and forward checkpoints
  void* work[2] = {nullptr, nullptr};
  void* work_base[2] = {nullptr, nullptr};  // their allocations (guarded like data)
  std::vector<void*> ckpt;
  size_t bytes() const { return (size_t(1) << n) * (dt == SV_C64 ? 8 : 16); }
};

namespace sv {

// Library-owned states (and the adjoint's work states) sit between two
// kGuardBytes regions filled with kGuardByte; sv_check_guards verifies them.
constexpr size_t kGuardBytes = 4096;
constexpr unsigned char kGuardByte = 0xA5;
// Allocates guard | bytes | guard, fills the guards; *data = base + guard.
sv_status alloc_guarded(size_t bytes, void** base, void** data);

sv_status ensure_partials(sv_state s, size_t doubles);
sv_status ensure_work(sv_state s, int which);

// ---- gate launchers (gate_kernels.cu) -----------------------------------------
// Applies matrix G on target bit positions tp[0..k-1] (tp[0] = MSB of tau)
// where all bit positions cp[0..nc-1] are 1.  Picks the specialised kernel
// from the matrix structure (phase-on-subspace, diagonal, real, swap,
// dense 1-qubit, generic k-qubit).  rc: the state's complex64 rounding
// context (feedback for gates without controls, dithered rounding of the
// 1-qubit kernels); null for plain rounding.
sv_status launch_gate(void* data, sv_dtype dt, int n, cudaStream_t st, int k, const int* tp,
                      int nc, const int* cp, const HostMatrix& G, RoundCtx* rc = nullptr);

sv_status launch_init(void* data, sv_dtype dt, int n, cudaStream_t st, uint64_t basis);

// ---- reductions (reduce_kernels.cu) --------------------------------------------
struct PauliDev {
  // terms after host preprocessing: coefficient times i^{#Y}, folded to
  // (cre, cim); the sign (-1)^popcount((x ^ xm) & zm) is applied per index.
  int nt;
  int nd;  // the first nd terms are diagonal (xm = 0)
  uint64_t xm[64];
  uint64_t zm[64];
  double cre[64];
  double cim[64];
  float cre32[64];  // the same, rounded once for complex64 states
  float cim32[64];
};
// Fills PauliDev chunks (64 terms each) from a host Pauli sum.
void pauli_chunks(const sv_pauli_sum* H, std::vector<PauliDev>* out);

// sum over blocks -> partials[0..blocks); returns the number of partials.
sv_status launch_norm_partials(sv_state s, double* partials, int* nparts);
sv_status launch_expval_partials(sv_state s, const PauliDev& P, double* partials, int* nparts);
// out = H in; if partials != NULL also Re<in|out> per block.
sv_status launch_apply_pauli(void* out, const void* in, sv_dtype dt, int n, cudaStream_t st,
                             const PauliDev& P, bool accumulate, double* partials,
                             int* nparts);
// <psi|H|psi> into the device double dst by staged passes (pauli_kernels.cu);
// SV_ERR_UNSUPPORTED with nothing launched when passes do not apply.
sv_status expval_staged(sv_state s, const sv_pauli_sum* H, double* dst);
// lambda = H psi (and <psi|H|psi> into energy_dst if not null) with the
// diagonal terms streamed; SV_ERR_UNSUPPORTED (nothing launched) where it
// does not apply (under 16 qubits, no diagonal term).
sv_status apply_pauli_staged(void* out, const void* in, sv_state s, const sv_pauli_sum* H,
                             double* energy_dst);
// Reads and clears the Pauli-pass status word (kWaitTimeout).
unsigned take_pauli_status();
// dst[j] = sum_{i<count} src[j * count + i] for j < slots (fixed order).
sv_status launch_finish(const double* src, int count, int slots, double* dst,
                        cudaStream_t st, bool add_to_dst);

// ---- fusion (planner.cu, fused_kernels.cu) ------------------------------------
// A gate as the fused kernels see it, in amplitude-index bit positions.
// FG_GRAD (reverse sweeps only): accumulate Im<lambda|P|psi> for generator
// `pauli` (1 X, 2 Y, 3 Z; 0: the Hermitian 2x2 in m) on bit t, restricted to
// the control bits cmask, into gradient slot `slot`; it precedes the
// un-applied gate whose derivative it gives.  ng > 1: ng gradients on the
// same uncontrolled bit evaluated at one place, generator i in gen[i] =
// (a, d, re b, im b) of [[a, b], [conj b, d]], slot gslots[i].
enum { FG_1Q = 0, FG_PHASE = 1, FG_SWAP = 2, FG_ALONE = 3, FG_GRAD = 4 };
constexpr int kGradPerOp = 4;
struct FGate {
  int type = FG_ALONE;
  int pauli = 0, slot = -1;  // FG_GRAD; an FG_ALONE gate of a reverse sweep with a gradient
  int ng = 1;                // FG_GRAD: gradients of this operation
  int gslots[kGradPerOp] = {};
  double gen[kGradPerOp][4] = {};
  uint64_t qmask = 0;  // every bit the gate touches (targets and controls)
  uint64_t cmask = 0;  // control bits (FG_1Q, FG_SWAP); all bits for FG_PHASE
  int t = 0, a = 0, b = 0;  // FG_1Q target bit; FG_SWAP bits
  cd m[4] = {};        // FG_1Q: 2x2 row-major; FG_PHASE: m[0] = phase
  int orig = -1;       // index of the (last merged) circuit gate
  std::vector<int> origs;  // every circuit gate folded into this one
};

struct FusedGroup {
  int k = 0;                 // staged-local bits of the group, ascending
  int bits[5] = {0, 0, 0, 0, 0};
  std::vector<int> ops;      // indices into the pass's gate list, in order
};

struct FusedPass {
  std::vector<int> S;        // staged bit positions, ascending; S[0..L) = 0..L-1
  int L = 0;
  std::vector<FGate> gates;  // the pass's gates (bits are global)
  std::vector<FusedGroup> groups;
};

struct FusionItem {
  bool is_pass = false;
  FusedPass pass;            // when is_pass
  int gate = -1;             // circuit gate index to run unfused otherwise
  int pauli = 0, slot = -1;  // reverse sweeps: the unfused gate's gradient, if any
};

struct FusionConfig {
  int fuse_k = 4;            // max qubits per register group
  int m = 13;                // staged bits per block
  int L = 5;                 // low bits staged as contiguous runs
  int max_ops = 200;         // gate capacity of one pass
  int max_grads = 200;       // gradient capacity of one pass (reverse sweeps)
  int max_groups = 64;       // group capacity of one pass
};

FusionConfig fusion_config(int n, sv_dtype dt, int fuse_k);
// Reverse sweeps stage two slices (psi, lambda) and hold two register tiles
// per thread: one staged bit fewer, register groups of at most 3 qubits.
FusionConfig fusion_config_reverse(int n, sv_dtype dt, int fuse_k);
// Plans `c` into passes and unfused gates; returns false (with an error
// set) if a matrix cannot be built.
bool plan_fusion(const sv_circuit* c, const double* theta, const FusionConfig& cfg,
                 std::vector<FusionItem>* out);
// Plan of the reverse sweep over gates [lo, hi): gates hi-1 .. lo as their
// adjoints, each parameterised gate preceded by its FG_GRAD; slot_of[i] is
// the gradient slot of circuit gate i (or -1).  Unfused items carry the
// circuit gate (to be un-applied) and its gradient slot.
bool plan_fusion_reverse(const sv_circuit* c, const double* theta, int lo, int hi,
                         const std::vector<int>& slot_of, const FusionConfig& cfg,
                         std::vector<FusionItem>* out);
// rc: the state's complex64 rounding context (null: plain rounding)
sv_status launch_fused_pass(void* data, sv_dtype dt, int n, cudaStream_t st,
                            const FusedPass& pass, RoundCtx* rc = nullptr);
// Reverse-sweep pass over psi and lambda (gradient operations write
// partials[slot * pstride + block], pstride >= the pass's block count; at
// most pstride blocks are launched).  fused_reverse_ok: the pass has a
// bulk-copy geometry (else the caller runs the unfused sweep).
bool fused_reverse_ok(sv_dtype dt, int n, const FusedPass& pass);
sv_status launch_fused_reverse_pass(void* psi, void* lam, sv_dtype dt, int n, cudaStream_t st,
                                    const FusedPass& pass, double* partials, int pstride);
// One bulk-copy pass armed for more bytes than it copies (its bounded waits
// give up; the state is unchanged); see sv_selftest_wait.
sv_status launch_wait_selftest(void* data, sv_dtype dt, int n, cudaStream_t st);
// Reads and clears the fused-pass device status word of the current device
// (kWaitTimeout = 1: a bounded wait inside a pass gave up).
unsigned take_fused_status();

// ---- Pauli-string rotations (evolve_kernels.cu) --------------------------------
// psi <- exp(-i a P) psi for the Pauli string P = (xm, zm) (mask convention
// of sv_pauli_sum); rc as in launch_gate.
sv_status launch_pauli_rotation(void* data, sv_dtype dt, int n, cudaStream_t st, uint64_t xm,
                                uint64_t zm, double a, RoundCtx* rc = nullptr);
// Reverse-sweep step of U = exp(-i theta P / 2): Im<lam|P|psi> into
// partials[0..nparts) (nparts = the 1-qubit adjoint's fixed grid), then
// psi, lam <- U^dagger psi, U^dagger lam.
sv_status launch_adjoint_pauli(void* psi, void* lam, sv_dtype dt, int n, cudaStream_t st,
                               uint64_t xm, uint64_t zm, double theta, double* partials,
                               int* nparts);

// ---- adjoint (adjoint_kernels.cu) ----------------------------------------------
// Un-applies U^dagger (given as matrix Gdag on bit tp, controls cp) on both
// psi and lam; if pauli in {1,2,3} (X, Y, Z generator) first accumulates
// Im<lam|P|psi> restricted to the control subspace into
// partials[0..nparts).
sv_status launch_adjoint_1q(void* psi, void* lam, sv_dtype dt, int n, cudaStream_t st, int tp,
                            int nc, const int* cp, const HostMatrix& Gdag, int pauli,
                            double* partials, int* nparts);

}  // namespace sv
