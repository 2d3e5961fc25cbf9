// C-ABI entry points of libsv (declared in include/sv.h): validation,
// gate-matrix construction in fp64 on the host, the gate-by-gate circuit
// loop (Sec. 2, Eq. 1 per gate), reductions and the adjoint gradient.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "sv_internal.cuh"

namespace sv {

std::atomic<uint64_t> g_launches{0};
static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

sv_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s launch failed: %s", what, cudaGetErrorString(e));
    return SV_ERR_CUDA;
  }
  return SV_OK;
}

// ---- per-launch profiling -------------------------------------------------------
namespace {
struct ProfRec {
  const char* name;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
std::vector<ProfRec> g_prof_recs;
size_t g_prof_used = 0;
}  // namespace

ProfScope::ProfScope(cudaStream_t s, const char* name) : st(s), slot(-1) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_prof_used == g_prof_recs.size()) {
    ProfRec r{name, nullptr, nullptr};
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
    g_prof_recs.push_back(r);
  }
  slot = (int)g_prof_used++;
  g_prof_recs[slot].name = name;
  cudaEventRecord(g_prof_recs[slot].a, st);
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEventRecord(g_prof_recs[slot].b, st);
}

// Gate matrices, fp64 (c = cos(a/2), s = sin(a/2)).
bool gate_matrix(const sv_gate& g, const double* theta, const double* pool, HostMatrix* out) {
  const double a = g.param >= 0 ? theta[g.param] : g.angle;
  const double c = std::cos(0.5 * a), s = std::sin(0.5 * a);
  const double r = 0.70710678118654752440;
  cd* m = out->m;
  out->k = 1;
  for (int e = 0; e < 4; ++e) m[e] = {0.0, 0.0};
  switch (g.kind) {
    case SV_GATE_H: m[0] = {r, 0}; m[1] = {r, 0}; m[2] = {r, 0}; m[3] = {-r, 0}; break;
    case SV_GATE_X: m[1] = {1, 0}; m[2] = {1, 0}; break;
    case SV_GATE_Y: m[1] = {0, -1}; m[2] = {0, 1}; break;
    case SV_GATE_Z: m[0] = {1, 0}; m[3] = {-1, 0}; break;
    case SV_GATE_RX: m[0] = {c, 0}; m[1] = {0, -s}; m[2] = {0, -s}; m[3] = {c, 0}; break;
    case SV_GATE_RY: m[0] = {c, 0}; m[1] = {-s, 0}; m[2] = {s, 0}; m[3] = {c, 0}; break;
    case SV_GATE_RZ: m[0] = {c, -s}; m[3] = {c, s}; break;
    case SV_GATE_U1: m[0] = {1, 0}; m[3] = {std::cos(a), std::sin(a)}; break;
    case SV_GATE_SWAP:
      out->k = 2;
      for (int e = 0; e < 16; ++e) m[e] = {0.0, 0.0};
      m[0] = {1, 0}; m[1 * 4 + 2] = {1, 0}; m[2 * 4 + 1] = {1, 0}; m[15] = {1, 0};
      break;
    case SV_GATE_MATRIX: {
      out->k = g.n_tar;
      const int d = 1 << g.n_tar;
      const double* p = pool + 2 * g.mat_off;
      for (int e = 0; e < d * d; ++e) m[e] = {p[2 * e], p[2 * e + 1]};
      break;
    }
    case SV_GATE_PAULI: {
      // c I - i s P, P[tau][tau'] = prod_j sigma_{L_j}[b_j(tau)][b_j(tau')]
      // with b_j the bit of target j (t_0 the most significant)
      if (g.n_tar < 1 || g.n_tar > SV_MAX_TARGETS) return false;
      out->k = g.n_tar;
      const int k = g.n_tar, d = 1 << k;
      static const cd sig[4][4] = {{{1, 0}, {0, 0}, {0, 0}, {1, 0}},
                                   {{0, 0}, {1, 0}, {1, 0}, {0, 0}},
                                   {{0, 0}, {0, -1}, {0, 1}, {0, 0}},
                                   {{1, 0}, {0, 0}, {0, 0}, {-1, 0}}};
      for (int r = 0; r < d; ++r)
        for (int q = 0; q < d; ++q) {
          cd p{1, 0};
          for (int j = 0; j < k; ++j) {
            const int L = (g.paulis >> (2 * j)) & 3;
            const int br = (r >> (k - 1 - j)) & 1, bq = (q >> (k - 1 - j)) & 1;
            const cd f = sig[L][br * 2 + bq];
            p = {p.re * f.re - p.im * f.im, p.re * f.im + p.im * f.re};
          }
          // c delta - i s p
          m[r * d + q] = {(r == q ? c : 0.0) + s * p.im, -s * p.re};
        }
      break;
    }
    default: return false;
  }
  return out->k == g.n_tar;
}

// Masks of a PAULI gate's string in amplitude-index bits (qubit q <-> bit
// n-1-q): X sets x, Z sets z, Y sets both.
void pauli_masks(int n, const sv_gate& g, uint64_t* xm, uint64_t* zm) {
  *xm = *zm = 0;
  for (int j = 0; j < g.n_tar; ++j) {
    const int L = (g.paulis >> (2 * j)) & 3;
    const uint64_t b = uint64_t(1) << (n - 1 - g.targets[j]);
    if (L == 1 || L == 2) *xm |= b;
    if (L == 2 || L == 3) *zm |= b;
  }
}

namespace {
bool fp32_number(double x) { return (double)(float)x == x; }
double sq32(cd z) {
  const double r = (float)z.re, i = (float)z.im;
  return r * r + i * i;
}
}  // namespace

void feedback_round(cd* m, int d, double* drift) {
  if (!drift) return;
  bool exact = true;
  for (int e = 0; e < d * d && exact; ++e) exact = fp32_number(m[e].re) && fp32_number(m[e].im);
  if (exact) return;
  const double f = std::exp(-0.5 * *drift);
  double t = 0.0;
  for (int e = 0; e < d * d; ++e) {
    m[e].re *= f;
    m[e].im *= f;
    t += sq32(m[e]);
  }
  *drift += std::log(t / d);
}

void feedback_round_diag(cd* dg, int d, double* drift, double mean_sq) {
  if (!drift) return;
  bool exact = true;
  for (int e = 0; e < d && exact; ++e) exact = fp32_number(dg[e].re) && fp32_number(dg[e].im);
  if (exact) return;
  const double f = std::exp(-0.5 * *drift);
  double t = 0.0;
  for (int e = 0; e < d; ++e) {
    dg[e].re *= f;
    dg[e].im *= f;
    t += sq32(dg[e]);
  }
  *drift += std::log(t / (d * mean_sq));
}

void feedback_round_pair(double* c, cd* k, double* drift) {
  if (!drift || (fp32_number(*c) && fp32_number(k->re) && fp32_number(k->im))) return;
  const double f = std::exp(-0.5 * *drift);
  *c *= f;
  k->re *= f;
  k->im *= f;
  const double cr = (float)*c;
  *drift += std::log(cr * cr + sq32(*k));
}

static void dagger(const HostMatrix& G, HostMatrix* D) {
  const int d = 1 << G.k;
  D->k = G.k;
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) D->m[r * d + c] = {G.m[c * d + r].re, -G.m[c * d + r].im};
}

// Gate i of c applied to the state in the forward direction: PAULI gates by
// the Pauli-rotation kernels (one pass, whatever the string), every other
// kind by its matrix (Eq. 1).  Rounding feedback from the state.
static sv_status apply_circuit_gate(sv_state s, const sv_circuit* c, int i,
                                    const double* theta) {
  const sv_gate& g = c->gates[i];
  if (g.kind == SV_GATE_PAULI) {
    uint64_t xm, zm;
    pauli_masks(s->n, g, &xm, &zm);
    const double a = g.param >= 0 ? theta[g.param] : g.angle;
    return launch_pauli_rotation(s->data, s->dt, s->n, s->stream, xm, zm, 0.5 * a, &s->rc);
  }
  static thread_local HostMatrix G;
  if (!gate_matrix(g, theta, c->mat_pool, &G)) {
    set_error("gate %d: cannot build matrix", i);
    return SV_ERR_INVALID;
  }
  int tp[SV_MAX_TARGETS], cp[SV_MAX_CONTROLS];
  for (int j = 0; j < g.n_tar; ++j) tp[j] = s->n - 1 - g.targets[j];
  for (int j = 0; j < g.n_ctrl; ++j) cp[j] = s->n - 1 - g.controls[j];
  return launch_gate(s->data, s->dt, s->n, s->stream, g.n_tar, tp, g.n_ctrl, cp, G, &s->rc);
}

// Reverse-sweep step for gate i of c on (psi, lam): un-apply it on both
// states; a parameterised gate first adds Im<lam|P|psi> into `part`
// (nullptr: no gradient).  PAULI strings by their own kernel, 1-qubit gates
// by the 1-qubit adjoint kernel, wider gates by their adjoint matrix.
static sv_status unapply_circuit_gate(sv_state s, void* psi, void* lam, const sv_circuit* c,
                                      int i, const double* theta, double* part) {
  const sv_gate& g = c->gates[i];
  if (g.kind == SV_GATE_PAULI) {
    uint64_t xm, zm;
    pauli_masks(s->n, g, &xm, &zm);
    const double a = g.param >= 0 ? theta[g.param] : g.angle;
    return launch_adjoint_pauli(psi, lam, s->dt, s->n, s->stream, xm, zm, a,
                                g.param >= 0 ? part : nullptr, nullptr);
  }
  static thread_local HostMatrix G, D;
  if (!gate_matrix(g, theta, c->mat_pool, &G)) {
    set_error("gate %d: cannot build matrix", i);
    return SV_ERR_INVALID;
  }
  dagger(G, &D);
  int tp[SV_MAX_TARGETS], cp[SV_MAX_CONTROLS];
  for (int j = 0; j < g.n_tar; ++j) tp[j] = s->n - 1 - g.targets[j];
  for (int j = 0; j < g.n_ctrl; ++j) cp[j] = s->n - 1 - g.controls[j];
  if (g.n_tar == 1) {
    const int pauli = (g.param < 0 || !part) ? 0
                      : g.kind == SV_GATE_RX ? 1
                      : g.kind == SV_GATE_RY ? 2
                                             : 3;
    return launch_adjoint_1q(psi, lam, s->dt, s->n, s->stream, tp[0], g.n_ctrl, cp, D, pauli,
                             pauli ? part : nullptr, nullptr);
  }
  sv_status st = launch_gate(psi, s->dt, s->n, s->stream, g.n_tar, tp, g.n_ctrl, cp, D);
  if (st == SV_OK) st = launch_gate(lam, s->dt, s->n, s->stream, g.n_tar, tp, g.n_ctrl, cp, D);
  return st;
}

sv_status ensure_partials(sv_state s, size_t doubles) {
  if (s->partials_cap >= doubles) return SV_OK;
  if (s->partials) cudaFree(s->partials);
  s->partials = nullptr;
  s->partials_cap = 0;
  SV_CUDA_TRY(cudaMalloc(&s->partials, doubles * sizeof(double)));
  s->partials_cap = doubles;
  return SV_OK;
}

sv_status alloc_guarded(size_t bytes, void** base, void** data) {
  *base = *data = nullptr;
  cudaError_t e = cudaMalloc(base, bytes + 2 * kGuardBytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *base = nullptr;
    set_error("allocation of %zu bytes: %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA;
  }
  char* b = static_cast<char*>(*base);
  e = cudaMemset(b, kGuardByte, kGuardBytes);
  if (e == cudaSuccess) e = cudaMemset(b + kGuardBytes + bytes, kGuardByte, kGuardBytes);
  if (e != cudaSuccess) {
    cudaFree(*base);
    *base = nullptr;
    set_error("guard fill: %s", cudaGetErrorString(e));
    return SV_ERR_CUDA;
  }
  *data = b + kGuardBytes;
  return SV_OK;
}

sv_status ensure_work(sv_state s, int which) {
  if (s->work[which]) return SV_OK;
  return alloc_guarded(s->bytes(), &s->work_base[which], &s->work[which]);
}

}  // namespace sv

using namespace sv;

// ---- validation ------------------------------------------------------------------
static bool valid_state(sv_state s) {
  if (!s || !s->data) {
    set_error("null state handle");
    return false;
  }
  return true;
}

static bool valid_qubits(int n, const int* t, int nt, const int* c, int nc) {
  if (nt < 1 || nt > SV_MAX_TARGETS) {
    set_error("n_tar = %d outside 1..%d", nt, SV_MAX_TARGETS);
    return false;
  }
  if (nc < 0 || nc > SV_MAX_CONTROLS || nt + nc > n) {
    set_error("n_ctrl = %d invalid for %d targets on %d qubits", nc, nt, n);
    return false;
  }
  if (!t || (nc > 0 && !c)) {
    set_error("null target or control array");
    return false;
  }
  uint64_t seen = 0;
  for (int j = 0; j < nt + nc; ++j) {
    const int q = j < nt ? t[j] : c[j - nt];
    if (q < 0 || q >= n) {
      set_error("qubit %d outside 0..%d", q, n - 1);
      return false;
    }
    if (seen & (uint64_t(1) << q)) {
      set_error("qubit %d repeated among targets and controls", q);
      return false;
    }
    seen |= uint64_t(1) << q;
  }
  return true;
}

static bool valid_circuit(sv_state s, const sv_circuit* c, const double* theta) {
  if (!c) {
    set_error("null circuit");
    return false;
  }
  if (c->n_qubits != s->n) {
    set_error("circuit has %d qubits, state has %d", c->n_qubits, s->n);
    return false;
  }
  if (c->n_gates < 0 || (c->n_gates > 0 && !c->gates) || c->n_params < 0) {
    set_error("bad gate list");
    return false;
  }
  if (c->n_params > 0 && !theta) {
    set_error("theta is NULL but the circuit has %d parameters", c->n_params);
    return false;
  }
  for (int i = 0; i < c->n_gates; ++i) {
    const sv_gate& g = c->gates[i];
    if (g.kind < SV_GATE_H || g.kind > SV_GATE_PAULI) {
      set_error("gate %d: unknown kind %d", i, g.kind);
      return false;
    }
    if (g.kind == SV_GATE_PAULI) {
      bool ok = g.n_tar >= 1 && g.n_tar <= SV_MAX_TARGETS && g.n_ctrl == 0 &&
                (g.paulis >> (2 * g.n_tar)) == 0;
      for (int j = 0; ok && j < g.n_tar; ++j) ok = ((g.paulis >> (2 * j)) & 3) != 0;
      if (!ok) {
        set_error("gate %d: PAULI takes 1..%d targets, a letter (X, Y, Z) for each and no "
                  "controls", i, SV_MAX_TARGETS);
        return false;
      }
    }
    const int want = g.kind == SV_GATE_SWAP                                ? 2
                     : (g.kind == SV_GATE_MATRIX || g.kind == SV_GATE_PAULI) ? -1
                                                                            : 1;
    if (want > 0 && g.n_tar != want) {
      set_error("gate %d: kind %d takes %d targets, got %d", i, g.kind, want, g.n_tar);
      return false;
    }
    if (!valid_qubits(s->n, g.targets, g.n_tar, g.controls, g.n_ctrl)) {
      char tmp[900];
      snprintf(tmp, sizeof(tmp), "gate %d: %s", i, sv_last_error());
      set_error("%s", tmp);
      return false;
    }
    if (g.param >= c->n_params || g.param < -1) {
      set_error("gate %d: parameter index %d outside 0..%d", i, g.param, c->n_params - 1);
      return false;
    }
    if (g.kind == SV_GATE_MATRIX && (!c->mat_pool || g.mat_off < 0)) {
      set_error("gate %d: MATRIX gate without a matrix pool entry", i);
      return false;
    }
  }
  return true;
}

static bool valid_pauli(sv_state s, const sv_pauli_sum* H) {
  if (!H || H->n_terms < 0 || H->n_terms > SV_MAX_PAULI_TERMS) {
    set_error("bad Pauli sum");
    return false;
  }
  if (H->n_terms > 0 && (!H->xmask || !H->zmask || !H->coeff)) {
    set_error("null Pauli sum arrays");
    return false;
  }
  const uint64_t lim = s->n >= 64 ? ~uint64_t(0) : (uint64_t(1) << s->n) - 1;
  for (int k = 0; k < H->n_terms; ++k)
    if ((H->xmask[k] | H->zmask[k]) & ~lim) {
      set_error("Pauli term %d has mask bits beyond qubit count %d", k, s->n);
      return false;
    }
  return true;
}

static void to_bits(int n, const int* q, int cnt, int* p) {
  for (int j = 0; j < cnt; ++j) p[j] = n - 1 - q[j];
}

// ---- handles -------------------------------------------------------------------------
static sv_status make_handle(void* ptr, bool owned, int n, sv_dtype dt, void* stream,
                             sv_state* out) {
  sv_state s = new sv_state_s();
  s->data = ptr;
  s->owned = owned;
  s->n = n;
  s->dt = dt;
  s->stream = (cudaStream_t)stream;
  cudaGetDevice(&s->device);
  // Controlled phase gates whose lowest bit is 2 or 3 touch alternate 32- or
  // 64-byte runs; with the default L2 fill granularity their reads fetch
  // whole lines (1.5x the bytes).  32-byte fills keep the touched runs only
  // and leave streaming kernels unchanged.  (A context limit: it ends with
  // the process.)
  {
    static std::once_flag l2once[64];
    if (s->device >= 0 && s->device < 64)
      std::call_once(l2once[s->device], [] {
        if (cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, 32) != cudaSuccess)
          cudaGetLastError();
      });
  }
  cudaError_t e = cudaMalloc(&s->dres, 64 * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&s->hres, 64 * sizeof(double));
  if (e != cudaSuccess) {
    set_error("handle buffers: %s", cudaGetErrorString(e));
    if (s->dres) cudaFree(s->dres);
    if (owned) cudaFree(ptr);
    delete s;
    return e == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA;
  }
  *out = s;
  return SV_OK;
}

extern "C" {

sv_status sv_alloc(int n_qubits, sv_dtype dtype, void* cuda_stream, sv_state* out) {
  if (!out || n_qubits < 1 || n_qubits > SV_MAX_QUBITS || (dtype != SV_C64 && dtype != SV_C128)) {
    set_error("sv_alloc: bad arguments (n_qubits = %d, dtype = %d)", n_qubits, (int)dtype);
    return SV_ERR_INVALID;
  }
  const size_t bytes = (size_t(1) << n_qubits) * (dtype == SV_C64 ? 8 : 16);
  void *base = nullptr, *p = nullptr;
  sv_status st = alloc_guarded(bytes, &base, &p);
  if (st) return st;
  st = make_handle(p, true, n_qubits, dtype, cuda_stream, out);
  if (st) {
    cudaFree(base);
    return st;
  }
  (*out)->base = base;
  return SV_OK;
}

sv_status sv_wrap(void* dev_ptr, int n_qubits, sv_dtype dtype, void* cuda_stream,
                  sv_state* out) {
  if (!out || !dev_ptr || n_qubits < 1 || n_qubits > SV_MAX_QUBITS ||
      (dtype != SV_C64 && dtype != SV_C128) || ((uintptr_t)dev_ptr & 15)) {
    set_error("sv_wrap: bad arguments");
    return SV_ERR_INVALID;
  }
  return make_handle(dev_ptr, false, n_qubits, dtype, cuda_stream, out);
}

sv_status sv_free(sv_state s) {
  if (!s) return SV_OK;
  cudaStreamSynchronize(s->stream);
  if (s->owned && s->base) cudaFree(s->base);
  if (s->partials) cudaFree(s->partials);
  if (s->dres) cudaFree(s->dres);
  if (s->hres) cudaFreeHost(s->hres);
  for (void* w : s->work_base)
    if (w) cudaFree(w);
  for (void* c : s->ckpt)
    if (c) cudaFree(c);
  delete s;
  return SV_OK;
}

sv_status sv_set_stream(sv_state s, void* cuda_stream) {
  if (!valid_state(s)) return SV_ERR_INVALID;
  s->stream = (cudaStream_t)cuda_stream;
  return SV_OK;
}

sv_status sv_set_rounding(sv_state s, int mode) {
  if (!valid_state(s)) return SV_ERR_INVALID;
  if (mode != SV_ROUNDING_DEFAULT && mode != SV_ROUNDING_DITHERED) {
    set_error("sv_set_rounding: mode %d is not SV_ROUNDING_DEFAULT or SV_ROUNDING_DITHERED", mode);
    return SV_ERR_INVALID;
  }
  s->rc.mode = mode;
  return SV_OK;
}

sv_status sv_info(sv_state s, void** dev_ptr, int* n_qubits, sv_dtype* dtype) {
  if (!valid_state(s)) return SV_ERR_INVALID;
  if (dev_ptr) *dev_ptr = s->data;
  if (n_qubits) *n_qubits = s->n;
  if (dtype) *dtype = s->dt;
  return SV_OK;
}

sv_status sv_init(sv_state s, uint64_t basis_index) {
  if (!valid_state(s)) return SV_ERR_INVALID;
  if (basis_index >> s->n) {
    set_error("sv_init: basis index beyond 2^%d", s->n);
    return SV_ERR_INVALID;
  }
  s->rc.reset();
  return launch_init(s->data, s->dt, s->n, s->stream, basis_index);
}

sv_status sv_host_alloc(size_t bytes, void** out) {
  if (!out || !bytes) {
    set_error("sv_host_alloc: null output or zero bytes");
    return SV_ERR_INVALID;
  }
  *out = nullptr;
  SV_CUDA_TRY(cudaHostAlloc(out, bytes, cudaHostAllocDefault));
  return SV_OK;
}

sv_status sv_host_free(void* p) {
  if (p) SV_CUDA_TRY(cudaFreeHost(p));
  return SV_OK;
}

sv_status sv_upload(sv_state s, const void* host) {
  if (!valid_state(s) || !host) return SV_ERR_INVALID;
  SV_CUDA_TRY(cudaMemcpyAsync(s->data, host, s->bytes(), cudaMemcpyHostToDevice, s->stream));
  s->rc.reset();
  return SV_OK;
}

sv_status sv_download(sv_state s, void* host) {
  if (!valid_state(s) || !host) return SV_ERR_INVALID;
  SV_CUDA_TRY(cudaMemcpyAsync(host, s->data, s->bytes(), cudaMemcpyDeviceToHost, s->stream));
  SV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return SV_OK;
}

sv_status sv_copy(sv_state dst, sv_state src) {
  if (!valid_state(dst) || !valid_state(src)) return SV_ERR_INVALID;
  if (dst->n != src->n || dst->dt != src->dt) {
    set_error("sv_copy: shape mismatch");
    return SV_ERR_INVALID;
  }
  if (dst->data == src->data) return SV_OK;
  SV_CUDA_TRY(cudaMemcpyAsync(dst->data, src->data, src->bytes(), cudaMemcpyDeviceToDevice,
                              dst->stream));
  const int mode = dst->rc.mode;
  dst->rc = src->rc;
  dst->rc.mode = mode;
  return SV_OK;
}

sv_status sv_apply_gate(sv_state s, const int* targets, int n_tar, const int* controls,
                        int n_ctrl, const double* matrix) {
  if (!valid_state(s)) return SV_ERR_INVALID;
  if (!valid_qubits(s->n, targets, n_tar, controls, n_ctrl)) return SV_ERR_INVALID;
  if (!matrix) {
    set_error("sv_apply_gate: null matrix");
    return SV_ERR_INVALID;
  }
  HostMatrix G;
  G.k = n_tar;
  const int d = 1 << n_tar;
  for (int e = 0; e < d * d; ++e) G.m[e] = {matrix[2 * e], matrix[2 * e + 1]};
  int tp[SV_MAX_TARGETS], cp[SV_MAX_CONTROLS];
  to_bits(s->n, targets, n_tar, tp);
  to_bits(s->n, controls, n_ctrl, cp);
  return launch_gate(s->data, s->dt, s->n, s->stream, n_tar, tp, n_ctrl, cp, G, &s->rc);
}

sv_status sv_apply_circuit(sv_state s, const sv_circuit* c, const double* theta, int fuse_k) {
  if (!valid_state(s)) return SV_ERR_INVALID;
  if (!valid_circuit(s, c, theta)) return SV_ERR_INVALID;
  if (fuse_k < 0 || fuse_k > 5 || fuse_k == 1) {
    set_error("fuse_k = %d: expected 0 (unfused) or 2..5", fuse_k);
    return SV_ERR_INVALID;
  }
  if (fuse_k > 0) {
    std::vector<FusionItem> plan;
    if (!plan_fusion(c, theta, fusion_config(s->n, s->dt, fuse_k), &plan)) return SV_ERR_INVALID;
    for (const FusionItem& it : plan) {
      sv_status st;
      if (it.is_pass) {
        st = launch_fused_pass(s->data, s->dt, s->n, s->stream, it.pass, &s->rc);
      } else {
        st = apply_circuit_gate(s, c, it.gate, theta);
      }
      if (st != SV_OK) return st;
    }
    return SV_OK;
  }
  for (int i = 0; i < c->n_gates; ++i) {
    sv_status st = apply_circuit_gate(s, c, i, theta);
    if (st != SV_OK) return st;
  }
  return SV_OK;
}

sv_status sv_fusion_plan(const sv_circuit* c, const double* theta, sv_dtype dtype, int fuse_k,
                         int32_t* order, int32_t* pass_of, int32_t* n_passes,
                         int32_t* staged_bits) {
  if (!c || !order || !pass_of || !n_passes || c->n_qubits < 1 ||
      c->n_qubits > SV_MAX_QUBITS || fuse_k < 2 || fuse_k > 5 ||
      (dtype != SV_C64 && dtype != SV_C128)) {
    set_error("sv_fusion_plan: bad arguments");
    return SV_ERR_INVALID;
  }
  sv_state_s probe;
  probe.n = c->n_qubits;
  probe.dt = dtype;
  probe.data = (void*)1;
  if (!valid_circuit(&probe, c, theta)) return SV_ERR_INVALID;
  const FusionConfig cfg = fusion_config(c->n_qubits, dtype, fuse_k);
  std::vector<FusionItem> plan;
  if (!plan_fusion(c, theta, cfg, &plan)) return SV_ERR_INVALID;
  int k = 0, p = 0;
  for (const FusionItem& it : plan) {
    if (it.is_pass) {
      for (const FusedGroup& g : it.pass.groups)
        for (int oi : g.ops)
          for (int o : it.pass.gates[oi].origs) {
            order[k] = o;
            pass_of[k++] = p;
          }
      if (staged_bits) {
        uint64_t m = 0;
        for (int b : it.pass.S) m |= uint64_t(1) << b;
        staged_bits[2 * p] = (int32_t)(m & 0xffffffffu);
        staged_bits[2 * p + 1] = (int32_t)(m >> 32);
      }
      ++p;
    } else {
      order[k] = it.gate;
      pass_of[k++] = -1;
    }
  }
  *n_passes = p;
  if (k != c->n_gates) {
    set_error("sv_fusion_plan: internal error, %d of %d gates planned", k, c->n_gates);
    return SV_ERR_INVALID;
  }
  return SV_OK;
}

static bool valid_grad_circuit(const sv_circuit* c);

sv_status sv_fusion_plan_reverse(const sv_circuit* c, const double* theta, sv_dtype dtype,
                                 int fuse_k, int lo, int hi, int32_t* events,
                                 int32_t* n_events, int32_t* n_passes) {
  if (!c || !events || !n_events || !n_passes || c->n_qubits < 1 ||
      c->n_qubits > SV_MAX_QUBITS || fuse_k < 2 || fuse_k > 5 ||
      (dtype != SV_C64 && dtype != SV_C128) || lo < 0 || hi < lo || hi > c->n_gates) {
    set_error("sv_fusion_plan_reverse: bad arguments");
    return SV_ERR_INVALID;
  }
  sv_state_s probe;
  probe.n = c->n_qubits;
  probe.dt = dtype;
  probe.data = (void*)1;
  if (!valid_circuit(&probe, c, theta) || !valid_grad_circuit(c)) return SV_ERR_INVALID;
  std::vector<int> slot_of(c->n_gates, -1), gate_of;
  for (int i = 0; i < c->n_gates; ++i)
    if (c->gates[i].param >= 0) {
      slot_of[i] = (int)gate_of.size();
      gate_of.push_back(i);
    }
  const FusionConfig cfg = fusion_config_reverse(c->n_qubits, dtype, fuse_k);
  std::vector<FusionItem> plan;
  if (!plan_fusion_reverse(c, theta, lo, hi, slot_of, cfg, &plan)) return SV_ERR_INVALID;
  const int cap = 2 * (hi - lo);
  int t = 0, p = 0, e = 0;
  auto emit = [&](int kind, int gate, int pass, int eval) {
    if (t < cap) {
      events[4 * t] = kind;
      events[4 * t + 1] = gate;
      events[4 * t + 2] = pass;
      events[4 * t + 3] = eval;
    }
    ++t;
  };
  for (const FusionItem& it : plan) {
    if (it.is_pass) {
      for (const FusedGroup& g : it.pass.groups)
        for (int oi : g.ops) {
          const FGate& f = it.pass.gates[oi];
          if (f.type == FG_GRAD) {
            for (int j = 0; j < f.ng; ++j)
              emit(1, gate_of[f.ng == 1 ? f.slot : f.gslots[j]], p, e);
            ++e;
          } else {
            for (int o : f.origs) emit(0, o, p, -1);
          }
        }
      ++p;
    } else {
      if (it.slot >= 0) emit(1, gate_of[it.slot], -1, e++);
      emit(0, it.gate, -1, -1);
    }
  }
  *n_events = t;
  *n_passes = p;
  if (t > cap) {
    set_error("sv_fusion_plan_reverse: internal error, %d events for %d gates", t, hi - lo);
    return SV_ERR_INVALID;
  }
  return SV_OK;
}

static sv_status norm_into(sv_state s, double* dst) {
  const int need = kRedMaxBlocks;
  sv_status st = ensure_partials(s, need);
  if (st) return st;
  int np = 0;
  st = launch_norm_partials(s, s->partials, &np);
  if (st) return st;
  return launch_finish(s->partials, np, 1, dst, s->stream, false);
}

sv_status sv_norm(sv_state s, double* out) {
  if (!valid_state(s) || !out) return SV_ERR_INVALID;
  sv_status st = norm_into(s, s->dres);
  if (st) return st;
  SV_CUDA_TRY(cudaMemcpyAsync(s->hres, s->dres, sizeof(double), cudaMemcpyDeviceToHost,
                              s->stream));
  SV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  *out = s->hres[0];
  return SV_OK;
}

static sv_status expval_into(sv_state s, const sv_pauli_sum* H, double* dst) {
  const sv_status staged = expval_staged(s, H, dst);
  if (staged != SV_ERR_UNSUPPORTED) return staged;
  std::vector<PauliDev> chunks;
  pauli_chunks(H, &chunks);
  if (chunks.empty()) {
    SV_CUDA_TRY(cudaMemsetAsync(dst, 0, sizeof(double), s->stream));
    return SV_OK;
  }
  const int g = red_blocks(uint64_t(1) << s->n);
  sv_status st = ensure_partials(s, (size_t)g * chunks.size());
  if (st) return st;
  int np = 0, total = 0;
  for (size_t i = 0; i < chunks.size(); ++i) {
    st = launch_expval_partials(s, chunks[i], s->partials + total, &np);
    if (st) return st;
    total += np;
  }
  return launch_finish(s->partials, total, 1, dst, s->stream, false);
}

sv_status sv_expval(sv_state s, const sv_pauli_sum* H, double* out) {
  if (!valid_state(s) || !out) return SV_ERR_INVALID;
  if (!valid_pauli(s, H)) return SV_ERR_INVALID;
  sv_status st = expval_into(s, H, s->dres);
  if (st) return st;
  SV_CUDA_TRY(cudaMemcpyAsync(s->hres, s->dres, sizeof(double), cudaMemcpyDeviceToHost,
                              s->stream));
  SV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  *out = s->hres[0];
  return SV_OK;
}

sv_status sv_expval_async(sv_state s, const sv_pauli_sum* H, double* dev_out) {
  if (!valid_state(s) || !dev_out) return SV_ERR_INVALID;
  if (!valid_pauli(s, H)) return SV_ERR_INVALID;
  return expval_into(s, H, dev_out);
}

static sv_status apply_pauli_into(void* out, const void* in, sv_state s, const sv_pauli_sum* H,
                                  double* energy_dst) {
  {
    const sv_status st = apply_pauli_staged(out, in, s, H, energy_dst);
    if (st != SV_ERR_UNSUPPORTED) return st;
  }
  std::vector<PauliDev> chunks;
  pauli_chunks(H, &chunks);
  if (chunks.empty()) {
    SV_CUDA_TRY(cudaMemsetAsync(out, 0, s->bytes(), s->stream));
    if (energy_dst) SV_CUDA_TRY(cudaMemsetAsync(energy_dst, 0, sizeof(double), s->stream));
    return SV_OK;
  }
  sv_status st = SV_OK;
  if (energy_dst) {
    st = ensure_partials(s, kRedMaxBlocks);
    if (st) return st;
  }
  int np = 0;
  for (size_t i = 0; i < chunks.size(); ++i) {
    const bool last = i + 1 == chunks.size();
    st = launch_apply_pauli(out, in, s->dt, s->n, s->stream, chunks[i], i > 0,
                            (last && energy_dst) ? s->partials : nullptr, &np);
    if (st) return st;
  }
  if (energy_dst) return launch_finish(s->partials, np, 1, energy_dst, s->stream, false);
  return SV_OK;
}

sv_status sv_apply_pauli_sum(sv_state out, sv_state in, const sv_pauli_sum* H) {
  if (!valid_state(out) || !valid_state(in)) return SV_ERR_INVALID;
  if (out == in || out->data == in->data || out->n != in->n || out->dt != in->dt) {
    set_error("sv_apply_pauli_sum: in and out must be distinct states of equal shape");
    return SV_ERR_INVALID;
  }
  if (!valid_pauli(in, H)) return SV_ERR_INVALID;
  {
    const sv_status st = apply_pauli_staged(out->data, in->data, in, H, nullptr);
    if (st != SV_ERR_UNSUPPORTED) return st;
  }
  std::vector<PauliDev> chunks;
  pauli_chunks(H, &chunks);
  if (chunks.empty()) {
    SV_CUDA_TRY(cudaMemsetAsync(out->data, 0, out->bytes(), in->stream));
    return SV_OK;
  }
  for (size_t i = 0; i < chunks.size(); ++i) {
    sv_status st = launch_apply_pauli(out->data, in->data, in->dt, in->n, in->stream, chunks[i],
                                      i > 0, nullptr, nullptr);
    if (st) return st;
  }
  return SV_OK;
}

// ---- adjoint gradient ------------------------------------------------------------------
static bool valid_grad_circuit(const sv_circuit* c) {
  for (int i = 0; i < c->n_gates; ++i) {
    const sv_gate& g = c->gates[i];
    if (g.param >= 0 && g.kind != SV_GATE_RX && g.kind != SV_GATE_RY && g.kind != SV_GATE_RZ &&
        g.kind != SV_GATE_PAULI) {
      set_error("gate %d: only RX, RY, RZ and PAULI gates may carry a parameter for gradients",
                i);
      return false;
    }
  }
  return true;
}

// Reverse sweep over gates [0, n_gates): work[0] holds psi_N, work[1] gets
// lambda = H psi_N.  ckpt/ckpt_gates: optional forward states to restore.
static sv_status reverse_sweep(sv_state s, const sv_circuit* c, const double* theta,
                               const sv_pauli_sum* H, const int32_t* ckpt_gates, int n_ckpt,
                               double* energy, double* grad) {
  void* psi = s->work[0];
  void* lam = s->work[1];
  int n_pg = 0;
  for (int i = 0; i < c->n_gates; ++i)
    if (c->gates[i].param >= 0) ++n_pg;
  const int grid = red_blocks(uint64_t(1) << (s->n >= 2 ? s->n - 2 : 0));
  // partials: n_pg * grid per-gate block sums, then n_pg slot sums; the
  // energy's block sums reuse the front before the first gate writes there
  sv_status st = ensure_partials(s, (size_t)n_pg * grid + n_pg + kRedMaxBlocks);
  if (st) return st;
  st = apply_pauli_into(lam, psi, s, H, s->dres);
  if (st) return st;
  double* slots = s->partials + (size_t)n_pg * grid;
  int slot = n_pg;
  int ck = n_ckpt - 1;
  for (int i = c->n_gates - 1; i >= 0; --i) {
    double* part = nullptr;
    if (c->gates[i].param >= 0) {
      --slot;
      part = s->partials + (size_t)slot * grid;
    }
    st = unapply_circuit_gate(s, psi, lam, c, i, theta, part);
    if (st) return st;
    if (ck >= 0 && ckpt_gates[ck] == i) {
      SV_CUDA_TRY(cudaMemcpyAsync(psi, s->ckpt[ck], s->bytes(), cudaMemcpyDeviceToDevice,
                                  s->stream));
      --ck;
    }
  }
  st = launch_finish(s->partials, grid, n_pg, slots, s->stream, false);
  if (st) return st;
  std::vector<double> gs(n_pg + 1);
  SV_CUDA_TRY(cudaMemcpyAsync(gs.data(), slots, n_pg * sizeof(double), cudaMemcpyDeviceToHost,
                              s->stream));
  SV_CUDA_TRY(cudaMemcpyAsync(s->hres, s->dres, sizeof(double), cudaMemcpyDeviceToHost,
                              s->stream));
  SV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  *energy = s->hres[0];
  for (int p = 0; p < c->n_params; ++p) grad[p] = 0.0;
  int k = 0;
  for (int i = 0; i < c->n_gates; ++i)
    if (c->gates[i].param >= 0) grad[c->gates[i].param] += gs[k++];
  return SV_OK;
}

sv_status sv_adjoint(sv_state s, const sv_circuit* c, const double* theta, const sv_pauli_sum* H,
                     double* energy, double* grad) {
  if (!valid_state(s) || !energy || !grad) return SV_ERR_INVALID;
  if (!valid_circuit(s, c, theta) || !valid_pauli(s, H) || !valid_grad_circuit(c))
    return SV_ERR_INVALID;
  sv_status st = ensure_work(s, 0);
  if (st == SV_OK) st = ensure_work(s, 1);
  if (st) return st;
  SV_CUDA_TRY(cudaMemcpyAsync(s->work[0], s->data, s->bytes(), cudaMemcpyDeviceToDevice,
                              s->stream));
  return reverse_sweep(s, c, theta, H, nullptr, 0, energy, grad);
}

sv_status sv_grad(sv_state s, const sv_circuit* c, const double* theta, const sv_pauli_sum* H,
                  const int32_t* checkpoint_gates, int n_checkpoints, double* energy,
                  double* grad) {
  if (!valid_state(s) || !energy || !grad) return SV_ERR_INVALID;
  if (!valid_circuit(s, c, theta) || !valid_pauli(s, H) || !valid_grad_circuit(c))
    return SV_ERR_INVALID;
  if (n_checkpoints < 0 || (n_checkpoints > 0 && !checkpoint_gates)) {
    set_error("sv_grad: bad checkpoint list");
    return SV_ERR_INVALID;
  }
  for (int k = 0; k < n_checkpoints; ++k)
    if (checkpoint_gates[k] < 0 || checkpoint_gates[k] >= c->n_gates ||
        (k > 0 && checkpoint_gates[k] <= checkpoint_gates[k - 1])) {
      set_error("sv_grad: checkpoint gates must increase within 0..%d", c->n_gates - 1);
      return SV_ERR_INVALID;
    }
  sv_status st = ensure_work(s, 0);
  if (st == SV_OK) st = ensure_work(s, 1);
  if (st) return st;
  while ((int)s->ckpt.size() < n_checkpoints) {
    void* p = nullptr;
    SV_CUDA_TRY(cudaMalloc(&p, s->bytes()));
    s->ckpt.push_back(p);
  }
  // forward, storing the state before each checkpoint gate
  int ck = 0;
  for (int i = 0; i < c->n_gates; ++i) {
    if (ck < n_checkpoints && checkpoint_gates[ck] == i) {
      SV_CUDA_TRY(cudaMemcpyAsync(s->ckpt[ck], s->data, s->bytes(), cudaMemcpyDeviceToDevice,
                                  s->stream));
      ++ck;
    }
    st = apply_circuit_gate(s, c, i, theta);
    if (st) return st;
  }
  SV_CUDA_TRY(cudaMemcpyAsync(s->work[0], s->data, s->bytes(), cudaMemcpyDeviceToDevice,
                              s->stream));
  return reverse_sweep(s, c, theta, H, checkpoint_gates, n_checkpoints, energy, grad);
}

sv_status sv_grad_fused(sv_state s, const sv_circuit* c, const double* theta,
                        const sv_pauli_sum* H, const int32_t* checkpoint_gates,
                        int n_checkpoints, int fuse_k, double* energy, double* grad) {
  if (fuse_k == 0)
    return sv_grad(s, c, theta, H, checkpoint_gates, n_checkpoints, energy, grad);
  if (!valid_state(s) || !energy || !grad) return SV_ERR_INVALID;
  if (!valid_circuit(s, c, theta) || !valid_pauli(s, H) || !valid_grad_circuit(c))
    return SV_ERR_INVALID;
  if (fuse_k < 2 || fuse_k > 5) {
    set_error("sv_grad_fused: fuse_k = %d: expected 0 or 2..5", fuse_k);
    return SV_ERR_INVALID;
  }
  if (n_checkpoints < 0 || (n_checkpoints > 0 && !checkpoint_gates)) {
    set_error("sv_grad_fused: bad checkpoint list");
    return SV_ERR_INVALID;
  }
  for (int k = 0; k < n_checkpoints; ++k)
    if (checkpoint_gates[k] < 0 || checkpoint_gates[k] >= c->n_gates ||
        (k > 0 && checkpoint_gates[k] <= checkpoint_gates[k - 1])) {
      set_error("sv_grad_fused: checkpoint gates must increase within 0..%d", c->n_gates - 1);
      return SV_ERR_INVALID;
    }
  sv_status st = ensure_work(s, 0);
  if (st == SV_OK) st = ensure_work(s, 1);
  if (st) return st;
  while ((int)s->ckpt.size() < n_checkpoints) {
    void* p = nullptr;
    SV_CUDA_TRY(cudaMalloc(&p, s->bytes()));
    s->ckpt.push_back(p);
  }
  // segments between checkpoints, fused separately (fusion reorders gates on
  // disjoint qubits, never across a checkpoint)
  std::vector<int> bounds(1, 0);
  for (int k = 0; k < n_checkpoints; ++k)
    if (checkpoint_gates[k] > bounds.back()) bounds.push_back(checkpoint_gates[k]);
  bounds.push_back(c->n_gates);
  auto ckpt_at = [&](int gate) {
    for (int k = 0; k < n_checkpoints; ++k)
      if (checkpoint_gates[k] == gate) return k;
    return -1;
  };
  for (size_t i = 0; i + 1 < bounds.size(); ++i) {
    const int k = ckpt_at(bounds[i]);
    if (k >= 0)
      SV_CUDA_TRY(cudaMemcpyAsync(s->ckpt[k], s->data, s->bytes(), cudaMemcpyDeviceToDevice,
                                  s->stream));
    sv_circuit sub = *c;
    sub.gates = c->gates + bounds[i];
    sub.n_gates = bounds[i + 1] - bounds[i];
    st = sv_apply_circuit(s, &sub, theta, fuse_k);
    if (st) return st;
  }
  SV_CUDA_TRY(cudaMemcpyAsync(s->work[0], s->data, s->bytes(), cudaMemcpyDeviceToDevice,
                              s->stream));
  // plan every reverse segment; without a bulk-copy geometry use the unfused sweep
  std::vector<int> slot_of(c->n_gates, -1);
  int n_pg = 0;
  for (int i = 0; i < c->n_gates; ++i)
    if (c->gates[i].param >= 0) slot_of[i] = n_pg++;
  const FusionConfig cfg = fusion_config_reverse(s->n, s->dt, fuse_k);
  std::vector<std::vector<FusionItem>> plans(bounds.size() - 1);
  bool fusable = s->n >= 10;
  for (size_t i = 0; fusable && i + 1 < bounds.size(); ++i) {
    if (!plan_fusion_reverse(c, theta, bounds[i], bounds[i + 1], slot_of, cfg, &plans[i]))
      return SV_ERR_INVALID;
    for (const FusionItem& it : plans[i])
      if (it.is_pass && !fused_reverse_ok(s->dt, s->n, it.pass)) fusable = false;
  }
  if (!fusable) return reverse_sweep(s, c, theta, H, checkpoint_gates, n_checkpoints, energy, grad);
  void* psi = s->work[0];
  void* lam = s->work[1];
  const int G = kRedMaxBlocks;  // partial slots per gradient (>= any pass's block count)
  st = ensure_partials(s, (size_t)n_pg * G + n_pg + kRedMaxBlocks);
  if (st) return st;
  st = apply_pauli_into(lam, psi, s, H, s->dres);
  if (st) return st;
  if (n_pg)
    SV_CUDA_TRY(cudaMemsetAsync(s->partials, 0, sizeof(double) * (size_t)n_pg * G, s->stream));
  double* slots = s->partials + (size_t)n_pg * G;
  for (size_t i = bounds.size() - 1; i-- > 0;) {
    for (const FusionItem& it : plans[i]) {
      if (it.is_pass) {
        st = launch_fused_reverse_pass(psi, lam, s->dt, s->n, s->stream, it.pass, s->partials, G);
      } else {
        st = unapply_circuit_gate(s, psi, lam, c, it.gate, theta,
                                  it.slot >= 0 ? s->partials + (size_t)it.slot * G : nullptr);
      }
      if (st) return st;
    }
    const int k = ckpt_at(bounds[i]);
    if (k >= 0)
      SV_CUDA_TRY(cudaMemcpyAsync(psi, s->ckpt[k], s->bytes(), cudaMemcpyDeviceToDevice,
                                  s->stream));
  }
  if (n_pg) {
    st = launch_finish(s->partials, G, n_pg, slots, s->stream, false);
    if (st) return st;
  }
  std::vector<double> gs(n_pg + 1);
  if (n_pg)
    SV_CUDA_TRY(cudaMemcpyAsync(gs.data(), slots, n_pg * sizeof(double), cudaMemcpyDeviceToHost,
                                s->stream));
  SV_CUDA_TRY(cudaMemcpyAsync(s->hres, s->dres, sizeof(double), cudaMemcpyDeviceToHost,
                              s->stream));
  SV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  if (take_fused_status()) {
    set_error("a fused pass gave up waiting for its bulk copies");
    return SV_ERR_TIMEOUT;
  }
  *energy = s->hres[0];
  for (int p = 0; p < c->n_params; ++p) grad[p] = 0.0;
  for (int i = 0; i < c->n_gates; ++i)
    if (slot_of[i] >= 0) grad[c->gates[i].param] += gs[slot_of[i]];
  return SV_OK;
}

sv_status sv_check_guards(sv_state s) {
  if (!valid_state(s)) return SV_ERR_INVALID;
  SV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  std::vector<unsigned char> h(kGuardBytes);
  struct Region {
    const void* base;
    const char* what;
  };
  const Region regions[] = {{s->owned ? s->base : nullptr, "state"},
                            {s->work_base[0], "adjoint work state psi"},
                            {s->work_base[1], "adjoint work state lambda"}};
  for (const Region& r : regions) {
    if (!r.base) continue;
    const char* b = static_cast<const char*>(r.base);
    const size_t offs[2] = {0, kGuardBytes + s->bytes()};
    for (size_t o : offs) {
      SV_CUDA_TRY(cudaMemcpy(h.data(), b + o, kGuardBytes, cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < kGuardBytes; ++i)
        if (h[i] != kGuardByte) {
          set_error("sv_check_guards: the %s guard %s the data was overwritten at byte %zu",
                    r.what, o ? "after" : "before", i);
          return SV_ERR_CUDA;
        }
    }
  }
  return SV_OK;
}

sv_status sv_selftest_wait(sv_state s) {
  if (!valid_state(s)) return SV_ERR_INVALID;
  return launch_wait_selftest(s->data, s->dt, s->n, s->stream);
}

sv_status sv_sync(sv_state s) {
  if (!valid_state(s)) return SV_ERR_INVALID;
  SV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  SV_CUDA_TRY(cudaGetLastError());
  if (take_fused_status() | take_pauli_status()) {
    set_error("a bulk-copy pass gave up waiting for its copies");
    return SV_ERR_TIMEOUT;
  }
  return SV_OK;
}

const char* sv_last_error(void) { return g_err; }

sv_status sv_profile_start(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_used = 0;
  g_prof_on.store(true);
  return SV_OK;
}

sv_status sv_profile_stop(char* buf, size_t len) {
  if (!buf || len == 0) {
    set_error("sv_profile_stop: null buffer");
    return SV_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on.store(false);
  std::map<std::string, std::pair<long, double>> agg;
  for (size_t i = 0; i < g_prof_used; ++i) {
    float ms = 0.f;
    SV_CUDA_TRY(cudaEventSynchronize(g_prof_recs[i].b));
    SV_CUDA_TRY(cudaEventElapsedTime(&ms, g_prof_recs[i].a, g_prof_recs[i].b));
    auto& e = agg[g_prof_recs[i].name];
    e.first += 1;
    e.second += ms;
  }
  g_prof_used = 0;
  std::string out;
  char line[256];
  for (auto& kv : agg) {
    snprintf(line, sizeof(line), "%s %ld %.6f\n", kv.first.c_str(), kv.second.first,
             kv.second.second);
    out += line;
  }
  if (out.size() + 1 > len) {
    set_error("sv_profile_stop: buffer of %zu bytes too small", len);
    return SV_ERR_INVALID;
  }
  memcpy(buf, out.c_str(), out.size() + 1);
  return SV_OK;
}

uint64_t sv_launch_count(void) { return g_launches.load(); }

int sv_version(void) { return 101; }

}  // extern "C"
