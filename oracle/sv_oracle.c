/*
 * CPU oracle for the Schroedinger state-vector method (Sec. 2, Eq. 1).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, complex128
 * definition that the GPU library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the
 * library never calls it and shares no code, header or table with it.
 *
 * What it computes, and where the paper states it:
 *   - a state of n qubits is 2^n complex amplitudes in the computational
 *     basis (Sec. 2);
 *   - a gate on n_tar targets is a 2^n_tar x 2^n_tar complex matrix G, and
 *     applying it replaces psi(tau, q) by sum_tau' G(tau, tau') psi(tau', q)
 *     (Sec. 2, Eq. 1);
 *   - controlled gates use the same rule on the part of the state where the
 *     controls are set (Sec. 2, the qibojit description of index
 *     generation for controlled and multi-target gates);
 *   - a circuit is its gates applied in order (Sec. 1: Schroedinger run time
 *     is linear in the number of gates).
 * Conventions the paper leaves open (one reading each, used everywhere):
 *   qubit q <-> amplitude-index bit n-1-q; tau = sum_j b(t_j) 2^(k-1-j);
 *   controls act on the all-ones subspace; matrices as listed in
 *   gate_matrix() below.
 *
 * Parity pins: every function here is pinned by tests/test_oracle_pins.py
 * against brute-force Kronecker operators, closed forms and invariants.
 *
 * orc_set_mutant() plants one known mistake at a time (used only by the
 * pin-sensitivity test); the default 0 is the plain definition.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { K_H = 0, K_X, K_Y, K_Z, K_RX, K_RY, K_RZ, K_U1, K_SWAP, K_MATRIX, K_PAULI };

static int g_threads = 1;
static int g_mutant = 0;

void orc_set_threads(int t) { g_threads = t > 0 ? t : 1; }
int orc_get_threads(void) { return g_threads; }
void orc_set_mutant(int m) { g_mutant = m; }
int orc_have_openmp(void) {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}

/* Gate matrices (row-major, G[r * d + c]).  c = cos(a/2), s = sin(a/2).
 *   H = [[1, 1], [1, -1]] / sqrt 2        X = [[0, 1], [1, 0]]
 *   Y = [[0, -i], [i, 0]]                 Z = diag(1, -1)
 *   RX(a) = exp(-i a X / 2) = [[c, -i s], [-i s, c]]
 *   RY(a) = exp(-i a Y / 2) = [[c, -s], [s, c]]
 *   RZ(a) = exp(-i a Z / 2) = diag(e^{-i a/2}, e^{i a/2})
 *   U1(a) = diag(1, e^{i a})
 *   SWAP on (t0, t1) exchanges |01> and |10>.
 * Returns the number of targets the kind expects (-1 for MATRIX: any). */
static int gate_matrix(int kind, double a, cplx* G) {
  const double r = 1.0 / sqrt(2.0);
  const double c = cos(a / 2.0), s = sin(a / 2.0);
  memset(G, 0, sizeof(cplx) * 16);
  switch (kind) {
    case K_H: G[0] = r; G[1] = r; G[2] = r; G[3] = -r; return 1;
    case K_X: G[1] = 1; G[2] = 1; return 1;
    case K_Y: G[1] = -I; G[2] = I; return 1;
    case K_Z: G[0] = 1; G[3] = -1; return 1;
    case K_RX:
      G[0] = c; G[1] = -I * s; G[2] = -I * s; G[3] = c;
      if (g_mutant == 4) { G[1] = I * s; G[2] = I * s; }
      return 1;
    case K_RY: G[0] = c; G[1] = -s; G[2] = s; G[3] = c; return 1;
    case K_RZ: G[0] = cexp(-I * a / 2.0); G[3] = cexp(I * a / 2.0); return 1;
    case K_U1: G[0] = 1; G[3] = cexp(I * a); return 1;
    case K_SWAP: G[0] = 1; G[1 * 4 + 2] = 1; G[2 * 4 + 1] = 1; G[15] = 1; return 2;
    default: return -1;
  }
}

void orc_init_basis(int n, cplx* psi, uint64_t x) {
  uint64_t dim = 1ull << n;
  memset(psi, 0, sizeof(cplx) * dim);
  psi[x] = 1.0;
}

/* Eq. (1): for every index x whose target bits are 0 and whose control bits
 * are 1, gather the 2^k amplitudes x | off[tau], multiply by G, scatter. */
int orc_apply(int n, cplx* psi, int k, const int* targets, int nc,
              const int* controls, const cplx* G) {
  if (n < 1 || n > 40 || k < 1 || k > 5 || nc < 0 || nc > 40) return 1;
  const uint64_t dim = 1ull << n;
  const int d = 1 << k;
  uint64_t tmask = 0, cmask = 0, off[32];
  for (int j = 0; j < k; ++j) {
    if (targets[j] < 0 || targets[j] >= n) return 1;
    tmask |= 1ull << (n - 1 - targets[j]);
  }
  for (int j = 0; j < nc; ++j) {
    if (controls[j] < 0 || controls[j] >= n) return 1;
    cmask |= 1ull << (n - 1 - controls[j]);
  }
  for (int tau = 0; tau < d; ++tau) {
    off[tau] = 0;
    for (int j = 0; j < k; ++j) {
      int bit = (g_mutant == 3) ? (tau >> j) & 1 : (tau >> (k - 1 - j)) & 1;
      off[tau] |= (uint64_t)bit << (n - 1 - targets[j]);
    }
  }
  const int64_t ndim = (int64_t)dim;
#pragma omp parallel for schedule(static) num_threads(g_threads) if (ndim >= (1 << 14))
  for (int64_t xi = 0; xi < ndim; ++xi) {
    uint64_t x = (uint64_t)xi;
    if (x & tmask) continue;
    if (g_mutant == 2) {
      if ((x & cmask) == cmask && cmask) continue;
    } else if ((x & cmask) != cmask) {
      continue;
    }
    cplx in[32], out[32];
    for (int tau = 0; tau < d; ++tau) in[tau] = psi[x | off[tau]];
    for (int r = 0; r < d; ++r) {
      cplx acc = 0;
      for (int c = 0; c < d; ++c)
        acc += (g_mutant == 1 ? G[c * d + r] : G[r * d + c]) * in[c];
      out[r] = acc;
    }
    for (int tau = 0; tau < d; ++tau) psi[x | off[tau]] = out[tau];
  }
  return 0;
}

int orc_pauli_rotation(int n, cplx* psi, int nops, const int* qubits, const char* letters,
                       double a);

/* A circuit applied gate by gate.  Gate g has kind[g], ntar[g] targets in
 * tar[5g..], nctl[g] controls in ctl[40g..], and either a parameter index
 * param[g] >= 0 (angle theta[param[g]]) or a fixed angle angle[g].  MATRIX
 * gates read 4^ntar entries of pool from mat_off[g].  PAULI gates are
 * exp(-i a P / 2) for the string with letter letters[5g + j] ('X', 'Y',
 * 'Z') on target j, applied by orc_pauli_rotation with angle a / 2; they
 * take no controls.  If shift_gate >= 0, that gate's angle is increased by
 * `shift` (parameter-shift evaluations). */
int orc_run(int n, cplx* psi, int ng, const int* kind, const int* ntar,
            const int* tar, const int* nctl, const int* ctl, const int* param,
            const double* angle, const int64_t* mat_off, const cplx* pool,
            const char* letters, const double* theta, int shift_gate, double shift) {
  cplx G[1024];
  for (int g = 0; g < ng; ++g) {
    const cplx* M = G;
    if (kind[g] == K_PAULI) {
      double a = param[g] >= 0 ? theta[param[g]] : angle[g];
      if (g == shift_gate) a += shift;
      if (nctl[g] != 0 || ntar[g] < 1 || ntar[g] > 5) return 1;
      int rc = orc_pauli_rotation(n, psi, ntar[g], tar + 5 * g, letters + 5 * g, 0.5 * a);
      if (rc) return rc;
      continue;
    }
    if (kind[g] == K_MATRIX) {
      M = pool + mat_off[g];
    } else {
      double a = param[g] >= 0 ? theta[param[g]] : angle[g];
      if (g == shift_gate) a += shift;
      int want = gate_matrix(kind[g], a, G);
      if (want != ntar[g]) return 1;
    }
    int rc = orc_apply(n, psi, ntar[g], tar + 5 * g, nctl[g], ctl + 40 * g, M);
    if (rc) return rc;
  }
  return 0;
}

/* sum_x conj(a_x) b_x by pairwise (recursive halving) summation in fp64. */
static cplx dot_pairwise(const cplx* a, const cplx* b, uint64_t lo, uint64_t hi) {
  if (hi - lo == 1) return conj(a[lo]) * b[lo];
  uint64_t mid = lo + (hi - lo) / 2;
  if (g_mutant == 5 && hi - lo == 2) return conj(a[lo]) * b[lo];
  return dot_pairwise(a, b, lo, mid) + dot_pairwise(a, b, mid, hi);
}

void orc_dot(int n, const cplx* a, const cplx* b, double* re, double* im) {
  cplx z = dot_pairwise(a, b, 0, 1ull << n);
  *re = creal(z);
  *im = cimag(z);
}

double orc_norm2(int n, const cplx* psi) {
  return creal(dot_pairwise(psi, psi, 0, 1ull << n));
}

/* <psi| H |psi> for H = sum_k coeff[k] P_k, P_k a product of single-qubit
 * Pauli matrices: letters[k * n + j] in {'X','Y','Z'} acts on qubit
 * qubits[k * n + j] for j < nops[k].  Each term is evaluated by applying
 * its Pauli factors to a copy of psi with orc_apply and taking the inner
 * product; term_re/term_im (if not NULL) receive <psi|P_k|psi>.
 * Returns 0 on success. */
int orc_expval(int n, const cplx* psi, int nterms, const double* coeff,
               const int* nops, const int* qubits, const char* letters,
               double* energy, double* term_re, double* term_im) {
  const uint64_t dim = 1ull << n;
  cplx* phi = (cplx*)malloc(sizeof(cplx) * dim);
  if (!phi) return 2;
  double e = 0.0;
  for (int k = 0; k < nterms; ++k) {
    memcpy(phi, psi, sizeof(cplx) * dim);
    for (int j = 0; j < nops[k]; ++j) {
      cplx P[16];
      char L = letters[k * n + j];
      int kind = L == 'X' ? K_X : L == 'Y' ? K_Y : L == 'Z' ? K_Z : -1;
      if (kind < 0) { free(phi); return 1; }
      gate_matrix(kind, 0.0, P);
      if (g_mutant == 6 && kind == K_Y) { P[1] = I; P[2] = -I; }
      int q = qubits[k * n + j];
      int rc = orc_apply(n, phi, 1, &q, 0, NULL, P);
      if (rc) { free(phi); return rc; }
    }
    cplx t = dot_pairwise(psi, phi, 0, dim);
    if (term_re) term_re[k] = creal(t);
    if (term_im) term_im[k] = cimag(t);
    e += coeff[k] * creal(t);
  }
  free(phi);
  *energy = e;
  return 0;
}

/* Measurement in the computational basis (Sec. 3: sampling of measurements).
 * The measured qubits q_0..q_{m-1} form the outcome r = sum_j b(q_j) 2^(m-1-j)
 * (q_0 the most significant bit), and P(r) = sum of |psi_x|^2 over every x
 * whose measured bits spell r. */
int orc_probabilities(int n, const cplx* psi, int m, const int* qubits, double* out) {
  if (m < 1 || m > n) return 1;
  for (int r = 0; r < (1 << m); ++r) out[r] = 0.0;
  for (uint64_t x = 0; x < (1ull << n); ++x) {
    int r = 0;
    for (int j = 0; j < m; ++j) r = (r << 1) | (int)((x >> (n - 1 - qubits[j])) & 1);
    out[r] += creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
  }
  return 0;
}

/* Inverse-CDF sampling: with c(x) = sum_{y <= x} |psi_y|^2 (ascending x, fp64)
 * and total = c(2^n - 1), shot s takes the smallest x with c(x) > u_s * total
 * for the given uniform u_s in [0, 1) and reports its measured bits. */
int orc_sample(int n, const cplx* psi, int m, const int* qubits, int nshots,
               const double* u, uint64_t* out) {
  if (m < 1 || m > n || n > 30) return 1;
  const uint64_t dim = 1ull << n;
  double* cdf = (double*)malloc(sizeof(double) * dim);
  if (!cdf) return 2;
  double acc = 0.0;
  for (uint64_t x = 0; x < dim; ++x) {
    acc += creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
    cdf[x] = acc;
  }
  for (int s = 0; s < nshots; ++s) {
    const double t = u[s] * acc;
    uint64_t lo = 0, hi = dim - 1;  /* smallest x with cdf[x] > t */
    while (lo < hi) {
      uint64_t mid = lo + (hi - lo) / 2;
      if (cdf[mid] > t) hi = mid; else lo = mid + 1;
    }
    uint64_t r = 0;
    for (int j = 0; j < m; ++j) r = (r << 1) | ((lo >> (n - 1 - qubits[j])) & 1);
    out[s] = r;
  }
  free(cdf);
  return 0;
}

/* Exact sampling.  Each amplitude contributes q(re) + q(im) with
 * q(v) = floor(v^2 * 2^120), an integer computed exactly from v's binary
 * significand and exponent; cumulative sums of q are exact 128-bit
 * integers, so the CDF does not depend on summation order.  A shot with
 * uniform u in [0, 1) takes T = floor(u * total) (exact) and the smallest x
 * whose cumulative sum exceeds T.  Requires sum |psi|^2 < 256. */
typedef unsigned __int128 u128;

static u128 q120(double v) {
  if (v == 0.0) return 0;
  int e;
  double f = frexp(fabs(v), &e);                 /* |v| = f 2^e, f in [0.5, 1) */
  uint64_t m = (uint64_t)ldexp(f, 53);           /* exact 53-bit significand */
  int sh = 2 * (e - 53) + 120;                   /* v^2 2^120 = m^2 2^sh */
  u128 m2 = (u128)m * m;                         /* < 2^106 */
  if (sh >= 0) return sh >= 22 ? (m2 << 22) << (sh - 22) : m2 << sh;
  return -sh >= 128 ? 0 : m2 >> -sh;
}

/* floor(u * t) for u in [0, 1) and t < 2^128, exactly */
static u128 frac_mul(double u, u128 t) {
  if (u <= 0.0) return 0;
  int e;
  double f = frexp(u, &e);
  uint64_t m = (uint64_t)ldexp(f, 53);           /* u = m 2^(e - 53), e <= 0 */
  const int s = 53 - e;                          /* >= 53 */
  const uint64_t t_hi = (uint64_t)(t >> 64), t_lo = (uint64_t)t;
  const u128 a = (u128)m * t_lo, b = (u128)m * t_hi;   /* m t = b 2^64 + a */
  /* (b 2^64 + a) >> s with a 192-bit intermediate */
  u128 lo = a + ((u128)(uint64_t)b << 64);
  uint64_t top = (uint64_t)(b >> 64) + (lo < a ? 1 : 0);  /* bits 128..191 */
  if (s >= 192) return 0;
  if (s >= 128) return (u128)(top >> (s - 128));
  if (s == 0) return lo;
  return (lo >> s) | ((u128)top << (128 - s));
}

int orc_sample_exact(int n, const cplx* psi, int m, const int* qubits, int nshots,
                     const double* u, uint64_t* out) {
  if (m < 1 || m > n || n > 30) return 1;
  const uint64_t dim = 1ull << n;
  u128* cdf = (u128*)malloc(sizeof(u128) * dim);
  if (!cdf) return 2;
  u128 acc = 0;
  for (uint64_t x = 0; x < dim; ++x) {
    acc += q120(creal(psi[x])) + q120(cimag(psi[x]));
    cdf[x] = acc;
  }
  for (int s = 0; s < nshots; ++s) {
    const u128 T = frac_mul(u[s], acc);
    uint64_t lo = 0, hi = dim - 1;  /* smallest x with cdf[x] > T */
    while (lo < hi) {
      uint64_t mid = lo + (hi - lo) / 2;
      if (cdf[mid] > T) hi = mid; else lo = mid + 1;
    }
    uint64_t r = 0;
    for (int j = 0; j < m; ++j) r = (r << 1) | ((lo >> (n - 1 - qubits[j])) & 1);
    out[s] = r;
  }
  free(cdf);
  return 0;
}

/* The exact total sum_x q(re) + q(im) as (hi, lo) 64-bit halves. */
void orc_exact_total(int n, const cplx* psi, uint64_t* hi, uint64_t* lo) {
  u128 acc = 0;
  for (uint64_t x = 0; x < (1ull << n); ++x) acc += q120(creal(psi[x])) + q120(cimag(psi[x]));
  *hi = (uint64_t)(acc >> 64);
  *lo = (uint64_t)acc;
}

/* exp(-i a P) psi for a Pauli string P (Sec. 3: Hamiltonians and time
 * evolution with the Trotter decomposition).  Since P^2 = I,
 * exp(-i a P) = cos(a) I - i sin(a) P; P psi is formed by applying the
 * string's single-qubit factors to a copy of psi with orc_apply. */
int orc_pauli_rotation(int n, cplx* psi, int nops, const int* qubits, const char* letters,
                       double a) {
  const uint64_t dim = 1ull << n;
  cplx* phi = (cplx*)malloc(sizeof(cplx) * dim);
  if (!phi) return 2;
  memcpy(phi, psi, sizeof(cplx) * dim);
  for (int j = 0; j < nops; ++j) {
    cplx P[16];
    const char L = letters[j];
    const int kind = L == 'X' ? K_X : L == 'Y' ? K_Y : L == 'Z' ? K_Z : -1;
    if (kind < 0) { free(phi); return 1; }
    gate_matrix(kind, 0.0, P);
    int q = qubits[j];
    int rc = orc_apply(n, phi, 1, &q, 0, NULL, P);
    if (rc) { free(phi); return rc; }
  }
  const double c = cos(a), s = sin(a);
  for (uint64_t x = 0; x < dim; ++x) psi[x] = c * psi[x] - I * s * phi[x];
  free(phi);
  return 0;
}
