// Pauli-string rotations and Trotterized time evolution (Sec. 3: Hamiltonian
// objects with a time-evolution solver using the Trotter decomposition; the
// same rotations build QAOA-style layers).
//
// For a Pauli string P with masks (xm, zm): P^2 = I, so
//     exp(-i a P) psi = cos(a) psi - i sin(a) P psi,
//     (P psi)_x = i^{#Y} (-1)^{popcount((x ^ xm) & zm)} psi_{x ^ xm}.
// Off-diagonal strings (xm != 0) update the pairs (x, x ^ xm) together (x
// with the highest bit of xm clear).  Diagonal strings (xm = 0) multiply
// psi_x by exp(-i a s(x)), s(x) = (-1)^{popcount(x & zm)}; a run of
// consecutive diagonal terms commutes, so one pass applies the whole run:
// psi_x *= exp(-i sum_k a_k s_k(x)).
#include <cmath>
#include <vector>

#include "sv_device.cuh"

namespace sv {
namespace {

constexpr int kEThreads = 256;
constexpr int kMaxDiag = 64;

struct DiagRun {
  int nt;
  uint64_t zm[kMaxDiag];
  double a[kMaxDiag];
};

// complex64 vectors (2 amplitudes), phases from an fp32 angle sum
__global__ void __launch_bounds__(kEThreads)
    kdiag_c64(float4* __restrict__ psi, uint64_t nvec, const __grid_constant__ DiagRun D) {
  constexpr int IT = 8;
  const uint64_t base = (uint64_t)blockIdx.x * (kEThreads * IT) + threadIdx.x;
  float4 v[IT];
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const uint64_t i = base + (uint64_t)it * kEThreads;
    if (i < nvec) v[it] = psi[i];
  }
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const uint64_t i = base + (uint64_t)it * kEThreads;
    if (i >= nvec) continue;
    float ph0 = 0.f, ph1 = 0.f;  // angle sums for amplitudes 2i and 2i+1
    for (int k = 0; k < D.nt; ++k) {
      const uint64_t z = D.zm[k];
      const float a = (float)D.a[k];
      const int p0 = __popcll((2 * i) & z) & 1;
      ph0 += p0 ? -a : a;
      const int p1 = p0 ^ (int)(z & 1);
      ph1 += p1 ? -a : a;
    }
    float s0, c0, s1, c1;
    sincosf(ph0, &s0, &c0);
    sincosf(ph1, &s1, &c1);
    float4 x = v[it];
    // multiply by exp(-i ph) = c - i s
    const float r0 = c0 * x.x + s0 * x.y, i0 = c0 * x.y - s0 * x.x;
    const float r1 = c1 * x.z + s1 * x.w, i1 = c1 * x.w - s1 * x.z;
    psi[i] = make_float4(r0, i0, r1, i1);
  }
}

__global__ void __launch_bounds__(kEThreads)
    kdiag_c128(double2* __restrict__ psi, uint64_t dim, const __grid_constant__ DiagRun D) {
  constexpr int IT = 8;
  const uint64_t base = (uint64_t)blockIdx.x * (kEThreads * IT) + threadIdx.x;
  double2 v[IT];
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const uint64_t i = base + (uint64_t)it * kEThreads;
    if (i < dim) v[it] = psi[i];
  }
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const uint64_t i = base + (uint64_t)it * kEThreads;
    if (i >= dim) continue;
    double ph = 0.0;
    for (int k = 0; k < D.nt; ++k) ph += (__popcll(i & D.zm[k]) & 1) ? -D.a[k] : D.a[k];
    double s, c;
    sincos(ph, &s, &c);
    const double2 x = v[it];
    psi[i] = make_double2(c * x.x + s * x.y, c * x.y - s * x.x);
  }
}

// off-diagonal string: pairs (x, y = x ^ xm), x with bit h = top bit of xm clear.
// coef = -i sin(a) i^{#Y}; (x', y') = (c x + coef sy y, c y + coef sx x),
// sy = (-1)^{popcount(y & zm)}, sx = (-1)^{popcount(x & zm)}.
template <typename R, typename T2>
__global__ void __launch_bounds__(kEThreads)
    kpair(T2* __restrict__ psi, uint64_t npairs, uint64_t lowmask, uint64_t xm, uint64_t zm,
          R c, R kr, R ki) {
  constexpr int IT = 8;
  const uint64_t base = (uint64_t)blockIdx.x * (kEThreads * IT) + threadIdx.x;
  uint64_t xs[IT];
  T2 a[IT], b[IT];
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const uint64_t u = base + (uint64_t)it * kEThreads;
    if (u < npairs) {
      xs[it] = ((u & ~lowmask) << 1) | (u & lowmask);
      a[it] = psi[xs[it]];
      b[it] = psi[xs[it] ^ xm];
    }
  }
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const uint64_t u = base + (uint64_t)it * kEThreads;
    if (u >= npairs) continue;
    const uint64_t x = xs[it], y = x ^ xm;
    const R sx = (__popcll(x & zm) & 1) ? R(-1) : R(1);
    const R sy = (__popcll(y & zm) & 1) ? R(-1) : R(1);
    const T2 p = a[it], q = b[it];
    T2 np, nq;
    // coef * sy * q and coef * sx * p with coef = kr + i ki
    np.x = c * p.x + sy * (kr * q.x - ki * q.y);
    np.y = c * p.y + sy * (kr * q.y + ki * q.x);
    nq.x = c * q.x + sx * (kr * p.x - ki * p.y);
    nq.y = c * q.y + sx * (kr * p.y + ki * p.x);
    psi[x] = np;
    psi[y] = nq;
  }
}

// the rotated state: device data, precision, qubits, stream and the
// complex64 rounding feedback (see feedback_round)
struct Target {
  void* data;
  sv_dtype dt;
  int n;
  cudaStream_t stream;
  RoundCtx* rc;
};

// Adjoint step of a Pauli-string rotation U = exp(-i theta P / 2) in a
// reverse sweep (P = i^{ny} X^xm Z^zm up to the sign convention above): each
// unit first adds its part of Im<lambda|P|psi> (the gradient of theta) and
// then un-applies U^dagger = c I + kappa P, c = cos(theta / 2),
// kappa = i sin(theta / 2) i^{ny}, on psi and lambda.  DIAG (xm = 0): a unit
// is one amplitude, (P v)_x = s(x) v_x; otherwise a unit is the pair
// (x, y = x ^ xm) with bit h = top bit of xm clear in x and
// (P v)_x = i^{ny} s(y) v_y, (P v)_y = i^{ny} s(x) v_x, s(v) =
// (-1)^{popcount(v & zm)}.  Per-thread sums: compensated in fp32 for
// complex64, fp64 for complex128; the block's fp64 sum goes to
// partials[blockIdx.x] (grid-stride loop, every block writes its slot).
template <typename R, typename T2, bool DIAG>
__global__ void __launch_bounds__(kEThreads)
    kadj_pauli(T2* __restrict__ psi, T2* __restrict__ lam, uint64_t units, uint64_t lowmask,
               uint64_t xm, uint64_t zm, int ny, R c, R kr, R ki, double* __restrict__ partials) {
  CompSum<R> acc;
  for (uint64_t u = (uint64_t)blockIdx.x * kEThreads + threadIdx.x; u < units;
       u += (uint64_t)gridDim.x * kEThreads) {
    if (DIAG) {
      const uint64_t x = u;
      T2 p = psi[x], l = lam[x];
      const R sx = (__popcll(x & zm) & 1) ? R(-1) : R(1);
      acc.add(sx * (l.x * p.y - l.y * p.x));  // Im conj(l) s p
      // v <- (c + s(x) kappa) v, kappa = (kr, ki)
      const R ar = c + sx * kr, ai = sx * ki;
      T2 np, nl;
      np.x = ar * p.x - ai * p.y;
      np.y = ar * p.y + ai * p.x;
      nl.x = ar * l.x - ai * l.y;
      nl.y = ar * l.y + ai * l.x;
      psi[x] = np;
      lam[x] = nl;
    } else {
      const uint64_t x = ((u & ~lowmask) << 1) | (u & lowmask), y = x ^ xm;
      const T2 px = psi[x], py = psi[y], lx = lam[x], ly = lam[y];
      const R sx = (__popcll(x & zm) & 1) ? R(-1) : R(1);
      const R sy = (__popcll(y & zm) & 1) ? R(-1) : R(1);
      // w = s(y) conj(lx) py + s(x) conj(ly) px; the unit adds Im(i^{ny} w)
      const R wr = sy * (lx.x * py.x + lx.y * py.y) + sx * (ly.x * px.x + ly.y * px.y);
      const R wi = sy * (lx.x * py.y - lx.y * py.x) + sx * (ly.x * px.y - ly.y * px.x);
      acc.add(ny == 0 ? wi : ny == 1 ? wr : ny == 2 ? -wi : -wr);
      T2 npx, npy, nlx, nly;
      npx.x = c * px.x + sy * (kr * py.x - ki * py.y);
      npx.y = c * px.y + sy * (kr * py.y + ki * py.x);
      npy.x = c * py.x + sx * (kr * px.x - ki * px.y);
      npy.y = c * py.y + sx * (kr * px.y + ki * px.x);
      nlx.x = c * lx.x + sy * (kr * ly.x - ki * ly.y);
      nlx.y = c * lx.y + sy * (kr * ly.y + ki * ly.x);
      nly.x = c * ly.x + sx * (kr * lx.x - ki * lx.y);
      nly.y = c * ly.y + sx * (kr * lx.y + ki * lx.x);
      psi[x] = npx;
      psi[y] = npy;
      lam[x] = nlx;
      lam[y] = nly;
    }
  }
  const double t = block_sum(acc.value());
  if (threadIdx.x == 0 && partials) partials[blockIdx.x] = t;
}

sv_status run_diag(const Target& s, const DiagRun& D) {
  if (D.nt == 0) return SV_OK;
  ProfScope prof(s.stream, s.dt == SV_C64 ? "kdiag_c64" : "kdiag_c128");
  if (s.dt == SV_C64) {
    const uint64_t nvec = uint64_t(1) << (s.n - 1);
    const unsigned g = (unsigned)((nvec + kEThreads * 8 - 1) / (kEThreads * 8));
    kdiag_c64<<<g, kEThreads, 0, s.stream>>>((float4*)s.data, nvec, D);
  } else {
    const uint64_t dim = uint64_t(1) << s.n;
    const unsigned g = (unsigned)((dim + kEThreads * 8 - 1) / (kEThreads * 8));
    kdiag_c128<<<g, kEThreads, 0, s.stream>>>((double2*)s.data, dim, D);
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return check_launch("diagonal rotation kernel");
}

sv_status run_pair(const Target& s, uint64_t xm, uint64_t zm, double a) {
  int h = 63;
  while (!((xm >> h) & 1)) --h;
  const uint64_t lowmask = (uint64_t(1) << h) - 1;
  const uint64_t npairs = uint64_t(1) << (s.n - 1);
  const int ny = __builtin_popcountll(xm & zm) & 3;
  // coef = -i sin(a) i^{ny}
  const double sa = std::sin(a), ca = std::cos(a);
  double kr = 0, ki = 0;
  switch (ny) {
    case 0: ki = -sa; break;        // -i s
    case 1: kr = sa; break;         // -i s * i = s
    case 2: ki = sa; break;         // -i s * -1 = i s
    default: kr = -sa; break;       // -i s * -i = -s
  }
  const unsigned g = (unsigned)((npairs + kEThreads * 8 - 1) / (kEThreads * 8));
  ProfScope prof(s.stream, s.dt == SV_C64 ? "kpair_c64" : "kpair_c128");
  if (s.dt == SV_C64) {
    // c I + k P with P^2 = I scales ||psi||^2 by |c|^2 + |k|^2 on every
    // state: round with the state's error feedback
    double c32 = ca;
    cd k32{kr, ki};
    feedback_round_pair(&c32, &k32, s.rc ? &s.rc->drift : nullptr);
    kpair<float, float2><<<g, kEThreads, 0, s.stream>>>((float2*)s.data, npairs, lowmask, xm, zm,
                                                        (float)c32, (float)k32.re, (float)k32.im);
  } else {
    kpair<double, double2><<<g, kEThreads, 0, s.stream>>>((double2*)s.data, npairs, lowmask, xm,
                                                          zm, ca, kr, ki);
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return check_launch("pair rotation kernel");
}

// Applies exp(-i a_k P_k) for the sequence (xm, zm, a), merging runs of
// consecutive diagonal terms into one pass.
sv_status run_sequence(const Target& s, const std::vector<uint64_t>& xm,
                       const std::vector<uint64_t>& zm, const std::vector<double>& a) {
  DiagRun D{};
  for (size_t k = 0; k < xm.size(); ++k) {
    if (xm[k] == 0) {
      if (D.nt == kMaxDiag) {
        sv_status st = run_diag(s, D);
        if (st) return st;
        D.nt = 0;
      }
      D.zm[D.nt] = zm[k];
      D.a[D.nt] = a[k];
      ++D.nt;
      continue;
    }
    sv_status st = run_diag(s, D);
    if (st) return st;
    D.nt = 0;
    st = run_pair(s, xm[k], zm[k], a[k]);
    if (st) return st;
  }
  return run_diag(s, D);
}

}  // namespace

sv_status launch_pauli_rotation(void* data, sv_dtype dt, int n, cudaStream_t st, uint64_t xm,
                                uint64_t zm, double a, RoundCtx* rc) {
  return run_sequence({data, dt, n, st, rc}, {xm}, {zm}, {a});
}

sv_status launch_adjoint_pauli(void* psi, void* lam, sv_dtype dt, int n, cudaStream_t st,
                               uint64_t xm, uint64_t zm, double theta, double* partials,
                               int* nparts) {
  // the same fixed grid as the 1-qubit adjoint kernels: every gate writes
  // the same number of partials
  const int grid = red_blocks(uint64_t(1) << (n >= 2 ? n - 2 : 0));
  const int ny = __builtin_popcountll(xm & zm) & 3;
  const double c = std::cos(0.5 * theta), sn = std::sin(0.5 * theta);
  // kappa = i sin(theta / 2) i^{ny}
  double kr = 0, ki = 0;
  switch (ny) {
    case 0: ki = sn; break;
    case 1: kr = -sn; break;
    case 2: ki = -sn; break;
    default: kr = sn; break;
  }
  const bool diag = xm == 0;
  uint64_t units = uint64_t(1) << n, lowmask = 0;
  if (!diag) {
    int h = 63;
    while (!((xm >> h) & 1)) --h;
    lowmask = (uint64_t(1) << h) - 1;
    units >>= 1;
  }
  ProfScope prof(st, dt == SV_C64 ? "kadj_pauli_c64" : "kadj_pauli_c128");
  if (dt == SV_C64) {
    if (diag)
      kadj_pauli<float, float2, true><<<grid, kEThreads, 0, st>>>(
          (float2*)psi, (float2*)lam, units, lowmask, xm, zm, ny, (float)c, (float)kr, (float)ki,
          partials);
    else
      kadj_pauli<float, float2, false><<<grid, kEThreads, 0, st>>>(
          (float2*)psi, (float2*)lam, units, lowmask, xm, zm, ny, (float)c, (float)kr, (float)ki,
          partials);
  } else {
    if (diag)
      kadj_pauli<double, double2, true><<<grid, kEThreads, 0, st>>>(
          (double2*)psi, (double2*)lam, units, lowmask, xm, zm, ny, c, kr, ki, partials);
    else
      kadj_pauli<double, double2, false><<<grid, kEThreads, 0, st>>>(
          (double2*)psi, (double2*)lam, units, lowmask, xm, zm, ny, c, kr, ki, partials);
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (nparts) *nparts = grid;
  return check_launch("adjoint Pauli rotation kernel");
}

}  // namespace sv

using namespace sv;

extern "C" {

sv_status sv_pauli_rotation(sv_state s, uint64_t xmask, uint64_t zmask, double theta) {
  if (!s || !s->data) {
    set_error("sv_pauli_rotation: null state");
    return SV_ERR_INVALID;
  }
  const uint64_t lim = (uint64_t(1) << s->n) - 1;
  if ((xmask | zmask) & ~lim || !std::isfinite(theta)) {
    set_error("sv_pauli_rotation: mask bits beyond %d qubits or non-finite angle", s->n);
    return SV_ERR_INVALID;
  }
  return run_sequence({s->data, s->dt, s->n, s->stream, &s->rc}, {xmask}, {zmask}, {theta});
}

sv_status sv_trotter(sv_state s, const sv_pauli_sum* H, double t, int steps, int order) {
  if (!s || !s->data || !H || H->n_terms < 0 || H->n_terms > SV_MAX_PAULI_TERMS ||
      (H->n_terms > 0 && (!H->xmask || !H->zmask || !H->coeff)) || steps < 1 ||
      (order != 1 && order != 2) || !std::isfinite(t)) {
    set_error("sv_trotter: bad arguments (steps >= 1, order 1 or 2)");
    return SV_ERR_INVALID;
  }
  const uint64_t lim = (uint64_t(1) << s->n) - 1;
  for (int k = 0; k < H->n_terms; ++k)
    if ((H->xmask[k] | H->zmask[k]) & ~lim) {
      set_error("sv_trotter: term %d has mask bits beyond %d qubits", k, s->n);
      return SV_ERR_INVALID;
    }
  const double dt = t / steps;
  std::vector<uint64_t> xm, zm;
  std::vector<double> a;
  for (int step = 0; step < steps; ++step) {
    if (order == 1) {
      for (int k = 0; k < H->n_terms; ++k) {
        xm.push_back(H->xmask[k]);
        zm.push_back(H->zmask[k]);
        a.push_back(H->coeff[k] * dt);
      }
    } else {
      for (int k = 0; k < H->n_terms; ++k) {
        xm.push_back(H->xmask[k]);
        zm.push_back(H->zmask[k]);
        a.push_back(0.5 * H->coeff[k] * dt);
      }
      for (int k = H->n_terms - 1; k >= 0; --k) {
        xm.push_back(H->xmask[k]);
        zm.push_back(H->zmask[k]);
        a.push_back(0.5 * H->coeff[k] * dt);
      }
    }
  }
  return run_sequence({s->data, s->dt, s->n, s->stream, &s->rc}, xm, zm, a);
}

}  // extern "C"
