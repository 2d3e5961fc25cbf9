// Adjoint reverse sweep for gradients of E(theta) = <psi|H|psi>.
//
// For a gate U_j = exp(-i theta_j P_j / 2) (RX, RY, RZ: P_j = X, Y, Z on
// one qubit), with psi_j the state after gate j and
// lambda_j = U_{j+1}^dagger ... U_N^dagger H psi_N,
//     dE/dtheta_j = 2 Re <lambda_j| dU_j/dtheta_j |psi_{j-1}>
//                 = Im <lambda_j| P_j |psi_j>.
// The sweep starts from psi_N and lambda_N = H psi_N and, for j = N..1,
// first accumulates Im<lambda|P_j|psi> and then un-applies U_j^dagger on
// both states.  One kernel does both for a 1-qubit gate: it reads the two
// states once and writes them once.  With controls, the generator acts on
// the control subspace only, which is exactly the set of units visited.
//
// Precision: the per-unit contribution is formed in the state's precision;
// complex64 threads accumulate it in a compensated fp32 sum, complex128
// threads in fp64; blocks and the fixed-order finish add in fp64.
#include <vector>

#include "sv_device.cuh"

namespace sv {
namespace {

// Per-thread compensated (Kahan) fp32 sum of the complex64 kernels' terms:
// GB300 issues fp64 instructions at a small fraction of the fp32 rate, so the
// per-unit additions stay in fp32 and the thread's s - c enters the fp64
// block sum once.
struct Kahan32 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Im( conj(l0) (P p)_0 + conj(l1) (P p)_1 ) for the pair (p0, p1) of one
// target qubit; PAULI 1 = X, 2 = Y, 3 = Z.
template <int PAULI, typename R>
__device__ __forceinline__ R im_lpp(R l0r, R l0i, R l1r, R l1i, R p0r, R p0i, R p1r, R p1i) {
  if (PAULI == 1) {  // (p1, p0)
    return (l0r * p1i - l0i * p1r) + (l1r * p0i - l1i * p0r);
  } else if (PAULI == 2) {  // (-i p1, i p0): Im(-i z) = -Re z, Im(i z) = Re z
    return -(l0r * p1r + l0i * p1i) + (l1r * p0r + l1i * p0i);
  } else {  // (p0, -p1)
    return (l0r * p0i - l0i * p0r) - (l1r * p1i - l1i * p1r);
  }
}

// complex64, target bit >= 1: vector pairs (lo, lo | tmask) in both states.
template <typename I, int PAULI>
__global__ void __launch_bounds__(kRedThreads)
    kadj_c64_pair(float4* __restrict__ psi, float4* __restrict__ lam, I n_units, Ins<I> ins,
                  I tmask, I cmask, int amp1_only, M2<float> g, double* __restrict__ partials) {
  Kahan32 acc;
  for (I u = (I)blockIdx.x * kRedThreads + threadIdx.x; u < n_units;
       u += (I)gridDim.x * kRedThreads) {
    const I lo = insert_zeros(u, ins) | cmask, hi = lo | tmask;
    float4 p0 = psi[lo], p1 = psi[hi], l0 = lam[lo], l1 = lam[hi];
    if (PAULI) {
      float c = im_lpp<PAULI>(l0.z, l0.w, l1.z, l1.w, p0.z, p0.w, p1.z, p1.w);
      if (!amp1_only) c += im_lpp<PAULI>(l0.x, l0.y, l1.x, l1.y, p0.x, p0.y, p1.x, p1.y);
      acc.add(c);
    }
    if (!amp1_only) {
      mv2<MK_DENSE>(g, p0.x, p0.y, p1.x, p1.y);
      mv2<MK_DENSE>(g, l0.x, l0.y, l1.x, l1.y);
    }
    mv2<MK_DENSE>(g, p0.z, p0.w, p1.z, p1.w);
    mv2<MK_DENSE>(g, l0.z, l0.w, l1.z, l1.w);
    psi[lo] = p0;
    psi[hi] = p1;
    lam[lo] = l0;
    lam[hi] = l1;
  }
  if (PAULI) {
    const double t = block_sum(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}

// complex64, target bit 0: the pair is (v.xy, v.zw) of one vector.
template <typename I, int PAULI>
__global__ void __launch_bounds__(kRedThreads)
    kadj_c64_in(float4* __restrict__ psi, float4* __restrict__ lam, I n_units, Ins<I> ins,
                I cmask, M2<float> g, double* __restrict__ partials) {
  Kahan32 acc;
  for (I u = (I)blockIdx.x * kRedThreads + threadIdx.x; u < n_units;
       u += (I)gridDim.x * kRedThreads) {
    const I v = insert_zeros(u, ins) | cmask;
    float4 p = psi[v], l = lam[v];
    if (PAULI) acc.add(im_lpp<PAULI>(l.x, l.y, l.z, l.w, p.x, p.y, p.z, p.w));
    mv2<MK_DENSE>(g, p.x, p.y, p.z, p.w);
    mv2<MK_DENSE>(g, l.x, l.y, l.z, l.w);
    psi[v] = p;
    lam[v] = l;
  }
  if (PAULI) {
    const double t = block_sum(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}

template <typename I, int PAULI>
__global__ void __launch_bounds__(kRedThreads)
    kadj_c128(double2* __restrict__ psi, double2* __restrict__ lam, I n_units, Ins<I> ins,
              I tmask, I cmask, M2<double> g, double* __restrict__ partials) {
  double acc = 0.0;
  for (I u = (I)blockIdx.x * kRedThreads + threadIdx.x; u < n_units;
       u += (I)gridDim.x * kRedThreads) {
    const I lo = insert_zeros(u, ins) | cmask, hi = lo | tmask;
    double2 p0 = psi[lo], p1 = psi[hi], l0 = lam[lo], l1 = lam[hi];
    if (PAULI) acc += im_lpp<PAULI>(l0.x, l0.y, l1.x, l1.y, p0.x, p0.y, p1.x, p1.y);
    mv2<MK_DENSE>(g, p0.x, p0.y, p1.x, p1.y);
    mv2<MK_DENSE>(g, l0.x, l0.y, l1.x, l1.y);
    psi[lo] = p0;
    psi[hi] = p1;
    lam[lo] = l0;
    lam[hi] = l1;
  }
  if (PAULI) {
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
  }
}

template <typename I, int PAULI>
void run_adj(void* psi, void* lam, sv_dtype dt, int n, cudaStream_t st, int tp, int nc,
             const int* cp, const HostMatrix& G, double* partials, int grid) {
  if (dt == SV_C64) {
    std::vector<int> vpos;
    I cmask = 0;
    int amp1_only = 0;
    for (int j = 0; j < nc; ++j) {
      if (cp[j] == 0) {
        amp1_only = 1;
      } else {
        vpos.push_back(cp[j] - 1);
        cmask |= I(1) << (cp[j] - 1);
      }
    }
    M2<float> g = to_m2<float>(G);
    if (tp == 0) {
      Ins<I> ins = make_ins<I>(vpos);
      const I nu = I(1) << (n - 1 - (int)vpos.size());
      kadj_c64_in<I, PAULI><<<grid, kRedThreads, 0, st>>>((float4*)psi, (float4*)lam, nu, ins,
                                                          cmask, g, partials);
    } else {
      vpos.push_back(tp - 1);
      Ins<I> ins = make_ins<I>(vpos);
      const I nu = I(1) << (n - 1 - (int)vpos.size());
      kadj_c64_pair<I, PAULI><<<grid, kRedThreads, 0, st>>>(
          (float4*)psi, (float4*)lam, nu, ins, I(1) << (tp - 1), cmask, amp1_only, g, partials);
    }
  } else {
    std::vector<int> pos{tp};
    I cmask = 0;
    for (int j = 0; j < nc; ++j) {
      pos.push_back(cp[j]);
      cmask |= I(1) << cp[j];
    }
    Ins<I> ins = make_ins<I>(pos);
    const I nu = I(1) << (n - (int)pos.size());
    kadj_c128<I, PAULI><<<grid, kRedThreads, 0, st>>>((double2*)psi, (double2*)lam, nu, ins,
                                                      I(1) << tp, cmask, to_m2<double>(G),
                                                      partials);
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

template <typename I>
void run_adj_p(void* psi, void* lam, sv_dtype dt, int n, cudaStream_t st, int tp, int nc,
               const int* cp, const HostMatrix& G, int pauli, double* partials, int grid) {
  ProfScope prof(st, dt == SV_C64 ? "kadj_c64" : "kadj_c128");
  switch (pauli) {
    case 1: run_adj<I, 1>(psi, lam, dt, n, st, tp, nc, cp, G, partials, grid); break;
    case 2: run_adj<I, 2>(psi, lam, dt, n, st, tp, nc, cp, G, partials, grid); break;
    case 3: run_adj<I, 3>(psi, lam, dt, n, st, tp, nc, cp, G, partials, grid); break;
    default: run_adj<I, 0>(psi, lam, dt, n, st, tp, nc, cp, G, partials, grid); break;
  }
}

}  // namespace


sv_status launch_adjoint_1q(void* psi, void* lam, sv_dtype dt, int n, cudaStream_t st, int tp,
                            int nc, const int* cp, const HostMatrix& Gdag, int pauli,
                            double* partials, int* nparts) {
  // fixed grid per state size, so every gate writes the same number of partials
  const int grid = red_blocks(uint64_t(1) << (n >= 2 ? n - 2 : 0));
  if (use_32bit_index(n, dt))
    run_adj_p<uint32_t>(psi, lam, dt, n, st, tp, nc, cp, Gdag, pauli, partials, grid);
  else
    run_adj_p<uint64_t>(psi, lam, dt, n, st, tp, nc, cp, Gdag, pauli, partials, grid);
  if (nparts) *nparts = grid;
  return check_launch("adjoint kernel");
}

}  // namespace sv
