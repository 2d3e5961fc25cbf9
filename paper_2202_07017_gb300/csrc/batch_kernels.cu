// Batched energies and adjoint gradients in one persistent launch.
//
// Many small variational circuits (Sec. 3: variational layers, VQE) are
// evaluated together: thread blocks pull items (a circuit, its parameters and
// its Pauli-sum Hamiltonian) from an atomic queue and run each item to the
// end inside the block - the forward pass from |0...0>, lambda = H psi and
// E = <psi|lambda>, then the adjoint reverse sweep (dE/dtheta_j =
// Im<lambda|P_j|psi> before U_j is un-applied on both states).  Each block
// owns one workspace slot of two states (2 x 2^nmax complex64), small enough
// to stay in L1/L2 while the block works on it.
//
// Gates are applied in register groups: the host list-schedules each
// circuit's gates into groups of at most k qubits; a thread pulls the 2^k
// amplitudes of a sub-block into registers, applies the group's gates in
// order (backward: their adjoints in reverse order) and writes them back, so
// the block synchronises once per group instead of once per gate.
//
// Precision: states and gate arithmetic in fp32; gate matrices from fp64
// sincos; the energy and every gradient accumulate per thread / per warp in
// compensated fp32 sums and across warps in fp64 (fixed order, so results
// repeat bit for bit; the single-block kernels - the cluster kernel keeps
// fp64 slots).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include <cooperative_groups.h>

#include "sv_device.cuh"

namespace sv {
namespace {

constexpr int kBMaxGates = 480;    // gates of one circuit (static smem stays < 48 KB)
constexpr int kBMaxParams = 256;   // parameters of one circuit
constexpr int kBMaxWarps = 16;     // 512 threads
constexpr int kBMaxTerms = 64;     // Pauli terms of one Hamiltonian
static_assert(SV_BATCH_MAX_QUBITS < 31, "term masks are packed in 31 bits");

struct BCirc {
  int n, ngates, gate0, ngroups, group0, nparams, nterms, term0;
  int ndiag;  // terms[term0 .. term0 + ndiag) are diagonal (no X or Y factor)
};
struct BGateDesc {
  int kind;   // SV_GATE_* (1-qubit kinds)
  int param;  // -1: fixed angle
  double angle;
};
struct BGroup {
  uint8_t k, bits[5];
  int32_t op0, op1;
};
struct BOp {
  uint8_t b0;     // group-local target index
  uint8_t cm;     // group-local control mask
  uint8_t pauli;  // generator for gradients: 0 none, 1 X, 2 Y, 3 Z
  uint8_t cls;    // arithmetic class of the 2x2 matrix (BC_*)
  int16_t param;  // parameter index or -1
  int16_t gi;     // gate index within the circuit (matrix table slot)
};
struct BTerm {
  uint64_t xm, zm;
  double cre, cim;  // coefficient times i^{#Y}
};

struct BatchArgs {
  const BCirc* circs;
  const BGateDesc* gates;
  const BGroup* groups;
  const BOp* ops;
  const BTerm* terms;
  const int* order;      // items, longest first
  const int* item_circ;  // circuit of each item
  const int* theta_off;  // parameter offset of each item
  int n_items, nmax;
  const double* theta;
  double* energy;
  double* grad;
  float2* work;          // gridDim.x slots of 2 x 2^nmax amplitudes
  int* queue;
};

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__host__ __device__ constexpr int lowbit_b(int r) { return (r & 1) ? 0 : 1 + lowbit_b(r >> 1); }

// Compensated (Kahan) fp32 sum: GB300 issues fp64 instructions at a small
// fraction of the fp32 rate, so per-operation and per-amplitude additions
// stay in fp32 and only s - c enters the fp64 totals.
__device__ __forceinline__ void ksum_add(float2& a, float x) {  // a = (s, c)
  const float y = x - a.y;
  const float t = a.x + y;
  a.y = (t - a.x) - y;
  a.x = t;
}
__device__ __forceinline__ double ksum_value(float2 a) { return (double)a.x - (double)a.y; }

// Arithmetic classes of a gate's 2x2 matrix: the work per pair drops from 16
// multiply-adds (dense) to 8 (real: H, X, RY; imaginary off-diagonal: Y, RX;
// diagonal: RZ), to 4 on one amplitude (phase: U1) or to a sign flip (Z, CZ).
enum { BC_DENSE = 0, BC_REAL = 1, BC_IMOFF = 2, BC_DIAG = 3, BC_PHASE = 4, BC_NEG = 5 };

// (a, b) <- M (a, b) for every register pair on group bit B (with controls cm
// when CTRL).
template <int K, int B, int CLS, bool CTRL>
__device__ __forceinline__ void pair_apply_c(const float* M, int cm, float (&re)[1 << K],
                                             float (&im)[1 << K]) {
  const float g0r = M[0], g0i = M[1], g1r = M[2], g1i = M[3];
  const float g2r = M[4], g2i = M[5], g3r = M[6], g3i = M[7];
#pragma unroll
  for (int r = 0; r < (1 << K); ++r) {
    if (r & (1 << B)) continue;
    if (CTRL && (r & cm) != cm) continue;
    const int r1 = r | (1 << B);
    const float ar = re[r], ai = im[r], br = re[r1], bi = im[r1];
    if (CLS == BC_NEG) {
      re[r1] = -br;
      im[r1] = -bi;
    } else if (CLS == BC_PHASE) {
      re[r1] = g3r * br - g3i * bi;
      im[r1] = g3r * bi + g3i * br;
    } else if (CLS == BC_DIAG) {
      re[r] = g0r * ar - g0i * ai;
      im[r] = g0r * ai + g0i * ar;
      re[r1] = g3r * br - g3i * bi;
      im[r1] = g3r * bi + g3i * br;
    } else if (CLS == BC_REAL) {
      re[r] = g0r * ar + g1r * br;
      im[r] = g0r * ai + g1r * bi;
      re[r1] = g2r * ar + g3r * br;
      im[r1] = g2r * ai + g3r * bi;
    } else if (CLS == BC_IMOFF) {
      re[r] = g0r * ar - g1i * bi;
      im[r] = g0r * ai + g1i * br;
      re[r1] = g3r * br - g2i * ai;
      im[r1] = g3r * bi + g2i * ar;
    } else {
      re[r] = g0r * ar - g0i * ai + g1r * br - g1i * bi;
      im[r] = g0r * ai + g0i * ar + g1r * bi + g1i * br;
      re[r1] = g2r * ar - g2i * ai + g3r * br - g3i * bi;
      im[r1] = g2r * ai + g2i * ar + g3r * bi + g3i * br;
    }
  }
}

// controlled phase / sign flip with the control mask CM fixed at compile time
// (no per-register mask tests)
template <int K, int B, int CLS, int CM>
__device__ __forceinline__ void pair_apply_cm(const float* M, float (&re)[1 << K],
                                              float (&im)[1 << K]) {
  if constexpr ((CM >> B) & 1) {
    return;  // a mask holding the target bit selects no pair (as the runtime test)
  } else {
    const float g3r = M[6], g3i = M[7];
#pragma unroll
    for (int r = 0; r < (1 << K); ++r) {
      if (r & (1 << B)) continue;
      if ((r & CM) != CM) continue;
      const int r1 = r | (1 << B);
      const float br = re[r1], bi = im[r1];
      if (CLS == BC_NEG) {
        re[r1] = -br;
        im[r1] = -bi;
      } else {
        re[r1] = g3r * br - g3i * bi;
        im[r1] = g3r * bi + g3i * br;
      }
    }
  }
}

template <int K, int B, int CLS>
__device__ __forceinline__ void pair_apply_ctrl(const float* M, int cm, float (&re)[1 << K],
                                                float (&im)[1 << K]) {
#define SV_CM_CASE(v)                                                       \
  case v:                                                                   \
    if constexpr (v < (1 << K)) pair_apply_cm<K, B, CLS, v>(M, re, im);     \
    break;
  switch (cm) {
    SV_CM_CASE(1) SV_CM_CASE(2) SV_CM_CASE(3) SV_CM_CASE(4) SV_CM_CASE(5)
    SV_CM_CASE(6) SV_CM_CASE(7) SV_CM_CASE(8) SV_CM_CASE(9) SV_CM_CASE(10)
    SV_CM_CASE(11) SV_CM_CASE(12) SV_CM_CASE(13) SV_CM_CASE(14) SV_CM_CASE(15)
    default: pair_apply_c<K, B, CLS, true>(M, cm, re, im); break;
  }
#undef SV_CM_CASE
}

template <int K, int B>
__device__ __forceinline__ void pair_apply(int cls, const float* M, int cm, float (&re)[1 << K],
                                           float (&im)[1 << K]) {
  if (cm) {
    switch (cls) {
      case BC_PHASE: pair_apply_ctrl<K, B, BC_PHASE>(M, cm, re, im); break;
      case BC_NEG: pair_apply_ctrl<K, B, BC_NEG>(M, cm, re, im); break;
      default: pair_apply_c<K, B, BC_DENSE, true>(M, cm, re, im); break;
    }
  } else {
    switch (cls) {
      case BC_REAL: pair_apply_c<K, B, BC_REAL, false>(M, 0, re, im); break;
      case BC_IMOFF: pair_apply_c<K, B, BC_IMOFF, false>(M, 0, re, im); break;
      case BC_DIAG: pair_apply_c<K, B, BC_DIAG, false>(M, 0, re, im); break;
      case BC_PHASE: pair_apply_c<K, B, BC_PHASE, false>(M, 0, re, im); break;
      case BC_NEG: pair_apply_c<K, B, BC_NEG, false>(M, 0, re, im); break;
      default: pair_apply_c<K, B, BC_DENSE, false>(M, 0, re, im); break;
    }
  }
}

// the adjoint of M (same arithmetic class) applied to the pairs
template <int K, int B>
__device__ __forceinline__ void pair_apply_dag(int cls, const float* M, int cm,
                                               float (&re)[1 << K], float (&im)[1 << K]) {
  // M^dagger = [[conj g0, conj g2], [conj g1, conj g3]]
  const float h[8] = {M[0], -M[1], M[4], -M[5], M[2], -M[3], M[6], -M[7]};
  pair_apply<K, B>(cls, h, cm, re, im);
}

// M^dagger on the pairs of two tiles (psi and lambda) behind one dispatch
template <int K, int B, int CLS, bool CTRL>
__device__ __forceinline__ void pair_apply_c2(const float* h, int cm, float (&pr)[1 << K],
                                              float (&pi)[1 << K], float (&lr)[1 << K],
                                              float (&li)[1 << K]) {
  pair_apply_c<K, B, CLS, CTRL>(h, cm, pr, pi);
  pair_apply_c<K, B, CLS, CTRL>(h, cm, lr, li);
}

template <int K, int B, int CLS, int CM>
__device__ __forceinline__ void pair_apply_cm2(const float* h, float (&pr)[1 << K],
                                               float (&pi)[1 << K], float (&lr)[1 << K],
                                               float (&li)[1 << K]) {
  pair_apply_cm<K, B, CLS, CM>(h, pr, pi);
  pair_apply_cm<K, B, CLS, CM>(h, lr, li);
}

template <int K, int B, int CLS>
__device__ __forceinline__ void pair_apply_ctrl2(const float* h, int cm, float (&pr)[1 << K],
                                                 float (&pi)[1 << K], float (&lr)[1 << K],
                                                 float (&li)[1 << K]) {
#define SV_CM_CASE(v)                                                            \
  case v:                                                                        \
    if constexpr (v < (1 << K)) pair_apply_cm2<K, B, CLS, v>(h, pr, pi, lr, li); \
    break;
  switch (cm) {
    SV_CM_CASE(1) SV_CM_CASE(2) SV_CM_CASE(3) SV_CM_CASE(4) SV_CM_CASE(5)
    SV_CM_CASE(6) SV_CM_CASE(7) SV_CM_CASE(8) SV_CM_CASE(9) SV_CM_CASE(10)
    SV_CM_CASE(11) SV_CM_CASE(12) SV_CM_CASE(13) SV_CM_CASE(14) SV_CM_CASE(15)
    default: pair_apply_c2<K, B, CLS, true>(h, cm, pr, pi, lr, li); break;
  }
#undef SV_CM_CASE
}

template <int K, int B>
__device__ __forceinline__ void pair_apply_dag2(int cls, const float* M, int cm,
                                                float (&pr)[1 << K], float (&pi)[1 << K],
                                                float (&lr)[1 << K], float (&li)[1 << K]) {
  const float h[8] = {M[0], -M[1], M[4], -M[5], M[2], -M[3], M[6], -M[7]};
  if (cm) {
    switch (cls) {
      case BC_PHASE: pair_apply_ctrl2<K, B, BC_PHASE>(h, cm, pr, pi, lr, li); break;
      case BC_NEG: pair_apply_ctrl2<K, B, BC_NEG>(h, cm, pr, pi, lr, li); break;
      default: pair_apply_c2<K, B, BC_DENSE, true>(h, cm, pr, pi, lr, li); break;
    }
  } else {
    switch (cls) {
      case BC_REAL: pair_apply_c2<K, B, BC_REAL, false>(h, 0, pr, pi, lr, li); break;
      case BC_IMOFF: pair_apply_c2<K, B, BC_IMOFF, false>(h, 0, pr, pi, lr, li); break;
      case BC_DIAG: pair_apply_c2<K, B, BC_DIAG, false>(h, 0, pr, pi, lr, li); break;
      case BC_PHASE: pair_apply_c2<K, B, BC_PHASE, false>(h, 0, pr, pi, lr, li); break;
      case BC_NEG: pair_apply_c2<K, B, BC_NEG, false>(h, 0, pr, pi, lr, li); break;
      default: pair_apply_c2<K, B, BC_DENSE, false>(h, 0, pr, pi, lr, li); break;
    }
  }
}

// sum over the pairs of Im( conj(l0) (P p)_0 + conj(l1) (P p)_1 )
template <int K, int B, int PAULI, bool CTRL>
__device__ __forceinline__ float pair_grad_c(int cm, const float (&pr)[1 << K],
                                             const float (&pi)[1 << K], const float (&lr)[1 << K],
                                             const float (&li)[1 << K]) {
  float acc = 0.f;
#pragma unroll
  for (int r = 0; r < (1 << K); ++r) {
    if (r & (1 << B)) continue;
    const int r1 = r | (1 << B);
    if (CTRL && (r & cm) != cm) continue;
    const float p0r = pr[r], p0i = pi[r], p1r = pr[r1], p1i = pi[r1];
    const float l0r = lr[r], l0i = li[r], l1r = lr[r1], l1i = li[r1];
    if (PAULI == 1)
      acc += (l0r * p1i - l0i * p1r) + (l1r * p0i - l1i * p0r);
    else if (PAULI == 2)
      acc += -(l0r * p1r + l0i * p1i) + (l1r * p0r + l1i * p0i);
    else
      acc += (l0r * p0i - l0i * p0r) - (l1r * p1i - l1i * p1r);
  }
  return acc;
}

template <int K, int B>
__device__ __forceinline__ float pair_grad(int pauli, int cm, const float (&pr)[1 << K],
                                           const float (&pi)[1 << K], const float (&lr)[1 << K],
                                           const float (&li)[1 << K]) {
  if (cm) {
    switch (pauli) {
      case 1: return pair_grad_c<K, B, 1, true>(cm, pr, pi, lr, li);
      case 2: return pair_grad_c<K, B, 2, true>(cm, pr, pi, lr, li);
      default: return pair_grad_c<K, B, 3, true>(cm, pr, pi, lr, li);
    }
  }
  switch (pauli) {
    case 1: return pair_grad_c<K, B, 1, false>(0, pr, pi, lr, li);
    case 2: return pair_grad_c<K, B, 2, false>(0, pr, pi, lr, li);
    default: return pair_grad_c<K, B, 3, false>(0, pr, pi, lr, li);
  }
}

#define SV_BIT_SWITCH(B, CALL) \
  switch (B) {                 \
    case 0: CALL(0); break;    \
    case 1: CALL(1); break;    \
    case 2: CALL(2); break;    \
    default: CALL(3); break;   \
  }

template <int K>
__device__ void group_offsets(const BGroup& g, int (&off)[1 << K], int (&lm)[K]) {
  off[0] = 0;
#pragma unroll
  for (int r = 1; r < (1 << K); ++r) off[r] = off[r & (r - 1)] | (1 << g.bits[lowbit_b(r)]);
#pragma unroll
  for (int i = 0; i < K; ++i) lm[i] = (1 << g.bits[i]) - 1;
}

// Storage order of a single-block item's states: amplitude x lives at
// swzb(x) = x ^ ((x >> 4) & 15).  The map is a bijection of [0, 2^n) for every
// n and linear over XOR, so swzb(b | off) = swzb(b) ^ swzb(off) for disjoint
// bits.  It spreads the 16 amplitudes of a 128-byte row over the row by the
// next four index bits: a warp whose lanes step over a register group's low
// bits then reaches 16 different 8-byte bank pairs instead of one.
__device__ __forceinline__ int swzb(int x) { return x ^ ((x >> 4) & 15); }

template <int K>
__device__ void group_offsets_swzb(const BGroup& g, int (&off)[1 << K], int (&lm)[K]) {
  off[0] = 0;
#pragma unroll
  for (int r = 1; r < (1 << K); ++r) off[r] = off[r & (r - 1)] ^ swzb(1 << g.bits[lowbit_b(r)]);
#pragma unroll
  for (int i = 0; i < K; ++i) lm[i] = (1 << g.bits[i]) - 1;
}

template <int K>
__device__ __forceinline__ int sub_base(int s, const int (&lm)[K], int kk) {
  int b = s;
#pragma unroll
  for (int i = 0; i < K; ++i)
    if (i < kk) b = ((b & ~lm[i]) << 1) | (b & lm[i]);
  return b;
}

// forward: psi <- group ops in order
template <int K>
__device__ void group_fwd(float2* psi, int n, const BGroup& g, const BOp* ops, const float* mats) {
  int off[1 << K], lm[K];
  group_offsets_swzb<K>(g, off, lm);
  const int kk = g.k;
  const int nsub = 1 << (n - kk);
  const int width = 1 << kk;
  for (int s = threadIdx.x; s < nsub; s += blockDim.x) {
    const int b = swzb(sub_base<K>(s, lm, kk));
    float re[1 << K], im[1 << K];
#pragma unroll
    for (int r = 0; r < (1 << K); ++r)
      if (r < width) {
        const float2 v = psi[b ^ off[r]];
        re[r] = v.x;
        im[r] = v.y;
      }
    for (int o = g.op0; o < g.op1; ++o) {
      const BOp op = ops[o];
      const float* M = mats + 8 * op.gi;
#define SV_FWD(BB) \
  if constexpr (BB < K) pair_apply<K, BB>(op.cls, M, op.cm, re, im)
      SV_BIT_SWITCH(op.b0, SV_FWD)
#undef SV_FWD
    }
#pragma unroll
    for (int r = 0; r < (1 << K); ++r)
      if (r < width) psi[b ^ off[r]] = make_float2(re[r], im[r]);
  }
}

// backward: for ops in reverse, gradient contribution then un-apply on both
template <int K>
__device__ void group_bwd(float2* psi, float2* lam, int n, const BGroup& g, const BOp* ops,
                          const float* mats, float2* wpart) {
  int off[1 << K], lm[K];
  group_offsets_swzb<K>(g, off, lm);
  const int kk = g.k;
  const int nsub = 1 << (n - kk);
  const int width = 1 << kk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // every lane of a warp runs the same number of iterations (warp sums)
  const int iters = (nsub + blockDim.x - 1) / blockDim.x;
  for (int it = 0; it < iters; ++it) {
    const int s = threadIdx.x + it * blockDim.x;
    const bool live = s < nsub;
    const int b = live ? swzb(sub_base<K>(s, lm, kk)) : 0;
    float pr[1 << K], pi[1 << K], lr[1 << K], li[1 << K];
#pragma unroll
    for (int r = 0; r < (1 << K); ++r) {
      pr[r] = pi[r] = lr[r] = li[r] = 0.f;
      if (live && r < width) {
        const float2 v = psi[b ^ off[r]], w = lam[b ^ off[r]];
        pr[r] = v.x;
        pi[r] = v.y;
        lr[r] = w.x;
        li[r] = w.y;
      }
    }
    for (int o = g.op1 - 1; o >= g.op0; --o) {
      const BOp op = ops[o];
      const float* M = mats + 8 * op.gi;
      if (op.pauli) {
        float c = 0.f;
#define SV_GRAD(BB) \
  if constexpr (BB < K) c = pair_grad<K, BB>(op.pauli, op.cm, pr, pi, lr, li)
        SV_BIT_SWITCH(op.b0, SV_GRAD)
#undef SV_GRAD
        c = warp_sum_f(c);
        if (lane == 0) ksum_add(wpart[warp * kBMaxParams + op.param], c);
      }
#define SV_BWD(BB) \
  if constexpr (BB < K) pair_apply_dag2<K, BB>(op.cls, M, op.cm, pr, pi, lr, li)
      SV_BIT_SWITCH(op.b0, SV_BWD)
#undef SV_BWD
    }
    if (live) {
#pragma unroll
      for (int r = 0; r < (1 << K); ++r)
        if (r < width) {
          psi[b ^ off[r]] = make_float2(pr[r], pi[r]);
          lam[b ^ off[r]] = make_float2(lr[r], li[r]);
        }
    }
  }
}

// SMS: the block also owns kBSmemStateBytes of dynamic shared memory and
// keeps psi there for items of up to 14 qubits (and lambda beside it for up
// to 13), the rest in its global workspace slot.
constexpr int kBSmemQubits = 14;
constexpr size_t kBSmemStateBytes = sizeof(float2) << kBSmemQubits;
// Every block also caches its item's operation and group descriptors in
// dynamic shared memory (they are read once per operation per sub-block).
constexpr size_t kBOpsBytes = sizeof(BOp) * kBMaxGates;
constexpr size_t kBGroupBytes = sizeof(BGroup) * kBMaxGates;
constexpr size_t kBTermBytes = sizeof(BTerm) * kBMaxTerms;
constexpr size_t kBCacheBytes = kBOpsBytes + kBGroupBytes + kBTermBytes + sizeof(float2) * kBMaxTerms;

template <int K, int MAXT, int MINB, bool SMS = false>
__global__ void __launch_bounds__(MAXT, MINB) kbatch(const BatchArgs A) {
  __shared__ float mats[8 * kBMaxGates];
  __shared__ float2 wpart[(MAXT / 32) * kBMaxParams];  // per warp and parameter: (sum, comp)
  __shared__ double red[MAXT / 32];
  __shared__ int s_item;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  BOp* sops = reinterpret_cast<BOp*>(dyn_smem);
  BGroup* sgrp = reinterpret_cast<BGroup*>(dyn_smem + kBOpsBytes);
  // per term: (swzb(x mask), z mask | parity of (x mask & z mask) << 31)
  int2* sterm = reinterpret_cast<int2*>(dyn_smem + kBOpsBytes + kBGroupBytes);
  // the terms' coefficients rounded to fp32 once per item (a conversion from
  // fp64 per term and amplitude would occupy GB300's slow fp64 pipe)
  float2* scoef = reinterpret_cast<float2*>(dyn_smem + kBOpsBytes + kBGroupBytes + kBTermBytes);
  float2* dyn_state = reinterpret_cast<float2*>(dyn_smem + kBCacheBytes);
  const int nwarps = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* const gpsi = A.work + (size_t)blockIdx.x * (size_t(2) << A.nmax);
  float2* const glam = gpsi + (size_t(1) << A.nmax);
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(A.queue, 1);
    __syncthreads();
    const int slot = s_item;
    if (slot >= A.n_items) break;
    const int item = A.order[slot];
    const BCirc C = A.circs[A.item_circ[item]];
    const double* th = A.theta + A.theta_off[item];
    const int dim = 1 << C.n;
    float2* psi = gpsi;
    float2* lam = glam;
    if constexpr (SMS) {
      if (C.n <= kBSmemQubits) psi = dyn_state;
      if (C.n < kBSmemQubits) lam = dyn_state + (1 << (kBSmemQubits - 1));
    }
    // gate matrices (fp64 trigonometry, rounded once), psi = |0...0>, zero partials
    for (int gi = threadIdx.x; gi < C.ngates; gi += blockDim.x) {
      const BGateDesc d = A.gates[C.gate0 + gi];
      const double a = d.param >= 0 ? th[d.param] : d.angle;
      double s, c;
      sincos(0.5 * a, &s, &c);
      double m[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      const double r2 = 0.70710678118654752440;
      switch (d.kind) {
        case SV_GATE_H: m[0] = r2; m[2] = r2; m[4] = r2; m[6] = -r2; break;
        case SV_GATE_X: m[2] = 1; m[4] = 1; break;
        case SV_GATE_Y: m[3] = -1; m[5] = 1; break;
        case SV_GATE_Z: m[0] = 1; m[6] = -1; break;
        case SV_GATE_RX: m[0] = c; m[3] = -s; m[5] = -s; m[6] = c; break;
        case SV_GATE_RY: m[0] = c; m[2] = -s; m[4] = s; m[6] = c; break;
        case SV_GATE_RZ: m[0] = c; m[1] = -s; m[6] = c; m[7] = s; break;
        default: {  // U1: diag(1, e^{ia})
          double sa, ca;
          sincos(a, &sa, &ca);
          m[0] = 1; m[6] = ca; m[7] = sa;
        }
      }
      for (int e = 0; e < 8; ++e) mats[8 * gi + e] = (float)m[e];
    }
    // |0...0>: swzb(0) = 0 and swzb maps every other index to a nonzero one
    for (int x = threadIdx.x; x < dim; x += blockDim.x) psi[x] = make_float2(x == 0 ? 1.f : 0.f, 0.f);
    for (int i = threadIdx.x; i < nwarps * kBMaxParams; i += blockDim.x)
      wpart[i] = make_float2(0.f, 0.f);
    {  // this item's groups and operations, operation indices rebased to the cache
      const int ng = C.ngroups;
      const int op_base = ng ? A.groups[C.group0].op0 : 0;
      const int nops = ng ? A.groups[C.group0 + ng - 1].op1 - op_base : 0;
      for (int i = threadIdx.x; i < nops; i += blockDim.x) sops[i] = A.ops[op_base + i];
      for (int i = threadIdx.x; i < ng; i += blockDim.x) {
        BGroup G = A.groups[C.group0 + i];
        G.op0 -= op_base;
        G.op1 -= op_base;
        sgrp[i] = G;
      }
      for (int t = threadIdx.x; t < C.nterms; t += blockDim.x) {
        const BTerm T = A.terms[C.term0 + t];
        const int xm = (int)T.xm, zm = (int)T.zm;  // n <= SV_BATCH_MAX_QUBITS < 31
        sterm[t] = make_int2(swzb(xm), (int)((unsigned)zm | ((unsigned)__popc(xm & zm) << 31)));
        scoef[t] = make_float2((float)T.cre, (float)T.cim);
      }
    }
    __syncthreads();
    // forward
    for (int gg = 0; gg < C.ngroups; ++gg) {
      group_fwd<K>(psi, C.n, sgrp[gg], sops, mats);
      __syncthreads();
    }
    // lambda = H psi, E = Re <psi|lambda> (logical index x, stored at swzb(x))
    float2 ek = make_float2(0.f, 0.f);
    for (int x = threadIdx.x; x < dim; x += blockDim.x) {
      const int px = swzb(x);
      const float2 a = psi[px];
      // sign of term t at x: parity of ((x ^ xm) & zm) = parity(x & zm) ^ parity(xm & zm)
      float dr = 0.f, di = 0.f;
      for (int t = 0; t < C.ndiag; ++t) {
        const int2 q = sterm[t];
        const float2 cf = scoef[t];
        if (__popc(x & q.y) & 1) {  // bit 31 (parity of xm & zm) is 0 here
          dr -= cf.x;
          di -= cf.y;
        } else {
          dr += cf.x;
          di += cf.y;
        }
      }
      float orr = dr * a.x - di * a.y, oi = dr * a.y + di * a.x;
      for (int t = C.ndiag; t < C.nterms; ++t) {
        const int2 q = sterm[t];
        const float2 b = psi[px ^ q.x];
        const float2 cf = scoef[t];
        const float sr = cf.x * b.x - cf.y * b.y, si = cf.x * b.y + cf.y * b.x;
        if ((__popc(x & q.y) + ((unsigned)q.y >> 31)) & 1) {
          orr -= sr;
          oi -= si;
        } else {
          orr += sr;
          oi += si;
        }
      }
      lam[px] = make_float2(orr, oi);
      ksum_add(ek, a.x * orr + a.y * oi);
    }
    double e = warp_sum_d(ksum_value(ek));
    if (lane == 0) red[warp] = e;
    __syncthreads();
    // reverse sweep
    for (int gg = C.ngroups - 1; gg >= 0; --gg) {
      group_bwd<K>(psi, lam, C.n, sgrp[gg], sops, mats, wpart);
      __syncthreads();
    }
    const int toff = A.theta_off[item];
    for (int p = threadIdx.x; p < C.nparams; p += blockDim.x) {
      double g = 0.0;
      for (int w = 0; w < nwarps; ++w) g += ksum_value(wpart[w * kBMaxParams + p]);
      A.grad[toff + p] = g;
    }
    if (threadIdx.x == 0) {
      double E = 0.0;
      for (int w = 0; w < nwarps; ++w) E += red[w];
      A.energy[item] = E;
    }
    __syncthreads();
  }
}

// ---- real-amplitude batches ------------------------------------------------------
// Gates whose matrices are real (H, X, Z, RY and their controlled forms)
// map |0...0> to real states, and a Hamiltonian whose terms are real
// matrices (coefficient times i^{#Y} real, as for the transverse-field Ising
// model) maps a real state to a real lambda = H psi.  A batch made only of
// such items runs psi and lambda as real vectors: half the bytes and half the
// multiply-adds of the complex kernel, and both states of an n = 14 item
// (2 x 64 KiB) in shared memory.  The only parameterised kind is then RY
// (generator Y), whose gradient Im<lambda|Y|psi> is the real sum of
// l1 p0 - l0 p1 over the pairs of its target bit.
//
// Storage order: amplitude x lives at swzr(x) = x ^ ((x >> 5) & 31), which
// spreads the 32 amplitudes of a 128-byte row over the row by the next five
// index bits (a bijection of [0, 2^n), linear over XOR).
__device__ __forceinline__ int swzr(int x) { return x ^ ((x >> 5) & 31); }

template <int K>
__device__ void group_offsets_swzr(const BGroup& g, int (&off)[1 << K], int (&lm)[K]) {
  off[0] = 0;
#pragma unroll
  for (int r = 1; r < (1 << K); ++r) off[r] = off[r & (r - 1)] ^ swzr(1 << g.bits[lowbit_b(r)]);
#pragma unroll
  for (int i = 0; i < K; ++i) lm[i] = (1 << g.bits[i]) - 1;
}

// (a, b) <- [[g0, g1], [g2, g3]] (a, b) on the pairs of group bit B (inside the
// group-local control mask cm when CTRL); NEG: b <- -b
template <int K, int B, bool NEG, bool CTRL>
__device__ __forceinline__ void re_pairs(float g0, float g1, float g2, float g3, int cm,
                                         float (&v)[1 << K]) {
#pragma unroll
  for (int r = 0; r < (1 << K); ++r) {
    if (r & (1 << B)) continue;
    if (CTRL && (r & cm) != cm) continue;
    const int r1 = r | (1 << B);
    if (NEG) {
      v[r1] = -v[r1];
    } else {
      const float a = v[r], b = v[r1];
      v[r] = g0 * a + g1 * b;
      v[r1] = g2 * a + g3 * b;
    }
  }
}

// sign flip under a control mask fixed at compile time (CZ and its kin)
template <int K, int B, int CM>
__device__ __forceinline__ void re_neg_cm(float (&v)[1 << K]) {
  if constexpr (!((CM >> B) & 1)) {
#pragma unroll
    for (int r = 0; r < (1 << K); ++r) {
      if (r & (1 << B)) continue;
      if ((r & CM) != CM) continue;
      v[r | (1 << B)] = -v[r | (1 << B)];
    }
  }
}

template <int K, int B>
__device__ __forceinline__ void re_neg(int cm, float (&v)[1 << K]) {
#define SV_RE_CM(c)                                          \
  case c:                                                    \
    if constexpr (c < (1 << K)) re_neg_cm<K, B, c>(v);       \
    break;
  switch (cm) {
    SV_RE_CM(0) SV_RE_CM(1) SV_RE_CM(2) SV_RE_CM(3) SV_RE_CM(4) SV_RE_CM(5) SV_RE_CM(6)
    SV_RE_CM(7) SV_RE_CM(8) SV_RE_CM(9) SV_RE_CM(10) SV_RE_CM(11) SV_RE_CM(12) SV_RE_CM(13)
    SV_RE_CM(14) SV_RE_CM(15) SV_RE_CM(16) SV_RE_CM(17) SV_RE_CM(18) SV_RE_CM(20)
    SV_RE_CM(24)
    default: re_pairs<K, B, true, true>(0.f, 0.f, 0.f, 0.f, cm, v); break;
  }
#undef SV_RE_CM
}

// operation (cls BC_REAL or BC_NEG) with matrix M (8 floats, re/im) or, when
// DAG, its transpose
template <int K, int B, bool DAG>
__device__ __forceinline__ void re_apply(const BOp& op, const float* M, float (&v)[1 << K]) {
  if (op.cls == BC_NEG) {
    re_neg<K, B>(op.cm, v);
    return;
  }
  const float g0 = M[0], g1 = DAG ? M[4] : M[2], g2 = DAG ? M[2] : M[4], g3 = M[6];
  if (op.cm)
    re_pairs<K, B, false, true>(g0, g1, g2, g3, op.cm, v);
  else
    re_pairs<K, B, false, false>(g0, g1, g2, g3, 0, v);
}

template <int K, int B>
__device__ __forceinline__ float re_grad(int cm, const float (&p)[1 << K], const float (&l)[1 << K]) {
  float acc = 0.f;
#pragma unroll
  for (int r = 0; r < (1 << K); ++r) {
    if (r & (1 << B)) continue;
    if ((r & cm) != cm) continue;
    const int r1 = r | (1 << B);
    acc = fmaf(l[r1], p[r], acc);
    acc = fmaf(-l[r], p[r1], acc);
  }
  return acc;
}

#define SV_RE_BITS(B, CALL) \
  switch (B) {              \
    case 0: CALL(0); break; \
    case 1: CALL(1); break; \
    case 2: CALL(2); break; \
    case 3: CALL(3); break; \
    default: CALL(4); break; \
  }

template <int K>
__device__ void group_fwd_re(float* psi, int n, const BGroup& g, const BOp* ops, const float* mats) {
  int off[1 << K], lm[K];
  group_offsets_swzr<K>(g, off, lm);
  const int kk = g.k;
  const int nsub = 1 << (n - kk);
  const int width = 1 << kk;
  for (int s = threadIdx.x; s < nsub; s += blockDim.x) {
    const int b = swzr(sub_base<K>(s, lm, kk));
    float v[1 << K];
#pragma unroll
    for (int r = 0; r < (1 << K); ++r) v[r] = r < width ? psi[b ^ off[r]] : 0.f;
    for (int o = g.op0; o < g.op1; ++o) {
      const BOp op = ops[o];
      const float* M = mats + 8 * op.gi;
#define SV_FWD_RE(BB) \
  if constexpr (BB < K) re_apply<K, BB, false>(op, M, v)
      SV_RE_BITS(op.b0, SV_FWD_RE)
#undef SV_FWD_RE
    }
#pragma unroll
    for (int r = 0; r < (1 << K); ++r)
      if (r < width) psi[b ^ off[r]] = v[r];
  }
}

template <int K>
__device__ void group_bwd_re(float* psi, float* lam, int n, const BGroup& g, const BOp* ops,
                             const float* mats, float2* wpart) {
  int off[1 << K], lm[K];
  group_offsets_swzr<K>(g, off, lm);
  const int kk = g.k;
  const int nsub = 1 << (n - kk);
  const int width = 1 << kk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // every lane of a warp runs the same number of iterations (warp sums)
  const int iters = (nsub + blockDim.x - 1) / blockDim.x;
  for (int it = 0; it < iters; ++it) {
    const int s = threadIdx.x + it * blockDim.x;
    const bool live = s < nsub;
    const int b = live ? swzr(sub_base<K>(s, lm, kk)) : 0;
    float p[1 << K], l[1 << K];
#pragma unroll
    for (int r = 0; r < (1 << K); ++r) {
      const bool in = live && r < width;
      p[r] = in ? psi[b ^ off[r]] : 0.f;
      l[r] = in ? lam[b ^ off[r]] : 0.f;
    }
    for (int o = g.op1 - 1; o >= g.op0; --o) {
      const BOp op = ops[o];
      const float* M = mats + 8 * op.gi;
      if (op.pauli) {  // RY: generator Y
        float c = 0.f;
#define SV_GRAD_RE(BB) \
  if constexpr (BB < K) c = re_grad<K, BB>(op.cm, p, l)
        SV_RE_BITS(op.b0, SV_GRAD_RE)
#undef SV_GRAD_RE
        c = warp_sum_f(c);
        if (lane == 0) ksum_add(wpart[warp * kBMaxParams + op.param], c);
      }
#define SV_BWD_RE(BB)                        \
  if constexpr (BB < K) {                    \
    re_apply<K, BB, true>(op, M, p);         \
    re_apply<K, BB, true>(op, M, l);         \
  }
      SV_RE_BITS(op.b0, SV_BWD_RE)
#undef SV_BWD_RE
    }
    if (live) {
#pragma unroll
      for (int r = 0; r < (1 << K); ++r)
        if (r < width) {
          psi[b ^ off[r]] = p[r];
          lam[b ^ off[r]] = l[r];
        }
    }
  }
}

// Real states in shared memory: psi for items up to kBSmemQubits + 1 qubits,
// lambda beside it up to kBSmemQubits; larger states in the block's global
// workspace slot (read as 4 x 2^nmax floats).
template <int K, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) kbatch_re(const BatchArgs A) {
  __shared__ float mats[8 * kBMaxGates];
  __shared__ float2 wpart[(MAXT / 32) * kBMaxParams];  // per warp and parameter: (sum, comp)
  __shared__ double red[MAXT / 32];
  __shared__ int s_item;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  BOp* sops = reinterpret_cast<BOp*>(dyn_smem);
  BGroup* sgrp = reinterpret_cast<BGroup*>(dyn_smem + kBOpsBytes);
  int2* sterm = reinterpret_cast<int2*>(dyn_smem + kBOpsBytes + kBGroupBytes);
  float* scoef = reinterpret_cast<float*>(dyn_smem + kBOpsBytes + kBGroupBytes + kBTermBytes);
  float* dyn_state = reinterpret_cast<float*>(dyn_smem + kBCacheBytes);
  constexpr int kSm = kBSmemQubits + 1;  // 2^15 floats = kBSmemStateBytes
  const int nwarps = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* const gpsi = reinterpret_cast<float*>(A.work + (size_t)blockIdx.x * (size_t(2) << A.nmax));
  float* const glam = gpsi + (size_t(1) << A.nmax);
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(A.queue, 1);
    __syncthreads();
    const int slot = s_item;
    if (slot >= A.n_items) break;
    const int item = A.order[slot];
    const BCirc C = A.circs[A.item_circ[item]];
    const double* th = A.theta + A.theta_off[item];
    const int dim = 1 << C.n;
    float* psi = C.n <= kSm ? dyn_state : gpsi;
    float* lam = C.n < kSm ? dyn_state + (1 << (kSm - 1)) : glam;
    // gate matrices (fp64 trigonometry, rounded once): real kinds only
    for (int gi = threadIdx.x; gi < C.ngates; gi += blockDim.x) {
      const BGateDesc d = A.gates[C.gate0 + gi];
      const double a = d.param >= 0 ? th[d.param] : d.angle;
      double s, c;
      sincos(0.5 * a, &s, &c);
      double m[4] = {1, 0, 0, 1};
      const double r2 = 0.70710678118654752440;
      switch (d.kind) {
        case SV_GATE_H: m[0] = r2; m[1] = r2; m[2] = r2; m[3] = -r2; break;
        case SV_GATE_X: m[0] = 0; m[1] = 1; m[2] = 1; m[3] = 0; break;
        case SV_GATE_Z: m[3] = -1; break;
        default: m[0] = c; m[1] = -s; m[2] = s; m[3] = c; break;  // RY
      }
      for (int e = 0; e < 4; ++e) {
        mats[8 * gi + 2 * e] = (float)m[e];
        mats[8 * gi + 2 * e + 1] = 0.f;
      }
    }
    for (int x = threadIdx.x; x < dim; x += blockDim.x) psi[x] = x == 0 ? 1.f : 0.f;
    for (int i = threadIdx.x; i < nwarps * kBMaxParams; i += blockDim.x)
      wpart[i] = make_float2(0.f, 0.f);
    {
      const int ng = C.ngroups;
      const int op_base = ng ? A.groups[C.group0].op0 : 0;
      const int nops = ng ? A.groups[C.group0 + ng - 1].op1 - op_base : 0;
      for (int i = threadIdx.x; i < nops; i += blockDim.x) sops[i] = A.ops[op_base + i];
      for (int i = threadIdx.x; i < ng; i += blockDim.x) {
        BGroup G = A.groups[C.group0 + i];
        G.op0 -= op_base;
        G.op1 -= op_base;
        sgrp[i] = G;
      }
      for (int t = threadIdx.x; t < C.nterms; t += blockDim.x) {
        const BTerm T = A.terms[C.term0 + t];
        const int xm = (int)T.xm, zm = (int)T.zm;
        sterm[t] = make_int2(swzr(xm), (int)((unsigned)zm | ((unsigned)__popc(xm & zm) << 31)));
        scoef[t] = (float)T.cre;  // a real batch has cim = 0
      }
    }
    __syncthreads();
    for (int gg = 0; gg < C.ngroups; ++gg) {
      group_fwd_re<K>(psi, C.n, sgrp[gg], sops, mats);
      __syncthreads();
    }
    // lambda = H psi, E = <psi|lambda>
    float2 ek = make_float2(0.f, 0.f);
    for (int x = threadIdx.x; x < dim; x += blockDim.x) {
      const int px = swzr(x);
      const float a = psi[px];
      float d = 0.f;
      for (int t = 0; t < C.ndiag; ++t) d += (__popc(x & sterm[t].y) & 1) ? -scoef[t] : scoef[t];
      float o = d * a;
      for (int t = C.ndiag; t < C.nterms; ++t) {
        const int2 q = sterm[t];
        const float sb = scoef[t] * psi[px ^ q.x];
        o += ((__popc(x & q.y) + ((unsigned)q.y >> 31)) & 1) ? -sb : sb;
      }
      lam[px] = o;
      ksum_add(ek, a * o);
    }
    double e = warp_sum_d(ksum_value(ek));
    if (lane == 0) red[warp] = e;
    __syncthreads();
    for (int gg = C.ngroups - 1; gg >= 0; --gg) {
      group_bwd_re<K>(psi, lam, C.n, sgrp[gg], sops, mats, wpart);
      __syncthreads();
    }
    const int toff = A.theta_off[item];
    for (int p = threadIdx.x; p < C.nparams; p += blockDim.x) {
      double g = 0.0;
      for (int w = 0; w < nwarps; ++w) g += ksum_value(wpart[w * kBMaxParams + p]);
      A.grad[toff + p] = g;
    }
    if (threadIdx.x == 0) {
      double E = 0.0;
      for (int w = 0; w < nwarps; ++w) E += red[w];
      A.energy[item] = E;
    }
    __syncthreads();
  }
}

// ---- two-block clusters: each item's states split over the pair ----------------------
// A cluster of two blocks (one per SM) runs one item at a time.  Block c
// holds the amplitudes whose top bit (n - 1) is c, of both psi and lambda: in
// its shared memory when n <= kClSmemQubits (2 x 64 KiB at n = 14), else in
// the cluster's global workspace slot.  A register group that does not touch
// bit n - 1 runs on each block's own half; a group that does ("split") gives
// each block half of the sub-blocks and reaches the partner's half through
// distributed shared memory (or global memory), with cluster barriers before
// and after.  Energy and gradient partials are summed per block, then block 0
// adds the partner's partials in a fixed order.
constexpr int kClSmemQubits = 14;
constexpr int kClThreads = 512;

// amplitude x of the whole state: its block's half, offset inside the half
struct Halves {
  float2* h0;
  float2* h1;
  int hn;  // qubits per half (n - 1)
  __device__ __forceinline__ float2& at(int x) const {
    return ((x >> hn) ? h1 : h0)[x & ((1 << hn) - 1)];
  }
};

template <int K>
__device__ __forceinline__ void cl_group_fwd(const Halves& P, float2* own, int rank, int n,
                                             bool split, const BGroup& g, const BOp* ops,
                                             const float* mats) {
  int off[1 << K], lm[K];
  group_offsets<K>(g, off, lm);
  const int kk = g.k, width = 1 << kk;
  if (!split) {
    const int nsub = 1 << (P.hn - kk);
    for (int s = threadIdx.x; s < nsub; s += kClThreads) {
      const int b = sub_base<K>(s, lm, kk);
      float re[1 << K], im[1 << K];
#pragma unroll
      for (int r = 0; r < (1 << K); ++r)
        if (r < width) {
          const float2 v = own[b | off[r]];
          re[r] = v.x;
          im[r] = v.y;
        }
      for (int o = g.op0; o < g.op1; ++o) {
        const BOp op = ops[o];
        const float* M = mats + 8 * op.gi;
#define SV_FWD(BB) \
  if constexpr (BB < K) pair_apply<K, BB>(op.cls, M, op.cm, re, im)
        SV_BIT_SWITCH(op.b0, SV_FWD)
#undef SV_FWD
      }
#pragma unroll
      for (int r = 0; r < (1 << K); ++r)
        if (r < width) own[b | off[r]] = make_float2(re[r], im[r]);
    }
  } else {
    const int nsub = 1 << (n - kk);  // sub-blocks s = rank, rank + 2, ...
    for (int s = rank + 2 * (int)threadIdx.x; s < nsub; s += 2 * kClThreads) {
      const int b = sub_base<K>(s, lm, kk);
      float re[1 << K], im[1 << K];
#pragma unroll
      for (int r = 0; r < (1 << K); ++r)
        if (r < width) {
          const float2 v = P.at(b | off[r]);
          re[r] = v.x;
          im[r] = v.y;
        }
      for (int o = g.op0; o < g.op1; ++o) {
        const BOp op = ops[o];
        const float* M = mats + 8 * op.gi;
#define SV_FWD(BB) \
  if constexpr (BB < K) pair_apply<K, BB>(op.cls, M, op.cm, re, im)
        SV_BIT_SWITCH(op.b0, SV_FWD)
#undef SV_FWD
      }
#pragma unroll
      for (int r = 0; r < (1 << K); ++r)
        if (r < width) P.at(b | off[r]) = make_float2(re[r], im[r]);
    }
  }
}

template <int K, bool split>
__device__ __forceinline__ void cl_group_bwd(const Halves& Pp, const Halves& Pl, float2* ownp,
                                             float2* ownl, int rank, int n, const BGroup& g,
                                             const BOp* ops, const float* mats, double* wpart) {
  int off[1 << K], lm[K];
  group_offsets<K>(g, off, lm);
  const int kk = g.k, width = 1 << kk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nsub = split ? 1 << (n - kk) : 1 << (Pp.hn - kk);
  const int first = split ? rank : 0, step = split ? 2 : 1;
  // every lane of a warp runs the same number of iterations (warp sums)
  const int mine = split ? (nsub - rank + 1) / 2 : nsub;
  const int iters = (mine + kClThreads - 1) / kClThreads;
  for (int it = 0; it < iters; ++it) {
    const int t = threadIdx.x + it * kClThreads;
    const bool live = t < mine;
    const int s = first + step * t;
    const int b = live ? sub_base<K>(s, lm, kk) : 0;
    float pr[1 << K], pi[1 << K], lr[1 << K], li[1 << K];
#pragma unroll
    for (int r = 0; r < (1 << K); ++r) {
      pr[r] = pi[r] = lr[r] = li[r] = 0.f;
      if (live && r < width) {
        const int x = b | off[r];
        float2 v, w;
        if constexpr (split) {
          v = Pp.at(x);
          w = Pl.at(x);
        } else {
          v = ownp[x];
          w = ownl[x];
        }
        pr[r] = v.x;
        pi[r] = v.y;
        lr[r] = w.x;
        li[r] = w.y;
      }
    }
    for (int o = g.op1 - 1; o >= g.op0; --o) {
      const BOp op = ops[o];
      const float* M = mats + 8 * op.gi;
      if (op.pauli) {
        float c = 0.f;
#define SV_GRAD(BB) \
  if constexpr (BB < K) c = pair_grad<K, BB>(op.pauli, op.cm, pr, pi, lr, li)
        SV_BIT_SWITCH(op.b0, SV_GRAD)
#undef SV_GRAD
        c = warp_sum_f(c);
        if (lane == 0) wpart[warp * kBMaxParams + op.param] += (double)c;
      }
#define SV_BWD(BB)                                   \
  if constexpr (BB < K) {                            \
    pair_apply_dag<K, BB>(op.cls, M, op.cm, pr, pi); \
    pair_apply_dag<K, BB>(op.cls, M, op.cm, lr, li); \
  }
      SV_BIT_SWITCH(op.b0, SV_BWD)
#undef SV_BWD
    }
    if (live) {
#pragma unroll
      for (int r = 0; r < (1 << K); ++r)
        if (r < width) {
          const int x = b | off[r];
          if constexpr (split) {
            Pp.at(x) = make_float2(pr[r], pi[r]);
            Pl.at(x) = make_float2(lr[r], li[r]);
          } else {
            ownp[x] = make_float2(pr[r], pi[r]);
            ownl[x] = make_float2(lr[r], li[r]);
          }
        }
    }
  }
}

__device__ __forceinline__ bool group_is_split(const BGroup& g, int hn) {
  if (hn < g.k) return true;
  for (int i = 0; i < g.k; ++i)
    if (g.bits[i] == hn) return true;
  return false;
}

// Dynamic shared memory: psi half, lambda half (2^13 amplitudes each), gate
// matrices, per-warp gradient partials.
constexpr size_t kClSmemBytes = (sizeof(float2) << kClSmemQubits) + sizeof(float) * 8 * kBMaxGates +
                                sizeof(double) * (kClThreads / 32) * kBMaxParams;

template <int K>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kClThreads, 1)
    kbatch_cl(const BatchArgs A) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char cl_smem[];
  float2* sh_psi = reinterpret_cast<float2*>(cl_smem);
  float2* sh_lam = sh_psi + (1 << (kClSmemQubits - 1));
  float* mats = reinterpret_cast<float*>(sh_lam + (1 << (kClSmemQubits - 1)));
  double* wpart = reinterpret_cast<double*>(mats + 8 * kBMaxGates);
  __shared__ double red[kClThreads / 32];
  __shared__ int s_item;
  const int rank = (int)cluster.block_rank();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int nwarps = kClThreads / 32;
  const size_t cid = blockIdx.x / 2;
  float2* gw = A.work + cid * (size_t(2) << A.nmax);  // global slot: psi, then lambda
  int* partner_item = cluster.map_shared_rank(&s_item, 1);
  while (true) {
    if (rank == 0 && threadIdx.x == 0) {
      const int v = atomicAdd(A.queue, 1);
      s_item = v;
      *partner_item = v;
    }
    cluster.sync();
    const int slot = s_item;
    if (slot >= A.n_items) break;
    const int item = A.order[slot];
    const BCirc C = A.circs[A.item_circ[item]];
    const double* th = A.theta + A.theta_off[item];
    const int n = C.n, hn = n - 1, hdim = 1 << hn;
    const bool in_smem = n <= kClSmemQubits;
    Halves Pp, Pl;
    Pp.hn = Pl.hn = hn;
    if (in_smem) {
      Pp.h0 = cluster.map_shared_rank(sh_psi, 0);
      Pp.h1 = cluster.map_shared_rank(sh_psi, 1);
      Pl.h0 = cluster.map_shared_rank(sh_lam, 0);
      Pl.h1 = cluster.map_shared_rank(sh_lam, 1);
    } else {
      Pp.h0 = gw;
      Pp.h1 = gw + hdim;
      Pl.h0 = gw + (size_t(1) << A.nmax);
      Pl.h1 = Pl.h0 + hdim;
    }
    float2* ownp = in_smem ? sh_psi : (rank ? Pp.h1 : Pp.h0);
    float2* ownl = in_smem ? sh_lam : (rank ? Pl.h1 : Pl.h0);
    for (int gi = threadIdx.x; gi < C.ngates; gi += kClThreads) {
      const BGateDesc d = A.gates[C.gate0 + gi];
      const double a = d.param >= 0 ? th[d.param] : d.angle;
      double sn, cs;
      sincos(0.5 * a, &sn, &cs);
      double m[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      const double r2 = 0.70710678118654752440;
      switch (d.kind) {
        case SV_GATE_H: m[0] = r2; m[2] = r2; m[4] = r2; m[6] = -r2; break;
        case SV_GATE_X: m[2] = 1; m[4] = 1; break;
        case SV_GATE_Y: m[3] = -1; m[5] = 1; break;
        case SV_GATE_Z: m[0] = 1; m[6] = -1; break;
        case SV_GATE_RX: m[0] = cs; m[3] = -sn; m[5] = -sn; m[6] = cs; break;
        case SV_GATE_RY: m[0] = cs; m[2] = -sn; m[4] = sn; m[6] = cs; break;
        case SV_GATE_RZ: m[0] = cs; m[1] = -sn; m[6] = cs; m[7] = sn; break;
        default: {  // U1: diag(1, e^{ia})
          double sa, ca;
          sincos(a, &sa, &ca);
          m[0] = 1; m[6] = ca; m[7] = sa;
        }
      }
      for (int e = 0; e < 8; ++e) mats[8 * gi + e] = (float)m[e];
    }
    for (int x = threadIdx.x; x < hdim; x += kClThreads)
      ownp[x] = make_float2(rank == 0 && x == 0 ? 1.f : 0.f, 0.f);
    for (int i = threadIdx.x; i < nwarps * kBMaxParams; i += kClThreads) wpart[i] = 0.0;
    __syncthreads();
    // forward
    bool synced = false;  // true right after a cluster barrier
    for (int gg = 0; gg < C.ngroups; ++gg) {
      const BGroup G = A.groups[C.group0 + gg];
      const bool split = group_is_split(G, hn);
      if (split && !synced) cluster.sync();
      cl_group_fwd<K>(Pp, ownp, rank, n, split, G, A.ops, mats);
      if (split) {
        cluster.sync();
        synced = true;
      } else {
        __syncthreads();
        synced = false;
      }
    }
    if (!synced) cluster.sync();
    // lambda = H psi on this block's half, E = Re <psi|lambda>
    double e = 0.0;
    for (int xl = threadIdx.x; xl < hdim; xl += kClThreads) {
      const int x = (rank << hn) | xl;
      float orr = 0.f, oi = 0.f;
      for (int t = 0; t < C.nterms; ++t) {
        const BTerm T = A.terms[C.term0 + t];
        const float2 b = Pp.at(x ^ (int)T.xm);
        const float cr = (float)T.cre, ci = (float)T.cim;
        const float sr = cr * b.x - ci * b.y, si = cr * b.y + ci * b.x;
        if (__popcll(((uint64_t)x ^ T.xm) & T.zm) & 1) {
          orr -= sr;
          oi -= si;
        } else {
          orr += sr;
          oi += si;
        }
      }
      ownl[xl] = make_float2(orr, oi);
      const float2 a = ownp[xl];
      e += (double)(a.x * orr + a.y * oi);
    }
    e = warp_sum_d(e);
    if (lane == 0) red[warp] = e;
    cluster.sync();  // lambda complete; nobody still reads the partner's psi
    // reverse sweep
    synced = true;
    for (int gg = C.ngroups - 1; gg >= 0; --gg) {
      const BGroup G = A.groups[C.group0 + gg];
      const bool split = group_is_split(G, hn);
      if (split && !synced) cluster.sync();
      if (split)
        cl_group_bwd<K, true>(Pp, Pl, ownp, ownl, rank, n, G, A.ops, mats, wpart);
      else
        cl_group_bwd<K, false>(Pp, Pl, ownp, ownl, rank, n, G, A.ops, mats, wpart);
      if (split) {
        cluster.sync();
        synced = true;
      } else {
        __syncthreads();
        synced = false;
      }
    }
    cluster.sync();  // both blocks' partials final
    if (rank == 0) {
      const double* pw = cluster.map_shared_rank(wpart, 1);
      const double* pred = cluster.map_shared_rank(red, 1);
      const int toff = A.theta_off[item];
      for (int p = threadIdx.x; p < C.nparams; p += kClThreads) {
        double g = 0.0;
        for (int w = 0; w < nwarps; ++w) g += wpart[w * kBMaxParams + p];
        for (int w = 0; w < nwarps; ++w) g += pw[w * kBMaxParams + p];
        A.grad[toff + p] = g;
      }
      if (threadIdx.x == 0) {
        double E = 0.0;
        for (int w = 0; w < nwarps; ++w) E += red[w];
        for (int w = 0; w < nwarps; ++w) E += pred[w];
        A.energy[item] = E;
      }
    }
    // the next item's barrier orders block 0's reads before block 1 reuses its partials
  }
}

}  // namespace
}  // namespace sv

// ---- host side: descriptors, autotuner, launches ---------------------------------
struct sv_batch_s {
  int n_items = 0, nmax = 0, total_params = 0;
  int k = 4, threads = 256, blocks = 0;  // chosen tile
  bool cluster = false;                  // two-block cluster kernel
  bool smem_states = false;              // single-block kernel with states in shared memory
  bool real = false;                     // real-amplitude kernel (kbatch_re)
  bool all_real = false;                 // every gate and term real: kbatch_re may run
  int sms = 152;
  // device buffers
  sv::BCirc* circs = nullptr;
  sv::BGateDesc* gates = nullptr;
  sv::BGroup* groups = nullptr;
  sv::BOp* ops = nullptr;
  sv::BTerm* terms = nullptr;
  int* order = nullptr;
  int* item_circ = nullptr;
  int* theta_off = nullptr;
  int* queue = nullptr;
  float2* work = nullptr;
  size_t work_slots = 0;
  std::vector<int> h_theta_off;
  // captured graph
  cudaGraphExec_t gexec = nullptr;
  const void* g_key[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace sv {
namespace {

struct HostPlan {
  std::vector<BCirc> circs;
  std::vector<BGateDesc> gates;
  std::vector<BGroup> groups;
  std::vector<BOp> ops;
  std::vector<BTerm> terms;
};

int popc64(uint64_t x) { return __builtin_popcountll(x); }

// List-schedule one circuit's gates (1-qubit kinds with controls) into groups
// of at most k qubits, as the fused pass planner does, without merging gates
// (every parameter keeps its own gate for the gradient).
bool plan_circuit(const sv_circuit* c, const sv_pauli_sum* H, int k, HostPlan* P) {
  const int n = c->n_qubits;
  BCirc C{};
  C.n = n;
  C.ngates = c->n_gates;
  C.gate0 = (int)P->gates.size();
  C.group0 = (int)P->groups.size();
  C.nparams = c->n_params;
  C.nterms = H->n_terms;
  C.term0 = (int)P->terms.size();
  std::vector<uint64_t> qm(c->n_gates);
  for (int i = 0; i < c->n_gates; ++i) {
    const sv_gate& g = c->gates[i];
    BGateDesc d{g.kind, g.param, g.angle};
    P->gates.push_back(d);
    uint64_t m = uint64_t(1) << (n - 1 - g.targets[0]);
    for (int j = 0; j < g.n_ctrl; ++j) m |= uint64_t(1) << (n - 1 - g.controls[j]);
    qm[i] = m;
  }
  std::vector<int> pending(c->n_gates);
  for (int i = 0; i < c->n_gates; ++i) pending[i] = i;
  while (!pending.empty()) {
    if (popc64(qm[pending[0]]) > k) return false;  // a gate wider than a group
    uint64_t gq = qm[pending[0]], acc = 0;
    std::vector<int> members, rest;
    for (int j : pending) {
      if (!(qm[j] & acc) && popc64(gq | qm[j]) <= k) {
        gq |= qm[j];
        members.push_back(j);
      } else {
        acc |= qm[j];
        rest.push_back(j);
      }
    }
    BGroup G{};
    int bits[64], nb = 0;
    for (int b = 0; b < n; ++b)
      if ((gq >> b) & 1) bits[nb++] = b;
    // pad narrow groups with free bits so every group has exactly min(k, n) bits
    for (int b = 0; b < n && nb < std::min(k, n); ++b)
      if (!((gq >> b) & 1)) {
        gq |= uint64_t(1) << b;
        bits[nb++] = b;
      }
    std::sort(bits, bits + nb);
    G.k = (uint8_t)nb;
    for (int i = 0; i < nb; ++i) G.bits[i] = (uint8_t)bits[i];
    G.op0 = (int32_t)P->ops.size();
    for (int j : members) {
      const sv_gate& g = c->gates[j];
      auto local = [&](int bit) {
        for (int i = 0; i < nb; ++i)
          if (bits[i] == bit) return i;
        return 0;
      };
      BOp op{};
      op.b0 = (uint8_t)local(n - 1 - g.targets[0]);
      for (int t = 0; t < g.n_ctrl; ++t) op.cm |= (uint8_t)(1 << local(n - 1 - g.controls[t]));
      op.pauli = g.param >= 0 ? (g.kind == SV_GATE_RX ? 1 : g.kind == SV_GATE_RY ? 2 : 3) : 0;
      switch (g.kind) {
        case SV_GATE_H: case SV_GATE_X: case SV_GATE_RY: op.cls = BC_REAL; break;
        case SV_GATE_Y: case SV_GATE_RX: op.cls = BC_IMOFF; break;
        case SV_GATE_RZ: op.cls = BC_DIAG; break;
        case SV_GATE_Z: op.cls = BC_NEG; break;
        case SV_GATE_U1: op.cls = BC_PHASE; break;
        default: op.cls = BC_DENSE;
      }
      op.param = (int16_t)g.param;
      op.gi = (int16_t)j;
      P->ops.push_back(op);
    }
    G.op1 = (int32_t)P->ops.size();
    P->groups.push_back(G);
    pending.swap(rest);
  }
  C.ngroups = (int)P->groups.size() - C.group0;
  // diagonal terms first: their coefficients combine per amplitude before
  // the one product with psi_x
  C.ndiag = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (int t = 0; t < H->n_terms; ++t) {
      const uint64_t xm = H->xmask[t], zm = H->zmask[t];
      if ((xm == 0) != (pass == 0)) continue;
      const int ny = popc64(xm & zm) & 3;
      const double cf = H->coeff[t];
      P->terms.push_back({xm, zm, ny == 0 ? cf : ny == 2 ? -cf : 0.0,
                          ny == 1 ? cf : ny == 3 ? -cf : 0.0});
      if (pass == 0) ++C.ndiag;
    }
  P->circs.push_back(C);
  return P->ops.size() < (size_t)0x7fffffff;
}

template <typename T>
sv_status upload(T** dst, const std::vector<T>& v) {
  const size_t bytes = std::max<size_t>(1, v.size()) * sizeof(T);
  SV_CUDA_TRY(cudaMalloc((void**)dst, bytes));
  if (!v.empty()) SV_CUDA_TRY(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SV_OK;
}

void free_batch(sv_batch b) {
  void* ptrs[] = {b->circs, b->gates, b->groups, b->ops, b->terms, b->order,
                  b->item_circ, b->theta_off, b->queue, b->work};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
}

typedef void (*BatchKernel)(const BatchArgs);
// Kernel variants by (group width, threads per block, resident blocks per
// SM): more resident blocks need fewer registers and less shared memory.
BatchKernel smem_kernel_for(int k) {
  return k == 2 ? kbatch<2, 512, 1, true> : k == 3 ? kbatch<3, 512, 1, true> : kbatch<4, 512, 1, true>;
}
BatchKernel kernel_for(int k, int threads, int per_sm) {
  if (threads >= 512) return k == 2 ? kbatch<2, 512, 1> : k == 3 ? kbatch<3, 512, 1> : kbatch<4, 512, 1>;
  if (threads <= 128) return k == 2 ? kbatch<2, 128, 8> : kbatch<3, 128, 8>;
  if (per_sm >= 4) return k == 2 ? kbatch<2, 256, 4> : kbatch<3, 256, 4>;
  return k == 2 ? kbatch<2, 256, 2> : k == 3 ? kbatch<3, 256, 2> : kbatch<4, 256, 2>;
}

// register groups of 2 or 3 qubits (4 would spill at 512 threads per block)
BatchKernel cluster_kernel_for(int k) { return k == 2 ? kbatch_cl<2> : kbatch_cl<3>; }

BatchKernel real_kernel_for(int k) {
  return k <= 3 ? kbatch_re<3, 512, 1> : k == 4 ? kbatch_re<4, 512, 1> : kbatch_re<5, 512, 1>;
}

sv_status launch_batch(sv_batch b, const double* theta, double* energy, double* grad,
                       cudaStream_t st, int k, int threads, int blocks, bool cl, bool sms,
                       bool re) {
  BatchArgs A;
  A.circs = b->circs;
  A.gates = b->gates;
  A.groups = b->groups;
  A.ops = b->ops;
  A.terms = b->terms;
  A.order = b->order;
  A.item_circ = b->item_circ;
  A.theta_off = b->theta_off;
  A.n_items = b->n_items;
  A.nmax = b->nmax;
  A.theta = theta;
  A.energy = energy;
  A.grad = grad;
  A.work = b->work;
  A.queue = b->queue;
  SV_CUDA_TRY(cudaMemsetAsync(b->queue, 0, sizeof(int), st));
  if (re) {
    BatchKernel kern = real_kernel_for(k);
    static bool attr[6] = {false, false, false, false, false, false};
    if (!attr[k]) {
      SV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(kBCacheBytes + kBSmemStateBytes)));
      attr[k] = true;
    }
    ProfScope prof(st, "kbatch_re");
    kern<<<blocks, 512, kBCacheBytes + kBSmemStateBytes, st>>>(A);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return check_launch("batch kernel (real amplitudes)");
  }
  if (cl) {
    BatchKernel kern = cluster_kernel_for(k);
    static bool attr[5] = {false, false, false, false, false};
    if (!attr[k]) {
      SV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kClSmemBytes));
      attr[k] = true;
    }
    ProfScope prof(st, "kbatch_cl");
    kern<<<blocks, kClThreads, kClSmemBytes, st>>>(A);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return check_launch("batch cluster kernel");
  }
  if (sms) {
    BatchKernel kern = smem_kernel_for(k);
    static bool attr[5] = {false, false, false, false, false};
    if (!attr[k]) {
      SV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(kBCacheBytes + kBSmemStateBytes)));
      attr[k] = true;
    }
    ProfScope prof(st, "kbatch_smem");
    kern<<<blocks, 512, kBCacheBytes + kBSmemStateBytes, st>>>(A);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return check_launch("batch kernel (shared-memory states)");
  }
  BatchKernel kern = kernel_for(k, threads, std::max(1, blocks / std::max(1, b->sms)));
  {
    // static (matrices, partials) + dynamic (descriptor cache) shared memory
    // can exceed the 48 KiB default: opt in once per kernel variant
    static std::mutex mu;
    static std::vector<BatchKernel> done;
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(done.begin(), done.end(), kern) == done.end()) {
      SV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kBCacheBytes));
      done.push_back(kern);
    }
  }
  ProfScope prof(st, "kbatch");
  kern<<<blocks, threads, kBCacheBytes, st>>>(A);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return check_launch("batch kernel");
}

}  // namespace
}  // namespace sv

using namespace sv;

extern "C" {

}  // extern "C"

// Checks every circuit and Hamiltonian against the batch kernel's limits;
// returns the largest qubit count and the widest gate (target + controls).
static sv_status validate_batch(const char* who, const sv_circuit* circuits,
                                const sv_pauli_sum* hamiltonians, int n_circuits, int* nmax_out,
                                int* width_out) {
  if (!circuits || !hamiltonians || n_circuits < 1) {
    set_error("%s: bad arguments", who);
    return SV_ERR_INVALID;
  }
  int nmax = 1, width = 1;  // widest gate: target plus controls
  for (int c = 0; c < n_circuits; ++c) {
    const sv_circuit& C = circuits[c];
    const sv_pauli_sum& H = hamiltonians[c];
    if (C.n_qubits < 1 || C.n_qubits > SV_BATCH_MAX_QUBITS || C.n_gates < 0 ||
        C.n_gates > kBMaxGates || C.n_params < 0 || C.n_params > kBMaxParams ||
        (C.n_gates > 0 && !C.gates)) {
      set_error("%s: circuit %d outside the batch limits (qubits <= %d, gates <= %d,"
                " parameters <= %d)", who, c, SV_BATCH_MAX_QUBITS, kBMaxGates, kBMaxParams);
      return SV_ERR_INVALID;
    }
    if (H.n_terms < 0 || H.n_terms > kBMaxTerms || (H.n_terms > 0 && (!H.xmask || !H.zmask || !H.coeff))) {
      set_error("%s: Hamiltonian %d must have 0..%d terms", who, c, kBMaxTerms);
      return SV_ERR_INVALID;
    }
    const uint64_t lim = (uint64_t(1) << C.n_qubits) - 1;
    for (int t = 0; t < H.n_terms; ++t)
      if ((H.xmask[t] | H.zmask[t]) & ~lim) {
        set_error("%s: Hamiltonian %d term %d has bits beyond %d qubits", who, c, t, C.n_qubits);
        return SV_ERR_INVALID;
      }
    for (int i = 0; i < C.n_gates; ++i) {
      const sv_gate& g = C.gates[i];
      const bool onequbit = g.kind >= SV_GATE_H && g.kind <= SV_GATE_U1 && g.n_tar == 1;
      bool ok = onequbit && g.n_ctrl >= 0 && g.n_ctrl <= 3 && g.param >= -1 && g.param < C.n_params;
      if (g.param >= 0 && g.kind != SV_GATE_RX && g.kind != SV_GATE_RY && g.kind != SV_GATE_RZ) ok = false;
      uint64_t seen = 0;
      for (int j = 0; ok && j < 1 + g.n_ctrl; ++j) {
        const int q = j == 0 ? g.targets[0] : g.controls[j - 1];
        if (q < 0 || q >= C.n_qubits || ((seen >> q) & 1)) ok = false;
        else seen |= uint64_t(1) << q;
      }
      if (!ok) {
        set_error("%s: circuit %d gate %d: the batch kernel takes 1-qubit kinds "
                  "(H X Y Z RX RY RZ U1) with up to 3 controls; parameters on RX/RY/RZ only", who, c, i);
        return SV_ERR_INVALID;
      }
    }
    nmax = std::max(nmax, C.n_qubits);
    for (int i = 0; i < C.n_gates; ++i) width = std::max(width, 1 + C.gates[i].n_ctrl);
  }
  *nmax_out = nmax;
  *width_out = width;
  return SV_OK;
}

extern "C" {

sv_status sv_batch_plan(const sv_circuit* circuits, const sv_pauli_sum* hamiltonians,
                        int n_circuits, int k, int32_t* groups_per_circuit) {
  int nmax = 0, width = 0;
  sv_status st = validate_batch("sv_batch_plan", circuits, hamiltonians, n_circuits, &nmax, &width);
  if (st) return st;
  if (k < 2 || k > 5 || k < width || !groups_per_circuit) {
    set_error("sv_batch_plan: group width %d must be in max(2, widest gate %d)..5", k, width);
    return SV_ERR_INVALID;
  }
  HostPlan P;
  for (int c = 0; c < n_circuits; ++c) {
    const size_t g0 = P.groups.size();
    if (!plan_circuit(&circuits[c], &hamiltonians[c], k, &P)) {
      set_error("sv_batch_plan: circuit %d does not fit groups of %d qubits", c, k);
      return SV_ERR_INVALID;
    }
    groups_per_circuit[c] = (int32_t)(P.groups.size() - g0);
  }
  return SV_OK;
}

sv_status sv_batch_create(const sv_circuit* circuits, const sv_pauli_sum* hamiltonians,
                          int n_circuits, const int32_t* item_circuit, int n_items, int tune,
                          sv_batch* out) {
  if (!item_circuit || !out || n_items < 1 || tune < 0 || tune > 4) {
    set_error("sv_batch_create: bad arguments");
    return SV_ERR_INVALID;
  }
  int nmax = 1, width = 1;
  {
    sv_status vs = validate_batch("sv_batch_create", circuits, hamiltonians, n_circuits, &nmax,
                                  &width);
    if (vs) return vs;
  }
  std::vector<int> ic(item_circuit, item_circuit + n_items), toff(n_items);
  int total = 0;
  for (int i = 0; i < n_items; ++i) {
    if (ic[i] < 0 || ic[i] >= n_circuits) {
      set_error("sv_batch_create: item %d names circuit %d of %d", i, ic[i], n_circuits);
      return SV_ERR_INVALID;
    }
    toff[i] = total;
    total += circuits[ic[i]].n_params;
  }
  sv_batch b = new sv_batch_s();
  b->n_items = n_items;
  b->nmax = nmax;
  b->total_params = total;
  b->h_theta_off = toff;
  // batch packing: longest items first (work ~ gates x 2^n)
  std::vector<int> order(n_items);
  for (int i = 0; i < n_items; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    const sv_circuit& A = circuits[ic[a]];
    const sv_circuit& C = circuits[ic[c]];
    return (double)A.n_gates * (1 << A.n_qubits) > (double)C.n_gates * (1 << C.n_qubits);
  });
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 152;
  // candidates: group width k, threads per block, blocks per SM
  struct Cand {
    int k, threads, per_sm;
    bool cl;          // two-block clusters (per_sm = 1, threads = kClThreads)
    bool sms = false; // states in shared memory up to 14 qubits (512 threads, 1 per SM)
    bool re = false;  // real amplitudes (kbatch_re, 512 threads, 1 per SM)
  };
  // real batch: every gate real (H, X, Z, RY, with controls) and every term a
  // real matrix (an even number of Y factors)
  bool all_real = true;
  for (int c = 0; c < n_circuits && all_real; ++c) {
    for (int i = 0; i < circuits[c].n_gates; ++i) {
      const int kd = circuits[c].gates[i].kind;
      if (kd != SV_GATE_H && kd != SV_GATE_X && kd != SV_GATE_Z && kd != SV_GATE_RY) all_real = false;
    }
    for (int t = 0; t < hamiltonians[c].n_terms; ++t)
      if (popc64(hamiltonians[c].xmask[t] & hamiltonians[c].zmask[t]) & 1) all_real = false;
  }
  b->all_real = all_real;
  std::vector<Cand> cands;
  if (tune == 4) {
    if (!all_real) {
      set_error("sv_batch_create: tune = 4 (real amplitudes) needs every gate real (H X Z RY)"
                " and every term with an even number of Y factors");
      delete b;
      return SV_ERR_INVALID;
    }
    cands.push_back({std::max(4, width), 512, 1, false, true, true});
  } else if (tune == 1) {
    if (all_real)
      for (int kr = std::max(3, width); kr <= 5; ++kr) cands.push_back({kr, 512, 1, false, true, true});
    const Cand all[] = {{2, 512, 1, false, true}, {3, 512, 1, false, true}, {4, 512, 1, false, true},
                        {2, kClThreads, 1, true}, {3, kClThreads, 1, true},
                        {2, 512, 1, false}, {3, 512, 1, false}, {4, 512, 1, false},
                        {2, 256, 2, false}, {3, 256, 2, false}, {4, 256, 2, false},
                        {2, 256, 4, false}, {3, 256, 4, false}, {2, 128, 8, false},
                        {3, 128, 8, false}};
    for (const Cand& c : all)
      if (c.k >= width) cands.push_back(c);
  } else if (tune == 2 && width <= 3) {
    cands.push_back({3, kClThreads, 1, true});
  } else if (tune == 3) {
    cands.push_back({std::max(4, width), 512, 1, false, true});
  } else {
    cands.push_back({std::max(4, width), 256, 2, false});
  }
  int max_per = 1;
  for (auto& c : cands) max_per = std::max(max_per, c.per_sm);
  b->work_slots = (size_t)sms * max_per;
  b->sms = sms;
  sv_status st = SV_OK;
  // plans per k are built on demand; start with the device buffers that do not depend on k
  st = upload(&b->order, order);
  if (!st) st = upload(&b->item_circ, ic);
  if (!st) st = upload(&b->theta_off, toff);
  if (!st) {
    cudaError_t e = cudaMalloc(&b->queue, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->work, b->work_slots * (sizeof(float2) << (nmax + 1)));
    if (e != cudaSuccess) {
      set_error("sv_batch_create: %s", cudaGetErrorString(e));
      st = e == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA;
    }
  }
  auto build_for_k = [&](int k) -> sv_status {
    HostPlan P;
    for (int c = 0; c < n_circuits; ++c)
      if (!plan_circuit(&circuits[c], &hamiltonians[c], k, &P)) {
        set_error("sv_batch_create: a gate does not fit a register group of %d qubits", k);
        return SV_ERR_INVALID;
      }
    void* olds[] = {b->circs, b->gates, b->groups, b->ops, b->terms};
    for (void* p : olds)
      if (p) cudaFree(p);
    b->circs = nullptr; b->gates = nullptr; b->groups = nullptr; b->ops = nullptr; b->terms = nullptr;
    sv_status s2 = upload(&b->circs, P.circs);
    if (!s2) s2 = upload(&b->gates, P.gates);
    if (!s2) s2 = upload(&b->groups, P.groups);
    if (!s2) s2 = upload(&b->ops, P.ops);
    if (!s2) s2 = upload(&b->terms, P.terms);
    return s2;
  };
  double* th = nullptr;
  double* en = nullptr;
  double* gr = nullptr;
  if (!st && cands.size() > 1) {
    // autotune on the real batch with arbitrary parameters (timing does not depend on them)
    std::vector<double> tv(std::max(1, total));
    for (size_t i = 0; i < tv.size(); ++i) tv[i] = 0.001 * (double)(i % 997);
    cudaError_t e = cudaMalloc(&th, tv.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&en, n_items * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&gr, tv.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(th, tv.data(), tv.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      set_error("sv_batch_create: tuning buffers: %s", cudaGetErrorString(e));
      st = SV_ERR_CUDA;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int built = -1;
    for (const Cand& c : cands) {
      if (st) break;
      if (c.k != built) {
        st = build_for_k(c.k);
        built = c.k;
        if (st) break;
      }
      const int blocks = c.cl ? 2 * (sms / 2) : sms * c.per_sm;
      st = launch_batch(b, th, en, gr, 0, c.k, c.threads, blocks, c.cl, c.sms, c.re);  // warm-up
      if (st) break;
      cudaEventRecord(e0, 0);
      st = launch_batch(b, th, en, gr, 0, c.k, c.threads, blocks, c.cl, c.sms, c.re);
      cudaEventRecord(e1, 0);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        set_error("sv_batch_create: tuning run failed: %s", cudaGetErrorString(cudaGetLastError()));
        st = SV_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        b->k = c.k;
        b->threads = c.threads;
        b->blocks = blocks;
        b->cluster = c.cl;
        b->smem_states = c.sms;
        b->real = c.re;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  } else if (!st) {
    b->k = cands[0].k;
    b->threads = cands[0].threads;
    b->cluster = cands[0].cl;
    b->smem_states = cands[0].sms;
    b->real = cands[0].re;
    b->blocks = cands[0].cl ? 2 * (sms / 2) : sms * cands[0].per_sm;
  }
  if (th) cudaFree(th);
  if (en) cudaFree(en);
  if (gr) cudaFree(gr);
  if (!st) st = build_for_k(b->k);
  if (!st) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      set_error("sv_batch_create: %s", cudaGetErrorString(e));
      st = SV_ERR_CUDA;
    }
  }
  if (st) {
    free_batch(b);
    delete b;
    return st;
  }
  *out = b;
  return SV_OK;
}

sv_status sv_batch_info(sv_batch b, int* k, int* threads, int* blocks, int* total_params) {
  if (!b) {
    set_error("sv_batch_info: null batch");
    return SV_ERR_INVALID;
  }
  if (k) *k = b->k;
  if (threads) *threads = b->threads;
  if (blocks) *blocks = b->blocks;
  if (total_params) *total_params = b->total_params;
  return SV_OK;
}

sv_status sv_batch_kernel(sv_batch b, int* cluster_size, int* smem_states, int* real_states) {
  if (!b || !cluster_size || !smem_states || !real_states) {
    set_error("sv_batch_kernel: bad arguments");
    return SV_ERR_INVALID;
  }
  *cluster_size = b->cluster ? 2 : 1;
  *smem_states = (b->cluster || b->smem_states || b->real) ? 1 : 0;
  *real_states = b->real ? 1 : 0;
  return SV_OK;
}

sv_status sv_batch_run(sv_batch b, const double* dev_theta, double* dev_energy, double* dev_grad,
                       void* cuda_stream) {
  if (!b || !dev_theta || !dev_energy || !dev_grad) {
    set_error("sv_batch_run: bad arguments");
    return SV_ERR_INVALID;
  }
  return launch_batch(b, dev_theta, dev_energy, dev_grad, (cudaStream_t)cuda_stream, b->k,
                      b->threads, b->blocks, b->cluster, b->smem_states, b->real);
}

sv_status sv_batch_run_graph(sv_batch b, const double* dev_theta, double* dev_energy,
                             double* dev_grad, void* cuda_stream) {
  if (!b || !dev_theta || !dev_energy || !dev_grad) {
    set_error("sv_batch_run_graph: bad arguments");
    return SV_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const void* key[4] = {dev_theta, dev_energy, dev_grad, cuda_stream};
  if (!b->gexec || memcmp(key, b->g_key, sizeof(key)) != 0) {
    if (b->gexec) {
      cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
    }
    cudaStream_t cap = nullptr;
    SV_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    sv_status s2 = SV_OK;
    if (e == cudaSuccess) {
      s2 = launch_batch(b, dev_theta, dev_energy, dev_grad, cap, b->k, b->threads, b->blocks,
                        b->cluster, b->smem_states, b->real);
      e = cudaStreamEndCapture(cap, &g);
    }
    if (e == cudaSuccess && s2 == SV_OK) e = cudaGraphInstantiate(&b->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess || s2 != SV_OK) {
      if (e != cudaSuccess) set_error("sv_batch_run_graph: capture: %s", cudaGetErrorString(e));
      b->gexec = nullptr;
      return s2 != SV_OK ? s2 : SV_ERR_CUDA;
    }
    memcpy(b->g_key, key, sizeof(key));
  }
  SV_CUDA_TRY(cudaGraphLaunch(b->gexec, st));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return SV_OK;
}

sv_status sv_batch_grad(const sv_circuit* circuits, const sv_pauli_sum* hamiltonians,
                        int n_circuits, const int32_t* item_circuit, int n_items,
                        const double* theta, void* cuda_stream, double* energies, double* grads) {
  if (!theta || !energies || !grads) {
    set_error("sv_batch_grad: null host arrays");
    return SV_ERR_INVALID;
  }
  sv_batch b = nullptr;
  sv_status st = sv_batch_create(circuits, hamiltonians, n_circuits, item_circuit, n_items, 0, &b);
  if (st) return st;
  const size_t np = std::max(1, b->total_params);
  double *th = nullptr, *en = nullptr, *gr = nullptr;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaMalloc(&th, np * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&en, n_items * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&gr, np * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(th, theta, b->total_params * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    st = sv_batch_run(b, th, en, gr, cuda_stream);
    if (!st) {
      e = cudaMemcpyAsync(energies, en, n_items * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(grads, gr, b->total_params * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
  }
  if (e != cudaSuccess && !st) {
    set_error("sv_batch_grad: %s", cudaGetErrorString(e));
    st = e == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA;
  }
  if (th) cudaFree(th);
  if (en) cudaFree(en);
  if (gr) cudaFree(gr);
  sv_batch_free(b);
  return st;
}

sv_status sv_batch_free(sv_batch b) {
  if (!b) return SV_OK;
  cudaDeviceSynchronize();
  free_batch(b);
  delete b;
  return SV_OK;
}

}  // extern "C"
