// Measurement in the computational basis (Sec. 3: sampling of measurements).
//
// Outcome of measuring qubits q_0..q_{m-1}: r = sum_j b(q_j) 2^(m-1-j)
// (q_0 the most significant bit), P(r) = sum of |psi_x|^2 over the x whose
// measured bits spell r.
//
// Arithmetic: every amplitude contributes q(re) + q(im), q(v) =
// floor(v^2 2^120), computed exactly from v's significand and exponent with
// integer instructions, and sums are exact 128-bit integers.  The CDF is
// therefore independent of summation order (GPU and CPU take identical
// integer decisions), and the kernels avoid the fp64 pipe, which on GB300
// issues too slowly to keep up with HBM for a per-amplitude fp64 square.
// The truncation costs at most 2^-120 per component (2^-85 over 2^34
// amplitudes).  States must satisfy sum |psi|^2 < 256.
//
// Probabilities: bin r is the set x = insert(e, measured bits) | bits(r),
// e < 2^(n-m); (bin, slice) blocks sum their slices, a finish adds the slices
// and rounds P = sum / 2^120 to fp64.
//
// Sampling for caller-given uniforms u (the random numbers are inputs):
// exact chunk sums (a warp per 1024 amplitudes, one HBM pass), an exact
// prefix scan of the chunk sums, then one warp per shot: T = floor(u *
// total) exactly, binary search for the first chunk prefix above T, and a
// scan of that chunk 32 amplitudes at a time (warp prefix sum) for the first
// x with c(x) > T.  Outcomes are projected onto the measured qubits (the
// marginal of a subset is the projection of full samples).
#include <algorithm>
#include <vector>

#include "sv_device.cuh"

namespace sv {
namespace {

constexpr int kChunkBits = 10;

struct U128 {
  uint64_t lo, hi;
};

__device__ __forceinline__ U128 add128(U128 a, U128 b) {
  U128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1 : 0);
  return r;
}

__device__ __forceinline__ bool gt128(U128 a, U128 b) {
  return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}

// x * 2^sh (sh >= 0) or floor(x / 2^-sh), for results below 2^128
__device__ __forceinline__ U128 shift128(U128 x, int sh) {
  if (sh > 0) {
    if (sh >= 128) return {0, 0};
    if (sh >= 64) return {0, x.lo << (sh - 64)};
    return {x.lo << sh, (x.hi << sh) | (x.lo >> (64 - sh))};
  }
  const int r = -sh;
  if (r == 0) return x;
  if (r >= 128) return {0, 0};
  if (r >= 64) return {x.hi >> (r - 64), 0};
  return {(x.lo >> r) | (x.hi << (64 - r)), x.hi >> r};
}

// q(v) = floor(v^2 2^120)
__device__ __forceinline__ U128 q120(float v) {
  const uint32_t b = __float_as_uint(v) & 0x7fffffffu;
  const int e = (int)(b >> 23);
  if (e == 0) return {0, 0};  // zero or subnormal: v^2 2^120 < 1
  const uint64_t m = (b & 0x7fffffu) | 0x800000u;  // v = m 2^(e - 150)
  return shift128(U128{m * m, 0}, 2 * (e - 150) + 120);
}

__device__ __forceinline__ U128 q120(double v) {
  const uint64_t b = (uint64_t)__double_as_longlong(v) & 0x7fffffffffffffffull;
  const int e = (int)(b >> 52);
  if (e == 0) return {0, 0};
  const uint64_t m = (b & 0xfffffffffffffull) | (1ull << 52);  // v = m 2^(e - 1075)
  return shift128(U128{m * m, __umul64hi(m, m)}, 2 * (e - 1075) + 120);
}

template <typename T2>
__device__ __forceinline__ U128 qamp(const T2 a) {
  return add128(q120(a.x), q120(a.y));
}

__device__ __forceinline__ U128 qvec(const float4 a) {
  return add128(add128(q120(a.x), q120(a.y)), add128(q120(a.z), q120(a.w)));
}
__device__ __forceinline__ U128 qvec(const double2 a) { return add128(q120(a.x), q120(a.y)); }

__device__ __forceinline__ U128 shfl_xor128(U128 v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.lo, o), __shfl_xor_sync(0xffffffffu, v.hi, o)};
}

__device__ __forceinline__ U128 warp_sum128(U128 v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = add128(v, shfl_xor128(v, o));
  return v;
}

// floor(u * t) for u in [0, 1), exactly (192-bit intermediate)
__device__ __forceinline__ U128 frac_mul(double u, U128 t) {
  if (!(u > 0.0)) return {0, 0};
  const uint64_t b = (uint64_t)__double_as_longlong(u);
  const int e = (int)(b >> 52);
  uint64_t m;
  int s;  // u = m 2^-s
  if (e == 0) {
    m = b & 0xfffffffffffffull;
    s = 1074;
  } else {
    m = (b & 0xfffffffffffffull) | (1ull << 52);
    s = 1075 - e;
  }
  // m t = w2 2^128 + w1 2^64 + w0
  const uint64_t w0 = m * t.lo, c0 = __umul64hi(m, t.lo);
  const uint64_t l1 = m * t.hi, h1 = __umul64hi(m, t.hi);
  const uint64_t w1 = c0 + l1;
  const uint64_t w2 = h1 + (w1 < c0 ? 1 : 0);
  if (s >= 192) return {0, 0};
  if (s >= 128) return {s == 128 ? w2 : w2 >> (s - 128), 0};
  if (s >= 64) {
    const int r = s - 64;
    if (r == 0) return {w1, w2};
    return {(w1 >> r) | (w2 << (64 - r)), w2 >> r};
  }
  if (s == 0) return {w0, w1};
  return {(w0 >> s) | (w1 << (64 - s)), (w1 >> s) | (w2 << (64 - s))};
}

// partials[r * slices + c] = exact sum over slice c of bin r
template <typename T2>
__global__ void __launch_bounds__(kRedThreads)
    kprob_slices(const T2* __restrict__ psi, Ins<uint64_t> rest, const int* __restrict__ mpos,
                 int m, uint64_t per_bin, int slices, U128* __restrict__ partials) {
  __shared__ U128 ws[kRedThreads / 32];
  const int r = blockIdx.x / slices, c = blockIdx.x % slices;
  uint64_t rbits = 0;
  for (int j = 0; j < m; ++j)
    if ((r >> (m - 1 - j)) & 1) rbits |= uint64_t(1) << mpos[j];
  const uint64_t len = (per_bin + slices - 1) / slices;
  const uint64_t e0 = (uint64_t)c * len, e1 = e0 + len < per_bin ? e0 + len : per_bin;
  U128 acc = {0, 0};
  constexpr int U = 8;  // loads in flight per thread
  for (uint64_t e = e0 + threadIdx.x; e < e1; e += (uint64_t)kRedThreads * U) {
    T2 v[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const uint64_t ek = e + (uint64_t)k * kRedThreads;
      if (ek < e1) v[k] = psi[insert_zeros(ek, rest) | rbits];
    }
#pragma unroll
    for (int k = 0; k < U; ++k)
      if (e + (uint64_t)k * kRedThreads < e1) acc = add128(acc, qamp(v[k]));
  }
  acc = warp_sum128(acc);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    U128 t = {0, 0};
    for (int w = 0; w < kRedThreads / 32; ++w) t = add128(t, ws[w]);
    partials[blockIdx.x] = t;
  }
}

// P(r) = (sum of the bin's slices) / 2^120, rounded to fp64
__global__ void kprob_finish(const U128* __restrict__ partials, int slices, uint64_t bins,
                             double* __restrict__ out) {
  const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= bins) return;
  U128 t = {0, 0};
  for (int c = 0; c < slices; ++c) t = add128(t, partials[r * slices + c]);
  out[r] = (__ull2double_rn(t.hi) * 18446744073709551616.0 + __ull2double_rn(t.lo)) *
           7.52316384526264005099991383822e-37;  // 2^-120
}

// sums[k] = exact sum over chunk k (2^vbits vectors of 16 bytes), a warp per chunk
template <typename V>
__global__ void __launch_bounds__(kRedThreads)
    kchunk_sums(const V* __restrict__ psi, int vbits, uint64_t K, U128* __restrict__ sums) {
  const uint64_t k = (uint64_t)blockIdx.x * (kRedThreads / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= K) return;
  const V* c = psi + (k << vbits);
  const int nv = 1 << vbits;
  U128 acc = {0, 0};
  constexpr int U = 16;
  for (int i0 = lane; i0 < nv; i0 += 32 * U) {
    V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (i0 + 32 * u < nv) v[u] = c[i0 + 32 * u];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (i0 + 32 * u < nv) acc = add128(acc, qvec(v[u]));
  }
  acc = warp_sum128(acc);
  if (lane == 0) sums[k] = acc;
}

// inclusive prefix sums in place (exact, so any order gives the same values)
__global__ void __launch_bounds__(1024) kscan(U128* __restrict__ v, uint64_t K) {
  __shared__ U128 tot[1024];
  const uint64_t seg = (K + 1023) / 1024;
  const uint64_t a = threadIdx.x * seg, b = a + seg < K ? a + seg : K;
  U128 s = {0, 0};
  for (uint64_t i = a; i < b; ++i) {
    s = add128(s, v[i]);
    v[i] = s;
  }
  tot[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    U128 run = {0, 0};
    for (int t = 0; t < 1024; ++t) {
      const U128 x = tot[t];
      tot[t] = run;
      run = add128(run, x);
    }
  }
  __syncthreads();
  const U128 off = tot[threadIdx.x];
  for (uint64_t i = a; i < b; ++i) v[i] = add128(v[i], off);
}

// Block-local inclusive scan of 1024 entries; the block's total goes to
// totals[blockIdx.x].
__global__ void __launch_bounds__(1024) kscan_local(U128* __restrict__ v, uint64_t K,
                                                    U128* __restrict__ totals) {
  __shared__ U128 ws[32];
  const uint64_t i = (uint64_t)blockIdx.x * 1024 + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  U128 x = i < K ? v[i] : U128{0, 0};
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const U128 y = {__shfl_up_sync(0xffffffffu, x.lo, o), __shfl_up_sync(0xffffffffu, x.hi, o)};
    if (lane >= o) x = add128(x, y);
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    U128 run = {0, 0};
    for (int k = 0; k < 32; ++k) {
      const U128 t = ws[k];
      ws[k] = run;
      run = add128(run, t);
    }
    totals[blockIdx.x] = run;
  }
  __syncthreads();
  x = add128(x, ws[w]);
  if (i < K) v[i] = x;
}

// v[i] += inclusive prefix of the totals of the blocks before i's block
__global__ void __launch_bounds__(1024) kscan_add(U128* __restrict__ v, uint64_t K,
                                                  const U128* __restrict__ scanned_totals) {
  const uint64_t i = (uint64_t)blockIdx.x * 1024 + threadIdx.x;
  if (blockIdx.x == 0 || i >= K) return;
  v[i] = add128(v[i], scanned_totals[blockIdx.x - 1]);
}

// One warp per shot.
template <typename T2>
__global__ void __launch_bounds__(kRedThreads)
    kshots(const T2* __restrict__ psi, int cbits, const U128* __restrict__ prefix, uint64_t K,
           const double* __restrict__ u, int64_t nshots, const int* __restrict__ mpos, int m,
           uint64_t* __restrict__ out) {
  const int64_t s = (int64_t)blockIdx.x * (kRedThreads / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= nshots) return;
  const U128 T = frac_mul(u[s], prefix[K - 1]);
  uint64_t lo = 0, hi = K - 1;  // first chunk whose prefix exceeds T
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (gt128(prefix[mid], T)) hi = mid; else lo = mid + 1;
  }
  U128 acc = lo ? prefix[lo - 1] : U128{0, 0};
  const uint64_t base = lo << cbits;
  const int len = 1 << cbits;
  uint64_t x = base + len - 1;
  for (int i0 = 0; i0 < len; i0 += 32) {
    const int i = i0 + lane;
    U128 incl = i < len ? qamp(psi[base + i]) : U128{0, 0};
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const U128 y = {__shfl_up_sync(0xffffffffu, incl.lo, o),
                      __shfl_up_sync(0xffffffffu, incl.hi, o)};
      if (lane >= o) incl = add128(incl, y);
    }
    const unsigned over = __ballot_sync(0xffffffffu, gt128(add128(acc, incl), T));
    if (over) {
      x = base + i0 + (__ffs(over) - 1);
      break;
    }
    acc = add128(acc, U128{__shfl_sync(0xffffffffu, incl.lo, 31),
                           __shfl_sync(0xffffffffu, incl.hi, 31)});
  }
  if (lane == 0) {
    uint64_t r = 0;
    for (int j = 0; j < m; ++j) r = (r << 1) | ((x >> mpos[j]) & 1);
    out[s] = r;
  }
}

}  // namespace
}  // namespace sv

using namespace sv;

static bool valid_measure(sv_state s, const int* qubits, int m, int maxm) {
  if (!s || !s->data || !qubits || m < 1 || m > s->n || m > maxm) {
    set_error("measurement: bad state or qubit list (1 <= n_meas <= min(n, %d))", maxm);
    return false;
  }
  uint64_t seen = 0;
  for (int j = 0; j < m; ++j) {
    if (qubits[j] < 0 || qubits[j] >= s->n || ((seen >> qubits[j]) & 1)) {
      set_error("measurement: qubit %d invalid or repeated", qubits[j]);
      return false;
    }
    seen |= uint64_t(1) << qubits[j];
  }
  return true;
}

extern "C" {

sv_status sv_probabilities(sv_state s, const int* qubits, int n_meas, double* out) {
  if (!valid_measure(s, qubits, n_meas, SV_MAX_MEASURE_PROBS) || !out) {
    if (!out) set_error("sv_probabilities: null output");
    return SV_ERR_INVALID;
  }
  const int n = s->n, m = n_meas;
  int mpos[64];
  std::vector<int> pos;
  for (int j = 0; j < m; ++j) {
    mpos[j] = n - 1 - qubits[j];
    pos.push_back(mpos[j]);
  }
  const uint64_t bins = uint64_t(1) << m, per_bin = uint64_t(1) << (n - m);
  const int slices = (int)std::max<uint64_t>(1, std::min<uint64_t>(2432 / bins, per_bin / 2048));
  const size_t nparts = bins * slices;
  // partials (2 doubles each), then the bins, then the measured positions
  sv_status st = ensure_partials(s, 2 * nparts + bins + 64);
  if (st) return st;
  U128* parts = reinterpret_cast<U128*>(s->partials);
  double* dbins = s->partials + 2 * nparts;
  int* dpos = reinterpret_cast<int*>(dbins + bins);
  SV_CUDA_TRY(cudaMemcpyAsync(dpos, mpos, sizeof(int) * m, cudaMemcpyHostToDevice, s->stream));
  const Ins<uint64_t> rest = make_ins<uint64_t>(pos);
  {
    ProfScope prof(s->stream, "kprob_slices");
    if (s->dt == SV_C64)
      kprob_slices<float2><<<(unsigned)nparts, kRedThreads, 0, s->stream>>>(
          (const float2*)s->data, rest, dpos, m, per_bin, slices, parts);
    else
      kprob_slices<double2><<<(unsigned)nparts, kRedThreads, 0, s->stream>>>(
          (const double2*)s->data, rest, dpos, m, per_bin, slices, parts);
    g_launches.fetch_add(1, std::memory_order_relaxed);
  }
  {
    ProfScope prof(s->stream, "kprob_finish");
    kprob_finish<<<(unsigned)((bins + 255) / 256), 256, 0, s->stream>>>(parts, slices, bins, dbins);
    g_launches.fetch_add(1, std::memory_order_relaxed);
  }
  st = check_launch("probabilities kernels");
  if (st) return st;
  SV_CUDA_TRY(cudaMemcpyAsync(out, dbins, sizeof(double) * bins, cudaMemcpyDeviceToHost, s->stream));
  SV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return SV_OK;
}

sv_status sv_sample(sv_state s, const int* qubits, int n_meas, int64_t n_shots,
                    const double* uniforms, uint64_t* out) {
  if (!valid_measure(s, qubits, n_meas, 64)) return SV_ERR_INVALID;
  if (n_shots < 0 || n_shots > SV_MAX_SHOTS || (n_shots > 0 && (!uniforms || !out))) {
    set_error("sv_sample: 0 <= n_shots <= %lld with host uniforms and outputs",
              (long long)SV_MAX_SHOTS);
    return SV_ERR_INVALID;
  }
  for (int64_t i = 0; i < n_shots; ++i)
    if (!(uniforms[i] >= 0.0 && uniforms[i] < 1.0)) {
      set_error("sv_sample: uniform %lld = %g outside [0, 1)", (long long)i, uniforms[i]);
      return SV_ERR_INVALID;
    }
  if (n_shots == 0) return SV_OK;
  const int n = s->n, m = n_meas;
  const int cbits = std::max(1, std::min(n, kChunkBits));
  const uint64_t K = uint64_t(1) << (n - cbits);
  int mpos[64];
  for (int j = 0; j < m; ++j) mpos[j] = n - 1 - qubits[j];
  // prefix[K] (2 doubles each), uniforms[n_shots], outcomes[n_shots], positions,
  // block totals of the scan
  const uint64_t nb = (K + 1023) / 1024;
  const size_t need = 2 * K + 2 * (size_t)n_shots + 64 + 2 * nb;
  sv_status st = ensure_partials(s, need);
  if (st) return st;
  U128* prefix = reinterpret_cast<U128*>(s->partials);
  double* du = s->partials + 2 * K;
  uint64_t* dout = reinterpret_cast<uint64_t*>(du + n_shots);
  int* dpos = reinterpret_cast<int*>(dout + n_shots);
  U128* btot = reinterpret_cast<U128*>(reinterpret_cast<double*>(dout + n_shots) + 64);
  SV_CUDA_TRY(cudaMemcpyAsync(dpos, mpos, sizeof(int) * m, cudaMemcpyHostToDevice, s->stream));
  SV_CUDA_TRY(cudaMemcpyAsync(du, uniforms, sizeof(double) * n_shots, cudaMemcpyHostToDevice,
                              s->stream));
  {
    ProfScope prof(s->stream, "kchunk_sums");
    const unsigned g = (unsigned)((K + kRedThreads / 32 - 1) / (kRedThreads / 32));
    if (s->dt == SV_C64)  // 2 amplitudes per 16-byte vector
      kchunk_sums<float4><<<g, kRedThreads, 0, s->stream>>>((const float4*)s->data, cbits - 1,
                                                            K, prefix);
    else
      kchunk_sums<double2><<<g, kRedThreads, 0, s->stream>>>((const double2*)s->data, cbits, K,
                                                             prefix);
    g_launches.fetch_add(1, std::memory_order_relaxed);
  }
  {
    ProfScope prof(s->stream, "kscan");
    if (nb == 1) {
      kscan<<<1, 1024, 0, s->stream>>>(prefix, K);
      g_launches.fetch_add(1, std::memory_order_relaxed);
    } else {
      kscan_local<<<(unsigned)nb, 1024, 0, s->stream>>>(prefix, K, btot);
      kscan<<<1, 1024, 0, s->stream>>>(btot, nb);
      kscan_add<<<(unsigned)nb, 1024, 0, s->stream>>>(prefix, K, btot);
      g_launches.fetch_add(3, std::memory_order_relaxed);
    }
  }
  {
    ProfScope prof(s->stream, "kshots");
    const unsigned g = (unsigned)((n_shots + kRedThreads / 32 - 1) / (kRedThreads / 32));
    if (s->dt == SV_C64)
      kshots<float2><<<g, kRedThreads, 0, s->stream>>>((const float2*)s->data, cbits, prefix, K,
                                                       du, n_shots, dpos, m, dout);
    else
      kshots<double2><<<g, kRedThreads, 0, s->stream>>>((const double2*)s->data, cbits, prefix,
                                                         K, du, n_shots, dpos, m, dout);
    g_launches.fetch_add(1, std::memory_order_relaxed);
  }
  st = check_launch("sampling kernels");
  if (st) return st;
  SV_CUDA_TRY(cudaMemcpyAsync(out, dout, sizeof(uint64_t) * n_shots, cudaMemcpyDeviceToHost,
                              s->stream));
  SV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return SV_OK;
}

}  // extern "C"
