// Measurement in the computational basis (Sec. 3: sampling of measurements).
//
// Outcome of measuring qubits q_0..q_{m-1}: r = sum_j b(q_j) 2^(m-1-j)
// (q_0 the most significant bit), P(r) = sum of |psi_x|^2 over the x whose
// measured bits spell r.
//
// Probabilities: bin r is the set x = insert(e, measured bits) | bits(r) for
// e < 2^(n-m); a grid of (bin, slice) blocks sums its slice in fp64 (thread,
// then block tree) and a fixed-order finish adds the slices: one HBM pass,
// bit-identical from call to call.
//
// Sampling by the inverse CDF c(x) = sum_{y <= x} |psi_y|^2 for caller-given
// uniforms u (the random numbers are inputs): fp64 sums of 1024-amplitude
// chunks (one HBM pass), an inclusive prefix scan of the chunk sums in fixed
// order, then per shot a binary search over the chunk prefixes for the first
// one above u * total and a scan inside that chunk for the first index whose
// running sum exceeds it.  Full outcomes x are projected onto the measured
// qubits (the marginal of a subset is the projection of full samples).
#include <algorithm>
#include <vector>

#include "sv_device.cuh"

namespace sv {
namespace {

constexpr int kChunkBits = 10;

template <typename T2>
__device__ __forceinline__ double prob(const T2 a) {
  return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}

// partials[r * slices + c] = sum over slice c of bin r
template <typename T2>
__global__ void __launch_bounds__(kRedThreads)
    kprob_slices(const T2* __restrict__ psi, Ins<uint64_t> rest, const int* __restrict__ mpos,
                 int m, uint64_t per_bin, int slices, double* __restrict__ partials) {
  const int r = blockIdx.x / slices, c = blockIdx.x % slices;
  uint64_t rbits = 0;
  for (int j = 0; j < m; ++j)
    if ((r >> (m - 1 - j)) & 1) rbits |= uint64_t(1) << mpos[j];
  const uint64_t len = (per_bin + slices - 1) / slices;
  const uint64_t e0 = (uint64_t)c * len, e1 = e0 + len < per_bin ? e0 + len : per_bin;
  double acc = 0.0;
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
      if (e + (uint64_t)k * kRedThreads < e1) acc += prob(v[k]);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// sums[k] = sum of |psi|^2 over chunk k (2^cbits amplitudes): one warp per
// chunk, 16-byte loads, a fixed shuffle tree per chunk.
__device__ __forceinline__ double prob4(const float4 a) {
  return (double)a.x * a.x + (double)a.y * a.y + ((double)a.z * a.z + (double)a.w * a.w);
}
__device__ __forceinline__ double prob4(const double2 a) { return a.x * a.x + a.y * a.y; }

template <typename V>
__global__ void __launch_bounds__(kRedThreads)
    kchunk_sums(const V* __restrict__ psi, int vbits, uint64_t K, double* __restrict__ sums) {
  const uint64_t k = (uint64_t)blockIdx.x * (kRedThreads / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= K) return;
  const V* c = psi + (k << vbits);
  const int nv = 1 << vbits;  // vectors per chunk
  double acc = 0.0;
  constexpr int U = 16;
  for (int i0 = lane; i0 < nv; i0 += 32 * U) {
    V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (i0 + 32 * u < nv) v[u] = c[i0 + 32 * u];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (i0 + 32 * u < nv) acc += prob4(v[u]);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) sums[k] = acc;
}

// inclusive prefix sums in place, one block of 1024 threads, fixed order
__global__ void __launch_bounds__(1024) kscan(double* __restrict__ v, uint64_t K) {
  __shared__ double tot[1024];
  const uint64_t seg = (K + 1023) / 1024;
  const uint64_t a = threadIdx.x * seg, b = a + seg < K ? a + seg : K;
  double s = 0.0;
  for (uint64_t i = a; i < b; ++i) {
    s += v[i];
    v[i] = s;
  }
  tot[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double run = 0.0;
    for (int t = 0; t < 1024; ++t) {
      const double x = tot[t];
      tot[t] = run;
      run += x;
    }
  }
  __syncthreads();
  const double off = tot[threadIdx.x];
  for (uint64_t i = a; i < b; ++i) v[i] += off;
}

// One warp per shot: binary search over the chunk prefixes, then the chunk
// is scanned 32 amplitudes at a time with a warp prefix sum.
template <typename T2>
__global__ void __launch_bounds__(kRedThreads)
    kshots(const T2* __restrict__ psi, int n, int cbits, const double* __restrict__ prefix,
           uint64_t K, const double* __restrict__ u, int64_t nshots,
           const int* __restrict__ mpos, int m, uint64_t* __restrict__ out) {
  const int64_t s = (int64_t)blockIdx.x * (kRedThreads / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= nshots) return;
  const double total = prefix[K - 1];
  const double t = u[s] * total;
  uint64_t lo = 0, hi = K - 1;  // first chunk whose prefix exceeds t
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (prefix[mid] > t) hi = mid; else lo = mid + 1;
  }
  double acc = lo ? prefix[lo - 1] : 0.0;
  const uint64_t base = lo << cbits;
  const int len = 1 << cbits;
  uint64_t x = base;
  int last_nonzero = -1;
  bool found = false;
  for (int i0 = 0; i0 < len && !found; i0 += 32) {
    const int i = i0 + lane;
    const double p = i < len ? prob(psi[base + i]) : 0.0;
    double incl = p;  // warp inclusive scan
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const unsigned nz = __ballot_sync(0xffffffffu, p > 0.0);
    if (nz) last_nonzero = i0 + 31 - __clz(nz);
    const unsigned over = __ballot_sync(0xffffffffu, acc + incl > t);
    if (over) {
      x = base + i0 + (__ffs(over) - 1);
      found = true;
    }
    acc += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (!found) x = base + (last_nonzero >= 0 ? last_nonzero : 0);  // t at the top after rounding
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
  int slices = (int)std::max<uint64_t>(1, std::min<uint64_t>(2432 / bins, per_bin / 256));
  if (slices < 1) slices = 1;
  const size_t nparts = bins * slices;
  // partials, then the bins, then the measured positions
  sv_status st = ensure_partials(s, nparts + bins + 64);
  if (st) return st;
  double* parts = s->partials;
  double* dbins = s->partials + nparts;
  int* dpos = reinterpret_cast<int*>(s->partials + nparts + bins);
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
  st = check_launch("probabilities kernel");
  if (st) return st;
  st = launch_finish(parts, slices, (int)bins, dbins, s->stream, false);
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
  // prefix[K], uniforms[n_shots], outcomes[n_shots], positions
  const size_t need = K + 2 * (size_t)n_shots + 64;
  sv_status st = ensure_partials(s, need);
  if (st) return st;
  double* prefix = s->partials;
  double* du = prefix + K;
  uint64_t* dout = reinterpret_cast<uint64_t*>(du + n_shots);
  int* dpos = reinterpret_cast<int*>(dout + n_shots);
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
    kscan<<<1, 1024, 0, s->stream>>>(prefix, K);
    g_launches.fetch_add(1, std::memory_order_relaxed);
  }
  {
    ProfScope prof(s->stream, "kshots");
    const unsigned g = (unsigned)((n_shots + kRedThreads / 32 - 1) / (kRedThreads / 32));
    if (s->dt == SV_C64)
      kshots<float2><<<g, kRedThreads, 0, s->stream>>>((const float2*)s->data, n, cbits, prefix, K,
                                                       du, n_shots, dpos, m, dout);
    else
      kshots<double2><<<g, kRedThreads, 0, s->stream>>>((const double2*)s->data, n, cbits, prefix,
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
