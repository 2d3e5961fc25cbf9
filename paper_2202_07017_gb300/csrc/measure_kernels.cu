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
  for (uint64_t e = e0 + threadIdx.x; e < e1; e += kRedThreads)
    acc += prob(psi[insert_zeros(e, rest) | rbits]);
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// sums[k] = sum of |psi|^2 over chunk k
template <typename T2>
__global__ void __launch_bounds__(kRedThreads)
    kchunk_sums(const T2* __restrict__ psi, int cbits, double* __restrict__ sums) {
  const uint64_t base = (uint64_t)blockIdx.x << cbits;
  double acc = 0.0;
  for (int i = threadIdx.x; i < (1 << cbits); i += kRedThreads) acc += prob(psi[base + i]);
  acc = block_sum(acc);
  if (threadIdx.x == 0) sums[blockIdx.x] = acc;
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

template <typename T2>
__global__ void __launch_bounds__(kRedThreads)
    kshots(const T2* __restrict__ psi, int n, int cbits, const double* __restrict__ prefix,
           uint64_t K, const double* __restrict__ u, int64_t nshots,
           const int* __restrict__ mpos, int m, uint64_t* __restrict__ out) {
  const int64_t s = (int64_t)blockIdx.x * kRedThreads + threadIdx.x;
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
  uint64_t x = base, last_nonzero = base;
  bool found = false;
  for (uint64_t i = 0; i < (uint64_t(1) << cbits); ++i) {
    const double p = prob(psi[base + i]);
    if (p > 0.0) last_nonzero = base + i;
    acc += p;
    if (acc > t) {
      x = base + i;
      found = true;
      break;
    }
  }
  if (!found) x = last_nonzero;  // t at the very top after rounding
  uint64_t r = 0;
  for (int j = 0; j < m; ++j) r = (r << 1) | ((x >> mpos[j]) & 1);
  out[s] = r;
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
  const int cbits = std::min(n, kChunkBits);
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
    if (s->dt == SV_C64)
      kchunk_sums<float2><<<(unsigned)K, kRedThreads, 0, s->stream>>>((const float2*)s->data,
                                                                        cbits, prefix);
    else
      kchunk_sums<double2><<<(unsigned)K, kRedThreads, 0, s->stream>>>((const double2*)s->data,
                                                                         cbits, prefix);
    g_launches.fetch_add(1, std::memory_order_relaxed);
  }
  {
    ProfScope prof(s->stream, "kscan");
    kscan<<<1, 1024, 0, s->stream>>>(prefix, K);
    g_launches.fetch_add(1, std::memory_order_relaxed);
  }
  {
    ProfScope prof(s->stream, "kshots");
    const unsigned g = (unsigned)((n_shots + kRedThreads - 1) / kRedThreads);
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
