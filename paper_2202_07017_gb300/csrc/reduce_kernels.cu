// Reductions over the state: <psi|psi>, <psi|H|psi> for a Pauli sum H
// (Sec. 3: Hamiltonians and VQE energies), and H psi.
//
// Precision: products in the state's precision, accumulation in fp64.  A
// thread sums its indices in fp64, a block reduces with warp shuffles and
// shared memory, and a second kernel sums the per-block partials in a fixed
// order, so a result is bit-identical from call to call (no atomics).
//
// A Pauli string P with masks (xm, zm) maps |b> to
// i^{#Y} (-1)^{popcount(b & zm)} |b ^ xm>, so
// (P psi)_x = i^{#Y} (-1)^{popcount((x ^ xm) & zm)} psi_{x ^ xm}.
// The host folds coeff * i^{#Y} into one complex coefficient per term.
#include <mutex>
#include <vector>

#include "sv_device.cuh"

namespace sv {

int red_blocks(uint64_t units) {
  const uint64_t b = (units + kRedThreads - 1) / kRedThreads;
  return (int)(b < (uint64_t)kRedMaxBlocks ? (b ? b : 1) : kRedMaxBlocks);
}

namespace {

// Per-thread sums.  complex64: a compensated (Kahan) fp32 sum (GB300 issues
// fp64 at a small fraction of the fp32 rate, so a conversion and an fp64 add
// per amplitude would bound the pass); the block then meets in fp64.
// complex128: plain fp64.
template <typename R>
struct ThreadSum {
  R s = 0, c = 0;
  __device__ __forceinline__ void add(R x) {
    if constexpr (sizeof(R) == 4) {
      const R y = x - c;
      const R t = s + y;
      c = (t - s) - y;
      s = t;
    } else {
      s += x;
    }
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

__global__ void __launch_bounds__(kRedThreads)
    knorm_c64(const float4* __restrict__ psi, uint64_t nvec, double* __restrict__ partials) {
  ThreadSum<float> acc;
#pragma unroll 4
  for (uint64_t v = (uint64_t)blockIdx.x * kRedThreads + threadIdx.x; v < nvec;
       v += (uint64_t)gridDim.x * kRedThreads) {
    const float4 a = psi[v];
    acc.add(a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w);
  }
  const double t = block_sum(acc.value());
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kRedThreads)
    knorm_c128(const double2* __restrict__ psi, uint64_t nvec, double* __restrict__ partials) {
  double acc = 0.0;
  for (uint64_t v = (uint64_t)blockIdx.x * kRedThreads + threadIdx.x; v < nvec;
       v += (uint64_t)gridDim.x * kRedThreads) {
    const double2 a = psi[v];
    acc += a.x * a.x + a.y * a.y;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// coefficient k of the chunk in the kernel's precision
template <typename R>
__device__ __forceinline__ R coef_re(const PauliDev& P, int k) {
  if constexpr (sizeof(R) == 4) return P.cre32[k]; else return P.cre[k];
}
template <typename R>
__device__ __forceinline__ R coef_im(const PauliDev& P, int k) {
  if constexpr (sizeof(R) == 4) return P.cim32[k]; else return P.cim[k];
}

// sum_x Re( c'_k s_k(x) conj(psi_x) psi_{x ^ xm_k} ) over this chunk's terms.
// The chunk's first P.nd terms are diagonal (xm = 0, real coefficients):
// their signed coefficients add up per index before one product with |psi_x|^2.
template <typename R, typename T2>
__global__ void __launch_bounds__(kRedThreads)
    kexpval(const T2* __restrict__ psi, uint64_t dim, const __grid_constant__ PauliDev P,
            double* __restrict__ partials) {
  ThreadSum<R> acc;
  for (uint64_t x = (uint64_t)blockIdx.x * kRedThreads + threadIdx.x; x < dim;
       x += (uint64_t)gridDim.x * kRedThreads) {
    const T2 a = psi[x];
    R d = 0;
    for (int k = 0; k < P.nd; ++k) {
      const R c = coef_re<R>(P, k);
      d += (__popcll(x & P.zm[k]) & 1) ? -c : c;
    }
    R sum = d * (a.x * a.x + a.y * a.y);
    for (int k = P.nd; k < P.nt; ++k) {
      const uint64_t xm = P.xm[k];
      const T2 b = psi[x ^ xm];
      const R zr = a.x * b.x + a.y * b.y;  // Re conj(a) b
      const R zi = a.x * b.y - a.y * b.x;  // Im conj(a) b
      const R t = coef_re<R>(P, k) * zr - coef_im<R>(P, k) * zi;
      sum += (__popcll((x ^ xm) & P.zm[k]) & 1) ? -t : t;
    }
    acc.add(sum);
  }
  const double t = block_sum(acc.value());
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// out_x (+)= sum_k c'_k s_k(x) psi_{x ^ xm_k}; optional partials of
// Re conj(psi_x) out_x (the energy, when this chunk completes out).
template <typename R, typename T2>
__global__ void __launch_bounds__(kRedThreads)
    kapply_pauli(T2* __restrict__ out, const T2* __restrict__ psi, uint64_t dim,
                 const __grid_constant__ PauliDev P, int accumulate,
                 double* __restrict__ partials) {
  ThreadSum<R> acc;
  for (uint64_t x = (uint64_t)blockIdx.x * kRedThreads + threadIdx.x; x < dim;
       x += (uint64_t)gridDim.x * kRedThreads) {
    R orr = 0, oi = 0;
    if (accumulate) {
      const T2 o = out[x];
      orr = o.x;
      oi = o.y;
    }
    const T2 a = psi[x];
    R d = 0;
    for (int k = 0; k < P.nd; ++k) {
      const R c = coef_re<R>(P, k);
      d += (__popcll(x & P.zm[k]) & 1) ? -c : c;
    }
    orr += d * a.x;
    oi += d * a.y;
    for (int k = P.nd; k < P.nt; ++k) {
      const uint64_t xm = P.xm[k];
      const T2 b = psi[x ^ xm];
      const R cr = coef_re<R>(P, k), ci = coef_im<R>(P, k);
      const R sr = cr * b.x - ci * b.y;
      const R si = cr * b.y + ci * b.x;
      if (__popcll((x ^ xm) & P.zm[k]) & 1) {
        orr -= sr;
        oi -= si;
      } else {
        orr += sr;
        oi += si;
      }
    }
    T2 o;
    o.x = orr;
    o.y = oi;
    out[x] = o;
    if (partials) acc.add(a.x * orr + a.y * oi);
  }
  if (partials) {
    const double t = block_sum(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kRedThreads)
    kfinish(const double* __restrict__ src, int count, double* __restrict__ dst, int add) {
  const double* s = src + (size_t)blockIdx.x * count;
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += kRedThreads) acc += s[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) dst[blockIdx.x] = add ? dst[blockIdx.x] + acc : acc;
}

}  // namespace

void pauli_chunks(const sv_pauli_sum* H, std::vector<PauliDev>* out) {
  out->clear();
  // diagonal terms (no X or Y factor) first, so that every chunk starts with
  // its diagonal terms; the sum does not depend on the order
  std::vector<int> order;
  for (int pass = 0; pass < 2; ++pass)
    for (int t = 0; t < H->n_terms; ++t)
      if ((H->xmask[t] == 0) == (pass == 0)) order.push_back(t);
  for (int k0 = 0; k0 < H->n_terms; k0 += 64) {
    PauliDev P{};
    P.nt = H->n_terms - k0 < 64 ? H->n_terms - k0 : 64;
    P.nd = 0;
    for (int j = 0; j < P.nt; ++j) {
      const int t = order[k0 + j];
      const uint64_t xm = H->xmask[t], zm = H->zmask[t];
      const int ny = __builtin_popcountll(xm & zm) & 3;
      const double c = H->coeff[t];
      P.xm[j] = xm;
      P.zm[j] = zm;
      // c * i^{ny}
      P.cre[j] = ny == 0 ? c : ny == 2 ? -c : 0.0;
      P.cim[j] = ny == 1 ? c : ny == 3 ? -c : 0.0;
      P.cre32[j] = (float)P.cre[j];
      P.cim32[j] = (float)P.cim[j];
      if (xm == 0 && P.nd == j) ++P.nd;
    }
    out->push_back(P);
  }
}

sv_status launch_norm_partials(sv_state s, double* partials, int* nparts) {
  ProfScope prof(s->stream, "knorm");
  if (s->dt == SV_C64) {
    const uint64_t nvec = s->n >= 1 ? (uint64_t(1) << (s->n - 1)) : 1;
    const int g = red_blocks(nvec);
    knorm_c64<<<g, kRedThreads, 0, s->stream>>>((const float4*)s->data, nvec, partials);
    *nparts = g;
  } else {
    const uint64_t nvec = uint64_t(1) << s->n;
    const int g = red_blocks(nvec);
    knorm_c128<<<g, kRedThreads, 0, s->stream>>>((const double2*)s->data, nvec, partials);
    *nparts = g;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return check_launch("norm kernel");
}

sv_status launch_expval_partials(sv_state s, const PauliDev& P, double* partials, int* nparts) {
  const uint64_t dim = uint64_t(1) << s->n;
  const int g = red_blocks(dim);
  ProfScope prof(s->stream, "kexpval");
  if (s->dt == SV_C64)
    kexpval<float, float2><<<g, kRedThreads, 0, s->stream>>>((const float2*)s->data, dim, P,
                                                             partials);
  else
    kexpval<double, double2><<<g, kRedThreads, 0, s->stream>>>((const double2*)s->data, dim, P,
                                                               partials);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  *nparts = g;
  return check_launch("expval kernel");
}

sv_status launch_apply_pauli(void* out, const void* in, sv_dtype dt, int n, cudaStream_t st,
                             const PauliDev& P, bool accumulate, double* partials,
                             int* nparts) {
  const uint64_t dim = uint64_t(1) << n;
  const int g = red_blocks(dim);
  ProfScope prof(st, "kapply_pauli");
  if (dt == SV_C64)
    kapply_pauli<float, float2><<<g, kRedThreads, 0, st>>>((float2*)out, (const float2*)in, dim,
                                                           P, accumulate ? 1 : 0, partials);
  else
    kapply_pauli<double, double2><<<g, kRedThreads, 0, st>>>(
        (double2*)out, (const double2*)in, dim, P, accumulate ? 1 : 0, partials);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (nparts) *nparts = g;
  return check_launch("apply_pauli kernel");
}

sv_status launch_finish(const double* src, int count, int slots, double* dst, cudaStream_t st,
                        bool add_to_dst) {
  if (slots <= 0) return SV_OK;
  ProfScope prof(st, "kfinish");
  kfinish<<<slots, kRedThreads, 0, st>>>(src, count, dst, add_to_dst ? 1 : 0);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return check_launch("finish kernel");
}

// ---- expectation value without any allocation ------------------------------------
// Some callers cannot allocate device memory when they need an energy: a
// serving process that hands the whole device to a caching allocator or a
// fixed arena up front (a cudaMalloc behind its back can fail or fragment),
// or code running where a failed allocation cannot be handled.
// sv_expval_noalloc serves them: the block partials of the reduction live in
// this fixed array, which every GPU that loads the library holds until the
// process exits.  It holds kNoAllocPartials doubles (152 KiB): red_blocks(2^n)
// <= 1216 partials per chunk of 64 terms, up to SV_NOALLOC_MAX_TERMS / 64 = 16
// chunks.  Every block writes its own slot before the finishing kernel reads
// it, so nothing has to start at zero; calls share the array, so calls that
// overlap on the GPU (different streams, or devices sharing a context) race.
constexpr int kNoAllocChunks = (SV_NOALLOC_MAX_TERMS + 63) / 64;
constexpr int kNoAllocPartials = kRedMaxBlocks * kNoAllocChunks;
static_assert(kNoAllocPartials >= kRedMaxBlocks * ((SV_NOALLOC_MAX_TERMS + 63) / 64),
              "scratch below one partial per block and chunk");
static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {};  // device address of the array, per device ordinal
}  // namespace

}  // namespace sv

extern "C" sv_status sv_expval_noalloc(const void* dev_state, int n_qubits, sv_dtype dtype,
                                       const sv_pauli_sum* H, double* dev_out,
                                       void* cuda_stream) {
  using namespace sv;
  if (!dev_state || !dev_out || n_qubits < 1 || n_qubits > SV_MAX_QUBITS ||
      (dtype != SV_C64 && dtype != SV_C128) || ((uintptr_t)dev_state & 15) || !H) {
    set_error("sv_expval_noalloc: bad state, output, qubit count or dtype");
    return SV_ERR_INVALID;
  }
  if (H->n_terms < 0 || H->n_terms > SV_NOALLOC_MAX_TERMS) {
    set_error("sv_expval_noalloc: %d terms, at most %d fit the fixed scratch array",
              H->n_terms, SV_NOALLOC_MAX_TERMS);
    return SV_ERR_INVALID;
  }
  if (H->n_terms > 0 && (!H->xmask || !H->zmask || !H->coeff)) {
    set_error("sv_expval_noalloc: null Pauli sum arrays");
    return SV_ERR_INVALID;
  }
  const uint64_t lim = (uint64_t(1) << n_qubits) - 1;
  for (int k = 0; k < H->n_terms; ++k)
    if ((H->xmask[k] | H->zmask[k]) & ~lim) {
      set_error("sv_expval_noalloc: term %d has mask bits beyond %d qubits", k, n_qubits);
      return SV_ERR_INVALID;
    }
  int dev = 0;
  SV_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) {
    set_error("sv_expval_noalloc: device ordinal %d out of range", dev);
    return SV_ERR_INVALID;
  }
  if (cuda_stream) {
    // the array's address is per device: the stream must run on the current one
    int sdev = -1;
    SV_CUDA_TRY(cudaStreamGetDevice((cudaStream_t)cuda_stream, &sdev));
    if (sdev != dev) {
      set_error("sv_expval_noalloc: the stream belongs to device %d, the current device is %d",
                sdev, dev);
      return SV_ERR_INVALID;
    }
  }
  double* scratch = nullptr;
  {
    // first call on a device: look up the array's device address (the host
    // symbol is only a stand-in and must never be passed to a kernel)
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
      if (e != cudaSuccess || !p) {
        set_error("sv_expval_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return SV_ERR_CUDA;
      }
      g_noalloc_ptr[dev] = (double*)p;
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (H->n_terms == 0) {
    SV_CUDA_TRY(cudaMemsetAsync(dev_out, 0, sizeof(double), st));
    return SV_OK;
  }
  const uint64_t dim = uint64_t(1) << n_qubits;
  const int g = red_blocks(dim);
  int total = 0;
  // the same term chunks as sv_expval (a host vector: no device memory)
  std::vector<PauliDev> chunks;
  pauli_chunks(H, &chunks);
  for (const PauliDev& P : chunks) {
    if (dtype == SV_C64)
      kexpval<float, float2><<<g, kRedThreads, 0, st>>>((const float2*)dev_state, dim, P,
                                                        scratch + total);
    else
      kexpval<double, double2><<<g, kRedThreads, 0, st>>>((const double2*)dev_state, dim, P,
                                                          scratch + total);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    total += g;
  }
  kfinish<<<1, kRedThreads, 0, st>>>(scratch, total, dev_out, 0);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return check_launch("sv_expval_noalloc kernels");
}
