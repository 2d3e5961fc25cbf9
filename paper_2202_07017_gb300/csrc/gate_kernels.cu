// Gate-application kernels: Eq. (1) of Sec. 2 applied in place.
//
// Index generation follows the paper's description of its JIT kernels
// (Sec. 2: indices generated on the fly with binary operations, modified for
// multi-target and controlled gates): a work unit u is turned into an
// amplitude (or 16-byte vector) index by inserting zero bits at the sorted
// target/control positions and OR-ing in the control ones.
//
// Data movement is designed for HBM3e: every access is a 16-byte vector
// (two complex64 or one complex128 amplitude); a 1-qubit gate on bit p >= 1
// (complex64) reads two coalesced streams 2^p amplitudes apart, a gate on
// bit 0 finds its pair inside one vector; diagonal gates whose matrix is
// diag(1, .., 1, phase) touch only the all-ones subspace.  The matrix
// structure picks the arithmetic variant (dense, diagonal, real, real
// diagonal with imaginary off-diagonal), which matters for complex128:
// GB300's fp64 rate is low enough that a dense complex 2x2 product per pair
// costs more than the HBM traffic.
#include <algorithm>
#include <cstdlib>
#include <type_traits>
#include <vector>

#include "sv_device.cuh"

namespace sv {
namespace {

constexpr int kThreads = 256;

// ---- phase multiply variants ---------------------------------------------------
enum { PK_GEN = 0, PK_NEG = 1, PK_I = 2, PK_MI = 3 };

template <int PK, typename R>
__device__ __forceinline__ void rot(R c, R s, R& re, R& im) {
  if (PK == PK_GEN) {
    R nr = c * re - s * im;
    R ni = s * re + c * im;
    re = nr;
    im = ni;
  } else if (PK == PK_NEG) {
    re = -re;
    im = -im;
  } else if (PK == PK_I) {
    R t = re;
    re = -im;
    im = t;
  } else {
    R t = re;
    re = im;
    im = -t;
  }
}

// ---- complex64 1-qubit, target bit >= 1: two coalesced streams --------------------
// DITHER: the outputs' final roundings are dithered (mv2_dither), keyed by
// the vector index and the launch's seed.
template <typename I>
__device__ __forceinline__ uint32_t unit_key(I v, uint32_t seed) {
  return mix32((uint32_t)v * 0x9E3779B1u ^ (uint32_t)((uint64_t)v >> 32) ^ seed);
}

template <typename I, int MK, int ITEMS, bool DITHER>
__global__ void __launch_bounds__(kThreads)
    k1q_c64_pair(float4* __restrict__ psi, I n_units, Ins<I> ins, I tmask, I cmask,
                 int amp1_only, M2<float> g, uint32_t seed) {
  const I base = (I)blockIdx.x * (I)(kThreads * ITEMS) + (I)threadIdx.x;
  I lo[ITEMS];
  float4 a[ITEMS], b[ITEMS];
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I u = base + (I)(it * kThreads);
    if (u < n_units) {
      lo[it] = insert_zeros(u, ins) | cmask;
      a[it] = psi[lo[it]];
      b[it] = psi[lo[it] | tmask];
    }
  }
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I u = base + (I)(it * kThreads);
    if (u < n_units) {
      float4 x = a[it], y = b[it];
      if constexpr (DITHER) {
        const uint32_t h = unit_key(lo[it], seed);
        if (!amp1_only) mv2_dither<MK>(g, x.x, x.y, y.x, y.y, h);
        mv2_dither<MK>(g, x.z, x.w, y.z, y.w, mix32(h));
      } else {
        if (!amp1_only) mv2<MK>(g, x.x, x.y, y.x, y.y);
        mv2<MK>(g, x.z, x.w, y.z, y.w);
      }
      psi[lo[it]] = x;
      psi[lo[it] | tmask] = y;
    }
  }
}

// ---- complex64 1-qubit, target bit 0: the pair shares one 16-byte vector ----------
template <typename I, int MK, int ITEMS, bool DITHER>
__global__ void __launch_bounds__(kThreads)
    k1q_c64_in(float4* __restrict__ psi, I n_units, Ins<I> ins, I cmask, M2<float> g,
               uint32_t seed) {
  const I base = (I)blockIdx.x * (I)(kThreads * ITEMS) + (I)threadIdx.x;
  I v[ITEMS];
  float4 a[ITEMS];
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I u = base + (I)(it * kThreads);
    if (u < n_units) {
      v[it] = insert_zeros(u, ins) | cmask;
      a[it] = psi[v[it]];
    }
  }
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I u = base + (I)(it * kThreads);
    if (u < n_units) {
      float4 x = a[it];
      if constexpr (DITHER)
        mv2_dither<MK>(g, x.x, x.y, x.z, x.w, unit_key(v[it], seed));
      else
        mv2<MK>(g, x.x, x.y, x.z, x.w);
      psi[v[it]] = x;
    }
  }
}

// ---- complex128 1-qubit: one amplitude per vector ---------------------------------
template <typename I, int MK, int ITEMS>
__global__ void __launch_bounds__(kThreads)
    k1q_c128_pair(double2* __restrict__ psi, I n_units, Ins<I> ins, I tmask, I cmask,
                  M2<double> g) {
  const I base = (I)blockIdx.x * (I)(kThreads * ITEMS) + (I)threadIdx.x;
  I lo[ITEMS];
  double2 a[ITEMS], b[ITEMS];
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I u = base + (I)(it * kThreads);
    if (u < n_units) {
      lo[it] = insert_zeros(u, ins) | cmask;
      a[it] = psi[lo[it]];
      b[it] = psi[lo[it] | tmask];
    }
  }
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I u = base + (I)(it * kThreads);
    if (u < n_units) {
      double2 x = a[it], y = b[it];
      mv2<MK>(g, x.x, x.y, y.x, y.y);
      psi[lo[it]] = x;
      psi[lo[it] | tmask] = y;
    }
  }
}

// ---- phase on the all-ones subspace of a bit mask (U1, Z, CZ, CU1, ...) ----------
template <typename I, int PK, int ITEMS>
__global__ void __launch_bounds__(kThreads)
    kphase_c64(float4* __restrict__ psi, I n_units, Ins<I> ins, I omask, int amp1_only,
               float c, float s) {
  const I base = (I)blockIdx.x * (I)(kThreads * ITEMS) + (I)threadIdx.x;
  I v[ITEMS];
  float4 a[ITEMS];
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I u = base + (I)(it * kThreads);
    if (u < n_units) {
      v[it] = insert_zeros(u, ins) | omask;
      a[it] = psi[v[it]];
    }
  }
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I u = base + (I)(it * kThreads);
    if (u < n_units) {
      float4 x = a[it];
      if (!amp1_only) rot<PK>(c, s, x.x, x.y);
      rot<PK>(c, s, x.z, x.w);
      psi[v[it]] = x;
    }
  }
}

template <typename I, int PK, int ITEMS>
__global__ void __launch_bounds__(kThreads)
    kphase_c128(double2* __restrict__ psi, I n_units, Ins<I> ins, I omask, double c,
                double s) {
  const I base = (I)blockIdx.x * (I)(kThreads * ITEMS) + (I)threadIdx.x;
  I v[ITEMS];
  double2 a[ITEMS];
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I u = base + (I)(it * kThreads);
    if (u < n_units) {
      v[it] = insert_zeros(u, ins) | omask;
      a[it] = psi[v[it]];
    }
  }
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I u = base + (I)(it * kThreads);
    if (u < n_units) {
      double2 x = a[it];
      rot<PK>(c, s, x.x, x.y);
      psi[v[it]] = x;
    }
  }
}

// ---- SWAP: exchange the (a=1,b=0) and (a=0,b=1) amplitudes ---------------------------
// complex64 with both bits >= 1: swap whole vectors (or only their odd
// amplitudes when a control sits on bit 0).
template <typename I, int ITEMS>
__global__ void __launch_bounds__(kThreads)
    kswap_c64_vv(float4* __restrict__ psi, I n_units, Ins<I> ins, I amask, I bmask, I cmask,
                 int amp1_only) {
  const I base = (I)blockIdx.x * (I)(kThreads * ITEMS) + (I)threadIdx.x;
  I p[ITEMS];
  float4 x[ITEMS], y[ITEMS];
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I u = base + (I)(it * kThreads);
    if (u < n_units) {
      p[it] = insert_zeros(u, ins) | cmask;
      x[it] = psi[p[it] | bmask];
      y[it] = psi[p[it] | amask];
    }
  }
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I u = base + (I)(it * kThreads);
    if (u < n_units) {
      float4 nx = y[it], ny = x[it];
      if (amp1_only) {
        nx.x = x[it].x; nx.y = x[it].y;
        ny.x = y[it].x; ny.y = y[it].y;
      }
      psi[p[it] | bmask] = nx;
      psi[p[it] | amask] = ny;
    }
  }
}

// complex64 with b = bit 0: vector v (a=0) holds (a0b0, a0b1), vector w (a=1)
// holds (a1b0, a1b1); exchange v's odd amplitude with w's even one.
template <typename I, int ITEMS>
__global__ void __launch_bounds__(kThreads)
    kswap_c64_v0(float4* __restrict__ psi, I n_units, Ins<I> ins, I amask, I cmask) {
  const I base = (I)blockIdx.x * (I)(kThreads * ITEMS) + (I)threadIdx.x;
  I p[ITEMS];
  float4 x[ITEMS], y[ITEMS];
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I u = base + (I)(it * kThreads);
    if (u < n_units) {
      p[it] = insert_zeros(u, ins) | cmask;
      x[it] = psi[p[it]];
      y[it] = psi[p[it] | amask];
    }
  }
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I u = base + (I)(it * kThreads);
    if (u < n_units) {
      float4 v = x[it], w = y[it];
      const float tz = v.z, tw = v.w;
      v.z = w.x;
      v.w = w.y;
      w.x = tz;
      w.y = tw;
      psi[p[it]] = v;
      psi[p[it] | amask] = w;
    }
  }
}

template <typename I, int ITEMS>
__global__ void __launch_bounds__(kThreads)
    kswap_c128(double2* __restrict__ psi, I n_units, Ins<I> ins, I amask, I bmask, I cmask) {
  const I base = (I)blockIdx.x * (I)(kThreads * ITEMS) + (I)threadIdx.x;
  I p[ITEMS];
  double2 x[ITEMS], y[ITEMS];
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I u = base + (I)(it * kThreads);
    if (u < n_units) {
      p[it] = insert_zeros(u, ins) | cmask;
      x[it] = psi[p[it] | bmask];
      y[it] = psi[p[it] | amask];
    }
  }
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I u = base + (I)(it * kThreads);
    if (u < n_units) {
      psi[p[it] | bmask] = y[it];
      psi[p[it] | amask] = x[it];
    }
  }
}

// ---- generic k-qubit dense gate (k <= 5), one index group per thread ---------------
template <int K, typename R, typename I>
struct GenParams {
  I off[1 << K];
  R gr[(1 << K) * (1 << K)];
  R gi[(1 << K) * (1 << K)];
};

template <int K, typename R, typename T2, typename I>
__global__ void __launch_bounds__(kThreads)
    kgen(T2* __restrict__ psi, I n_units, Ins<I> ins, I cmask, const __grid_constant__ GenParams<K, R, I> p) {
  constexpr int D = 1 << K;
  const I u = (I)blockIdx.x * (I)kThreads + (I)threadIdx.x;
  if (u >= n_units) return;
  const I b = insert_zeros(u, ins) | cmask;
  R ar[D], ai[D];
#pragma unroll
  for (int t = 0; t < D; ++t) {
    const T2 v = psi[b | p.off[t]];
    ar[t] = v.x;
    ai[t] = v.y;
  }
#pragma unroll
  for (int r = 0; r < D; ++r) {
    R sr = 0, si = 0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const R gr = p.gr[r * D + c], gi = p.gi[r * D + c];
      sr += gr * ar[c] - gi * ai[c];
      si += gr * ai[c] + gi * ar[c];
    }
    T2 o;
    o.x = sr;
    o.y = si;
    psi[b | p.off[r]] = o;
  }
}

template <typename I, int ITEMS>
__global__ void kinit_c64(float4* __restrict__ psi, I n_vec, I bvec, int slot) {
  const I base = (I)blockIdx.x * (I)(kThreads * ITEMS) + (I)threadIdx.x;
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I v = base + (I)(it * kThreads);
    if (v < n_vec) {
      float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      if (v == bvec) {
        if (slot) z.z = 1.f; else z.x = 1.f;
      }
      psi[v] = z;
    }
  }
}

template <typename I, int ITEMS>
__global__ void kinit_c128(double2* __restrict__ psi, I n_vec, I bvec) {
  const I base = (I)blockIdx.x * (I)(kThreads * ITEMS) + (I)threadIdx.x;
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const I v = base + (I)(it * kThreads);
    if (v < n_vec) psi[v] = make_double2(v == bvec ? 1.0 : 0.0, 0.0);
  }
}

// ---- host side -------------------------------------------------------------------
// Amplitude vectors per thread: kernels that read two streams (pairs, SWAP)
// keep 2 x ITEMS vectors in flight, single-stream kernels (bit-0 pairs,
// phases, init) ITEMS vectors.  Measured on GB300 at n = 30 (complex64):
// ITEMS = 8 for both families brings the 1-qubit kernel from 5.9 to
// 6.8 TB/s (the copy bandwidth) and the controlled-U1 kernel from 3.6 to
// 6.6 TB/s; fewer vectors in flight leave HBM latency exposed.
// SV_ITEMS_PAIR / SV_ITEMS_SINGLE (1, 2, 4, 8) override the defaults.
int env_items(const char* name, int dflt) {
  const char* e = getenv(name);
  const int x = e ? atoi(e) : dflt;
  return (x == 1 || x == 2 || x == 4 || x == 8) ? x : dflt;
}
int items_pair() {
  static const int v = env_items("SV_ITEMS_PAIR", 8);
  return v;
}
int items_single() {
  static const int v = env_items("SV_ITEMS_SINGLE", 8);
  return v;
}

template <typename F>
void with_items(int items, F&& f) {
  switch (items) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 8: f(std::integral_constant<int, 8>{}); break;
    default: f(std::integral_constant<int, 4>{}); break;
  }
}

template <typename I>
unsigned grid_for(I n_units, int items) {
  const uint64_t per = (uint64_t)kThreads * items;
  return (unsigned)(((uint64_t)n_units + per - 1) / per);
}

bool is_zero(cd z) { return z.re == 0.0 && z.im == 0.0; }
bool is_one(cd z) { return z.re == 1.0 && z.im == 0.0; }

int classify2(const HostMatrix& G) {
  cd g00 = G.at(0, 0), g01 = G.at(0, 1), g10 = G.at(1, 0), g11 = G.at(1, 1);
  if (is_zero(g01) && is_zero(g10)) return MK_DIAG;
  if (g00.im == 0 && g01.im == 0 && g10.im == 0 && g11.im == 0) return MK_REAL;
  if (g00.im == 0 && g11.im == 0 && g01.re == 0 && g10.re == 0) return MK_IMOFF;
  return MK_DENSE;
}

int phase_kind(cd ph) {
  if (ph.re == -1.0 && ph.im == 0.0) return PK_NEG;
  if (ph.re == 0.0 && ph.im == 1.0) return PK_I;
  if (ph.re == 0.0 && ph.im == -1.0) return PK_MI;
  return PK_GEN;
}

template <typename... KArgs, typename... Args>
void launch_k(void (*kern)(KArgs...), const char* name, unsigned grid, cudaStream_t st,
              Args... args) {
  if (grid == 0) return;
  ProfScope prof(st, name);
  kern<<<grid, kThreads, 0, st>>>(args...);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

// Splits control bit positions for complex64 vectors: bit 0 selects the odd
// amplitude of each vector (amp1_only), bits >= 1 become vector-index bits.
template <typename I>
void split_c64(const int* bits, int nb, std::vector<int>* vpos, I* vmask, int* amp1_only) {
  for (int j = 0; j < nb; ++j) {
    if (bits[j] == 0) {
      *amp1_only = 1;
    } else {
      vpos->push_back(bits[j] - 1);
      *vmask |= I(1) << (bits[j] - 1);
    }
  }
}

template <typename I, int MK>
void run_1q_c64(float4* psi, int n, cudaStream_t st, int t, int nc, const int* cp,
                const M2<float>& g, uint32_t seed) {
  std::vector<int> vpos;
  I cmask = 0;
  int amp1_only = 0;
  split_c64<I>(cp, nc, &vpos, &cmask, &amp1_only);
  if (t == 0) {
    Ins<I> ins = make_ins<I>(vpos);
    const I nu = I(1) << (n - 1 - (int)vpos.size());
    with_items(items_single(), [&](auto it) {
      constexpr int IT = decltype(it)::value;
      if (seed)
        launch_k(k1q_c64_in<I, MK, IT, true>, "k1q_c64_in", grid_for(nu, IT), st, psi, nu, ins,
                 cmask, g, seed);
      else
        launch_k(k1q_c64_in<I, MK, IT, false>, "k1q_c64_in", grid_for(nu, IT), st, psi, nu, ins,
                 cmask, g, seed);
    });
  } else {
    vpos.push_back(t - 1);
    Ins<I> ins = make_ins<I>(vpos);
    const I tmask = I(1) << (t - 1);
    const I nu = I(1) << (n - 1 - (int)vpos.size());
    with_items(items_pair(), [&](auto it) {
      constexpr int IT = decltype(it)::value;
      if (seed)
        launch_k(k1q_c64_pair<I, MK, IT, true>, "k1q_c64_pair", grid_for(nu, IT), st, psi, nu,
                 ins, tmask, cmask, amp1_only, g, seed);
      else
        launch_k(k1q_c64_pair<I, MK, IT, false>, "k1q_c64_pair", grid_for(nu, IT), st, psi, nu,
                 ins, tmask, cmask, amp1_only, g, seed);
    });
  }
}

template <typename I, int MK>
void run_1q_c128(double2* psi, int n, cudaStream_t st, int t, int nc, const int* cp,
                 const M2<double>& g) {
  std::vector<int> pos{t};
  I cmask = 0;
  for (int j = 0; j < nc; ++j) {
    pos.push_back(cp[j]);
    cmask |= I(1) << cp[j];
  }
  Ins<I> ins = make_ins<I>(pos);
  const I tmask = I(1) << t;
  const I nu = I(1) << (n - (int)pos.size());
  with_items(items_pair(), [&](auto it) {
    constexpr int IT = decltype(it)::value;
    launch_k(k1q_c128_pair<I, MK, IT>, "k1q_c128_pair", grid_for(nu, IT), st, psi, nu, ins,
             tmask, cmask, g);
  });
}

template <typename I>
void run_1q(void* data, sv_dtype dt, int n, cudaStream_t st, int t, int nc, const int* cp,
            const HostMatrix& G, uint32_t seed) {
  const int mk = classify2(G);
  if (dt == SV_C64) {
    float4* psi = (float4*)data;
    M2<float> g = to_m2<float>(G);
    switch (mk) {
      case MK_DIAG: run_1q_c64<I, MK_DIAG>(psi, n, st, t, nc, cp, g, seed); break;
      case MK_REAL: run_1q_c64<I, MK_REAL>(psi, n, st, t, nc, cp, g, seed); break;
      case MK_IMOFF: run_1q_c64<I, MK_IMOFF>(psi, n, st, t, nc, cp, g, seed); break;
      default: run_1q_c64<I, MK_DENSE>(psi, n, st, t, nc, cp, g, seed); break;
    }
  } else {
    double2* psi = (double2*)data;
    M2<double> g = to_m2<double>(G);
    switch (mk) {
      case MK_DIAG: run_1q_c128<I, MK_DIAG>(psi, n, st, t, nc, cp, g); break;
      case MK_REAL: run_1q_c128<I, MK_REAL>(psi, n, st, t, nc, cp, g); break;
      case MK_IMOFF: run_1q_c128<I, MK_IMOFF>(psi, n, st, t, nc, cp, g); break;
      default: run_1q_c128<I, MK_DENSE>(psi, n, st, t, nc, cp, g); break;
    }
  }
}

template <typename I, int PK>
void run_phase_pk(void* data, sv_dtype dt, int n, cudaStream_t st, const std::vector<int>& bits,
                  cd ph) {
  if (dt == SV_C64) {
    float4* psi = (float4*)data;
    std::vector<int> vpos;
    I omask = 0;
    int amp1_only = 0;
    split_c64<I>(bits.data(), (int)bits.size(), &vpos, &omask, &amp1_only);
    Ins<I> ins = make_ins<I>(vpos);
    const I nu = I(1) << (n - 1 - (int)vpos.size());
    const float c = (float)ph.re, s = (float)ph.im;
    with_items(items_single(), [&](auto it) {
      constexpr int IT = decltype(it)::value;
      launch_k(kphase_c64<I, PK, IT>, "kphase_c64", grid_for(nu, IT), st, psi, nu, ins, omask,
               amp1_only, c, s);
    });
  } else {
    double2* psi = (double2*)data;
    I omask = 0;
    for (int b : bits) omask |= I(1) << b;
    Ins<I> ins = make_ins<I>(bits);
    const I nu = I(1) << (n - (int)bits.size());
    with_items(items_single(), [&](auto it) {
      constexpr int IT = decltype(it)::value;
      launch_k(kphase_c128<I, PK, IT>, "kphase_c128", grid_for(nu, IT), st, psi, nu, ins, omask,
               ph.re, ph.im);
    });
  }
}

template <typename I>
void run_phase(void* data, sv_dtype dt, int n, cudaStream_t st, const std::vector<int>& bits,
               cd ph) {
  switch (phase_kind(ph)) {
    case PK_NEG: run_phase_pk<I, PK_NEG>(data, dt, n, st, bits, ph); break;
    case PK_I: run_phase_pk<I, PK_I>(data, dt, n, st, bits, ph); break;
    case PK_MI: run_phase_pk<I, PK_MI>(data, dt, n, st, bits, ph); break;
    default: run_phase_pk<I, PK_GEN>(data, dt, n, st, bits, ph); break;
  }
}

template <typename I>
void run_swap(void* data, sv_dtype dt, int n, cudaStream_t st, int a, int b, int nc,
              const int* cp) {
  if (a < b) std::swap(a, b);  // a > b
  if (dt == SV_C64) {
    float4* psi = (float4*)data;
    std::vector<int> vpos;
    I cmask = 0;
    int amp1_only = 0;
    split_c64<I>(cp, nc, &vpos, &cmask, &amp1_only);
    const I amask = I(1) << (a - 1);
    if (b == 0) {
      vpos.push_back(a - 1);
      Ins<I> ins = make_ins<I>(vpos);
      const I nu = I(1) << (n - 1 - (int)vpos.size());
      with_items(items_pair(), [&](auto it) {
        constexpr int IT = decltype(it)::value;
        launch_k(kswap_c64_v0<I, IT>, "kswap_c64_v0", grid_for(nu, IT), st, psi, nu, ins, amask,
                 cmask);
      });
    } else {
      const I bmask = I(1) << (b - 1);
      vpos.push_back(a - 1);
      vpos.push_back(b - 1);
      Ins<I> ins = make_ins<I>(vpos);
      const I nu = I(1) << (n - 1 - (int)vpos.size());
      with_items(items_pair(), [&](auto it) {
        constexpr int IT = decltype(it)::value;
        launch_k(kswap_c64_vv<I, IT>, "kswap_c64_vv", grid_for(nu, IT), st, psi, nu, ins, amask,
                 bmask, cmask, amp1_only);
      });
    }
  } else {
    double2* psi = (double2*)data;
    std::vector<int> pos{a, b};
    I cmask = 0;
    for (int j = 0; j < nc; ++j) {
      pos.push_back(cp[j]);
      cmask |= I(1) << cp[j];
    }
    Ins<I> ins = make_ins<I>(pos);
    const I amask = I(1) << a, bmask = I(1) << b;
    const I nu = I(1) << (n - (int)pos.size());
    with_items(items_pair(), [&](auto it) {
      constexpr int IT = decltype(it)::value;
      launch_k(kswap_c128<I, IT>, "kswap_c128", grid_for(nu, IT), st, psi, nu, ins, amask, bmask,
               cmask);
    });
  }
}

template <int K, typename R, typename I>
GenParams<K, R, I> gen_params(const int* tp, const HostMatrix& G) {
  constexpr int D = 1 << K;
  GenParams<K, R, I> p;
  for (int t = 0; t < D; ++t) {
    I o = 0;
    for (int j = 0; j < K; ++j)
      if ((t >> (K - 1 - j)) & 1) o |= I(1) << tp[j];
    p.off[t] = o;
  }
  for (int e = 0; e < D * D; ++e) {
    p.gr[e] = (R)G.m[e].re;
    p.gi[e] = (R)G.m[e].im;
  }
  return p;
}

template <int K, typename I>
void run_gen_k(void* data, sv_dtype dt, int n, cudaStream_t st, const int* tp, int nc,
               const int* cp, const HostMatrix& G) {
  std::vector<int> pos(tp, tp + K);
  I cmask = 0;
  for (int j = 0; j < nc; ++j) {
    pos.push_back(cp[j]);
    cmask |= I(1) << cp[j];
  }
  Ins<I> ins = make_ins<I>(pos);
  const I nu = I(1) << (n - (int)pos.size());
  const unsigned grid = grid_for(nu, 1);
  if (dt == SV_C64)
    launch_k(kgen<K, float, float2, I>, "kgen_c64", grid, st, (float2*)data, nu, ins, cmask,
             gen_params<K, float, I>(tp, G));
  else
    launch_k(kgen<K, double, double2, I>, "kgen_c128", grid, st, (double2*)data, nu, ins, cmask,
             gen_params<K, double, I>(tp, G));
}

template <typename I>
void run_gen(void* data, sv_dtype dt, int n, cudaStream_t st, int k, const int* tp, int nc,
             const int* cp, const HostMatrix& G) {
  switch (k) {
    case 1: run_gen_k<1, I>(data, dt, n, st, tp, nc, cp, G); break;
    case 2: run_gen_k<2, I>(data, dt, n, st, tp, nc, cp, G); break;
    case 3: run_gen_k<3, I>(data, dt, n, st, tp, nc, cp, G); break;
    case 4: run_gen_k<4, I>(data, dt, n, st, tp, nc, cp, G); break;
    default: run_gen_k<5, I>(data, dt, n, st, tp, nc, cp, G); break;
  }
}

bool is_swap(const HostMatrix& G) {
  if (G.k != 2) return false;
  static const int perm[4] = {0, 2, 1, 3};
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      cd z = G.at(r, c);
      if (c == perm[r] ? !is_one(z) : !is_zero(z)) return false;
    }
  return true;
}

template <typename I>
void dispatch(void* data, sv_dtype dt, int n, cudaStream_t st, int k, const int* tp, int nc,
              const int* cp, const HostMatrix& G, uint32_t seed) {
  const int d = 1 << k;
  bool diag = true, ones = true;
  for (int r = 0; r < d && diag; ++r)
    for (int c = 0; c < d; ++c)
      if (r != c && !is_zero(G.at(r, c))) {
        diag = false;
        break;
      }
  if (diag) {
    for (int r = 0; r + 1 < d; ++r)
      if (!is_one(G.at(r, r))) ones = false;
    if (ones) {
      const cd ph = G.at(d - 1, d - 1);
      if (is_one(ph)) return;  // identity
      std::vector<int> bits(tp, tp + k);
      bits.insert(bits.end(), cp, cp + nc);
      run_phase<I>(data, dt, n, st, bits, ph);
      return;
    }
  }
  if (k == 2 && is_swap(G)) {
    run_swap<I>(data, dt, n, st, tp[0], tp[1], nc, cp);
    return;
  }
  if (k == 1) {
    run_1q<I>(data, dt, n, st, tp[0], nc, cp, G, seed);
    return;
  }
  run_gen<I>(data, dt, n, st, k, tp, nc, cp, G);
}

}  // namespace

bool use_32bit_index(int n, sv_dtype dt) {
  // vectors are 2 amplitudes (complex64) or 1 (complex128); unit counters
  // and vector indices stay below 2^31 with 32-bit arithmetic.
  return dt == SV_C64 ? n <= 32 : n <= 31;
}

sv_status launch_gate(void* data, sv_dtype dt, int n, cudaStream_t st, int k, const int* tp,
                      int nc, const int* cp, const HostMatrix& G, RoundCtx* rc) {
  // complex64 without controls: round with the state's error feedback.
  // Phases on a subspace (diag(1, .., 1, ph)) act on part of the state only
  // and keep plain rounding; the structure tests below see the unscaled G.
  // Complex64 matrices with entries that are not fp32 numbers get a
  // dithered final rounding in the 1-qubit kernels (seed != 0).
  const HostMatrix* Gp = &G;
  static thread_local HostMatrix Gs;
  uint32_t seed = 0;
  const int d = 1 << k;
  if (rc && dt == SV_C64) {
    for (int e = 0; e < d * d && !seed; ++e)
      if ((double)(float)G.m[e].re != G.m[e].re || (double)(float)G.m[e].im != G.m[e].im)
        seed = rc->next_seed();
  }
  if (rc && dt == SV_C64 && nc == 0) {
    bool phase_only = true;
    for (int r = 0; r < d && phase_only; ++r)
      for (int c = 0; c < d; ++c)
        if ((r != c && !is_zero(G.at(r, c))) || (r == c && r + 1 < d && !is_one(G.at(r, c)))) {
          phase_only = false;
          break;
        }
    if (!phase_only) {
      Gs.k = k;
      for (int e = 0; e < d * d; ++e) Gs.m[e] = G.m[e];
      feedback_round(Gs.m, d, &rc->drift);
      Gp = &Gs;
    }
  }
  if (use_32bit_index(n, dt))
    dispatch<uint32_t>(data, dt, n, st, k, tp, nc, cp, *Gp, seed);
  else
    dispatch<uint64_t>(data, dt, n, st, k, tp, nc, cp, *Gp, seed);
  return check_launch("gate kernel");
}

sv_status launch_init(void* data, sv_dtype dt, int n, cudaStream_t st, uint64_t basis) {
  if (dt == SV_C64) {
    const uint64_t nvec = uint64_t(1) << (n - 1);  // n >= 1: 2^(n-1) vectors of 2 amplitudes
    if (use_32bit_index(n, dt)) {
      const uint32_t nu = (uint32_t)nvec;
      launch_k(kinit_c64<uint32_t, 4>, "kinit_c64", grid_for(nu, 4), st, (float4*)data, nu,
               (uint32_t)(basis >> 1), (int)(basis & 1));
    } else {
      launch_k(kinit_c64<uint64_t, 4>, "kinit_c64", grid_for(nvec, 4), st, (float4*)data, nvec,
               basis >> 1, (int)(basis & 1));
    }
  } else {
    const uint64_t nvec = uint64_t(1) << n;
    if (use_32bit_index(n, dt)) {
      const uint32_t nu = (uint32_t)nvec;
      launch_k(kinit_c128<uint32_t, 4>, "kinit_c128", grid_for(nu, 4), st, (double2*)data, nu,
               (uint32_t)basis);
    } else {
      launch_k(kinit_c128<uint64_t, 4>, "kinit_c128", grid_for(nvec, 4), st, (double2*)data, nvec,
               basis);
    }
  }
  return check_launch("init kernel");
}

}  // namespace sv
