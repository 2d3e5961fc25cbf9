// Device-side helpers shared by the kernel translation units: on-the-fly
// index generation by zero-bit insertion (Sec. 2: indices generated with
// binary operations), 2x2 complex products and the fp64 block reduction.
#pragma once

#include <algorithm>
#include <vector>

#include "sv_internal.cuh"

namespace sv {

template <typename I>
struct Ins {
  int m;
  I low[40];  // low[i] = 2^p_i - 1, p_i ascending (positions in the final index)
};

template <typename I>
inline Ins<I> make_ins(std::vector<int> pos) {
  std::sort(pos.begin(), pos.end());
  Ins<I> s{};
  s.m = (int)pos.size();
  for (int i = 0; i < s.m; ++i) s.low[i] = (I(1) << pos[i]) - 1;
  return s;
}

// Insert a 0 bit at every position of `s`, lowest first.
template <typename I>
__device__ __forceinline__ I insert_zeros(I u, const Ins<I>& s) {
  for (int i = 0; i < s.m; ++i) {
    const I lm = s.low[i];
    u = ((u & ~lm) << 1) | (u & lm);
  }
  return u;
}

// 2x2 complex matrix G00, G01, G10, G11 (real and imaginary parts apart).
template <typename R>
struct M2 {
  R r[4];
  R i[4];
};

template <typename R>
inline M2<R> to_m2(const HostMatrix& G) {
  M2<R> m;
  for (int e = 0; e < 4; ++e) {
    m.r[e] = (R)G.m[e].re;
    m.i[e] = (R)G.m[e].im;
  }
  return m;
}

// Arithmetic variants of (a, b) <- G (a, b); fewer products where the
// matrix structure allows (fp64 throughput is scarce on GB300).
enum { MK_DENSE = 0, MK_DIAG = 1, MK_REAL = 2, MK_IMOFF = 3 };

template <int MK, typename R>
__device__ __forceinline__ void mv2(const M2<R>& g, R& ar, R& ai, R& br, R& bi) {
  R nar, nai, nbr, nbi;
  if (MK == MK_DENSE) {
    nar = g.r[0] * ar - g.i[0] * ai + g.r[1] * br - g.i[1] * bi;
    nai = g.r[0] * ai + g.i[0] * ar + g.r[1] * bi + g.i[1] * br;
    nbr = g.r[2] * ar - g.i[2] * ai + g.r[3] * br - g.i[3] * bi;
    nbi = g.r[2] * ai + g.i[2] * ar + g.r[3] * bi + g.i[3] * br;
  } else if (MK == MK_DIAG) {
    nar = g.r[0] * ar - g.i[0] * ai;
    nai = g.r[0] * ai + g.i[0] * ar;
    nbr = g.r[3] * br - g.i[3] * bi;
    nbi = g.r[3] * bi + g.i[3] * br;
  } else if (MK == MK_REAL) {
    nar = g.r[0] * ar + g.r[1] * br;
    nai = g.r[0] * ai + g.r[1] * bi;
    nbr = g.r[2] * ar + g.r[3] * br;
    nbi = g.r[2] * ai + g.r[3] * bi;
  } else {  // [[r0, i*i1], [i*i2, r3]]
    nar = g.r[0] * ar - g.i[1] * bi;
    nai = g.r[0] * ai + g.i[1] * br;
    nbr = g.r[3] * br - g.i[2] * ai;
    nbi = g.r[3] * bi + g.i[2] * ar;
  }
  ar = nar;
  ai = nai;
  br = nbr;
  bi = nbi;
}

// ---- complex64: dithered rounding ---------------------------------------------
// Round-to-nearest errors of identical inputs are identical.  In states with
// many equal amplitudes (uniform superpositions, the iterates of Grover's
// search) every amplitude of such a class makes the same rounding error at
// every gate, and ||psi||^2 moves by the same relative amount each time: a
// drift linear in the gate count (measured 3e-8 per Grover iteration at
// n = 20).  Complex64 gate kernels therefore add, inside each output's
// fused multiply-add chain before its final rounding, a pseudo-random term
// rho (|a| + |b|) with |rho| <= 2^-24 and zero mean, keyed by the amplitude
// index and a per-launch seed: the final rounding becomes dithered (its
// error random, with zero mean, from amplitude to amplitude) and equal
// amplitudes leave the gate distinct in their last bit, so later roundings
// are uncorrelated as well.  The added error is of the size of one rounding.
//
// mix32: the "lowbias32" integer hash (C. Wellons, hash-prospector, 2018).
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// byte i of h as an odd integer in -255..255 times 2^-32 (|rho| < 2^-24,
// mean 0 over uniform bytes)
__device__ __forceinline__ float dither_rho(uint32_t h, int i) {
  const int b = (int)(int8_t)(h >> (8 * i));
  return (float)(2 * b + 1) * 2.3283064365386963e-10f;
}

// (a, b) <- G (a, b) in fp32 with the final rounding of each of the four
// outputs dithered by rho_i (|a| + |b|) of its own component.
template <int MK>
__device__ __forceinline__ void mv2_dither(const M2<float>& g, float& ar, float& ai, float& br,
                                           float& bi, uint32_t h) {
  const float dr0 = dither_rho(h, 0) * (fabsf(ar) + fabsf(br));
  const float di0 = dither_rho(h, 1) * (fabsf(ai) + fabsf(bi));
  const float dr1 = dither_rho(h, 2) * (fabsf(ar) + fabsf(br));
  const float di1 = dither_rho(h, 3) * (fabsf(ai) + fabsf(bi));
  float nar, nai, nbr, nbi;
  if (MK == MK_DENSE) {
    nar = fmaf(g.r[0], ar, fmaf(-g.i[0], ai, fmaf(g.r[1], br, fmaf(-g.i[1], bi, dr0))));
    nai = fmaf(g.r[0], ai, fmaf(g.i[0], ar, fmaf(g.r[1], bi, fmaf(g.i[1], br, di0))));
    nbr = fmaf(g.r[2], ar, fmaf(-g.i[2], ai, fmaf(g.r[3], br, fmaf(-g.i[3], bi, dr1))));
    nbi = fmaf(g.r[2], ai, fmaf(g.i[2], ar, fmaf(g.r[3], bi, fmaf(g.i[3], br, di1))));
  } else if (MK == MK_DIAG) {
    nar = fmaf(g.r[0], ar, fmaf(-g.i[0], ai, dr0));
    nai = fmaf(g.r[0], ai, fmaf(g.i[0], ar, di0));
    nbr = fmaf(g.r[3], br, fmaf(-g.i[3], bi, dr1));
    nbi = fmaf(g.r[3], bi, fmaf(g.i[3], br, di1));
  } else if (MK == MK_REAL) {
    nar = fmaf(g.r[0], ar, fmaf(g.r[1], br, dr0));
    nai = fmaf(g.r[0], ai, fmaf(g.r[1], bi, di0));
    nbr = fmaf(g.r[2], ar, fmaf(g.r[3], br, dr1));
    nbi = fmaf(g.r[2], ai, fmaf(g.r[3], bi, di1));
  } else {  // [[r0, i*i1], [i*i2, r3]]
    nar = fmaf(g.r[0], ar, fmaf(-g.i[1], bi, dr0));
    nai = fmaf(g.r[0], ai, fmaf(g.i[1], br, di0));
    nbr = fmaf(g.r[3], br, fmaf(-g.i[2], ai, dr1));
    nbi = fmaf(g.r[3], bi, fmaf(g.i[2], ar, di1));
  }
  ar = nar;
  ai = nai;
  br = nbr;
  bi = nbi;
}

// A thread's running sum: compensated (Kahan) in fp32 for complex64 kernels
// (GB300 issues fp64 at a small fraction of the fp32 rate, so the per-unit
// additions stay in fp32 and s - c meets the fp64 block sum once), plain fp64
// for complex128.
template <typename R>
struct CompSum {
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

// Sum over the block (fixed order); the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[32];
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

bool use_32bit_index(int n, sv_dtype dt);

}  // namespace sv
