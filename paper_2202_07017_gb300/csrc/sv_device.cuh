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
