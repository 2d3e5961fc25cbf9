// Fused qubit-block pass: one HBM round trip for many gates.
//
// A pass stages m amplitude-index bits S (the L lowest bits, as contiguous
// runs of 2^L amplitudes, plus m - L high bits).  A thread block holds one
// 2^m-amplitude slice (all other bits fixed by the slice id) in shared
// memory, applies the pass's register groups one after another, and writes
// the slice back.  In a group every thread pulls 2^k amplitudes that differ
// only in the group's k bits into registers, applies the group's gates there
// (Eq. 1 of Sec. 2 for each gate, with compile-time register indices) and
// pushes them back, so shared memory is touched once per group rather than
// once per gate.
//
// Staging: the slice is a box of a rank-2..5 tensor view of the state
// (128-byte rows; the low run; up to three runs of consecutive staged high
// bits as further dimensions; any remaining staged bits enumerated as
// separate boxes), moved by bulk tensor copies (TMA) whose completion is
// signalled on an mbarrier; blocks are persistent, one per resident slot.
// Passes whose geometry does not fit a box use the fallback kernel, which
// stages with 16-byte loads by all threads.
//
// Shared-memory layout: local amplitude j (bit i of j <-> staged bit
// order[i]) lives at slot j with the 16-byte chunks of every 128-byte row
// XOR-permuted by the row index mod 8 - the TMA 128-byte swizzle, applied
// in software by the fallback kernel - which spreads the strided
// register-group accesses of a warp over the banks.
#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <numeric>

#include "slice_geom.cuh"
#include "sv_device.cuh"
#include "tma.cuh"

namespace sv {
namespace {

constexpr int kFThreads = 256;
constexpr int kFMaxOps = 200;
constexpr int kFMaxGroups = 64;
constexpr int kFMaxLayers = 128;
constexpr int kFCoefBytes = 12288;  // layer coefficients of one pass

template <typename R>
struct FOpDev {
  uint8_t type, b0, b1, cmask;  // group-local bit indices and control mask
  uint8_t cls;                  // FG_1Q: MK_* arithmetic class; FG_PHASE: 1 if the phase is -1
  uint8_t pad[3];
  R m[8];                       // FG_1Q: G00 G01 G10 G11 (re, im); FG_PHASE: m[0..1]
};

// One layer of a layered group: a scaled real rotation on every group bit i
// with bit i of rot set, a dense 2x2 on every bit with bit i of u1 set (the
// 2x2s act on different bits and commute), then a diagonal over the group's
// 2^k local indices (dk: 0 none, 1 real, 2 complex).  The rotation on bit i
// is S = [[1, -t], [t, 1]], |t| <= 1: one FMA per output component.
// Coefficients at coef[off...]: the rotations' t in slots 0..3 by bit (if
// rot), the 2x2s in bit order
// (8 values each, row-major re/im), then the diagonal (2^k real or 2^k re/im
// pairs).
struct FLayerDev {
  uint8_t u1, dk;
  uint16_t off;
  uint8_t rot, pad8;
  uint16_t pad;
};

template <typename R>
struct FusedParams {
  CUtensorMap tmap;   // TMA view of the state (64-byte aligned)
  CUtensorMap tmap2;  // reverse sweeps: the same view of lambda
  Ins<uint64_t> blk;  // zero bits at every staged position: block id -> base index
  int m, L, nh;
  uint8_t hpos[32];   // staged bits above the low run, in local order
  // TMA geometry: coordinate d >= 1 of a box at base index a is
  // (a mod 2^thi[d]) >> tlo[d]; box k adds software bits swpos[j] for the
  // set bits j of k and lands at k * box_bytes in shared memory
  int rank, nsw, ncopies;
  uint8_t tlo[5], thi[5], swpos[12];
  uint32_t box_bytes, slice_bytes;
  uint32_t extra_tx;  // 0; the bounded-wait self-test arms the barrier for more bytes
  uint32_t dseed;     // complex64 forward passes: seed of the dithered rounding (0: none)
  int ngroups;
  int ngrad;            // reverse sweeps: gradient operations of the pass
  int gslot[kFMaxOps];  // their gradient slots
  uint8_t gk[kFMaxGroups];
  uint8_t gbits[kFMaxGroups][5];
  uint16_t gop[kFMaxGroups + 1];
  uint8_t gkind[kFMaxGroups];        // 1, 2: the group runs as layers glay[g]..glay[g+1] (2: no dense 2x2)
  uint8_t gxm[kFMaxGroups];          // layer programs: register relabelling the stores undo
  uint16_t glay[kFMaxGroups + 1];
  int ncoef;                         // coefficients in coef[] (elements of R)
  FLayerDev layers[kFMaxLayers];
  R coef[kFCoefBytes / sizeof(R)];
  FOpDev<R> ops[kFMaxOps];
};

template <typename R>
struct Cplx2;
template <>
struct Cplx2<float> {
  typedef float2 T;
};
template <>
struct Cplx2<double> {
  typedef double2 T;
};

template <typename R>
__device__ __forceinline__ int swz(int j);
template <>
__device__ __forceinline__ int swz<float>(int j) {
  return j ^ (((j >> 4) & 7) << 1);
}
template <>
__device__ __forceinline__ int swz<double>(int j) {
  return j ^ ((j >> 3) & 7);
}

__host__ __device__ constexpr int lowbit(int r) { return (r & 1) ? 0 : 1 + lowbit(r >> 1); }

// ---- register-level gate application -------------------------------------------
// Every operation acts on NS register tiles at once (1 for forward passes;
// psi and lambda for reverse sweeps), so one dispatch serves both states.
// (a, b) <- G (a, b) on every register pair of group bit B; CTRL: only where
// the group-local control mask is set; MK: arithmetic class of G.
template <int KG, int B, int MK, bool CTRL, int NS, typename R>
__device__ __forceinline__ void ap1(const FOpDev<R>& op, R (&re)[NS][1 << KG],
                                    R (&im)[NS][1 << KG]) {
  const int cm = op.cmask;
  M2<R> g;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    g.r[e] = op.m[2 * e];
    g.i[e] = op.m[2 * e + 1];
  }
#pragma unroll
  for (int q = 0; q < NS; ++q)
#pragma unroll
    for (int r = 0; r < (1 << KG); ++r) {
      if (r & (1 << B)) continue;
      if (CTRL && (r & cm) != cm) continue;
      const int r1 = r | (1 << B);
      mv2<MK, R>(g, re[q][r], im[q][r], re[q][r1], im[q][r1]);
    }
}

template <int KG, int B, int NS, typename R>
__device__ __forceinline__ void ap1_cls(const FOpDev<R>& op, R (&re)[NS][1 << KG],
                                        R (&im)[NS][1 << KG]) {
  if constexpr (NS == 2 && KG >= 4) {
    // two 16-amplitude tiles: one dense form only (the class-specific
    // variants raise register pressure past the 2-blocks-per-SM budget; the
    // un-applied products of a reverse sweep are mostly dense anyway)
    if (op.cmask)
      ap1<KG, B, MK_DENSE, true, NS>(op, re, im);
    else
      ap1<KG, B, MK_DENSE, false, NS>(op, re, im);
    return;
  }
  if (op.cmask) {
    ap1<KG, B, MK_DENSE, true, NS>(op, re, im);
    return;
  }
  switch (op.cls) {
    case MK_REAL: ap1<KG, B, MK_REAL, false, NS>(op, re, im); break;
    case MK_IMOFF: ap1<KG, B, MK_IMOFF, false, NS>(op, re, im); break;
    case MK_DIAG: ap1<KG, B, MK_DIAG, false, NS>(op, re, im); break;
    default: ap1<KG, B, MK_DENSE, false, NS>(op, re, im); break;
  }
}

// phase on the registers whose index has every bit of the compile-time
// group mask CM set: a sign flip (NEG) or multiplication by (c, s)
template <int KG, int CM, bool NEG, int NS, typename R>
__device__ __forceinline__ void phase_cm(R c, R s, R (&re)[NS][1 << KG], R (&im)[NS][1 << KG]) {
#pragma unroll
  for (int q = 0; q < NS; ++q)
#pragma unroll
    for (int r = 0; r < (1 << KG); ++r) {
      if ((r & CM) != CM) continue;
      if (NEG) {
        re[q][r] = -re[q][r];
        im[q][r] = -im[q][r];
      } else {
        const R xr = re[q][r], xi = im[q][r];
        re[q][r] = c * xr - s * xi;
        im[q][r] = s * xr + c * xi;
      }
    }
}

// the runtime mask as a compile-time one (no per-register mask tests)
template <int KG, bool NEG, int NS, typename R>
__device__ __forceinline__ void phase_op(int cm, R c, R s, R (&re)[NS][1 << KG],
                                         R (&im)[NS][1 << KG]) {
#define SV_PHASE_CASE(v) \
  case v:                \
    if constexpr (v < (1 << KG)) phase_cm<KG, v, NEG, NS>(c, s, re, im); \
    break;
  switch (cm) {
    SV_PHASE_CASE(0) SV_PHASE_CASE(1) SV_PHASE_CASE(2) SV_PHASE_CASE(3)
    SV_PHASE_CASE(4) SV_PHASE_CASE(5) SV_PHASE_CASE(6) SV_PHASE_CASE(7)
    SV_PHASE_CASE(8) SV_PHASE_CASE(9) SV_PHASE_CASE(10) SV_PHASE_CASE(11)
    SV_PHASE_CASE(12) SV_PHASE_CASE(13) SV_PHASE_CASE(14) SV_PHASE_CASE(15)
    default: break;
  }
#undef SV_PHASE_CASE
}

template <int KG, int B0, int B1, int NS, typename R>
__device__ __forceinline__ void apswap(int cm, R (&re)[NS][1 << KG], R (&im)[NS][1 << KG]) {
#pragma unroll
  for (int q = 0; q < NS; ++q)
#pragma unroll
    for (int r = 0; r < (1 << KG); ++r) {
      if (!((r >> B0) & 1) || ((r >> B1) & 1)) continue;
      if ((r & cm) != cm) continue;
      const int r2 = r ^ (1 << B0) ^ (1 << B1);
      const R tr = re[q][r], ti = im[q][r];
      re[q][r] = re[q][r2];
      im[q][r] = im[q][r2];
      re[q][r2] = tr;
      im[q][r2] = ti;
    }
}

template <int KG, int NS, typename R>
__device__ __forceinline__ void apply_op(const FOpDev<R>& op, R (&re)[NS][1 << KG],
                                         R (&im)[NS][1 << KG]) {
  static_assert(KG <= 4, "group masks beyond 4 bits");
  if (op.type == FG_1Q) {
    switch (op.b0) {
      case 0: ap1_cls<KG, 0, NS>(op, re, im); break;
      case 1: if constexpr (KG > 1) ap1_cls<KG, 1, NS>(op, re, im); break;
      case 2: if constexpr (KG > 2) ap1_cls<KG, 2, NS>(op, re, im); break;
      default: if constexpr (KG > 3) ap1_cls<KG, 3, NS>(op, re, im); break;
    }
  } else if (op.type == FG_PHASE) {
    if constexpr (NS == 2 && KG >= 4) {
      const int cm = op.cmask;
      if (op.cls) {  // sign flips of the common two-bit masks (CZ) at compile time
        switch (cm) {
          case 3: phase_cm<KG, 3, true, NS>(R(0), R(0), re, im); return;
          case 5: phase_cm<KG, 5, true, NS>(R(0), R(0), re, im); return;
          case 6: phase_cm<KG, 6, true, NS>(R(0), R(0), re, im); return;
          case 9: phase_cm<KG, 9, true, NS>(R(0), R(0), re, im); return;
          case 10: phase_cm<KG, 10, true, NS>(R(0), R(0), re, im); return;
          case 12: phase_cm<KG, 12, true, NS>(R(0), R(0), re, im); return;
          default: break;
        }
      }
      const R c = op.cls ? R(-1) : op.m[0], sn = op.cls ? R(0) : op.m[1];
#pragma unroll
      for (int q = 0; q < NS; ++q)
#pragma unroll
        for (int r = 0; r < (1 << KG); ++r) {
          if ((r & cm) != cm) continue;
          const R xr = re[q][r], xi = im[q][r];
          re[q][r] = c * xr - sn * xi;
          im[q][r] = sn * xr + c * xi;
        }
      return;
    }
    if (op.cls)  // phase -1 (Z, CZ): a sign flip
      phase_op<KG, true, NS>(op.cmask, R(0), R(0), re, im);
    else
      phase_op<KG, false, NS>(op.cmask, op.m[0], op.m[1], re, im);
  } else {  // FG_SWAP, b0 < b1
    if constexpr (KG >= 2) {
      const int cm = op.cmask, key = op.b0 * 8 + op.b1;
      switch (key) {
        case 0 * 8 + 1: apswap<KG, 0, 1, NS>(cm, re, im); break;
        case 0 * 8 + 2: if constexpr (KG > 2) apswap<KG, 0, 2, NS>(cm, re, im); break;
        case 1 * 8 + 2: if constexpr (KG > 2) apswap<KG, 1, 2, NS>(cm, re, im); break;
        case 0 * 8 + 3: if constexpr (KG > 3) apswap<KG, 0, 3, NS>(cm, re, im); break;
        case 1 * 8 + 3: if constexpr (KG > 3) apswap<KG, 1, 3, NS>(cm, re, im); break;
        case 2 * 8 + 3: if constexpr (KG > 3) apswap<KG, 2, 3, NS>(cm, re, im); break;
        default: break;
      }
    }
  }
}

template <int KG, typename R>
__device__ __forceinline__ void run_group(typename Cplx2<R>::T* sm, int m, const uint8_t* gb,
                                          const FOpDev<R>* ops, int o0, int o1) {
  typedef typename Cplx2<R>::T V2;
  constexpr int D = 1 << KG;
  // the swizzle is linear over XOR and b, off[r] have disjoint bits, so
  // swz(b | off[r]) = swz(b) ^ swz(off[r]): one XOR per access
  int soff[D];
  soff[0] = 0;
#pragma unroll
  for (int r = 1; r < D; ++r) soff[r] = soff[r & (r - 1)] ^ swz<R>(1 << gb[lowbit(r)]);
  int lm[KG];
#pragma unroll
  for (int i = 0; i < KG; ++i) lm[i] = (1 << gb[i]) - 1;
  const int nsub = 1 << (m - KG);
  for (int s = threadIdx.x; s < nsub; s += kFThreads) {
    int b = s;
#pragma unroll
    for (int i = 0; i < KG; ++i) b = ((b & ~lm[i]) << 1) | (b & lm[i]);
    const int sb = swz<R>(b);
    R re[1][D], im[1][D];
#pragma unroll
    for (int r = 0; r < D; ++r) {
      const V2 v = sm[sb ^ soff[r]];
      re[0][r] = v.x;
      im[0][r] = v.y;
    }
    for (int o = o0; o < o1; ++o) apply_op<KG, 1, R>(ops[o], re, im);
#pragma unroll
    for (int r = 0; r < D; ++r) {
      V2 v;
      v.x = re[0][r];
      v.y = im[0][r];
      sm[sb ^ soff[r]] = v;
    }
  }
}

// (a, b) <- G (a, b) on every register pair of compile-time group bit B,
// G read from shared memory (8 values, 16-byte aligned)
template <int KG, int B, typename R>
__device__ __forceinline__ void dense_bit(const R* c, R (&re)[1 << KG], R (&im)[1 << KG]) {
  M2<R> g;
  if constexpr (sizeof(R) == 4) {
    const float4 x = reinterpret_cast<const float4*>(c)[0];
    const float4 y = reinterpret_cast<const float4*>(c)[1];
    g.r[0] = x.x; g.i[0] = x.y; g.r[1] = x.z; g.i[1] = x.w;
    g.r[2] = y.x; g.i[2] = y.y; g.r[3] = y.z; g.i[3] = y.w;
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const double2 x = reinterpret_cast<const double2*>(c)[e];
      g.r[e] = x.x;
      g.i[e] = x.y;
    }
  }
#pragma unroll
  for (int r = 0; r < (1 << KG); ++r) {
    if (r & (1 << B)) continue;
    const int r1 = r | (1 << B);
    mv2<MK_DENSE, R>(g, re[r], im[r], re[r1], im[r1]);
  }
}

// (a, b) <- S (a, b) on every register pair of group bit B, S the scaled
// rotation [[1, -t], [t, 1]] (F false) or [[t, -1], [1, t]] (F true)
template <int KG, int B, bool F, typename R>
__device__ __forceinline__ void rot_bit(R t, R (&re)[1 << KG], R (&im)[1 << KG]) {
#pragma unroll
  for (int r = 0; r < (1 << KG); ++r) {
    if (r & (1 << B)) continue;
    const int r1 = r | (1 << B);
    const R a = re[r], b = im[r], c = re[r1], d = im[r1];
    if constexpr (F) {
      re[r] = fma(t, a, -c);
      im[r] = fma(t, b, -d);
      re[r1] = fma(t, c, a);
      im[r1] = fma(t, d, b);
    } else {
      re[r] = fma(-t, c, a);
      im[r] = fma(-t, d, b);
      re[r1] = fma(t, a, c);
      im[r1] = fma(t, b, d);
    }
  }
}

// the four rotation slots of a layer (16-byte aligned)
template <typename R>
__device__ __forceinline__ void load_tau4(const R* c, R (&tv)[4]) {
  if constexpr (sizeof(R) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(c);
    tv[0] = v.x;
    tv[1] = v.y;
    tv[2] = v.z;
    tv[3] = v.w;
  } else {
    const double2 v0 = reinterpret_cast<const double2*>(c)[0];
    const double2 v1 = reinterpret_cast<const double2*>(c)[1];
    tv[0] = v0.x;
    tv[1] = v0.y;
    tv[2] = v1.x;
    tv[3] = v1.y;
  }
}

// S(t) on group bit i of a register tile, i a compile-time index after unrolling
template <int KG, typename R>
__device__ __forceinline__ void rot_bit_at(int i, const R (&tv)[4], R (&re)[1 << KG],
                                           R (&im)[1 << KG]) {
  if (i == 0) rot_bit<KG, 0, false, R>(tv[0], re, im);
  if constexpr (KG > 1) if (i == 1) rot_bit<KG, (KG > 1 ? 1 : 0), false, R>(tv[KG > 1 ? 1 : 0], re, im);
  if constexpr (KG > 2) if (i == 2) rot_bit<KG, (KG > 2 ? 2 : 0), false, R>(tv[KG > 2 ? 2 : 0], re, im);
  if constexpr (KG > 3) if (i == 3) rot_bit<KG, (KG > 3 ? 3 : 0), false, R>(tv[KG > 3 ? 3 : 0], re, im);
}

// dense_bit with the final rounding of every output dithered (mv2_dither),
// pair r keyed by mix32(h + r): complex64 only
template <int KG, int B>
__device__ __forceinline__ void dense_bit_dither(const float* c, float (&re)[1 << KG],
                                                 float (&im)[1 << KG], uint32_t h) {
  M2<float> g;
  const float4 x = reinterpret_cast<const float4*>(c)[0];
  const float4 y = reinterpret_cast<const float4*>(c)[1];
  g.r[0] = x.x; g.i[0] = x.y; g.r[1] = x.z; g.i[1] = x.w;
  g.r[2] = y.x; g.i[2] = y.y; g.r[3] = y.z; g.i[3] = y.w;
#pragma unroll
  for (int r = 0; r < (1 << KG); ++r) {
    if (r & (1 << B)) continue;
    const int r1 = r | (1 << B);
    mv2_dither<MK_DENSE>(g, re[r], im[r], re[r1], im[r1], mix32(h + (uint32_t)r));
  }
}

// The group as a layer program (see FLayerDev): no per-gate dispatch, every
// register index fixed at compile time.
// slot offset of register r: XOR of the swizzled group-bit offsets sw[i]
// over the set bits i of r (at most two 3-input XORs)
template <int KG>
__device__ __forceinline__ int reg_off(int r, const int (&sw)[KG]) {
  int o = 0;
#pragma unroll
  for (int i = 0; i < KG; ++i)
    if ((r >> i) & 1) o ^= sw[i];
  return o;
}

// DITHER (complex64): every dense 2x2 rounds its outputs with dither (see
// mv2_dither), keyed by dseed and the sub-block.
// xm: the program's final register relabelling (register r holds group
// index r ^ xm; stored back at its place).
template <int KG, typename R, bool TABLE, bool DITHER = false>
__device__ __forceinline__ void run_layers(typename Cplx2<R>::T* sm, int m, const uint8_t* gb,
                                           const FLayerDev* lay, int l0, int l1, const R* coef,
                                           uint32_t dseed = 0, int xm = 0) {
  typedef typename Cplx2<R>::T V2;
  constexpr int D = 1 << KG;
  int sw[KG];
#pragma unroll
  for (int i = 0; i < KG; ++i) sw[i] = swz<R>(1 << gb[i]);
  const int xoff = reg_off<KG>(xm, sw);
  int soff[TABLE ? D : 1];
  if constexpr (TABLE) {
    soff[0] = 0;
#pragma unroll
    for (int r = 1; r < D; ++r) soff[r] = soff[r & (r - 1)] ^ sw[lowbit(r)];
  }
  auto off = [&](int r) -> int {
    if constexpr (TABLE)
      return soff[r];
    else
      return reg_off<KG>(r, sw);
  };
  int lm[KG];
#pragma unroll
  for (int i = 0; i < KG; ++i) lm[i] = (1 << gb[i]) - 1;
  const int nsub = 1 << (m - KG);
  for (int s = threadIdx.x; s < nsub; s += kFThreads) {
    int b = s;
#pragma unroll
    for (int i = 0; i < KG; ++i) b = ((b & ~lm[i]) << 1) | (b & lm[i]);
    const int sb = swz<R>(b);
    R re[D], im[D];
#pragma unroll
    for (int r = 0; r < D; ++r) {
      const V2 v = sm[sb ^ off(r)];
      re[r] = v.x;
      im[r] = v.y;
    }
    uint32_t h = 0;
    if constexpr (DITHER) h = mix32(dseed + (uint32_t)s * 0x9E3779B1u);
    for (int l = l0; l < l1; ++l) {
      const FLayerDev L = lay[l];
      const R* c = coef + L.off;
      if (L.rot) {
        R tv[4];
        load_tau4<R>(c, tv);
        if (L.rot == (1 << KG) - 1) {  // every bit: one straight-line block
#pragma unroll
          for (int i = 0; i < KG; ++i) rot_bit_at<KG, R>(i, tv, re, im);
        } else {
#pragma unroll
          for (int i = 0; i < KG; ++i)
            if (L.rot & (1 << i)) rot_bit_at<KG, R>(i, tv, re, im);
        }
        c += 4;
      }
#pragma unroll
      for (int i = 0; i < KG; ++i) {
        if (L.u1 & (1 << i)) {
          if constexpr (DITHER && sizeof(R) == 4) {
            h = mix32(h + (uint32_t)(l * KG + i));
            if (i == 0) dense_bit_dither<KG, 0>(c, re, im, h);
            if constexpr (KG > 1) if (i == 1) dense_bit_dither<KG, (KG > 1 ? 1 : 0)>(c, re, im, h);
            if constexpr (KG > 2) if (i == 2) dense_bit_dither<KG, (KG > 2 ? 2 : 0)>(c, re, im, h);
            if constexpr (KG > 3) if (i == 3) dense_bit_dither<KG, (KG > 3 ? 3 : 0)>(c, re, im, h);
            c += 8;
            continue;
          }
          if (i == 0) dense_bit<KG, 0, R>(c, re, im);
          if constexpr (KG > 1) if (i == 1) dense_bit<KG, (KG > 1 ? 1 : 0), R>(c, re, im);
          if constexpr (KG > 2) if (i == 2) dense_bit<KG, (KG > 2 ? 2 : 0), R>(c, re, im);
          if constexpr (KG > 3) if (i == 3) dense_bit<KG, (KG > 3 ? 3 : 0), R>(c, re, im);
          c += 8;
        }
      }
      // diagonal: 16-byte loads of the entries
      typedef typename Cplx2<R>::T V2c;
      if (L.dk == 1) {
        if constexpr (sizeof(R) == 4) {
#pragma unroll
          for (int r = 0; r < D; r += 4) {
            const float4 d = *reinterpret_cast<const float4*>(c + r);
            const float dd[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
            for (int e = 0; e < 4 && r + e < D; ++e) {
              re[r + e] *= dd[e];
              im[r + e] *= dd[e];
            }
          }
        } else {
#pragma unroll
          for (int r = 0; r < D; r += 2) {
            const double2 d = *reinterpret_cast<const double2*>(c + r);
            re[r] *= d.x;
            im[r] *= d.x;
            if (r + 1 < D) {
              re[r + 1] *= d.y;
              im[r + 1] *= d.y;
            }
          }
        }
      } else if (L.dk == 2) {
#pragma unroll
        for (int r = 0; r < D; ++r) {
          const V2c d = *reinterpret_cast<const V2c*>(c + 2 * r);
          const R xr = re[r], xi = im[r];
          re[r] = d.x * xr - d.y * xi;
          im[r] = d.x * xi + d.y * xr;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < D; ++r) {
      V2 v;
      v.x = re[r];
      v.y = im[r];
      sm[sb ^ off(r) ^ xoff] = v;
    }
  }
}

// Two sub-blocks per thread (s and s + kFThreads: a slice of 2^13 amplitudes
// in 4-qubit groups) through one layer program in rotation form (no dense
// 2x2: the registers of two tiles fit beside the rotations, not beside the
// 2x2 coefficients) together: each layer's coefficients are read once for
// both, and the two tiles' operations are independent, so a warp has twice
// the arithmetic in flight between the dependent steps of one tile
// (rotation on bit 0, then bit 1, ..., then the diagonal).
// The registers hold each amplitude as a (re, im) pair, so the rotation's
// four FMAs per register pair - every one scaling both parts of an amplitude
// by the same t - issue as two paired fp32 FMAs (fma.rn.f32x2): half the
// instructions for the same arithmetic.  Complex64 only.
template <int KG, int B>
__device__ __forceinline__ void rot_bit2p(float t, float2 (&v)[2][1 << KG]) {
  const float2 tp = make_float2(t, t), tn = make_float2(-t, -t);
#pragma unroll
  for (int r = 0; r < (1 << KG); ++r) {
    if (r & (1 << B)) continue;
    const int r1 = r | (1 << B);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const float2 a = v[u][r], c = v[u][r1];
      v[u][r] = __ffma2_rn(tn, c, a);   // a - t c
      v[u][r1] = __ffma2_rn(tp, a, c);  // t a + c
    }
  }
}

template <int KG>
__device__ __forceinline__ void rot_bit2p_at(int i, const float (&tv)[4], float2 (&v)[2][1 << KG]) {
  if (i == 0) rot_bit2p<KG, 0>(tv[0], v);
  if constexpr (KG > 1) if (i == 1) rot_bit2p<KG, (KG > 1 ? 1 : 0)>(tv[KG > 1 ? 1 : 0], v);
  if constexpr (KG > 2) if (i == 2) rot_bit2p<KG, (KG > 2 ? 2 : 0)>(tv[KG > 2 ? 2 : 0], v);
  if constexpr (KG > 3) if (i == 3) rot_bit2p<KG, (KG > 3 ? 3 : 0)>(tv[KG > 3 ? 3 : 0], v);
}

template <int KG>
__device__ __forceinline__ void run_layers_x2(float2* sm, const uint8_t* gb, const FLayerDev* lay,
                                              int l0, int l1, const float* coef, int xm) {
  constexpr int D = 1 << KG;
  int sw[KG], lm[KG];
#pragma unroll
  for (int i = 0; i < KG; ++i) {
    sw[i] = swz<float>(1 << gb[i]);
    lm[i] = (1 << gb[i]) - 1;
  }
  int sb[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    int b = threadIdx.x + u * kFThreads;
#pragma unroll
    for (int i = 0; i < KG; ++i) b = ((b & ~lm[i]) << 1) | (b & lm[i]);
    sb[u] = swz<float>(b);
  }
  float2 v[2][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int u = 0; u < 2; ++u) v[u][r] = sm[sb[u] ^ reg_off<KG>(r, sw)];
  for (int l = l0; l < l1; ++l) {
    const FLayerDev L = lay[l];
    const float* c = coef + L.off;
    if (L.rot) {
      float tv[4];
      load_tau4<float>(c, tv);
      if (L.rot == (1 << KG) - 1) {  // every bit: one straight-line block
#pragma unroll
        for (int i = 0; i < KG; ++i) rot_bit2p_at<KG>(i, tv, v);
      } else {
#pragma unroll
        for (int i = 0; i < KG; ++i)
          if (L.rot & (1 << i)) rot_bit2p_at<KG>(i, tv, v);
      }
      c += 4;
    }
    if (L.dk == 1) {
#pragma unroll
      for (int r = 0; r < D; ++r) {
        const float2 d = make_float2(c[r], c[r]);
#pragma unroll
        for (int u = 0; u < 2; ++u) v[u][r] = __fmul2_rn(d, v[u][r]);
      }
    } else if (L.dk == 2) {
#pragma unroll
      for (int r = 0; r < D; ++r) {
        const float2 d = *reinterpret_cast<const float2*>(c + 2 * r);
        const float2 dr = make_float2(d.x, d.x), di = make_float2(-d.y, d.y);
#pragma unroll
        for (int u = 0; u < 2; ++u) {  // (dr xr - di xi, dr xi + di xr)
          const float2 x = v[u][r];
          v[u][r] = __ffma2_rn(di, make_float2(x.y, x.x), __fmul2_rn(dr, x));
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      int sbr = sb[u] ^ reg_off<KG>(xm, sw);
      asm volatile("mov.b32 %0, %1;" : "=r"(sbr) : "r"(sbr));  // store addresses recomputed
      sm[sbr ^ reg_off<KG>(r, sw)] = v[u][r];
    }
}

// ---- the pass kernel ------------------------------------------------------------
// KGF: register-group width of every group of the pass (the planner pads
// groups to it); 3 resident blocks per SM for complex64, 2 for complex128.
template <typename R, int KGF>
__global__ void __launch_bounds__(kFThreads, sizeof(R) == 4 ? 3 : 2)
    kfused(typename Cplx2<R>::T* __restrict__ psi, uint64_t n_blocks,
           const __grid_constant__ FusedParams<R> P) {
  typedef typename Cplx2<R>::T V2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V2* sm = reinterpret_cast<V2*>(smem_raw);
  const int M = 1 << P.m;
  uint64_t* runoff = reinterpret_cast<uint64_t*>(sm + M);
  const int L = P.L;
  const int nruns = 1 << (P.m - L);
  R* csm = reinterpret_cast<R*>(runoff + ((nruns + 1) & ~1));
  for (int i = threadIdx.x; i < P.ncoef; i += kFThreads) csm[i] = P.coef[i];
  for (int r = threadIdx.x; r < nruns; r += kFThreads) {
    uint64_t o = 0;
    for (int i = 0; i < P.nh; ++i)
      if ((r >> i) & 1) o |= uint64_t(1) << P.hpos[i];
    runoff[r] = o;
  }
  __syncthreads();
  // 16-byte chunks: 2 amplitudes (complex64) or 1 (complex128)
  constexpr int APC = sizeof(R) == 4 ? 2 : 1;
  constexpr int LAPC = APC == 2 ? 1 : 0;
  const int lcr = L - LAPC;  // log2 chunks per run
  const int nch = M / APC;
  constexpr int U = 4;  // 16-byte loads in flight per thread while staging
  for (uint64_t blk = blockIdx.x; blk < n_blocks; blk += gridDim.x) {
    const uint64_t base = insert_zeros(blk, P.blk);
    for (int c0 = threadIdx.x; c0 < nch; c0 += kFThreads * U) {
      float4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = c0 + u * kFThreads;
        if (c < nch) {
          const int run = c >> lcr, w = c & ((1 << lcr) - 1);
          const uint64_t amp = base | runoff[run] | ((uint64_t)w << LAPC);
          v[u] = reinterpret_cast<const float4*>(psi)[amp >> LAPC];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = c0 + u * kFThreads;
        if (c < nch) {
          const int run = c >> lcr, w = c & ((1 << lcr) - 1);
          const int j = (run << L) | (w << LAPC);
          *reinterpret_cast<float4*>(&sm[swz<R>(j)]) = v[u];
        }
      }
    }
    __syncthreads();
    for (int g = 0; g < P.ngroups; ++g) {
      const uint8_t* gb = P.gbits[g];
      if (P.gkind[g])
        run_layers<KGF, R, true>(sm, P.m, gb, P.layers, P.glay[g], P.glay[g + 1], csm, 0,
                                 P.gxm[g]);
      else
        run_group<KGF, R>(sm, P.m, gb, P.ops, P.gop[g], P.gop[g + 1]);
      __syncthreads();
    }
    for (int c0 = threadIdx.x; c0 < nch; c0 += kFThreads * U) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = c0 + u * kFThreads;
        if (c < nch) {
          const int run = c >> lcr, w = c & ((1 << lcr) - 1);
          const int j = (run << L) | (w << LAPC);
          const uint64_t amp = base | runoff[run] | ((uint64_t)w << LAPC);
          reinterpret_cast<float4*>(psi)[amp >> LAPC] =
              *reinterpret_cast<const float4*>(&sm[swz<R>(j)]);
        }
      }
    }
    __syncthreads();
  }
}

// ---- the TMA-staged pass kernel ---------------------------------------------------
__device__ unsigned g_fused_status = 0;  // kWaitTimeout: a bounded wait gave up

template <typename R>
__device__ __forceinline__ void box_coords(const FusedParams<R>& P, uint64_t base, int k, int* c) {
  uint64_t a = base;
  for (int j = 0; j < P.nsw; ++j)
    if ((k >> j) & 1) a |= uint64_t(1) << P.swpos[j];
  c[0] = 0;
#pragma unroll
  for (int d = 1; d < 5; ++d)
    c[d] = d < P.rank ? (int)((a & ((uint64_t(1) << P.thi[d]) - 1)) >> P.tlo[d]) : 0;
}

template <typename R>
__device__ __forceinline__ void issue_load(const FusedParams<R>& P, uint32_t dst, const int* c,
                                           uint32_t bar) {
  switch (P.rank) {
    case 2: tma_load<2>(dst, &P.tmap, c, bar); break;
    case 3: tma_load<3>(dst, &P.tmap, c, bar); break;
    case 4: tma_load<4>(dst, &P.tmap, c, bar); break;
    default: tma_load<5>(dst, &P.tmap, c, bar); break;
  }
}

template <typename R>
__device__ __forceinline__ void issue_prefetch(const FusedParams<R>& P, const CUtensorMap* map,
                                               const int* c) {
  switch (P.rank) {
    case 2: tma_prefetch<2>(map, c); break;
    case 3: tma_prefetch<3>(map, c); break;
    case 4: tma_prefetch<4>(map, c); break;
    default: tma_prefetch<5>(map, c); break;
  }
}

// The block's next slice (blk + gridDim.x) into L2 while this one is worked
// on: its load then waits on L2 rather than HBM.  Warp 0; both views for
// reverse sweeps.
template <typename R>
__device__ __forceinline__ void prefetch_next(const FusedParams<R>& P, uint64_t blk,
                                              uint64_t n_blocks, int lane, bool two) {
  const uint64_t nb = blk + gridDim.x;
  if (nb >= n_blocks) return;
  const uint64_t nbase = insert_zeros(nb, P.blk);
  for (int k = lane; k < P.ncopies; k += 32) {
    int c[5];
    box_coords(P, nbase, k, c);
    issue_prefetch(P, &P.tmap, c);
    if (two) issue_prefetch(P, &P.tmap2, c);
  }
}

template <typename R>
__device__ __forceinline__ void issue_store(const FusedParams<R>& P, uint32_t src, const int* c) {
  switch (P.rank) {
    case 2: tma_store<2>(&P.tmap, c, src); break;
    case 3: tma_store<3>(&P.tmap, c, src); break;
    case 4: tma_store<4>(&P.tmap, c, src); break;
    default: tma_store<5>(&P.tmap, c, src); break;
  }
}

// Persistent: block b handles slices b, b + gridDim.x, ...  Warp 0 moves the
// slice: waits until its earlier stores have read the buffer, arms the
// mbarrier with the slice's byte count and issues the box loads; every
// thread waits for the phase (bounded), runs the groups, makes its writes
// visible to the async proxy, and warp 0 issues the box stores.
// MODE: 0 every group a gate list, 1 mixed, 3 every group a layer program
// (shared-memory addresses recomputed per access instead of tabulated), 4 as
// 3 with every dense 2x2 rounded with dither (complex64, dithered rounding
// selected for the state)
template <typename R, int KGF, int MINB, int MODE>
__global__ void __launch_bounds__(kFThreads, MINB)
    kfused_tma(uint64_t n_blocks, const __grid_constant__ FusedParams<R> P) {
  typedef typename Cplx2<R>::T V2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t sbuf = (raw + 1023u) & ~1023u;  // the 128-byte swizzle repeats every 1024 bytes
  V2* sm = reinterpret_cast<V2*>(smem_raw + (sbuf - raw));
  const uint32_t barp = smem_addr(&bar);
  const int lane = threadIdx.x & 31;
  R* csm = reinterpret_cast<R*>(smem_raw + (sbuf - raw) + P.slice_bytes);
  for (int i = threadIdx.x; i < P.ncoef; i += kFThreads) csm[i] = P.coef[i];
  // the layer table beside the coefficients: read per layer by every thread,
  // from shared memory rather than the parameter space
  FLayerDev* lsm = reinterpret_cast<FLayerDev*>(csm + ((P.ncoef + 1) & ~1));
  for (int i = threadIdx.x; i < P.glay[P.ngroups]; i += kFThreads) lsm[i] = P.layers[i];
  if (threadIdx.x == 0) {
    mbar_init(barp, 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  uint32_t parity = 0;
  for (uint64_t blk = blockIdx.x; blk < n_blocks; blk += gridDim.x) {
    const uint64_t base = insert_zeros(blk, P.blk);
    if (threadIdx.x < 32) {
      bulk_wait_read_all();
      __syncwarp();
      if (lane == 0) mbar_arrive_expect_tx(barp, P.slice_bytes + P.extra_tx);
      __syncwarp();
      for (int k = lane; k < P.ncopies; k += 32) {
        int c[5];
        box_coords(P, base, k, c);
        issue_load(P, sbuf + (uint32_t)k * P.box_bytes, c, barp);
      }
      prefetch_next(P, blk, n_blocks, lane, false);
    }
    const bool ok = mbar_wait_bounded(barp, parity);
    parity ^= 1;
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicOr(&g_fused_status, kWaitTimeout);
      break;
    }
    for (int g = 0; g < P.ngroups; ++g) {
      if (MODE == 4)
        run_layers<KGF, R, false, true>(
            sm, P.m, P.gbits[g], lsm, P.glay[g], P.glay[g + 1], csm,
            mix32(P.dseed ^ (uint32_t)blk ^ ((uint32_t)(blk >> 32) + (uint32_t)g * 0x85ebca6bu)));
      else if (MODE == 3 && KGF == 4 && sizeof(R) == 4 && P.m == 13 && P.gkind[g] == 2) {
        if constexpr (sizeof(R) == 4)  // two sub-blocks per thread (complex64 slices)
          run_layers_x2<KGF>(sm, P.gbits[g], lsm, P.glay[g], P.glay[g + 1], csm, P.gxm[g]);
      } else if (MODE == 3)
        run_layers<KGF, R, false>(sm, P.m, P.gbits[g], lsm, P.glay[g], P.glay[g + 1], csm, 0,
                                  P.gxm[g]);
      else if (MODE == 1 && P.gkind[g])
        run_layers<KGF, R, true>(sm, P.m, P.gbits[g], lsm, P.glay[g], P.glay[g + 1], csm, 0,
                                 P.gxm[g]);
      else
        run_group<KGF, R>(sm, P.m, P.gbits[g], P.ops, P.gop[g], P.gop[g + 1]);
      if (g + 1 < P.ngroups) __syncthreads();
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x < 32) {
      for (int k = lane; k < P.ncopies; k += 32) {
        int c[5];
        box_coords(P, base, k, c);
        issue_store(P, sbuf + (uint32_t)k * P.box_bytes, c);
      }
      bulk_commit();
    }
  }
  if (threadIdx.x < 32) bulk_wait_all();
}

// ---- reverse sweep pass: psi and lambda together ---------------------------------------
// Gradient of U = exp(-i theta P / 2) at its place in the reverse sweep:
// Im <lambda|P|psi> (P a Pauli, or for pauli = 0 the Hermitian generator
// [[a, b], [conj b, d]] in gm = (a, d, re b, im b) that a pending un-apply
// W turns P into: W^dagger P W) over the register pairs of group bit B inside the
// control mask cm, in the state's precision (a thread's 2^(KG-1) pairs;
// the warp's sum is then added to an fp64 accumulator).
template <int KG, int B, typename R>
__device__ __forceinline__ R grad_pairs(int pauli, int cm, const R* gm, const R (&pr)[1 << KG],
                                        const R (&pi)[1 << KG], const R (&lr)[1 << KG],
                                        const R (&li)[1 << KG]) {
  R acc = 0;
  const R ga = gm[0], gd = gm[1], gbr = gm[2], gbi = gm[3];
#pragma unroll
  for (int r = 0; r < (1 << KG); ++r) {
    if (r & (1 << B)) continue;
    if ((r & cm) != cm) continue;
    const int r1 = r | (1 << B);
    const R p0r = pr[r], p0i = pi[r], p1r = pr[r1], p1i = pi[r1];
    const R l0r = lr[r], l0i = li[r], l1r = lr[r1], l1i = li[r1];
    R c;
    if (pauli == 0) {  // M = [[a, b], [conj b, d]]: terms of conj(l_r) M_rs p_s
      const R z00i = l0r * p0i - l0i * p0r, z11i = l1r * p1i - l1i * p1r;
      const R z01r = l0r * p1r + l0i * p1i, z01i = l0r * p1i - l0i * p1r;
      const R z10r = l1r * p0r + l1i * p0i, z10i = l1r * p0i - l1i * p0r;
      c = ga * z00i + gd * z11i + gbr * (z01i + z10i) + gbi * (z01r - z10r);
    } else if (pauli == 1)  // P psi = (p1, p0)
      c = (l0r * p1i - l0i * p1r) + (l1r * p0i - l1i * p0r);
    else if (pauli == 2)  // (-i p1, i p0)
      c = -(l0r * p1r + l0i * p1i) + (l1r * p0r + l1i * p0i);
    else  // (p0, -p1)
      c = (l0r * p0i - l0i * p0r) - (l1r * p1i - l1i * p1r);
    acc += c;
  }
  return acc;
}

// The four real sums that every generator [[a, b], [conj b, d]] on group
// bit B needs: with z_rs = conj(l_r) p_s over the pairs inside cm,
// Im<lambda|M|psi> = a Im z00 + d Im z11 + re b Im(z01 + z10) + im b Re(z01 - z10).
// Several gradients on one bit then cost these 12 FMAs per pair once.
template <int KG, int B, bool CTRL, typename R>
__device__ __forceinline__ void grad_quad(int cm, const R (&pr)[1 << KG], const R (&pi)[1 << KG],
                                          const R (&lr)[1 << KG], const R (&li)[1 << KG],
                                          R (&q)[4]) {
#pragma unroll
  for (int r = 0; r < (1 << KG); ++r) {
    if (r & (1 << B)) continue;
    if (CTRL && (r & cm) != cm) continue;
    const int r1 = r | (1 << B);
    const R p0r = pr[r], p0i = pi[r], p1r = pr[r1], p1i = pi[r1];
    const R l0r = lr[r], l0i = li[r], l1r = lr[r1], l1i = li[r1];
    q[0] = fma(l0r, p0i, q[0]);
    q[0] = fma(-l0i, p0r, q[0]);
    q[1] = fma(l1r, p1i, q[1]);
    q[1] = fma(-l1i, p1r, q[1]);
    q[2] = fma(l0r, p1i, q[2]);
    q[2] = fma(-l0i, p1r, q[2]);
    q[2] = fma(l1r, p0i, q[2]);
    q[2] = fma(-l1i, p0r, q[2]);
    q[3] = fma(l0r, p1r, q[3]);
    q[3] = fma(l0i, p1i, q[3]);
    q[3] = fma(-l1r, p0r, q[3]);
    q[3] = fma(-l1i, p0i, q[3]);
  }
}

template <int KG, bool CTRL, typename R>
__device__ __forceinline__ void grad_quad_at(int b, int cm, const R (&pr)[1 << KG],
                                             const R (&pi)[1 << KG], const R (&lr)[1 << KG],
                                             const R (&li)[1 << KG], R (&q)[4]) {
  switch (b) {
    case 0: grad_quad<KG, 0, CTRL, R>(cm, pr, pi, lr, li, q); break;
    case 1: if constexpr (KG > 1) grad_quad<KG, (KG > 1 ? 1 : 0), CTRL, R>(cm, pr, pi, lr, li, q); break;
    case 2: if constexpr (KG > 2) grad_quad<KG, (KG > 2 ? 2 : 0), CTRL, R>(cm, pr, pi, lr, li, q); break;
    default: if constexpr (KG > 3) grad_quad<KG, (KG > 3 ? 3 : 0), CTRL, R>(cm, pr, pi, lr, li, q); break;
  }
}

// Warp sums of v[0..3] in 6 shuffles: afterwards lane 8 i holds the sum of
// v[i] (lanes split the values by lane bits 4 and 3, then reduce the rest).
template <typename R>
__device__ __forceinline__ R warp_sum4(const R (&v)[4], int lane) {
  const bool h4 = lane & 16, h3 = lane & 8;
  R a = h4 ? v[2] : v[0], b = h4 ? v[3] : v[1];
  const R sa = h4 ? v[0] : v[2], sb = h4 ? v[1] : v[3];
  a += __shfl_xor_sync(0xffffffffu, sa, 16);
  b += __shfl_xor_sync(0xffffffffu, sb, 16);
  R w = h3 ? b : a;
  w += __shfl_xor_sync(0xffffffffu, h3 ? a : b, 8);
  w += __shfl_xor_sync(0xffffffffu, w, 4);
  w += __shfl_xor_sync(0xffffffffu, w, 2);
  w += __shfl_xor_sync(0xffffffffu, w, 1);
  return w;
}

// Per-warp gradient accumulator: a compensated (Kahan) sum in the state's
// precision - GB300 issues fp64 instructions at a small fraction of the fp32
// rate, so the per-sub-block additions avoid fp64; the block converts s - c
// to fp64 once at the end.
template <typename R>
struct KahanAcc {
  R s, c;
};

template <typename R>
__device__ __forceinline__ void kahan_add(KahanAcc<R>& a, R x) {
  const R y = x - a.c;
  const R t = a.s + y;
  a.c = (t - a.s) - y;
  a.s = t;
}

// One register group over both slices: gradient operations accumulate into
// this warp's slots gw[0..ngrad), every other operation is applied to psi
// and lambda.  All lanes of a warp run the same iterations (warp sums).
template <int KG, typename R>
__device__ __forceinline__ void run_group_adj(typename Cplx2<R>::T* smp,
                                              typename Cplx2<R>::T* sml, int m,
                                              const uint8_t* gb, const FOpDev<R>* ops, int o0,
                                              int o1, const R* gcoef, KahanAcc<R>* gw) {
  typedef typename Cplx2<R>::T V2;
  constexpr int D = 1 << KG;
  // register offsets: a table for up to 8 registers, else XORs of the
  // swizzled bit offsets at each access (frees 16 registers for the tiles)
  constexpr bool kTable = KG <= 3;
  int sw[KG];
  int soff[kTable ? D : 1];
  if constexpr (kTable) {
    soff[0] = 0;
#pragma unroll
    for (int r = 1; r < D; ++r) soff[r] = soff[r & (r - 1)] ^ swz<R>(1 << gb[lowbit(r)]);
  } else {
#pragma unroll
    for (int i = 0; i < KG; ++i) sw[i] = swz<R>(1 << gb[i]);
  }
#define SV_ADJ_OFF(r) (kTable ? soff[kTable ? (r) : 0] : reg_off<KG>((r), sw))
  int lm[KG];
#pragma unroll
  for (int i = 0; i < KG; ++i) lm[i] = (1 << gb[i]) - 1;
  const int nsub = 1 << (m - KG);
  // reverse slices hold at most 2^12 amplitudes: one sub-block per thread for 4-qubit groups
  const int iters = KG >= 4 ? 1 : (nsub + kFThreads - 1) / kFThreads;
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < iters; ++it) {
    const int s = threadIdx.x + it * kFThreads;
    const bool live = s < nsub;
    int b = live ? s : 0;
#pragma unroll
    for (int i = 0; i < KG; ++i) b = ((b & ~lm[i]) << 1) | (b & lm[i]);
    const int sb = swz<R>(b);
    R re[2][D], im[2][D];  // [0] psi, [1] lambda
#pragma unroll
    for (int r = 0; r < D; ++r) {
      const V2 v = smp[sb ^ SV_ADJ_OFF(r)], w = sml[sb ^ SV_ADJ_OFF(r)];
      re[0][r] = v.x;
      im[0][r] = v.y;
      re[1][r] = w.x;
      im[1][r] = w.y;
    }
    R(&pr)[D] = re[0];
    R(&pi)[D] = im[0];
    R(&lr)[D] = re[1];
    R(&li)[D] = im[1];
    for (int o = o0; o < o1; ++o) {
      const FOpDev<R>& op = ops[o];
      if (op.type == FG_GRAD) {
        const int j0 = op.pad[0] | (op.pad[1] << 8), ng = op.pad[2];
        const int cm = op.cmask, pa = op.cls;
        if (ng == 1 && pa != 0) {  // one Pauli generator: 4 FMAs per pair
          R c = 0;
          if (live) {
            switch (op.b0) {
              case 0: c = grad_pairs<KG, 0, R>(pa, cm, op.m, pr, pi, lr, li); break;
              case 1: if constexpr (KG > 1) c = grad_pairs<KG, (KG > 1 ? 1 : 0), R>(pa, cm, op.m, pr, pi, lr, li); break;
              case 2: if constexpr (KG > 2) c = grad_pairs<KG, (KG > 2 ? 2 : 0), R>(pa, cm, op.m, pr, pi, lr, li); break;
              default: if constexpr (KG > 3) c = grad_pairs<KG, (KG > 3 ? 3 : 0), R>(pa, cm, op.m, pr, pi, lr, li); break;
            }
          }
#pragma unroll
          for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
          if (lane == 0) kahan_add(gw[j0], c);
        } else {  // general generator(s): the four sums, then each gradient from them
          R q[4] = {0, 0, 0, 0};
          if (live) {
            if (cm)
              grad_quad_at<KG, true, R>(op.b0, cm, pr, pi, lr, li, q);
            else
              grad_quad_at<KG, false, R>(op.b0, cm, pr, pi, lr, li, q);
          }
          if (ng == 1) {
            R c = op.m[0] * q[0] + op.m[1] * q[1] + op.m[2] * q[2] + op.m[3] * q[3];
#pragma unroll
            for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
            if (lane == 0) kahan_add(gw[j0], c);
          } else {
            R v[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const R* gm = gcoef + 4 * (j0 + (i < ng ? i : 0));
              const R c = gm[0] * q[0] + gm[1] * q[1] + gm[2] * q[2] + gm[3] * q[3];
              v[i] = i < ng ? c : R(0);
            }
            const R w = warp_sum4<R>(v, lane);
            if ((lane & 7) == 0 && (lane >> 3) < ng) kahan_add(gw[j0 + (lane >> 3)], w);
          }
        }
      } else {
        apply_op<KG, 2, R>(op, re, im);
      }
    }
    if (live) {
#pragma unroll
      for (int r = 0; r < D; ++r) {
        V2 v, w;
        v.x = pr[r];
        v.y = pi[r];
        w.x = lr[r];
        w.y = li[r];
        int o2;
        if constexpr (kTable) {
          o2 = sb ^ soff[kTable ? r : 0];
        } else {
          // an opaque copy of sb: the store addresses are recomputed here
          // instead of being kept live from the loads across every operation
          // (16 registers that pushed the 4-qubit tiles into spills)
          int sbr = sb;
          asm volatile("mov.b32 %0, %1;" : "=r"(sbr) : "r"(sb));
          o2 = sbr ^ reg_off<KG>(r, sw);
        }
        smp[o2] = v;
        sml[o2] = w;
      }
    }
  }
#undef SV_ADJ_OFF
}

template <int RANK>
__device__ __forceinline__ void load_pair(uint32_t d1, uint32_t d2, const CUtensorMap* m1,
                                          const CUtensorMap* m2, const int* c, uint32_t bar) {
  tma_load<RANK>(d1, m1, c, bar);
  tma_load<RANK>(d2, m2, c, bar);
}

template <int RANK>
__device__ __forceinline__ void store_pair(uint32_t s1, uint32_t s2, const CUtensorMap* m1,
                                           const CUtensorMap* m2, const int* c) {
  tma_store<RANK>(m1, c, s1);
  tma_store<RANK>(m2, c, s2);
}

// Shared memory of a reverse-sweep block after its two slices: the per-warp
// gradient accumulators, then the operation list, then the gradient
// generators (each part 16-byte aligned).
template <typename R>
__host__ __device__ constexpr size_t adj_ops_offset(int ngrad) {
  return (sizeof(KahanAcc<R>) * (kFThreads / 32) * (size_t)ngrad + 15) & ~size_t(15);
}
template <typename R>
__host__ __device__ constexpr size_t adj_coef_offset(int ngrad, int nops) {
  return (adj_ops_offset<R>(ngrad) + sizeof(FOpDev<R>) * (size_t)nops + 15) & ~size_t(15);
}
template <typename R>
__host__ __device__ constexpr size_t adj_tail_bytes(int ngrad, int nops) {
  return adj_coef_offset<R>(ngrad, nops) + sizeof(R) * 4 * (size_t)ngrad;
}

// Reverse-sweep pass: as kfused_tma, staging the psi slice (tmap) and the
// lambda slice (tmap2) on one mbarrier.  Gradient sums: per warp and
// gradient operation a compensated sum in shared memory, then per block
// (warps in order, fp64) into partials[gslot[j] * pstride + blockIdx.x].
template <typename R, int KGF, int MINB>
__global__ void __launch_bounds__(kFThreads, MINB)
    kfused_adj(uint64_t n_blocks, const __grid_constant__ FusedParams<R> P,
               double* __restrict__ partials, int pstride) {
  typedef typename Cplx2<R>::T V2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t sbuf = (raw + 1023u) & ~1023u;
  const uint32_t sbuf2 = sbuf + P.slice_bytes;  // slice bytes are a multiple of 1024
  V2* smp = reinterpret_cast<V2*>(smem_raw + (sbuf - raw));
  V2* sml = reinterpret_cast<V2*>(smem_raw + (sbuf2 - raw));
  KahanAcc<R>* gacc = reinterpret_cast<KahanAcc<R>*>(smem_raw + (sbuf2 - raw) + P.slice_bytes);
  constexpr int nw = kFThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < nw * P.ngrad; i += kFThreads) gacc[i] = KahanAcc<R>{0, 0};
  // the operation list and the gradient generators beside the accumulators:
  // every thread reads them per operation, from shared memory rather than
  // the parameter space
  unsigned char* tail = reinterpret_cast<unsigned char*>(gacc);
  FOpDev<R>* osm = reinterpret_cast<FOpDev<R>*>(tail + adj_ops_offset<R>(P.ngrad));
  R* gsm = reinterpret_cast<R*>(tail + adj_coef_offset<R>(P.ngrad, P.gop[P.ngroups]));
  for (int i = threadIdx.x; i < P.gop[P.ngroups]; i += kFThreads) osm[i] = P.ops[i];
  for (int i = threadIdx.x; i < 4 * P.ngrad; i += kFThreads) gsm[i] = P.coef[i];
  const uint32_t barp = smem_addr(&bar);
  if (threadIdx.x == 0) {
    mbar_init(barp, 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  uint32_t parity = 0;
  for (uint64_t blk = blockIdx.x; blk < n_blocks; blk += gridDim.x) {
    const uint64_t base = insert_zeros(blk, P.blk);
    if (threadIdx.x < 32) {
      bulk_wait_read_all();
      __syncwarp();
      if (lane == 0) mbar_arrive_expect_tx(barp, 2 * P.slice_bytes);
      __syncwarp();
      for (int k = lane; k < P.ncopies; k += 32) {
        int c[5];
        box_coords(P, base, k, c);
        const uint32_t off = (uint32_t)k * P.box_bytes;
        switch (P.rank) {
          case 2: load_pair<2>(sbuf + off, sbuf2 + off, &P.tmap, &P.tmap2, c, barp); break;
          case 3: load_pair<3>(sbuf + off, sbuf2 + off, &P.tmap, &P.tmap2, c, barp); break;
          case 4: load_pair<4>(sbuf + off, sbuf2 + off, &P.tmap, &P.tmap2, c, barp); break;
          default: load_pair<5>(sbuf + off, sbuf2 + off, &P.tmap, &P.tmap2, c, barp); break;
        }
      }
      prefetch_next(P, blk, n_blocks, lane, true);
    }
    const bool ok = mbar_wait_bounded(barp, parity);
    parity ^= 1;
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicOr(&g_fused_status, kWaitTimeout);
      break;
    }
    for (int g = 0; g < P.ngroups; ++g) {
      run_group_adj<KGF, R>(smp, sml, P.m, P.gbits[g], osm, P.gop[g], P.gop[g + 1], gsm,
                            gacc + warp * P.ngrad);
      if (g + 1 < P.ngroups) __syncthreads();
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x < 32) {
      for (int k = lane; k < P.ncopies; k += 32) {
        int c[5];
        box_coords(P, base, k, c);
        const uint32_t off = (uint32_t)k * P.box_bytes;
        switch (P.rank) {
          case 2: store_pair<2>(sbuf + off, sbuf2 + off, &P.tmap, &P.tmap2, c); break;
          case 3: store_pair<3>(sbuf + off, sbuf2 + off, &P.tmap, &P.tmap2, c); break;
          case 4: store_pair<4>(sbuf + off, sbuf2 + off, &P.tmap, &P.tmap2, c); break;
          default: store_pair<5>(sbuf + off, sbuf2 + off, &P.tmap, &P.tmap2, c); break;
        }
      }
      bulk_commit();
    }
  }
  if (threadIdx.x < 32) bulk_wait_all();
  __syncthreads();
  for (int j = threadIdx.x; j < P.ngrad; j += kFThreads) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) {
      const KahanAcc<R> a = gacc[w * P.ngrad + j];
      t += (double)a.s - (double)a.c;
    }
    partials[(size_t)P.gslot[j] * pstride + blockIdx.x] = t;
  }
}

}  // namespace

// ---- host: local order, TMA geometry, parameters -----------------------------------
// TMA view of the state in 8-byte words (w = 1 or 2 per amplitude, lw =
// log2 w): dim 0 = the 16 words of a 128-byte row, dim 1 = rows (amplitude
// bits [4 - lw, thi[1])), dims 2.. = chosen runs of staged bits, each
// spanning up to the next chosen run (the last up to n).  Box: the whole row,
// the low run, the chosen runs.  Fails (fallback kernel) if the low run is
// shorter than a row or a box is smaller than 1024 bytes.
bool tma_geometry(const std::vector<int>& S, int L, int n, int lw, TmaGeom* g) {
  const int lo1 = 4 - lw;  // amplitude bits inside one row
  if (L < lo1 || n > 34) return false;
  const int d1 = std::min(L - lo1, 8);  // rows of the low run in one box (box dim <= 256)
  struct Run {
    int start, len;
  };
  std::vector<int> hi;
  for (int b : S)
    if (b >= lo1 + d1) hi.push_back(b);
  std::vector<Run> runs;
  for (size_t i = 0; i < hi.size();) {
    size_t j = i;
    while (j + 1 < hi.size() && hi[j + 1] == hi[j] + 1 && (int)(j + 1 - i) < 8) ++j;
    runs.push_back({hi[i], (int)(j - i + 1)});
    i = j + 1;
  }
  std::vector<int> idx(runs.size());
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return runs[a].len > runs[b].len; });
  std::vector<Run> chosen;
  std::vector<char> is_chosen(runs.size(), 0);
  for (size_t i = 0; i < idx.size() && i < 3; ++i) is_chosen[idx[i]] = 1;
  for (size_t i = 0; i < runs.size(); ++i)
    if (is_chosen[i]) chosen.push_back(runs[i]);
  if (chosen.size() > 3) return false;
  g->rank = 2 + (int)chosen.size();
  g->dims[0] = 16;
  g->box[0] = 16;
  g->tlo[1] = lo1;
  g->thi[1] = chosen.empty() ? n : chosen[0].start;
  g->dims[1] = uint64_t(1) << (g->thi[1] - lo1);
  g->box[1] = 1u << d1;
  g->strides[0] = 128;
  int bits = lo1 + d1;
  for (size_t i = 0; i < chosen.size(); ++i) {
    const int d = 2 + (int)i;
    g->tlo[d] = chosen[i].start;
    g->thi[d] = i + 1 < chosen.size() ? chosen[i + 1].start : n;
    g->dims[d] = uint64_t(1) << (g->thi[d] - g->tlo[d]);
    g->box[d] = 1u << chosen[i].len;
    g->strides[d - 1] = (uint64_t(8) << lw) << chosen[i].start;
    bits += chosen[i].len;
  }
  g->box_bits = bits;
  if (bits + lw + 3 < 10) return false;  // box of >= 1024 bytes keeps every box 1024-aligned
  g->order.clear();
  g->sw.clear();
  for (int b = 0; b < lo1 + d1; ++b) g->order.push_back(b);
  for (const Run& r : chosen)
    for (int b = r.start; b < r.start + r.len; ++b) g->order.push_back(b);
  for (size_t i = 0; i < runs.size(); ++i)
    if (!is_chosen[i])
      for (int b = runs[i].start; b < runs[i].start + runs[i].len; ++b) {
        g->order.push_back(b);
        g->sw.push_back(b);
      }
  return (int)g->order.size() == (int)S.size() && g->sw.size() <= 12;
}

// Host check of the geometry against the kernel's coordinate formula for
// the given slice: every box lies inside the tensor, its start address is the
// slice base with the box's software bits, and the boxes' local indices map
// one-to-one onto the slice's amplitudes.
bool verify_tma(const TmaGeom& g, const std::vector<int>& S, int n, int lw, uint64_t blk) {
  std::vector<int> sorted = S;
  std::sort(sorted.begin(), sorted.end());
  uint64_t base = 0;  // insert zeros at the staged bits into blk
  {
    uint64_t u = blk;
    int ui = 0;
    for (int b = 0; b < n; ++b) {
      if (std::binary_search(sorted.begin(), sorted.end(), b)) continue;
      if ((u >> ui) & 1) base |= uint64_t(1) << b;
      ++ui;
    }
  }
  const int ncop = 1 << (int)g.sw.size();
  const uint64_t word = uint64_t(8);
  for (int k = 0; k < ncop; ++k) {
    uint64_t a = base;
    for (size_t j = 0; j < g.sw.size(); ++j)
      if ((k >> j) & 1) a |= uint64_t(1) << g.sw[j];
    uint64_t bytes = 0;
    for (int d = 1; d < g.rank; ++d) {
      const uint64_t c = (a & ((uint64_t(1) << g.thi[d]) - 1)) >> g.tlo[d];
      if (c > 0x7fffffffull || c + g.box[d] > g.dims[d]) return false;
      bytes += c * g.strides[d - 1];
    }
    if (bytes != (a << lw) * word) return false;
  }
  // local index -> amplitude offset is a bijection onto the staged bits
  uint64_t all = 0;
  for (int b : g.order) {
    if (all & (uint64_t(1) << b)) return false;
    all |= uint64_t(1) << b;
  }
  for (int b : S)
    if (!(all & (uint64_t(1) << b))) return false;
  return true;
}

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
  });
  return fn;
}

bool build_slice(const TmaGeom& g, const std::vector<int>& S, int n, int lw, void* data,
                 SliceDev* d) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(data) & 15) || g.rank < 2 || g.rank > 5) return false;
  if (!verify_tma(g, S, n, lw, 0) ||
      !verify_tma(g, S, n, lw, (uint64_t(1) << (n - (int)S.size())) - 1))
    return false;
  cuuint64_t dims[5], strides[4];
  cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
  for (int k = 0; k < g.rank; ++k) {
    dims[k] = g.dims[k];
    box[k] = g.box[k];
    if (k + 1 < g.rank) strides[k] = g.strides[k];
  }
  const uint64_t run_bytes = uint64_t(g.box[1]) * 128;
  const CUtensorMapL2promotion prom = run_bytes >= 256 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B
                                                       : CU_TENSOR_MAP_L2_PROMOTION_L2_128B;
  if (fn(&d->tmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, (cuuint32_t)g.rank, data, dims, strides, box,
         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, prom,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  if ((int)g.sw.size() > 12 || (int)S.size() > 24) return false;
  *reinterpret_cast<Ins<uint64_t>*>(&d->blk) = make_ins<uint64_t>(S);
  d->m = (int)S.size();
  d->rank = g.rank;
  for (int k = 0; k < 5; ++k) {
    d->tlo[k] = (uint8_t)g.tlo[k];
    d->thi[k] = (uint8_t)g.thi[k];
  }
  d->nsw = (int)g.sw.size();
  for (int j = 0; j < d->nsw; ++j) d->swpos[j] = (uint8_t)g.sw[j];
  d->ncopies = 1 << d->nsw;
  d->box_bytes = (uint32_t)((8u << lw) << g.box_bits);
  d->slice_bytes = d->box_bytes * (uint32_t)d->ncopies;
  return true;
}

namespace {

template <typename R>
bool build_tma(const TmaGeom& g, void* data, FusedParams<R>* P, CUtensorMap* map = nullptr) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(data) & 15)) return false;
  if (!map) map = &P->tmap;
  cuuint64_t dims[5], strides[4];
  cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
  for (int d = 0; d < g.rank; ++d) {
    dims[d] = g.dims[d];
    box[d] = g.box[d];
    if (d + 1 < g.rank) strides[d] = g.strides[d];
  }
  // the low run is 2^L amplitudes: fetch from DRAM at up to 256 bytes
  const uint64_t run_bytes = uint64_t(g.box[1]) * 128;
  const CUtensorMapL2promotion prom = run_bytes >= 256 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B
                                                       : CU_TENSOR_MAP_L2_PROMOTION_L2_128B;
  if (fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, (cuuint32_t)g.rank, data, dims, strides, box,
         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, prom,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  P->rank = g.rank;
  for (int d = 0; d < 5; ++d) {
    P->tlo[d] = (uint8_t)g.tlo[d];
    P->thi[d] = (uint8_t)g.thi[d];
  }
  P->nsw = (int)g.sw.size();
  if (P->nsw > 12) return false;
  for (int j = 0; j < P->nsw; ++j) P->swpos[j] = (uint8_t)g.sw[j];
  P->ncopies = 1 << P->nsw;
  P->box_bytes = (uint32_t)((sizeof(R) * 2) << g.box_bits);
  P->slice_bytes = P->box_bytes * (uint32_t)P->ncopies;
  return true;
}

// Rewrites group g, if its gates are uncontrolled 1-qubit gates and diagonal
// gates (phases on subspaces, controlled diagonal 1-qubit gates), as a layer
// program: a 1-qubit gate joins the open layer unless the layer's diagonal
// already touches its bit (then a new layer starts); consecutive 1-qubit
// gates on one bit multiply; diagonal gates multiply into the layer's
// diagonal.  All products in fp64; the coefficients are rounded with the
// state's error feedback (drift; the layers' 2x2s and diagonals act on the
// whole state).  With rotform every dense 2x2 is split into a scaled real
// rotation between diagonals (see rotation_form below).  Returns 0 (and
// leaves nl, nc) if the group keeps its gate list, 2 for a layer program in
// rotation form throughout, 1 for one with dense 2x2s.
template <typename R>
int layer_group(const FusedPass& pass, int g, const int* pos_of, FusedParams<R>* P, int* nlp,
                int* ncp, double* drift, bool rotform) {
  struct LayerH {
    int u1 = 0, dtouch = 0;
    int rot = 0, form = 0;  // rotation form: bits with scaled rotations tau[i]
    double tau[5] = {0, 0, 0, 0, 0};
    double msq = 1.0;  // exact mean squared modulus of Dg
    cd U[5][4];
    cd Dg[32];
    LayerH() {
      for (int r = 0; r < 32; ++r) Dg[r] = {1.0, 0.0};
    }
    bool empty() const { return !u1 && !dtouch; }
  };
  auto cmul = [](cd a, cd b) { return cd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; };
  auto cdiv = [](cd x, cd y) {
    const double d = y.re * y.re + y.im * y.im;
    return cd{(x.re * y.re + x.im * y.im) / d, (x.im * y.re - x.re * y.im) / d};
  };
  auto scl = [](cd x, double f) { return cd{x.re * f, x.im * f}; };
  // U = diag(a) S diag(b), S = [[1, -tau], [tau, 1]] (form 0, |u00| >= |u01|)
  // or [[tau, -1], [1, tau]] (form 1), tau <= 1 (a ZYZ Euler split:
  // U = e^{i phi} RZ RY RZ with RY = cos [[1, -tan], [tan, 1]]).  False if U
  // is not unitary or the split does not reproduce it to 1e-12.
  auto decompose = [&](const cd* u, cd* a, cd* b, double* tau, int* form) {
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        double re = 0, im = 0;
        for (int r = 0; r < 2; ++r) {  // (U^dagger U)_ij
          const cd x = u[r * 2 + i], y = u[r * 2 + j];
          re += x.re * y.re + x.im * y.im;
          im += x.re * y.im - x.im * y.re;
        }
        if (std::fabs(re - (i == j ? 1.0 : 0.0)) > 1e-12 || std::fabs(im) > 1e-12) return false;
      }
    const double c = std::hypot(u[0].re, u[0].im), s = std::hypot(u[1].re, u[1].im);
    if (c >= s) {
      *form = 0;
      *tau = s / c;
      a[0] = u[0];
      b[0] = {1.0, 0.0};
      if (s == 0) {
        b[1] = {1.0, 0.0};
        a[1] = u[3];
      } else {
        b[1] = scl(cdiv(u[1], scl(a[0], *tau)), -1.0);
        a[1] = cdiv(u[3], b[1]);
      }
    } else {
      *form = 1;
      *tau = c / s;
      b[1] = {1.0, 0.0};
      a[0] = scl(u[1], -1.0);
      if (c == 0) {
        b[0] = {1.0, 0.0};
        a[1] = u[2];
      } else {
        b[0] = cdiv(u[0], scl(a[0], *tau));
        a[1] = cdiv(u[2], b[0]);
      }
    }
    const double S[4] = {*form ? *tau : 1.0, -(*form ? 1.0 : *tau), *form ? 1.0 : *tau,
                         *form ? *tau : 1.0};
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        const cd v = scl(cmul(a[i], b[j]), S[i * 2 + j]);
        if (std::fabs(v.re - u[i * 2 + j].re) > 1e-12 || std::fabs(v.im - u[i * 2 + j].im) > 1e-12)
          return false;
      }
    return true;
  };
  // The layers in rotation form: each dense 2x2 of layer l becomes
  // A_l S_l B_l; diagonals commute, so B_0 runs first as a diagonal-only
  // layer and layer l becomes the rotations S_l and the one diagonal
  // E_l = B_{l+1} Dg_l A_l.  tau is rounded to the state's precision and A
  // rescaled so that A S B stays unitary in fp64 (the rounding moves the
  // rotation angle, not the norm).  False (nothing changed) if some 2x2 is
  // not unitary.
  auto rotation_form = [&](const std::vector<LayerH>& in, int k, std::vector<LayerH>* out,
                           int* xmask) {
    const int D = 1 << k;
    const size_t NL = in.size();
    std::vector<std::array<cd, 32>> A(NL), B(NL);
    std::vector<LayerH> mid(NL);
    for (size_t l = 0; l < NL; ++l) {
      for (int r = 0; r < D; ++r) A[l][r] = B[l][r] = {1.0, 0.0};
      const LayerH& h = in[l];
      LayerH& o = mid[l];
      o.rot = h.u1;
      for (int t = 0; t < k; ++t) {
        if (!((h.u1 >> t) & 1)) continue;
        cd a[2], b[2];
        double tau;
        int f;
        if (!decompose(h.U[t], a, b, &tau, &f)) return false;
        const double tr = (double)(R)tau;
        const double sc = std::sqrt((1.0 + tau * tau) / (1.0 + tr * tr));
        a[0] = scl(a[0], sc);
        a[1] = scl(a[1], sc);
        o.tau[t] = tr;
        if (f) o.form |= 1 << t;
        for (int r = 0; r < D; ++r) {
          A[l][r] = cmul(A[l][r], a[(r >> t) & 1]);
          B[l][r] = cmul(B[l][r], b[(r >> t) & 1]);
        }
      }
    }
    out->clear();
    bool id = true;
    for (int r = 0; r < D; ++r)
      if (B[0][r].re != 1.0 || B[0][r].im != 0.0) id = false;
    if (!id) {
      LayerH f0;
      for (int r = 0; r < D; ++r) f0.Dg[r] = B[0][r];
      out->push_back(f0);
    }
    for (size_t l = 0; l < NL; ++l) {
      LayerH o = mid[l];
      double msq = 0.0;
      for (int r = 0; r < D; ++r) {
        cd e = cmul(in[l].Dg[r], A[l][r]);
        if (l + 1 < NL) e = cmul(B[l + 1][r], e);
        o.Dg[r] = e;
        msq += e.re * e.re + e.im * e.im;
      }
      o.msq = msq / D;
      out->push_back(o);
    }
    // One rotation shape on the device: [[t, -1], [1, t]] = X Z S(-t) with
    // S(t) = [[1, -t], [t, 1]].  X on a bit relabels the registers instead of
    // moving them (mask M: register p holds logical index p ^ M; X S(t) X =
    // S(-t), so a rotation on a flipped bit negates t); the layer's X's come
    // after its rotations (other bits commute), and X Z = -Z X puts -Z into
    // the layer's diagonal, which is then read at p ^ M.  The group's stores
    // undo M.
    int M = 0;
    for (LayerH& o : *out) {
      const int F = o.form;
      for (int t = 0; t < k; ++t)
        if ((o.rot >> t) & 1)
          o.tau[t] *= (((F ^ M) >> t) & 1) ? -1.0 : 1.0;
      cd Dl[32];
      for (int r = 0; r < D; ++r) {
        Dl[r] = o.Dg[r];
        for (int t = 0; t < k; ++t)
          if ((F >> t) & 1) Dl[r] = scl(Dl[r], ((r >> t) & 1) ? 1.0 : -1.0);  // -Z_t
      }
      M ^= F;
      for (int p = 0; p < D; ++p) o.Dg[p] = Dl[p ^ M];
      o.form = 0;
    }
    *xmask = M;
    return true;
  };
  int& nl = *nlp;
  int& nc = *ncp;
  const int cap = (int)(sizeof(P->coef) / sizeof(R));
  {
    const FusedGroup& grp = pass.groups[g];
    const int k = grp.k, D = 1 << k;
    // convertible: uncontrolled or diagonal 1-qubit gates and phases only
    bool conv = true;
    for (int oi : grp.ops) {
      const FGate& f = pass.gates[oi];
      const bool diag1 = f.type == FG_1Q && f.m[1].re == 0 && f.m[1].im == 0 && f.m[2].re == 0 &&
                         f.m[2].im == 0;
      if (!(f.type == FG_PHASE || (f.type == FG_1Q && (f.cmask == 0 || diag1)))) conv = false;
    }
    if (!conv) return 0;
    int lb[5];
    for (int i = 0; i < k; ++i) lb[i] = pos_of[pass.S[grp.bits[i]]];
    std::sort(lb, lb + k);
    auto gl = [&](int bit) {
      for (int i = 0; i < k; ++i)
        if (lb[i] == pos_of[bit]) return i;
      return -1;
    };
    auto glmask = [&](uint64_t mask) {
      int r = 0;
      for (int b = 0; b < 64; ++b)
        if ((mask >> b) & 1) r |= 1 << gl(b);
      return r;
    };
    std::vector<LayerH> L(1);
    int gxm = 0;  // the rotation form's final register relabelling
    bool ok = true;
    for (int oi : grp.ops) {
      const FGate& f = pass.gates[oi];
      LayerH* cur = &L.back();
      if (f.type == FG_1Q) {
        const int t = gl(f.t), cm = glmask(f.cmask);
        const bool diag = f.m[1].re == 0 && f.m[1].im == 0 && f.m[2].re == 0 && f.m[2].im == 0;
        if (diag) {
          for (int r = 0; r < D; ++r)
            if ((r & cm) == cm) cur->Dg[r] = cmul(((r >> t) & 1) ? f.m[3] : f.m[0], cur->Dg[r]);
          cur->dtouch |= cm | (1 << t);
        } else if (cm == 0) {
          if ((cur->dtouch >> t) & 1) {
            L.emplace_back();
            cur = &L.back();
          }
          if ((cur->u1 >> t) & 1) {
            cd r4[4];
            for (int i = 0; i < 2; ++i)
              for (int j = 0; j < 2; ++j) {
                const cd a = cmul(f.m[i * 2], cur->U[t][j]), b = cmul(f.m[i * 2 + 1], cur->U[t][2 + j]);
                r4[i * 2 + j] = {a.re + b.re, a.im + b.im};
              }
            for (int e = 0; e < 4; ++e) cur->U[t][e] = r4[e];
          } else {
            for (int e = 0; e < 4; ++e) cur->U[t][e] = f.m[e];
            cur->u1 |= 1 << t;
          }
        } else {
          ok = false;
        }
      } else if (f.type == FG_PHASE) {
        const int cm = glmask(f.cmask);
        for (int r = 0; r < D; ++r)
          if ((r & cm) == cm) cur->Dg[r] = cmul(f.m[0], cur->Dg[r]);
        cur->dtouch |= cm;
      } else {
        ok = false;
      }
      if (!ok) break;
    }
    if (!ok) return 0;
    if (L.back().empty()) L.pop_back();
    if (rotform) {
      std::vector<LayerH> R2;
      int xm = 0;
      if (rotation_form(L, k, &R2, &xm)) {
        L.swap(R2);
        gxm = xm;
      }
    }
    // coefficient count and capacity
    int need = 0;
    std::vector<int> dks;
    for (const LayerH& h : L) {
      bool one = true, real = true;
      for (int r = 0; r < D; ++r) {
        if (h.Dg[r].re != 1.0 || h.Dg[r].im != 0.0) one = false;
        if (h.Dg[r].im != 0.0) real = false;
      }
      const int dk = one ? 0 : real ? 1 : 2;
      dks.push_back(dk);
      need += h.rot ? 4 : 0;
      need += 8 * __builtin_popcount(h.u1);
      need += dk == 0 ? 0 : dk == 1 ? D : 2 * D;
      need = (need + 3) & ~3;  // 16-byte alignment of the next layer (float)
    }
    if (nl + (int)L.size() > kFMaxLayers || nc + need > cap) return 0;
    double* fb = sizeof(R) == 4 ? drift : nullptr;
    for (size_t li = 0; li < L.size(); ++li) {
      LayerH& h = L[li];
      FLayerDev& d = P->layers[nl++];
      d.u1 = (uint8_t)h.u1;
      d.dk = (uint8_t)dks[li];
      d.off = (uint16_t)nc;
      d.rot = (uint8_t)h.rot;
      d.pad8 = 0;
      d.pad = 0;
      if (h.rot) {  // tau of bit i in slot i (0 where bit i has no rotation)
        for (int i = 0; i < 4; ++i) P->coef[nc++] = ((h.rot >> i) & 1) ? (R)h.tau[i] : R(0);
      }
      for (int i = 0; i < k; ++i)
        if ((h.u1 >> i) & 1) {
          feedback_round(h.U[i], 2, fb);
          for (int e = 0; e < 4; ++e) {
            P->coef[nc++] = (R)h.U[i][e].re;
            P->coef[nc++] = (R)h.U[i][e].im;
          }
        }
      if (dks[li] == 1) {  // real entries (+-1 in gate-list form: exact)
        feedback_round_diag(h.Dg, D, fb, h.msq);
        for (int r = 0; r < D; ++r) P->coef[nc++] = (R)h.Dg[r].re;
      } else if (dks[li] == 2) {
        feedback_round_diag(h.Dg, D, fb, h.msq);
        for (int r = 0; r < D; ++r) {
          P->coef[nc++] = (R)h.Dg[r].re;
          P->coef[nc++] = (R)h.Dg[r].im;
        }
      }
      while (nc & 3) P->coef[nc++] = 0;
    }
    bool dense = false;
    for (const LayerH& h : L) dense = dense || h.u1 != 0;
    P->gxm[g] = (uint8_t)gxm;
    return dense ? 1 : 2;
  }
}

// order: the staged bits in local order (order[0..L) = 0..L-1).  forward:
// a forward pass (groups may become layer programs; complex64 coefficients of
// operations on the whole state are rounded with the error feedback drift);
// otherwise a reverse-sweep pass (gate lists, plain rounding).
template <typename R>
bool build_params(const FusedPass& pass, const std::vector<int>& order, FusedParams<R>* P,
                  bool forward = true, double* drift = nullptr, bool rotform = false) {
  P->ngrad = 0;
  P->extra_tx = 0;
  P->dseed = 0;
  const std::vector<int>& S = pass.S;
  P->m = (int)S.size();
  P->L = pass.L;
  P->nh = P->m - pass.L;
  if (P->m > 24 || P->nh > 32 || (int)order.size() != P->m) return false;
  *reinterpret_cast<Ins<uint64_t>*>(&P->blk) = make_ins<uint64_t>(S);
  for (int i = 0; i < P->nh; ++i) P->hpos[i] = (uint8_t)order[pass.L + i];
  int pos_of[64];
  for (int b = 0; b < 64; ++b) pos_of[b] = 0;
  for (int i = 0; i < P->m; ++i) pos_of[order[i]] = i;
  if ((int)pass.groups.size() > kFMaxGroups) return false;
  P->ngroups = (int)pass.groups.size();
  int nop = 0;
  for (int g = 0; g < P->ngroups; ++g) {
    const FusedGroup& grp = pass.groups[g];
    // the group's bits in local order, ascending (zero-bit insertion order)
    int lb[5];
    for (int i = 0; i < grp.k; ++i) lb[i] = pos_of[S[grp.bits[i]]];
    std::sort(lb, lb + grp.k);
    P->gk[g] = (uint8_t)grp.k;
    for (int i = 0; i < 5; ++i) P->gbits[g][i] = (uint8_t)(i < grp.k ? lb[i] : 0);
    P->gop[g] = (uint16_t)nop;
    // global bit -> index within the group
    auto gl = [&](int bit) {
      for (int i = 0; i < grp.k; ++i)
        if (lb[i] == pos_of[bit]) return i;
      return -1;
    };
    auto glmask = [&](uint64_t mask) {
      int r = 0;
      for (int b = 0; b < 64; ++b)
        if ((mask >> b) & 1) r |= 1 << gl(b);
      return r;
    };
    for (int oi : grp.ops) {
      if (nop >= kFMaxOps) return false;
      const FGate& f = pass.gates[oi];
      FOpDev<R>& o = P->ops[nop++];
      o.type = (uint8_t)f.type;
      o.b0 = o.b1 = 0;
      o.cmask = (uint8_t)glmask(f.cmask);
      o.cls = 0;
      o.pad[0] = o.pad[1] = o.pad[2] = 0;
      for (int e = 0; e < 8; ++e) o.m[e] = 0;
      if (f.type == FG_1Q) {
        o.b0 = (uint8_t)gl(f.t);
        const cd* g = f.m;
        auto z = [](cd x) { return x.re == 0.0 && x.im == 0.0; };
        if (z(g[1]) && z(g[2]))
          o.cls = MK_DIAG;
        else if (g[0].im == 0 && g[1].im == 0 && g[2].im == 0 && g[3].im == 0)
          o.cls = MK_REAL;
        else if (g[0].im == 0 && g[3].im == 0 && g[1].re == 0 && g[2].re == 0)
          o.cls = MK_IMOFF;
        else
          o.cls = MK_DENSE;
        for (int e = 0; e < 4; ++e) {
          o.m[2 * e] = (R)f.m[e].re;
          o.m[2 * e + 1] = (R)f.m[e].im;
        }
      } else if (f.type == FG_PHASE) {
        o.m[0] = (R)f.m[0].re;
        o.m[1] = (R)f.m[0].im;
        o.cls = (f.m[0].re == -1.0 && f.m[0].im == 0.0) ? 1 : 0;
      } else if (f.type == FG_GRAD) {
        // generator(s) on bit t within the control mask; first local gradient
        // index in pad[0..1], count in pad[2]
        o.b0 = (uint8_t)gl(f.t);
        o.cls = (uint8_t)(f.ng == 1 ? f.pauli : 0);
        if (f.ng == 1 && !f.pauli) {  // Hermitian generator [[a, b], [conj b, d]]
          o.m[0] = (R)f.m[0].re;
          o.m[1] = (R)f.m[3].re;
          o.m[2] = (R)f.m[1].re;
          o.m[3] = (R)f.m[1].im;
        }
        const int j = P->ngrad;
        if (f.ng < 1 || f.ng > kGradPerOp || j + f.ng > kFMaxOps) return false;
        P->ngrad += f.ng;
        o.pad[0] = (uint8_t)(j & 0xff);
        o.pad[1] = (uint8_t)(j >> 8);
        o.pad[2] = (uint8_t)f.ng;
        if (f.ng == 1) {
          P->gslot[j] = f.slot;
        } else {  // generators of the shared evaluation in coef[4 j ...]
          for (int i = 0; i < f.ng; ++i) {
            P->gslot[j + i] = f.gslots[i];
            for (int e = 0; e < 4; ++e) P->coef[4 * (j + i) + e] = (R)f.gen[i][e];
          }
        }
      } else {
        const int x = gl(f.a), y = gl(f.b);
        o.b0 = (uint8_t)std::min(x, y);
        o.b1 = (uint8_t)std::max(x, y);
      }
    }
  }
  P->gop[P->ngroups] = (uint16_t)nop;
  if (forward && P->ngrad == 0) {
    // groups in application order, so the feedback sees the roundings in the
    // order they act on the state
    int nl = 0, nc = 0;
    double* fb = sizeof(R) == 4 ? drift : nullptr;
    for (int g = 0; g < P->ngroups; ++g) {
      P->glay[g] = (uint16_t)nl;
      P->gxm[g] = 0;
      P->gkind[g] = (uint8_t)layer_group(pass, g, pos_of, P, &nl, &nc, fb, rotform);
      if (P->gkind[g] || !fb) continue;
      const FusedGroup& grp = pass.groups[g];
      for (size_t j = 0; j < grp.ops.size(); ++j) {
        const FGate& f = pass.gates[grp.ops[j]];
        if (f.type != FG_1Q || f.cmask) continue;
        cd gm[4] = {f.m[0], f.m[1], f.m[2], f.m[3]};
        feedback_round(gm, 2, fb);
        FOpDev<R>& o = P->ops[P->gop[g] + j];
        for (int e = 0; e < 4; ++e) {
          o.m[2 * e] = (R)gm[e].re;
          o.m[2 * e + 1] = (R)gm[e].im;
        }
      }
    }
    P->glay[P->ngroups] = (uint16_t)nl;
    P->ncoef = nc;
  } else {  // reverse sweeps run gate lists; coef[] holds gradient generators
    for (int g = 0; g <= P->ngroups; ++g) P->glay[g] = 0;
    for (int g = 0; g < P->ngroups; ++g) P->gkind[g] = P->gxm[g] = 0;
    P->ncoef = 4 * P->ngrad;
  }
  return true;
}

template <typename R>
struct PassKernels {
  typedef void (*Lsu)(typename Cplx2<R>::T*, uint64_t, const FusedParams<R>);
  typedef void (*Tma)(uint64_t, const FusedParams<R>);
  static Lsu lsu(int kg) {
    return kg <= 1 ? kfused<R, 1> : kg == 2 ? kfused<R, 2> : kg == 3 ? kfused<R, 3> : kfused<R, 4>;
  }
  template <int KG, int MINB>
  static Tma pick(int mode) {
    if constexpr (sizeof(R) == 4)
      if (mode == 4) return kfused_tma<R, KG, MINB, 4>;
    return mode == 3   ? kfused_tma<R, KG, MINB, 3>
           : mode == 1 ? kfused_tma<R, KG, MINB, 1>
                       : kfused_tma<R, KG, MINB, 0>;
  }
  // mode 0: gate lists, 1: mixed, 3: layer programs only.  Measured on
  // GB300 (complex64, 4-bit groups): layer programs run fastest with the
  // register budget of 2 blocks per SM, gate lists with 3.
  static Tma tma(int kg, int mode) {
    constexpr int MB = sizeof(R) == 4 ? 3 : 2;
    if (kg == 4) return mode >= 3 ? pick<4, 2>(mode) : pick<4, MB>(mode);
    return kg <= 1 ? pick<1, MB>(mode) : kg == 2 ? pick<2, MB>(mode) : pick<3, MB>(mode);
  }
};

template <typename R>
sv_status run_pass(void* data, int n, cudaStream_t st, const FusedPass& pass, RoundCtx* rc) {
  double* drift = rc ? &rc->drift : nullptr;
  static FusedParams<R> P;  // ~8-15 KB: kept off the stack; launches are serialised per call
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  const int kg = pass.groups.empty() ? 1 : pass.groups[0].k;
  for (const FusedGroup& g : pass.groups)
    if (g.k != kg) {
      set_error("fused pass: groups of unequal width");
      return SV_ERR_INVALID;
    }
  const int lw = sizeof(R) == 4 ? 0 : 1;
  TmaGeom geo;
  bool tma = tma_geometry(pass.S, pass.L, n, lw, &geo);
  std::vector<int> order = tma ? geo.order : pass.S;
  const double drift0 = drift ? *drift : 0.0;
  // layer programs in rotation form, except where every dense 2x2 is to be
  // rounded with dither (that mode keeps the dense form)
  const bool dither_all = sizeof(R) == 4 && rc && rc->mode == SV_ROUNDING_DITHERED;
  if (!build_params(pass, order, &P, true, drift, !dither_all)) {
    set_error("fused pass exceeds kernel capacity");
    return SV_ERR_INVALID;
  }
  if (tma && !(verify_tma(geo, pass.S, n, lw, 0) &&
               verify_tma(geo, pass.S, n, lw, (uint64_t(1) << (n - (int)pass.S.size())) - 1))) {
    set_error("fused pass: inconsistent bulk-copy geometry");
    return SV_ERR_INVALID;
  }
  if (tma) tma = build_tma(geo, data, &P);
  if (!tma && order != pass.S && drift) *drift = drift0;  // rebuilt below
  if (!tma && order != pass.S && !build_params(pass, pass.S, &P, true, drift, !dither_all)) {
    set_error("fused pass exceeds kernel capacity");
    return SV_ERR_INVALID;
  }
  if (dither_all) P.dseed = rc->next_seed();
  const uint64_t nblk = uint64_t(1) << (n - P.m);
  const size_t amp = sizeof(R) * 2;
  ProfScope prof(st, sizeof(R) == 4 ? (tma ? "kfused_tma_c64" : "kfused_c64")
                                    : (tma ? "kfused_tma_c128" : "kfused_c128"));
  if (tma) {
    int nlay = 0;
    for (int g = 0; g < P.ngroups; ++g) nlay += P.gkind[g] != 0;
    const int mode = nlay == 0 ? 0 : nlay == P.ngroups ? (dither_all ? 4 : 3) : 1;
    typename PassKernels<R>::Tma kern = PassKernels<R>::tma(kg, mode);
    const size_t smem = (amp << P.m) + 1024 + sizeof(R) * (size_t)((P.ncoef + 1) & ~1) +
                        sizeof(FLayerDev) * (size_t)P.glay[P.ngroups];
    // resident blocks per SM for this kernel and shared-memory size
    static std::map<std::pair<const void*, size_t>, int> resident;
    int& res = resident[{reinterpret_cast<const void*>(kern), smem}];
    if (!res) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res, kern, kFThreads, smem) != cudaSuccess ||
          res < 1) {
        cudaGetLastError();
        res = 1;
      }
    }
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t grid = std::min<uint64_t>(nblk, (uint64_t)sms * res);
    kern<<<(unsigned)grid, kFThreads, smem, st>>>(nblk, P);
  } else {
    typename PassKernels<R>::Lsu kern = PassKernels<R>::lsu(kg);
    const size_t smem = (amp << P.m) + (sizeof(uint64_t) * (((size_t(1) << (P.m - P.L)) + 1) & ~size_t(1))) +
                        sizeof(R) * (size_t)P.ncoef;
    static bool attr_set[5] = {false, false, false, false, false};
    if (!attr_set[kg]) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr_set[kg] = true;
    }
    const uint64_t grid = std::min<uint64_t>(nblk, 152 * 16);
    kern<<<(unsigned)grid, kFThreads, smem, st>>>(
        reinterpret_cast<typename Cplx2<R>::T*>(data), nblk, P);
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return check_launch("fused pass kernel");
}

template <typename R>
bool adj_pass_ok(int n, const FusedPass& pass) {
  TmaGeom geo;
  return tma_geometry(pass.S, pass.L, n, sizeof(R) == 4 ? 0 : 1, &geo);
}

template <typename R>
sv_status run_adj_pass(void* psi, void* lam, int n, cudaStream_t st, const FusedPass& pass,
                       double* partials, int pstride) {
  static FusedParams<R> P;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  const int kg = pass.groups.empty() ? 1 : pass.groups[0].k;
  for (const FusedGroup& g : pass.groups)
    if (g.k != kg) {
      set_error("fused reverse pass: groups of unequal width");
      return SV_ERR_INVALID;
    }
  const int lw = sizeof(R) == 4 ? 0 : 1;
  TmaGeom geo;
  if (!tma_geometry(pass.S, pass.L, n, lw, &geo) || !build_params(pass, geo.order, &P, false) ||
      !verify_tma(geo, pass.S, n, lw, 0) ||
      !verify_tma(geo, pass.S, n, lw, (uint64_t(1) << (n - (int)pass.S.size())) - 1) ||
      !build_tma(geo, psi, &P) || !build_tma(geo, lam, &P, &P.tmap2)) {
    set_error("fused reverse pass: no bulk-copy geometry for this pass");
    return SV_ERR_UNSUPPORTED;
  }
  typedef void (*Kern)(uint64_t, const FusedParams<R>, double*, int);
  constexpr int MB = sizeof(R) == 4 ? 3 : 1;
  constexpr int KMAX = sizeof(R) == 4 ? 4 : 3;  // two 2^k tiles of complex128 above 3 spill
  if (kg > KMAX) {
    set_error("fused reverse pass: register groups wider than %d qubits", KMAX);
    return SV_ERR_INVALID;
  }
  if (kg >= 4 && (1 << (P.m - kg)) > kFThreads) {  // the kernel runs one sub-block per thread
    set_error("fused reverse pass: slice of 2^%d amplitudes too large for 4-qubit groups", P.m);
    return SV_ERR_INVALID;
  }
  const Kern kern = kg <= 1   ? kfused_adj<R, 1, MB>
                    : kg == 2 ? kfused_adj<R, 2, MB>
                    : kg == 3 ? kfused_adj<R, 3, MB>
                              : kfused_adj<R, (KMAX > 3 ? 4 : 3), 2>;
  const size_t smem = 1024 + 2 * (size_t)P.slice_bytes + adj_tail_bytes<R>(P.ngrad, P.gop[P.ngroups]);
  static std::map<std::pair<const void*, size_t>, int> resident;
  int& res = resident[{reinterpret_cast<const void*>(kern), smem}];
  if (!res) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res, kern, kFThreads, smem) != cudaSuccess ||
        res < 1) {
      cudaGetLastError();
      res = 1;
    }
  }
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t nblk = uint64_t(1) << (n - P.m);
  const uint64_t grid = std::min<uint64_t>({nblk, (uint64_t)sms * res, (uint64_t)pstride});
  ProfScope prof(st, sizeof(R) == 4 ? "kfused_adj_c64" : "kfused_adj_c128");
  kern<<<(unsigned)grid, kFThreads, smem, st>>>(nblk, P, partials, pstride);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return check_launch("fused reverse pass kernel");
}

static_assert(sizeof(FusedParams<double>) <= 32000, "kernel parameters above the launch limit");
static_assert(4 * kFMaxOps * sizeof(double) <= kFCoefBytes, "gradient generators exceed coef[]");
static_assert(sizeof(FusedParams<float>) <= 32000, "kernel parameters above the launch limit");

}  // namespace

bool fused_reverse_ok(sv_dtype dt, int n, const FusedPass& pass) {
  return dt == SV_C64 ? adj_pass_ok<float>(n, pass) : adj_pass_ok<double>(n, pass);
}

sv_status launch_fused_reverse_pass(void* psi, void* lam, sv_dtype dt, int n, cudaStream_t st,
                                    const FusedPass& pass, double* partials, int pstride) {
  return dt == SV_C64 ? run_adj_pass<float>(psi, lam, n, st, pass, partials, pstride)
                      : run_adj_pass<double>(psi, lam, n, st, pass, partials, pstride);
}

sv_status launch_fused_pass(void* data, sv_dtype dt, int n, cudaStream_t st,
                            const FusedPass& pass, RoundCtx* rc) {
  return dt == SV_C64 ? run_pass<float>(data, n, st, pass, rc)
                      : run_pass<double>(data, n, st, pass, nullptr);
}

// Bounded-wait self-test: one pass over the state with no gates whose
// mbarrier expects 16 bytes more than its slice, so no phase completes; every
// block gives up after the wait limit, records the timeout and exits before
// storing anything.  The state is unchanged.
template <typename R>
sv_status selftest_wait(void* data, int n, cudaStream_t st) {
  static FusedParams<R> P;
  FusedPass pass;
  const int m = std::min(n, 10);
  for (int b = 0; b < m; ++b) pass.S.push_back(b);
  pass.L = m;
  const int lw = sizeof(R) == 4 ? 0 : 1;
  TmaGeom geo;
  if (n < 10 || !tma_geometry(pass.S, pass.L, n, lw, &geo) || !build_params(pass, geo.order, &P) ||
      !build_tma(geo, data, &P)) {
    set_error("bounded-wait self-test: needs a state of at least 10 qubits");
    return SV_ERR_INVALID;
  }
  P.extra_tx = 16;
  typedef void (*Kern)(uint64_t, const FusedParams<R>);
  const Kern kern = kfused_tma<R, 1, sizeof(R) == 4 ? 3 : 2, 0>;
  const size_t smem = ((sizeof(R) * 2) << P.m) + 1024;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  const uint64_t nblk = uint64_t(1) << (n - P.m);
  kern<<<(unsigned)std::min<uint64_t>(nblk, 152), kFThreads, smem, st>>>(nblk, P);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return check_launch("bounded-wait self-test kernel");
}

sv_status launch_wait_selftest(void* data, sv_dtype dt, int n, cudaStream_t st) {
  return dt == SV_C64 ? selftest_wait<float>(data, n, st) : selftest_wait<double>(data, n, st);
}

unsigned take_fused_status() {
  unsigned v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_fused_status, sizeof(v)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (v) cudaMemcpyToSymbol(g_fused_status, &zero, sizeof(zero));
  return v;
}

}  // namespace sv
