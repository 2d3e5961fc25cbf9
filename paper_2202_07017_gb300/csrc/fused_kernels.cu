// Fused qubit-block pass: one HBM round trip for many gates.
//
// A pass stages m amplitude-index bits S (the L lowest bits, as contiguous
// runs of 2^L amplitudes, plus m - L high bits).  A thread block loads one
// 2^m-amplitude slice (all other bits fixed by the block id) into shared
// memory with coalesced 16-byte loads, applies the pass's register groups
// one after another, and writes the slice back.  In a group every thread
// pulls 2^k amplitudes that differ only in the group's k bits into
// registers, applies the group's gates there (Eq. 1 of Sec. 2 for each
// gate, with compile-time register indices) and pushes them back, so shared
// memory is touched once per group rather than once per gate.
//
// Shared-memory layout: local amplitude j (bit i of j <-> staged bit S[i])
// lives at slot j XOR-swizzled in bits 1..3 by bits 4..6 (complex64; bit 0
// kept so a 16-byte vector of two amplitudes stays contiguous) or in bits
// 0..2 by bits 3..5 (complex128), which spreads the strided register-group
// accesses of a warp over the banks.
#include <algorithm>

#include "sv_device.cuh"

namespace sv {
namespace {

constexpr int kFThreads = 256;
constexpr int kFMaxOps = 200;
constexpr int kFMaxGroups = 64;

template <typename R>
struct FOpDev {
  uint8_t type, b0, b1, cmask;  // group-local bit indices and control mask
  uint8_t cls;                  // FG_1Q: MK_* arithmetic class; FG_PHASE: 1 if the phase is -1
  uint8_t pad[3];
  R m[8];                       // FG_1Q: G00 G01 G10 G11 (re, im); FG_PHASE: m[0..1]
};

template <typename R>
struct FusedParams {
  Ins<uint64_t> blk;  // zero bits at every staged position: block id -> base index
  int m, L, nh;
  uint8_t hpos[32];   // staged bits above the low run, ascending
  int ngroups;
  uint8_t gk[kFMaxGroups];
  uint8_t gbits[kFMaxGroups][5];
  uint16_t gop[kFMaxGroups + 1];
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
// (a, b) <- G (a, b) on every register pair of group bit B; CTRL: only where
// the group-local control mask is set; MK: arithmetic class of G.
template <int KG, int B, int MK, bool CTRL, typename R>
__device__ __forceinline__ void ap1(const FOpDev<R>& op, R (&re)[1 << KG], R (&im)[1 << KG]) {
  const int cm = op.cmask;
  M2<R> g;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    g.r[e] = op.m[2 * e];
    g.i[e] = op.m[2 * e + 1];
  }
#pragma unroll
  for (int r = 0; r < (1 << KG); ++r) {
    if (r & (1 << B)) continue;
    if (CTRL && (r & cm) != cm) continue;
    const int r1 = r | (1 << B);
    mv2<MK, R>(g, re[r], im[r], re[r1], im[r1]);
  }
}

template <int KG, int B, typename R>
__device__ __forceinline__ void ap1_cls(const FOpDev<R>& op, R (&re)[1 << KG], R (&im)[1 << KG]) {
  if (op.cmask) {
    ap1<KG, B, MK_DENSE, true>(op, re, im);
    return;
  }
  switch (op.cls) {
    case MK_REAL: ap1<KG, B, MK_REAL, false>(op, re, im); break;
    case MK_IMOFF: ap1<KG, B, MK_IMOFF, false>(op, re, im); break;
    case MK_DIAG: ap1<KG, B, MK_DIAG, false>(op, re, im); break;
    default: ap1<KG, B, MK_DENSE, false>(op, re, im); break;
  }
}

template <int KG, int B0, int B1, typename R>
__device__ __forceinline__ void apswap(int cm, R (&re)[1 << KG], R (&im)[1 << KG]) {
#pragma unroll
  for (int r = 0; r < (1 << KG); ++r) {
    if (!((r >> B0) & 1) || ((r >> B1) & 1)) continue;
    if ((r & cm) != cm) continue;
    const int r2 = r ^ (1 << B0) ^ (1 << B1);
    const R tr = re[r], ti = im[r];
    re[r] = re[r2];
    im[r] = im[r2];
    re[r2] = tr;
    im[r2] = ti;
  }
}

template <int KG, typename R>
__device__ __forceinline__ void apply_op(const FOpDev<R>& op, R (&re)[1 << KG],
                                         R (&im)[1 << KG]) {
  if (op.type == FG_1Q) {
    switch (op.b0) {
      case 0: ap1_cls<KG, 0>(op, re, im); break;
      case 1: if constexpr (KG > 1) ap1_cls<KG, 1>(op, re, im); break;
      case 2: if constexpr (KG > 2) ap1_cls<KG, 2>(op, re, im); break;
      case 3: if constexpr (KG > 3) ap1_cls<KG, 3>(op, re, im); break;
      default: if constexpr (KG > 4) ap1_cls<KG, 4>(op, re, im); break;
    }
  } else if (op.type == FG_PHASE) {
    const int cm = op.cmask;
    if (op.cls) {  // phase -1 (Z, CZ): a sign flip
#pragma unroll
      for (int r = 0; r < (1 << KG); ++r) {
        if ((r & cm) != cm) continue;
        re[r] = -re[r];
        im[r] = -im[r];
      }
    } else {
      const R c = op.m[0], s = op.m[1];
#pragma unroll
      for (int r = 0; r < (1 << KG); ++r) {
        if ((r & cm) != cm) continue;
        const R xr = re[r], xi = im[r];
        re[r] = c * xr - s * xi;
        im[r] = s * xr + c * xi;
      }
    }
  } else {  // FG_SWAP, b0 < b1
    if constexpr (KG >= 2) {
      const int cm = op.cmask, key = op.b0 * 8 + op.b1;
      switch (key) {
        case 0 * 8 + 1: apswap<KG, 0, 1>(cm, re, im); break;
        case 0 * 8 + 2: if constexpr (KG > 2) apswap<KG, 0, 2>(cm, re, im); break;
        case 1 * 8 + 2: if constexpr (KG > 2) apswap<KG, 1, 2>(cm, re, im); break;
        case 0 * 8 + 3: if constexpr (KG > 3) apswap<KG, 0, 3>(cm, re, im); break;
        case 1 * 8 + 3: if constexpr (KG > 3) apswap<KG, 1, 3>(cm, re, im); break;
        case 2 * 8 + 3: if constexpr (KG > 3) apswap<KG, 2, 3>(cm, re, im); break;
        case 0 * 8 + 4: if constexpr (KG > 4) apswap<KG, 0, 4>(cm, re, im); break;
        case 1 * 8 + 4: if constexpr (KG > 4) apswap<KG, 1, 4>(cm, re, im); break;
        case 2 * 8 + 4: if constexpr (KG > 4) apswap<KG, 2, 4>(cm, re, im); break;
        case 3 * 8 + 4: if constexpr (KG > 4) apswap<KG, 3, 4>(cm, re, im); break;
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
    R re[D], im[D];
#pragma unroll
    for (int r = 0; r < D; ++r) {
      const V2 v = sm[sb ^ soff[r]];
      re[r] = v.x;
      im[r] = v.y;
    }
    for (int o = o0; o < o1; ++o) apply_op<KG, R>(ops[o], re, im);
#pragma unroll
    for (int r = 0; r < D; ++r) {
      V2 v;
      v.x = re[r];
      v.y = im[r];
      sm[sb ^ soff[r]] = v;
    }
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
      const int o0 = P.gop[g], o1 = P.gop[g + 1];
      run_group<KGF, R>(sm, P.m, gb, P.ops, o0, o1);
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

template <typename R>
bool build_params(const FusedPass& pass, FusedParams<R>* P) {
  const std::vector<int>& S = pass.S;
  P->m = (int)S.size();
  P->L = pass.L;
  P->nh = P->m - pass.L;
  if (P->m > 24 || P->nh > 32) return false;
  *reinterpret_cast<Ins<uint64_t>*>(&P->blk) = make_ins<uint64_t>(S);
  for (int i = 0; i < P->nh; ++i) P->hpos[i] = (uint8_t)S[pass.L + i];
  if ((int)pass.groups.size() > kFMaxGroups) return false;
  P->ngroups = (int)pass.groups.size();
  int nop = 0;
  for (int g = 0; g < P->ngroups; ++g) {
    const FusedGroup& grp = pass.groups[g];
    P->gk[g] = (uint8_t)grp.k;
    for (int i = 0; i < 5; ++i) P->gbits[g][i] = (uint8_t)grp.bits[i];
    P->gop[g] = (uint16_t)nop;
    // global bit -> group-local index
    auto gl = [&](int bit) {
      const int loc = (int)(std::lower_bound(S.begin(), S.end(), bit) - S.begin());
      for (int i = 0; i < grp.k; ++i)
        if (grp.bits[i] == loc) return i;
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
      } else {
        const int x = gl(f.a), y = gl(f.b);
        o.b0 = (uint8_t)std::min(x, y);
        o.b1 = (uint8_t)std::max(x, y);
      }
    }
  }
  P->gop[P->ngroups] = (uint16_t)nop;
  return true;
}

template <typename R>
sv_status run_pass(void* data, int n, cudaStream_t st, const FusedPass& pass) {
  FusedParams<R> P;
  if (!build_params(pass, &P)) {
    set_error("fused pass exceeds kernel capacity");
    return SV_ERR_INVALID;
  }
  const size_t smem = (sizeof(R) * 2 << P.m) + (sizeof(uint64_t) << (P.m - P.L));
  const int kg = pass.groups.empty() ? 1 : pass.groups[0].k;
  for (const FusedGroup& g : pass.groups)
    if (g.k != kg) {
      set_error("fused pass: groups of unequal width");
      return SV_ERR_INVALID;
    }
  typedef void (*Kern)(typename Cplx2<R>::T*, uint64_t, const FusedParams<R>);
  Kern kern = kg <= 1 ? kfused<R, 1> : kg == 2 ? kfused<R, 2> : kg == 3 ? kfused<R, 3> : kfused<R, 4>;
  static bool attr_set[5] = {false, false, false, false, false};
  if (!attr_set[kg]) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set[kg] = true;
  }
  const uint64_t nblk = uint64_t(1) << (n - P.m);
  const uint64_t grid = std::min<uint64_t>(nblk, 152 * 16);
  ProfScope prof(st, sizeof(R) == 4 ? "kfused_c64" : "kfused_c128");
  kern<<<(unsigned)grid, kFThreads, smem, st>>>(
      reinterpret_cast<typename Cplx2<R>::T*>(data), nblk, P);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return check_launch("fused pass kernel");
}

}  // namespace

sv_status launch_fused_pass(void* data, sv_dtype dt, int n, cudaStream_t st,
                            const FusedPass& pass) {
  return dt == SV_C64 ? run_pass<float>(data, n, st, pass) : run_pass<double>(data, n, st, pass);
}

}  // namespace sv
