// <psi|H|psi> for a Pauli sum H = sum_k c_k P_k (Sec. 3: Hamiltonians and
// VQE energies), in few reads of the state.
//
// Diagonal terms (Z strings) in one streaming read (kdiag_energy): a thread
// loads a register tile of amplitudes that differ in a few low bits and an
// unrolled bit, and the 2^t-point Walsh-Hadamard transform of p_r = |psi_r|^2
// gives sum_r (-1)^{popcount(r & rho)} p_r for every z pattern rho on the
// tile's bits; the other z bits of a term split into thread bits (a sign per
// thread, summed per key) and iteration bits (a sign per loop trip), so that
// every diagonal term costs a few operations per tile, not a parity per
// amplitude.
//
// Off-diagonal terms in staged passes (kpauli_energy): every thread block
// holds one 2^m-amplitude slice of the state in shared memory (bulk tensor
// copies, as the fused gate passes do) and reads it back in register tiles of
// 16 amplitudes that differ in four staged bits (a "group").  A term whose x
// bits lie in one group pairs register r with r ^ mu inside the tile (X or Y
// on one bit through the tile's pair sums, other shapes through partners
// read from the slice), its z bits giving a sign per tile (staged bits), per
// slice (unstaged bits) and per pair (group bits).  A pass of single-X terms
// only (a transverse field, a QAOA mixer) takes the lean kernel
// kpauli_xbits, which keeps per-bit pair sums in registers for the whole
// launch and weighs them once.  The planner covers the x bits by passes that
// stage the low rows plus up to m - 4 high bits each; terms it cannot place
// (more than four x bits, or x bits too far apart) go to the per-amplitude
// kernel.
//
// Precision: products in the state's precision; per-thread compensated fp32
// sums (complex64) or fp64 (complex128); blocks meet in fp64 and a
// fixed-order finish adds the blocks, so results repeat bit for bit.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "slice_geom.cuh"
#include "sv_device.cuh"
#include "tma.cuh"

namespace sv {
namespace {

constexpr int kPThreads = 512;
constexpr int kPMaxTerms = 96;
constexpr int kPMaxGroups = 16;
constexpr int kPG = 4;  // bits of a register tile

// kind of an off-diagonal term inside its group
enum { PT_GENERAL = 0, PT_XBIT = 1, PT_YBIT = 2 };

template <typename R>
struct PTermDev {
  uint64_t zglob;  // z bits at unstaged positions (global bit positions)
  uint32_t zloc;   // z bits at staged positions outside the group (local positions)
  uint8_t mu;      // x bits on the group's bits (bit i <-> gbits[i]); 0: diagonal
  uint8_t zeta;    // z bits on the group's bits
  uint8_t kind;    // PT_XBIT / PT_YBIT: one x bit `bit` and zeta 0 / zeta = mu
  uint8_t bit;
  R cre, cim;      // c_k i^{#Y}
};

template <typename R>
struct PauliPassDev {
  SliceDev geo;
  int ngroups;
  uint8_t gbits[kPMaxGroups][kPG];  // local bit positions of each group, ascending
  int nt;                           // terms of the pass
  int xstart[kPMaxGroups + 1];      // off-diagonal terms of group g: [xstart[g], xstart[g + 1])
  uint8_t gmaska[kPMaxGroups];      // group bits with PT_XBIT terms (their sums A_i are formed)
  uint8_t gmaskb[kPMaxGroups];      // group bits with PT_YBIT terms (B_i)
  PTermDev<R> terms[kPMaxTerms];
};

template <typename R>
struct Cplx2P;
template <>
struct Cplx2P<float> {
  typedef float2 T;
};
template <>
struct Cplx2P<double> {
  typedef double2 T;
};

// the slice layout of the fused passes: 128-byte swizzle of 16-byte chunks
template <typename R>
__device__ __forceinline__ int pswz(int j);
template <>
__device__ __forceinline__ int pswz<float>(int j) {
  return j ^ (((j >> 4) & 7) << 1);
}
template <>
__device__ __forceinline__ int pswz<double>(int j) {
  return j ^ ((j >> 3) & 7);
}

__device__ __forceinline__ void slice_load(const SliceDev& P, uint32_t dst, const int* c,
                                           uint32_t bar) {
  switch (P.rank) {
    case 2: tma_load<2>(dst, &P.tmap, c, bar); break;
    case 3: tma_load<3>(dst, &P.tmap, c, bar); break;
    case 4: tma_load<4>(dst, &P.tmap, c, bar); break;
    default: tma_load<5>(dst, &P.tmap, c, bar); break;
  }
}

// Per group bit i of a tile: A_i = sum Re conj(psi_r) psi_r', B_i = sum
// Im conj(psi_r) psi_r' over the pairs r (bit i clear), r' = r | 2^i, for the
// bits in ma / mb.  A term X on that bit contributes 2 c A_i, a term Y
// 2 c B_i (c = c_k i^{#Y}, (P psi)_x = i^{#Y} (-1)^{popcount((x ^ xm) & zm)}
// psi_{x ^ xm}).
template <typename R>
__device__ __forceinline__ void bit_sums(const R (&re)[16], const R (&im)[16], int ma, int mb,
                                         R (&A)[4], R (&B)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    R a = 0, b = 0;
    if ((ma >> i) & 1) {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        if (r & (1 << i)) continue;
        const int q = r | (1 << i);
        a = fma(re[r], re[q], a);
        a = fma(im[r], im[q], a);
      }
    }
    if ((mb >> i) & 1) {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        if (r & (1 << i)) continue;
        const int q = r | (1 << i);
        b = fma(re[r], im[q], b);
        b = fma(-im[r], re[q], b);
      }
    }
    A[i] = a;
    B[i] = b;
  }
}

template <typename R>
__device__ __forceinline__ R pick4(const R (&v)[4], int i) {
  return i == 0 ? v[0] : i == 1 ? v[1] : i == 2 ? v[2] : v[3];
}

// Re(c sum_r (-1)^{popcount((r ^ mu) & zeta)} conj(psi_r) psi_{r ^ mu}) for a
// general term, the partners read from the slice: slot(r ^ mu) =
// slot(r) ^ off_mu (the swizzled offsets are linear over XOR).
template <typename R, typename V2>
__device__ __forceinline__ R xgeneral(int mu, int zeta, R cre, R cim, const V2* sm, int sb,
                                      const int (&soff)[16], int offmu, const R (&re)[16],
                                      const R (&im)[16]) {
  R tr = 0, ti = 0;
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const V2 w = sm[sb ^ soff[r] ^ offmu];
    const R a = re[r] * w.x + im[r] * w.y;
    const R b = re[r] * w.y - im[r] * w.x;
    if (__popc((r ^ mu) & zeta) & 1) {
      tr -= a;
      ti -= b;
    } else {
      tr += a;
      ti += b;
    }
  }
  return cre * tr - cim * ti;
}

template <typename R>
__device__ __forceinline__ void issue_slice(const SliceDev& G, uint64_t blk, uint32_t dst,
                                            uint32_t barp, int lane) {
  const uint64_t base = insert_zeros(blk, G.blk);
  if (lane == 0) mbar_arrive_expect_tx(barp, G.slice_bytes);
  __syncwarp();
  for (int k = lane; k < G.ncopies; k += 32) {
    int c[5];
    slice_box_coords(G, base, k, c);
    slice_load(G, dst + (uint32_t)k * G.box_bytes, c, barp);
  }
}

// Persistent, one block per SM: block b reads slices b, b + gridDim.x, ...
// into two buffers, the next slice's bulk copies in flight while the current
// one is evaluated; every wait is bounded (a block that gives up records the
// timeout, waits for its copies still in flight and stops).  The groups only
// read shared memory.
template <typename R>
__global__ void __launch_bounds__(kPThreads, 1)
    kpauli_energy(uint64_t n_blocks, const __grid_constant__ PauliPassDev<R> P,
                  double* __restrict__ partials, unsigned* __restrict__ status) {
  typedef typename Cplx2P<R>::T V2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ R cs_re[kPMaxTerms], cs_im[kPMaxTerms];
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t sbuf0 = (raw + 1023u) & ~1023u;
  const uint32_t sbuf[2] = {sbuf0, sbuf0 + P.geo.slice_bytes};  // slice bytes: multiples of 1024
  const uint32_t barp[2] = {smem_addr(&bars[0]), smem_addr(&bars[1])};
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(barp[0], 1);
    mbar_init(barp[1], 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  CompSum<R> acc;
  uint32_t parity[2] = {0, 0};
  bool pending[2] = {false, false};
  const int nsub = 1 << (P.geo.m - kPG);
  if (threadIdx.x < 32 && (uint64_t)blockIdx.x < n_blocks)
    issue_slice<R>(P.geo, blockIdx.x, sbuf[0], barp[0], lane);
  pending[0] = (uint64_t)blockIdx.x < n_blocks;
  int it = 0;
  for (uint64_t blk = blockIdx.x; blk < n_blocks; blk += gridDim.x, ++it) {
    const int cur = it & 1, nxt = cur ^ 1;
    const uint64_t nb = blk + gridDim.x;
    if (nb < n_blocks) {  // the other buffer was released by the last __syncthreads
      if (threadIdx.x < 32) issue_slice<R>(P.geo, nb, sbuf[nxt], barp[nxt], lane);
      pending[nxt] = true;
    }
    // the slice's signed coefficients: (-1)^{popcount(base & unstaged z bits)} c_k
    const uint64_t base = insert_zeros(blk, P.geo.blk);
    for (int k = threadIdx.x; k < P.nt; k += kPThreads) {
      const bool neg = __popcll(base & P.terms[k].zglob) & 1;
      cs_re[k] = neg ? -P.terms[k].cre : P.terms[k].cre;
      cs_im[k] = neg ? -P.terms[k].cim : P.terms[k].cim;
    }
    const bool ok = mbar_wait_bounded(barp[cur], parity[cur]);
    parity[cur] ^= 1;
    pending[cur] = false;
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicOr(status, kWaitTimeout);
      break;
    }
    const V2* sm = reinterpret_cast<const V2*>(smem_raw + (sbuf[cur] - raw));
    for (int g = 0; g < P.ngroups; ++g) {
      const uint8_t* gb = P.gbits[g];
      int soff[16];
      soff[0] = 0;
#pragma unroll
      for (int r = 1; r < 16; ++r) {
        const int i = __ffs(r) - 1;
        soff[r] = soff[r & (r - 1)] ^ pswz<R>(1 << gb[i]);
      }
      const int ma = P.gmaska[g], mb = P.gmaskb[g];
      const int x0 = P.xstart[g], x1 = P.xstart[g + 1];
      for (int s = threadIdx.x; s < nsub; s += kPThreads) {
        uint32_t b = (uint32_t)s;
#pragma unroll
        for (int i = 0; i < kPG; ++i) {
          const uint32_t lm = (1u << gb[i]) - 1;
          b = ((b & ~lm) << 1) | (b & lm);
        }
        const int sb = pswz<R>((int)b);
        R re[16], im[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          const V2 v = sm[sb ^ soff[r]];
          re[r] = v.x;
          im[r] = v.y;
        }
        R e = 0;
        R A[4], B[4];
        bit_sums<R>(re, im, ma, mb, A, B);
        for (int k = x0; k < x1; ++k) {
          const PTermDev<R>& t = P.terms[k];
          R v;
          if (t.kind == PT_XBIT) {
            v = 2 * cs_re[k] * pick4<R>(A, t.bit);
          } else if (t.kind == PT_YBIT) {
            v = 2 * cs_im[k] * pick4<R>(B, t.bit);
          } else {
            int offmu = 0;
#pragma unroll
            for (int i = 0; i < kPG; ++i)
              if ((t.mu >> i) & 1) offmu ^= pswz<R>(1 << gb[i]);
            v = xgeneral<R, V2>(t.mu, t.zeta, cs_re[k], cs_im[k], sm, sb, soff, offmu, re, im);
          }
          e += (__popc(b & t.zloc) & 1) ? -v : v;
        }
        acc.add(e);
      }
    }
    __syncthreads();  // every thread is done with this buffer and the coefficients
  }
  // copies still in flight (a block that gave up): wait for them, bounded
  for (int j = 0; j < 2; ++j)
    if (pending[j]) mbar_wait_bounded(barp[j], parity[j]);
  const double t = block_sum(acc.value());
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// ---- X terms without signs: a lean staged pass ------------------------------------------
// A pass whose terms are all single X factors (no Z or Y anywhere: the
// transverse field of an Ising chain, the QAOA mixer) needs no per-tile sign:
// E = sum_k 2 c_k sum_tiles A_{bit k}.  Each thread keeps the pair sums of
// every group bit in registers (at most kXGroups groups of four bits) across
// all its slices and weighs them by the coefficients once at the end.
constexpr int kXGroups = 4;

struct XPassDev {
  SliceDev geo;
  int ngroups;
  uint8_t gbits[kXGroups][kPG];  // local bit positions, ascending
  double w[kPG * kXGroups];      // 2 sum c_k over the terms on bit i of group g, at 4 g + i
};

// pair sums A_i of one group over the tile (all four bits)
template <typename R>
__device__ __forceinline__ void xsums(const R (&re)[16], const R (&im)[16], R (&A)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    R a = 0;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      if (r & (1 << i)) continue;
      a = fma(re[r], re[r | (1 << i)], a);
      a = fma(im[r], im[r | (1 << i)], a);
    }
    A[i] = a;
  }
}

// Three slice buffers: the copies of the next two slices are in flight while
// the current one is read.
constexpr int kXBuf = 3;

template <typename R>
__global__ void __launch_bounds__(kPThreads, 1)
    kpauli_xbits(uint64_t n_blocks, const __grid_constant__ XPassDev P,
                 double* __restrict__ partials, unsigned* __restrict__ status) {
  typedef typename Cplx2P<R>::T V2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kXBuf];   // full: the slice's bytes have landed
  __shared__ __align__(8) uint64_t ebars[kXBuf];  // empty: every warp is done with it
  constexpr int kWarps = kPThreads / 32;
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t sbuf0 = (raw + 1023u) & ~1023u;  // slice bytes: multiples of 1024
  const uint32_t sbytes = P.geo.slice_bytes;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int j = 0; j < kXBuf; ++j) {
      mbar_init(smem_addr(&bars[j]), 1);
      mbar_init(smem_addr(&ebars[j]), kWarps);
    }
    fence_proxy_async_smem();
  }
  __syncthreads();
  CompSum<R> acc[kPG * kXGroups];
  // bit j: buffer j.  used: filled before (its refill waits until every warp
  // released the previous fill); eparity: phase of its empty barrier
  uint32_t parity = 0, pending = 0, used = 0, eparity = 0;
  const int nsub = 1 << (P.geo.m - kPG);
  for (int j = 0; j < kXBuf - 1; ++j) {
    const uint64_t b = blockIdx.x + (uint64_t)j * gridDim.x;
    if (b < n_blocks) {
      if (threadIdx.x < 32)
        issue_slice<R>(P.geo, b, sbuf0 + (uint32_t)j * sbytes, smem_addr(&bars[j]), lane);
      pending |= 1u << j;
      used |= 1u << j;
    }
  }
  int cur = 0;
  for (uint64_t blk = blockIdx.x; blk < n_blocks; blk += gridDim.x) {
    // slice blk + (kXBuf - 1) grid strides into the buffer of the previous
    // iteration, once all warps have released it: no block-wide barrier, the
    // other warps run on into the slices already loaded
    const int nxt = cur == 0 ? kXBuf - 1 : cur - 1;
    const uint64_t nb = blk + (uint64_t)(kXBuf - 1) * gridDim.x;
    if (nb < n_blocks) {
      if (threadIdx.x < 32) {
        bool free_ok = true;
        if ((used >> nxt) & 1)
          free_ok = mbar_wait_bounded(smem_addr(&ebars[nxt]), (eparity >> nxt) & 1);
        if (free_ok)
          issue_slice<R>(P.geo, nb, sbuf0 + (uint32_t)nxt * sbytes, smem_addr(&bars[nxt]), lane);
        else if (lane == 0)
          atomicOr(status, kWaitTimeout);
      }
      if ((used >> nxt) & 1) eparity ^= 1u << nxt;
      used |= 1u << nxt;
      pending |= 1u << nxt;
    }
    const bool ok = mbar_wait_bounded(smem_addr(&bars[cur]), (parity >> cur) & 1);
    parity ^= 1u << cur;
    pending &= ~(1u << cur);
    if (!ok) {  // this warp stops; the others give up at their own bounded waits
      if (lane == 0) atomicOr(status, kWaitTimeout);
      break;
    }
    const V2* sm = reinterpret_cast<const V2*>(smem_raw + (sbuf0 + (uint32_t)cur * sbytes - raw));
#pragma unroll
    for (int g = 0; g < kXGroups; ++g) {
      if (g >= P.ngroups) break;
      const uint8_t* gb = P.gbits[g];
      int sw[kPG];
#pragma unroll
      for (int i = 0; i < kPG; ++i) sw[i] = pswz<R>(1 << gb[i]);
      for (int s = threadIdx.x; s < nsub; s += kPThreads) {
        uint32_t b = (uint32_t)s;
#pragma unroll
        for (int i = 0; i < kPG; ++i) {
          const uint32_t lm = (1u << gb[i]) - 1;
          b = ((b & ~lm) << 1) | (b & lm);
        }
        const int sb = pswz<R>((int)b);
        R re[16], im[16];
        if (sizeof(R) == 4 && gb[0] == 0 && gb[3] == 3) {
          // the tile is one 128-byte row: amplitudes 2q, 2q + 1 share a
          // 16-byte chunk at chunk (q ^ row swizzle), read as one vector
          // (a warp's 32 rows then spread over all banks)
          const float4* sm4 = reinterpret_cast<const float4*>(sm);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 v = sm4[(sb >> 1) ^ q];
            re[2 * q] = v.x;
            im[2 * q] = v.y;
            re[2 * q + 1] = v.z;
            im[2 * q + 1] = v.w;
          }
        } else {
#pragma unroll
          for (int r = 0; r < 16; ++r) {
            int o = 0;
#pragma unroll
            for (int i = 0; i < kPG; ++i)
              if ((r >> i) & 1) o ^= sw[i];
            const V2 v = sm[sb ^ o];
            re[r] = v.x;
            im[r] = v.y;
          }
        }
        R A[4];
        xsums<R>(re, im, A);
#pragma unroll
        for (int i = 0; i < kPG; ++i) acc[kPG * g + i].add(A[i]);
      }
    }
    __syncwarp();  // this warp is done with the buffer
    if (lane == 0) mbar_arrive(smem_addr(&ebars[cur]));
    cur = cur + 1 == kXBuf ? 0 : cur + 1;
  }
  // copies still in flight (a block that gave up): wait for them, bounded
  for (int j = 0; j < kXBuf; ++j)
    if ((pending >> j) & 1) mbar_wait_bounded(smem_addr(&bars[j]), (parity >> j) & 1);
  double e = 0.0;
#pragma unroll
  for (int q = 0; q < kPG * kXGroups; ++q) e += P.w[q] * acc[q].value();
  e = block_sum(e);
  if (threadIdx.x == 0) partials[blockIdx.x] = e;
}

// ---- diagonal terms: one streaming read -----------------------------------------------
// The diagonal part of H, E_d = sum_x |psi_x|^2 d(x), d(x) = sum_k c_k
// (-1)^{popcount(x & z_k)}, read with coalesced 16-byte loads and no shared
// memory.  Thread t of T = 2^tb threads reads the vectors t + T (u + 8 J),
// u = 0..7 unrolled, J = 0, 1, ...: the amplitude-index bits split into the
// tile bits (the bit inside a complex64 vector and u: 16 amplitudes per
// tile, complex128 8), the thread bits (fixed for the thread) and the
// iteration bits J.  A term's sign is the product of its parts on the three,
// so for every key (its z pattern rho on the tile bits, its z mask zJ on the
// iteration bits) a thread accumulates sum_J (-1)^{popcount(J & zJ)} W[rho],
// W the Walsh-Hadamard transform of the tile's |psi|^2; at the end each term
// takes c_k (-1)^{popcount(t & z_k's thread bits)} times its key's sum.  A
// launch serves up to kDKeys keys (terms that share a key share its sum).
constexpr int kDKeys = 16;
constexpr int kDTerms = 64;
constexpr int kDThreads = 256;

template <typename R>
struct DiagDev {
  int nk, nk0;          // keys; keys[0..nk0) have rho = 0
  uint8_t rho[kDKeys];  // z pattern on the tile bits
  uint32_t zj[kDKeys];  // z mask on the iteration bits
  int nt;
  uint8_t key[kDTerms];     // key of term k
  uint32_t zt[kDTerms];     // z mask on the thread bits
  R c[kDTerms];             // coefficient
  int tb;                   // log2 threads
  uint32_t jmax;            // iterations per thread
};

// 16-way pick by a runtime index without register-array indexing
template <typename R, int N>
__device__ __forceinline__ R pick(const R (&w)[N], int i) {
  R v = w[0];
#pragma unroll
  for (int r = 1; r < N; ++r) v = (i == r) ? w[r] : v;
  return v;
}

template <typename R>
__global__ void __launch_bounds__(kDThreads, 3)
    kdiag_energy(const typename Cplx2P<R>::T* __restrict__ psi, const __grid_constant__ DiagDev<R> D,
                 double* __restrict__ partials) {
  typedef typename Cplx2P<R>::T V2;
  constexpr bool C64 = sizeof(R) == 4;
  constexpr int NT = C64 ? 16 : 8;  // amplitudes of a tile
  __shared__ double sacc[kDKeys][kDThreads];
  const uint32_t t = blockIdx.x * kDThreads + threadIdx.x;
  const uint64_t T = uint64_t(1) << D.tb;
  CompSum<R> acc[kDKeys];
  for (uint32_t J = 0; J < D.jmax; ++J) {
    R w[NT];
    if constexpr (C64) {
      const float4* v4 = reinterpret_cast<const float4*>(psi);
      float4 a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = v4[t + T * (uint64_t)(u + 8 * J)];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        w[2 * u] = a[u].x * a[u].x + a[u].y * a[u].y;
        w[2 * u + 1] = a[u].z * a[u].z + a[u].w * a[u].w;
      }
    } else {
      V2 a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = psi[t + T * (uint64_t)(u + 8 * J)];
#pragma unroll
      for (int u = 0; u < 8; ++u) w[u] = a[u].x * a[u].x + a[u].y * a[u].y;
    }
#pragma unroll
    for (int i = 0; (1 << i) < NT; ++i)
#pragma unroll
      for (int r = 0; r < NT; ++r) {
        if (r & (1 << i)) continue;
        const R x = w[r], y = w[r | (1 << i)];
        w[r] = x + y;
        w[r | (1 << i)] = x - y;
      }
#pragma unroll
    for (int q = 0; q < kDKeys; ++q) {
      if (q >= D.nk) break;
      const R v = q < D.nk0 ? w[0] : pick<R, NT>(w, D.rho[q]);
      acc[q].add((__popc(J & D.zj[q]) & 1) ? -v : v);
    }
  }
#pragma unroll
  for (int q = 0; q < kDKeys; ++q) sacc[q][threadIdx.x] = acc[q].value();
  double e = 0.0;
  for (int k = 0; k < D.nt; ++k) {
    const double v = (double)D.c[k] * sacc[D.key[k]][threadIdx.x];
    e += (__popc(t & D.zt[k]) & 1) ? -v : v;
  }
  e = block_sum(e);
  if (threadIdx.x == 0) partials[blockIdx.x] = e;
}

// lambda = D psi for the diagonal part D = diag(d), d(x) = sum_k c_k
// (-1)^{popcount(x & z_k)} (Sec. 3: H psi for the adjoint sweep), in one
// streaming read and write, with the tiles of kdiag_energy.  Per thread the
// key coefficients C_q = sum over the key's terms of c_k (-1)^{popcount(t &
// zt_k)} are formed once; per loop trip J the signed C_q gather into v[rho]
// and the tile's diagonal is the Walsh-Hadamard transform d_r = sum_rho
// (-1)^{popcount(r & rho)} v_rho.  accumulate: out += D psi (a later chunk of
// keys).  partials (or null): per block sum_x d(x) |psi_x|^2, this chunk's
// part of <psi|D|psi>.
template <typename R>
__global__ void __launch_bounds__(kDThreads, 2)
    kdiag_apply(typename Cplx2P<R>::T* __restrict__ out,
                const typename Cplx2P<R>::T* __restrict__ psi, const __grid_constant__ DiagDev<R> D,
                int accumulate, double* __restrict__ partials) {
  typedef typename Cplx2P<R>::T V2;
  constexpr bool C64 = sizeof(R) == 4;
  constexpr int NT = C64 ? 16 : 8;  // amplitudes of a tile
  __shared__ R cq[kDKeys][kDThreads];
  const uint32_t t = blockIdx.x * kDThreads + threadIdx.x;
  const uint64_t T = uint64_t(1) << D.tb;
#pragma unroll
  for (int q = 0; q < kDKeys; ++q) cq[q][threadIdx.x] = R(0);
  for (int k = 0; k < D.nt; ++k) {
    const R c = D.c[k];
    cq[D.key[k]][threadIdx.x] += (__popc(t & D.zt[k]) & 1) ? -c : c;
  }
  CompSum<R> acc;
  for (uint32_t J = 0; J < D.jmax; ++J) {
    R v[NT];
#pragma unroll
    for (int r = 0; r < NT; ++r) v[r] = R(0);
    for (int q = 0; q < D.nk; ++q) {
      const R c = cq[q][threadIdx.x];
      const R sv = (__popc(J & D.zj[q]) & 1) ? -c : c;
      if (q < D.nk0) {
        v[0] += sv;
      } else {
        const int rho = D.rho[q];
#pragma unroll
        for (int r = 1; r < NT; ++r) v[r] += (rho == r) ? sv : R(0);
      }
    }
#pragma unroll
    for (int i = 0; (1 << i) < NT; ++i)
#pragma unroll
      for (int r = 0; r < NT; ++r) {
        if (r & (1 << i)) continue;
        const R x = v[r], y = v[r | (1 << i)];
        v[r] = x + y;
        v[r | (1 << i)] = x - y;
      }
    if constexpr (C64) {
      const float4* p4 = reinterpret_cast<const float4*>(psi);
      float4* o4 = reinterpret_cast<float4*>(out);
      float4 a[8], b[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = p4[t + T * (uint64_t)(u + 8 * J)];
      if (accumulate) {
#pragma unroll
        for (int u = 0; u < 8; ++u) b[u] = o4[t + T * (uint64_t)(u + 8 * J)];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float d0 = v[2 * u], d1 = v[2 * u + 1];
        float4 w = make_float4(d0 * a[u].x, d0 * a[u].y, d1 * a[u].z, d1 * a[u].w);
        if (accumulate) {
          w.x += b[u].x;
          w.y += b[u].y;
          w.z += b[u].z;
          w.w += b[u].w;
        }
        o4[t + T * (uint64_t)(u + 8 * J)] = w;
        if (partials) {
          acc.add(d0 * (a[u].x * a[u].x + a[u].y * a[u].y));
          acc.add(d1 * (a[u].z * a[u].z + a[u].w * a[u].w));
        }
      }
    } else {
      V2 a[8], b[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = psi[t + T * (uint64_t)(u + 8 * J)];
      if (accumulate) {
#pragma unroll
        for (int u = 0; u < 8; ++u) b[u] = out[t + T * (uint64_t)(u + 8 * J)];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        V2 w;
        w.x = v[u] * a[u].x;
        w.y = v[u] * a[u].y;
        if (accumulate) {
          w.x += b[u].x;
          w.y += b[u].y;
        }
        out[t + T * (uint64_t)(u + 8 * J)] = w;
        if (partials) acc.add(v[u] * (a[u].x * a[u].x + a[u].y * a[u].y));
      }
    }
  }
  if (partials) {
    const double e = block_sum(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = e;
  }
}

__device__ unsigned g_pauli_status = 0;

// ---- host: pass planning -------------------------------------------------------
struct TermH {
  uint64_t xm, zm;
  double cre, cim;
};

struct PassH {
  std::vector<int> S;                 // staged bits, ascending
  int L = 0;
  std::vector<std::vector<int>> groups;  // global bits of each group (kPG of them)
  std::vector<std::vector<int>> xt;   // off-diagonal terms per group
};

int popc64(uint64_t x) { return __builtin_popcountll(x); }

// Group for the x bits xb inside S: an existing group containing them, else
// the aligned block of four staged positions that holds them (positions
// 4j..4j+3; the last block is the top four, so ceil(|S| / 4) blocks cover S
// whatever order the terms come in), else kPG bits: xb plus the nearest
// staged bits above (then below).
int group_for(PassH* p, uint64_t xb) {
  for (size_t g = 0; g < p->groups.size(); ++g) {
    uint64_t gm = 0;
    for (int b : p->groups[g]) gm |= uint64_t(1) << b;
    if ((xb & ~gm) == 0) return (int)g;
  }
  if ((int)p->groups.size() >= kPMaxGroups || popc64(xb) > kPG) return -1;
  const int ns = (int)p->S.size();
  if (ns < kPG) return -1;
  int lo_i = ns, hi_i = -1;
  for (int i = 0; i < ns; ++i)
    if ((xb >> p->S[i]) & 1) {
      lo_i = std::min(lo_i, i);
      hi_i = std::max(hi_i, i);
    }
  std::vector<int> bits;
  const int start = std::min(lo_i / kPG * kPG, ns - kPG);
  if (hi_i < start + kPG) {
    bits.assign(p->S.begin() + start, p->S.begin() + start + kPG);
  } else {
    for (int b = 0; b < 64; ++b)
      if ((xb >> b) & 1) bits.push_back(b);
    const int lo = bits[0];
    std::vector<int> cand;
    for (int b : p->S)
      if (b >= lo && !((xb >> b) & 1)) cand.push_back(b);
    for (auto it = p->S.rbegin(); it != p->S.rend(); ++it)
      if (*it < lo && !((xb >> *it) & 1)) cand.push_back(*it);
    for (size_t i = 0; i < cand.size() && (int)bits.size() < kPG; ++i) bits.push_back(cand[i]);
    if ((int)bits.size() < kPG) return -1;
    std::sort(bits.begin(), bits.end());
  }
  p->groups.push_back(bits);
  p->xt.emplace_back();
  return (int)p->groups.size() - 1;
}

// Plans passes over the n-qubit state for the off-diagonal terms T, with m
// staged bits per slice and lo1 bits per 128-byte row: pass 0 stages bits
// 0..m-1 and takes every term whose x bits lie there; later passes stage the
// row bits plus the lowest x bits still uncovered.  Terms that fit no pass
// go to `rest`.  At most kPMaxTerms terms per pass (further passes repeat a
// staged set).
void plan_passes(int n, int m, int lo1, const std::vector<TermH>& T, std::vector<PassH>* out,
                 std::vector<int>* rest) {
  out->clear();
  rest->clear();
  std::vector<int> pend(T.size());
  for (int k = 0; k < (int)T.size(); ++k) pend[k] = k;
  PassH p0;
  for (int b = 0; b < m; ++b) p0.S.push_back(b);
  p0.L = m;
  const uint64_t low = (uint64_t(1) << m) - 1;
  auto add_pass = [&](PassH& p, const std::vector<int>& cands, std::vector<int>* left) {
    int count = 0;
    for (int k : cands) {
      const uint64_t xb = T[k].xm;
      uint64_t sm = 0;
      for (int b : p.S) sm |= uint64_t(1) << b;
      int g = (xb & ~sm) == 0 && count < kPMaxTerms ? group_for(&p, xb) : -1;
      if (g < 0) {
        left->push_back(k);
        continue;
      }
      p.xt[g].push_back(k);
      ++count;
    }
  };
  // pass 0: the terms with x bits among the low m bits (repeated while they
  // exceed one pass's capacity)
  {
    std::vector<int> cand, others;
    for (int k : pend) ((T[k].xm & ~low) == 0 ? cand : others).push_back(k);
    while (!cand.empty()) {
      PassH p = p0;
      std::vector<int> left;
      add_pass(p, cand, &left);
      if (left.size() == cand.size()) {  // nothing fits: the per-amplitude kernel takes them
        for (int k : left) rest->push_back(k);
        break;
      }
      out->push_back(p);
      cand.clear();
      for (int k : left) (popc64(T[k].xm) > kPG ? *rest : cand).push_back(k);
    }
    pend.swap(others);
  }
  // later passes: the row bits plus the lowest uncovered x bits
  while (!pend.empty()) {
    std::vector<int> xbits;
    for (int k : pend)
      for (int b = lo1; b < n; ++b)
        if ((T[k].xm >> b) & 1) xbits.push_back(b);
    std::sort(xbits.begin(), xbits.end());
    xbits.erase(std::unique(xbits.begin(), xbits.end()), xbits.end());
    PassH p;
    for (int b = 0; b < lo1; ++b) p.S.push_back(b);
    p.L = lo1;
    // fill with the lowest uncovered x bits, then extend the top run
    for (int b : xbits)
      if ((int)p.S.size() < m && b >= lo1) p.S.push_back(b);
    for (int b = lo1; (int)p.S.size() < m && b < n; ++b)
      if (std::find(p.S.begin(), p.S.end(), b) == p.S.end()) p.S.push_back(b);
    std::sort(p.S.begin(), p.S.end());
    std::vector<int> left;
    add_pass(p, pend, &left);
    if (left.size() == pend.size()) {  // nothing fits: the per-amplitude kernel takes them
      for (int k : left) rest->push_back(k);
      break;
    }
    out->push_back(p);
    pend.swap(left);
  }
}

template <typename R>
bool build_pass(const PassH& p, const std::vector<TermH>& T, const TmaGeom& geo, int n,
                void* data, PauliPassDev<R>* P) {
  const int lw = sizeof(R) == 4 ? 0 : 1;
  if (!build_slice(geo, p.S, n, lw, data, &P->geo)) return false;
  int pos_of[64];
  for (int b = 0; b < 64; ++b) pos_of[b] = -1;
  for (size_t i = 0; i < geo.order.size(); ++i) pos_of[geo.order[i]] = (int)i;
  if ((int)p.groups.size() > kPMaxGroups) return false;
  P->ngroups = (int)p.groups.size();
  std::vector<std::vector<int>> glocal(p.groups.size());
  for (size_t g = 0; g < p.groups.size(); ++g) {
    for (int b : p.groups[g]) glocal[g].push_back(pos_of[b]);
    std::sort(glocal[g].begin(), glocal[g].end());
    for (int i = 0; i < kPG; ++i) P->gbits[g][i] = (uint8_t)glocal[g][i];
  }
  uint64_t smask = 0;
  for (int b : p.S) smask |= uint64_t(1) << b;
  // a term as group g sees it
  auto make = [&](int k, int g) {
    PTermDev<R> d{};
    const TermH& t = T[k];
    uint32_t zloc = 0;
    uint8_t mu = 0, zeta = 0;
    for (int b = 0; b < 64; ++b) {
      if (!((smask >> b) & 1)) continue;
      const int lp = pos_of[b];
      int gi = -1;
      for (int i = 0; i < kPG; ++i)
        if (glocal[g][i] == lp) gi = i;
      if (gi >= 0) {
        if ((t.xm >> b) & 1) mu |= (uint8_t)(1 << gi);
        if ((t.zm >> b) & 1) zeta |= (uint8_t)(1 << gi);
      } else if ((t.zm >> b) & 1) {
        zloc |= 1u << lp;
      }
    }
    d.zglob = t.zm & ~smask;
    d.zloc = zloc;
    d.mu = mu;
    d.zeta = zeta;
    d.kind = PT_GENERAL;
    d.bit = 0;
    if (__builtin_popcount(mu) == 1) {
      d.bit = (uint8_t)__builtin_ctz(mu);
      if (zeta == 0) d.kind = PT_XBIT;
      if (zeta == mu) d.kind = PT_YBIT;
    }
    d.cre = (R)t.cre;
    d.cim = (R)t.cim;
    return d;
  };
  int nt = 0;
  for (size_t g = 0; g < p.groups.size(); ++g) {
    P->xstart[g] = nt;
    P->gmaska[g] = P->gmaskb[g] = 0;
    for (int k : p.xt[g]) {
      if (nt >= kPMaxTerms) return false;
      P->terms[nt] = make(k, (int)g);
      if (P->terms[nt].kind == PT_XBIT) P->gmaska[g] |= (uint8_t)(1 << P->terms[nt].bit);
      if (P->terms[nt].kind == PT_YBIT) P->gmaskb[g] |= (uint8_t)(1 << P->terms[nt].bit);
      ++nt;
    }
  }
  P->xstart[p.groups.size()] = nt;
  P->nt = nt;
  return true;
}

// The lean form of a pass when every term is a single X factor on a group
// bit with no z bits anywhere and a real coefficient, in at most kXGroups
// groups.
template <typename R>
bool lean_pass(const PauliPassDev<R>& P, XPassDev* X) {
  if (P.ngroups > kXGroups) return false;
  *X = XPassDev{};
  X->geo = P.geo;
  X->ngroups = P.ngroups;
  for (int g = 0; g < P.ngroups; ++g) {
    for (int i = 0; i < kPG; ++i) X->gbits[g][i] = P.gbits[g][i];
    for (int k = P.xstart[g]; k < P.xstart[g + 1]; ++k) {
      const PTermDev<R>& t = P.terms[k];
      if (t.kind != PT_XBIT || t.zglob || t.zloc || t.cim != 0) return false;
      X->w[kPG * g + t.bit] += 2.0 * (double)t.cre;
    }
  }
  return true;
}

// The diagonal terms of T (x mask 0) as launches of kdiag_energy /
// kdiag_apply: up to kDKeys keys (tile pattern rho, iteration mask zJ) and
// kDTerms terms each, keys with rho = 0 first; tb thread bits.
void diag_chunks(int n, bool c64, const std::vector<TermH>& T, int tb,
                 std::vector<DiagDev<float>>* dfs, std::vector<DiagDev<double>>* dds) {
  std::vector<DiagDev<double>> chunks;  // built in fp64, converted below
  DiagDev<double> cur{};
  std::map<std::pair<int, uint32_t>, int> keys;
  auto flush = [&]() {
    if (cur.nt == 0) return;
    // keys with rho = 0 first
    std::vector<int> order;
    for (int q = 0; q < cur.nk; ++q)
      if (cur.rho[q] == 0) order.push_back(q);
    for (int q = 0; q < cur.nk; ++q)
      if (cur.rho[q] != 0) order.push_back(q);
    DiagDev<double> d = cur;
    std::vector<int> pos(cur.nk);
    for (int i = 0; i < cur.nk; ++i) {
      pos[order[i]] = i;
      d.rho[i] = cur.rho[order[i]];
      d.zj[i] = cur.zj[order[i]];
    }
    d.nk0 = 0;
    while (d.nk0 < d.nk && d.rho[d.nk0] == 0) ++d.nk0;
    for (int k = 0; k < d.nt; ++k) d.key[k] = (uint8_t)pos[cur.key[k]];
    chunks.push_back(d);
    cur = DiagDev<double>{};
    keys.clear();
  };
  for (int k = 0; k < (int)T.size(); ++k) {
    if (T[k].xm != 0) continue;
    const uint64_t zm = T[k].zm;
    int rho;
    uint32_t zt, zj;
    if (c64) {
      rho = (int)((zm & 1) | (((zm >> (tb + 1)) & 7) << 1));
      zt = (uint32_t)((zm >> 1) & ((uint64_t(1) << tb) - 1));
      zj = (uint32_t)(zm >> (tb + 4));
    } else {
      rho = (int)((zm >> tb) & 7);
      zt = (uint32_t)(zm & ((uint64_t(1) << tb) - 1));
      zj = (uint32_t)(zm >> (tb + 3));
    }
    const std::pair<int, uint32_t> kk{rho, zj};
    if (cur.nt == kDTerms || (!keys.count(kk) && cur.nk == kDKeys)) flush();
    auto it = keys.find(kk);
    int q;
    if (it == keys.end()) {
      q = cur.nk++;
      cur.rho[q] = (uint8_t)rho;
      cur.zj[q] = zj;
      keys[kk] = q;
    } else {
      q = it->second;
    }
    cur.key[cur.nt] = (uint8_t)q;
    cur.zt[cur.nt] = zt;
    cur.c[cur.nt] = T[k].cre;
    ++cur.nt;
  }
  flush();
  const uint32_t jmax = (uint32_t)(uint64_t(1) << (n - (c64 ? 1 : 0) - 3 - tb));
  for (DiagDev<double>& d : chunks) {
    d.tb = tb;
    d.jmax = jmax;
    if (c64) {
      DiagDev<float> f{};
      f.nk = d.nk;
      f.nk0 = d.nk0;
      for (int q = 0; q < kDKeys; ++q) {
        f.rho[q] = d.rho[q];
        f.zj[q] = d.zj[q];
      }
      f.nt = d.nt;
      for (int k = 0; k < kDTerms; ++k) {
        f.key[k] = d.key[k];
        f.zt[k] = d.zt[k];
        f.c[k] = (float)d.c[k];
      }
      f.tb = d.tb;
      f.jmax = d.jmax;
      dfs->push_back(f);
    } else {
      dds->push_back(d);
    }
  }
}

}  // namespace

// <psi|H|psi> of the state into the device double dst by staged passes:
// each pass's blocks write partial sums, the terms no pass takes go to the
// per-amplitude kernel, and one fixed-order finish adds everything.
// SV_ERR_UNSUPPORTED (nothing launched) when the state is too small for
// passes or a pass has no bulk-copy geometry: the caller takes the
// per-amplitude kernel for everything.
sv_status expval_staged(sv_state s, const sv_pauli_sum* H, double* dst) {
  const bool c64 = s->dt == SV_C64;
  const int lw = c64 ? 0 : 1, lo1 = 4 - lw;
  if (s->n < 16 || H->n_terms == 0) return SV_ERR_UNSUPPORTED;
  const int m = std::min(c64 ? 13 : 12, s->n - 8);
  std::vector<TermH> T(H->n_terms);
  for (int k = 0; k < H->n_terms; ++k) {
    const uint64_t xm = H->xmask[k], zm = H->zmask[k];
    const int ny = popc64(xm & zm) & 3;
    const double c = H->coeff[k];
    T[k] = {xm, zm, ny == 0 ? c : ny == 2 ? -c : 0.0, ny == 1 ? c : ny == 3 ? -c : 0.0};
  }
  // diagonal terms: streaming launches of up to kDKeys keys / kDTerms terms
  // thread bits: enough blocks for many waves over the SMs (2^20 threads at
  // n >= 27), at least 8 loop trips per thread where the state allows
  const int tb = std::min(20, std::max(8, s->n - (c64 ? 4 : 3) - 3));
  std::vector<DiagDev<float>> dfs;
  std::vector<DiagDev<double>> dds;
  diag_chunks(s->n, c64, T, tb, &dfs, &dds);
  const size_t ndiag = c64 ? dfs.size() : dds.size();
  // off-diagonal terms: staged passes
  std::vector<TermH> Toff;
  std::vector<int> off_index;
  for (int k = 0; k < H->n_terms; ++k)
    if (T[k].xm != 0) {
      Toff.push_back(T[k]);
      off_index.push_back(k);
    }
  std::vector<PassH> passes;
  std::vector<int> rest_off, rest;
  plan_passes(s->n, m, lo1, Toff, &passes, &rest_off);
  for (int k : rest_off) rest.push_back(off_index[k]);
  if (passes.empty() && ndiag == 0) return SV_ERR_UNSUPPORTED;
  std::vector<TmaGeom> geos(passes.size());
  for (size_t i = 0; i < passes.size(); ++i)
    if (!tma_geometry(passes[i].S, passes[i].L, s->n, lw, &geos[i])) return SV_ERR_UNSUPPORTED;
  std::vector<PauliDev> chunks;
  std::vector<uint64_t> rxm, rzm;
  std::vector<double> rcf;
  if (!rest.empty()) {
    for (int k : rest) {
      rxm.push_back(H->xmask[k]);
      rzm.push_back(H->zmask[k]);
      rcf.push_back(H->coeff[k]);
    }
    sv_pauli_sum sub{(int32_t)rest.size(), rxm.data(), rzm.data(), rcf.data()};
    pauli_chunks(&sub, &chunks);
  }
  sv_status st =
      ensure_partials(s, ndiag * ((size_t(1) << tb) / kDThreads) +
                             (passes.size() + chunks.size()) * (size_t)kRedMaxBlocks);
  if (st) return st;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = 2 * (size_t(8) << lw << m) + 1024;  // two slice buffers
  const uint64_t nblk = uint64_t(1) << (s->n - m);
  static std::mutex mu;
  static PauliPassDev<float> Pf;
  static PauliPassDev<double> Pd;
  static std::map<std::pair<const void*, size_t>, int> resident;
  std::lock_guard<std::mutex> lk(mu);
  unsigned* status = nullptr;
  if (cudaGetSymbolAddress((void**)&status, g_pauli_status) != cudaSuccess) {
    cudaGetLastError();
    return SV_ERR_UNSUPPORTED;
  }
  // every pass's geometry first: nothing is launched unless all of them build
  std::vector<PauliPassDev<float>> pf;
  std::vector<PauliPassDev<double>> pd;
  for (size_t i = 0; i < passes.size(); ++i) {
    const bool ok = c64 ? build_pass<float>(passes[i], Toff, geos[i], s->n, s->data, &Pf)
                        : build_pass<double>(passes[i], Toff, geos[i], s->n, s->data, &Pd);
    if (!ok) return SV_ERR_UNSUPPORTED;
    if (c64)
      pf.push_back(Pf);
    else
      pd.push_back(Pd);
  }
  std::vector<XPassDev> lean(passes.size());
  std::vector<char> is_lean(passes.size());
  for (size_t i = 0; i < passes.size(); ++i)
    is_lean[i] = c64 ? lean_pass<float>(pf[i], &lean[i]) : lean_pass<double>(pd[i], &lean[i]);
  const size_t smem_x = kXBuf * (size_t(8) << lw << m) + 1024;  // the lean kernel's buffers
  auto grid_of = [&](const void* kern, size_t bytes, int nbuf) -> uint64_t {
    int& res = resident[{kern, bytes}];
    if (!res) {
      // the largest slice any pass stages (the attribute is per kernel, not per size)
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(nbuf * (size_t(8) << lw << (c64 ? 13 : 12)) + 1024));
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res, kern, kPThreads, bytes) !=
              cudaSuccess ||
          res < 1) {
        cudaGetLastError();
        res = 1;
      }
    }
    return std::min<uint64_t>({nblk, (uint64_t)sms * res, (uint64_t)kRedMaxBlocks});
  };
  int total = 0;
  const unsigned dgrid = (unsigned)((uint64_t(1) << tb) / kDThreads);  // <= 4096
  for (size_t i = 0; i < ndiag; ++i) {
    ProfScope prof(s->stream, c64 ? "kdiag_energy_c64" : "kdiag_energy_c128");
    if (c64)
      kdiag_energy<float><<<dgrid, kDThreads, 0, s->stream>>>((const float2*)s->data, dfs[i],
                                                               s->partials + total);
    else
      kdiag_energy<double><<<dgrid, kDThreads, 0, s->stream>>>((const double2*)s->data, dds[i],
                                                                s->partials + total);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    st = check_launch("diagonal-term kernel");
    if (st) return st;
    total += (int)dgrid;
  }
  for (size_t i = 0; i < passes.size(); ++i) {
    uint64_t grid;
    if (is_lean[i]) {
      ProfScope prof(s->stream, c64 ? "kpauli_xbits_c64" : "kpauli_xbits_c128");
      if (c64) {
        grid = grid_of((const void*)kpauli_xbits<float>, smem_x, kXBuf);
        kpauli_xbits<float><<<(unsigned)grid, kPThreads, smem_x, s->stream>>>(
            nblk, lean[i], s->partials + total, status);
      } else {
        grid = grid_of((const void*)kpauli_xbits<double>, smem_x, kXBuf);
        kpauli_xbits<double><<<(unsigned)grid, kPThreads, smem_x, s->stream>>>(
            nblk, lean[i], s->partials + total, status);
      }
    } else {
      ProfScope prof(s->stream, c64 ? "kpauli_energy_c64" : "kpauli_energy_c128");
      if (c64) {
        grid = grid_of((const void*)kpauli_energy<float>, smem, 2);
        kpauli_energy<float><<<(unsigned)grid, kPThreads, smem, s->stream>>>(
            nblk, pf[i], s->partials + total, status);
      } else {
        grid = grid_of((const void*)kpauli_energy<double>, smem, 2);
        kpauli_energy<double><<<(unsigned)grid, kPThreads, smem, s->stream>>>(
            nblk, pd[i], s->partials + total, status);
      }
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    st = check_launch("Pauli-sum pass kernel");
    if (st) return st;
    total += (int)grid;
  }
  for (const PauliDev& P : chunks) {
    int np1 = 0;
    st = launch_expval_partials(s, P, s->partials + total, &np1);
    if (st) return st;
    total += np1;
  }
  return launch_finish(s->partials, total, 1, dst, s->stream, false);
}

// lambda = H psi into out, and <psi|H|psi> into the device double energy_dst
// if it is not null: the diagonal terms by the streaming kdiag_apply, the
// other terms by the per-amplitude kernel adding on top (its last launch
// forms the energy of the whole lambda).  SV_ERR_UNSUPPORTED (nothing
// launched) for states under 16 qubits or sums without diagonal terms.
sv_status apply_pauli_staged(void* out, const void* in, sv_state s, const sv_pauli_sum* H,
                             double* energy_dst) {
  const bool c64 = s->dt == SV_C64;
  if (s->n < 16 || H->n_terms == 0) return SV_ERR_UNSUPPORTED;
  std::vector<TermH> T;
  std::vector<uint64_t> rxm, rzm;
  std::vector<double> rcf;
  for (int k = 0; k < H->n_terms; ++k) {
    if (H->xmask[k] == 0) {
      T.push_back({0, H->zmask[k], H->coeff[k], 0.0});
    } else {
      rxm.push_back(H->xmask[k]);
      rzm.push_back(H->zmask[k]);
      rcf.push_back(H->coeff[k]);
    }
  }
  if (T.empty()) return SV_ERR_UNSUPPORTED;
  const int tb = std::min(20, std::max(8, s->n - (c64 ? 4 : 3) - 3));
  std::vector<DiagDev<float>> dfs;
  std::vector<DiagDev<double>> dds;
  diag_chunks(s->n, c64, T, tb, &dfs, &dds);
  const size_t ndiag = c64 ? dfs.size() : dds.size();
  std::vector<PauliDev> chunks;
  if (!rxm.empty()) {
    sv_pauli_sum sub{(int32_t)rxm.size(), rxm.data(), rzm.data(), rcf.data()};
    pauli_chunks(&sub, &chunks);
  }
  const unsigned dgrid = (unsigned)((uint64_t(1) << tb) / kDThreads);
  const bool diag_energy = energy_dst && chunks.empty();
  const size_t need = diag_energy ? ndiag * dgrid : energy_dst ? (size_t)kRedMaxBlocks : 0;
  sv_status st = need ? ensure_partials(s, need) : SV_OK;
  if (st) return st;
  int total = 0;
  for (size_t i = 0; i < ndiag; ++i) {
    ProfScope prof(s->stream, c64 ? "kdiag_apply_c64" : "kdiag_apply_c128");
    double* part = diag_energy ? s->partials + total : nullptr;
    if (c64)
      kdiag_apply<float><<<dgrid, kDThreads, 0, s->stream>>>(
          (float2*)out, (const float2*)in, dfs[i], i > 0 ? 1 : 0, part);
    else
      kdiag_apply<double><<<dgrid, kDThreads, 0, s->stream>>>(
          (double2*)out, (const double2*)in, dds[i], i > 0 ? 1 : 0, part);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    st = check_launch("diagonal apply kernel");
    if (st) return st;
    if (diag_energy) total += (int)dgrid;
  }
  int np = 0;
  for (size_t i = 0; i < chunks.size(); ++i) {
    const bool last = i + 1 == chunks.size();
    st = launch_apply_pauli(out, in, s->dt, s->n, s->stream, chunks[i], true,
                            (last && energy_dst) ? s->partials : nullptr, &np);
    if (st) return st;
  }
  if (energy_dst)
    return launch_finish(s->partials, diag_energy ? total : np, 1, energy_dst, s->stream, false);
  return SV_OK;
}

unsigned take_pauli_status() {
  unsigned v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_pauli_status, sizeof(v)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (v) cudaMemcpyToSymbol(g_pauli_status, &zero, sizeof(zero));
  return v;
}

static_assert(sizeof(PauliPassDev<double>) <= 32000, "kernel parameters above the launch limit");

}  // namespace sv
