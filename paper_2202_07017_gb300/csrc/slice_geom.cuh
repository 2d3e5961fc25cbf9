// Bulk-copy (TMA) geometry of a staged slice of the state: the m staged
// amplitude-index bits S of a pass (the low run 0..L-1 plus high bits) are
// one or more boxes of a rank-2..5 tensor view of the state.  Shared by the
// fused gate passes and the Pauli-sum passes.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include <vector>

#include "sv_device.cuh"

namespace sv {

// TMA view of the state in 8-byte words (w = 1 or 2 per amplitude, lw =
// log2 w): dim 0 = the 16 words of a 128-byte row, dim 1 = rows, dims 2.. =
// chosen runs of staged bits; staged bits beyond three runs are enumerated
// as separate boxes (sw).  order: the staged bits in local (shared-memory)
// order.
struct TmaGeom {
  int rank = 0;
  int tlo[5] = {0, 0, 0, 0, 0}, thi[5] = {0, 0, 0, 0, 0};
  uint64_t dims[5] = {0, 0, 0, 0, 0}, strides[4] = {0, 0, 0, 0};
  uint32_t box[5] = {0, 0, 0, 0, 0};
  std::vector<int> order;  // staged bits in local (shared-memory) order
  std::vector<int> sw;     // staged bits enumerated as separate boxes
  int box_bits = 0;        // log2 amplitudes per box
};

bool tma_geometry(const std::vector<int>& S, int L, int n, int lw, TmaGeom* g);
// Host check of the geometry against the kernels' coordinate formula for
// slice blk (boxes inside the tensor, start addresses, bijection).
bool verify_tma(const TmaGeom& g, const std::vector<int>& S, int n, int lw, uint64_t blk);

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn();

// The copy geometry a kernel needs for one pass over `data`: the tensor
// map, zero-bit insertion at the staged bits (slice id -> base index), the
// coordinate recipe and the sizes.  Box k of the slice at base index a lands
// at k * box_bytes in shared memory; coordinate d >= 1 of a box is
// (a mod 2^thi[d]) >> tlo[d], a with the software bits swpos[j] of k added.
struct SliceDev {
  CUtensorMap tmap;  // 64-byte aligned
  Ins<uint64_t> blk;
  int m, rank, nsw, ncopies;
  uint8_t tlo[5], thi[5], swpos[12];
  uint32_t box_bytes, slice_bytes;
};

// Fills d for the staged set S (ascending, S[0..L) = 0..L-1) of an n-qubit
// state at data with 8 << lw bytes per amplitude, after checking the
// geometry on the host for the first and the last slice.  false: no
// bulk-copy geometry (the caller takes another path).
bool build_slice(const TmaGeom& g, const std::vector<int>& S, int n, int lw, void* data,
                 SliceDev* d);

__device__ __forceinline__ void slice_box_coords(const SliceDev& P, uint64_t base, int k, int* c) {
  uint64_t a = base;
  for (int j = 0; j < P.nsw; ++j)
    if ((k >> j) & 1) a |= uint64_t(1) << P.swpos[j];
  c[0] = 0;
#pragma unroll
  for (int d = 1; d < 5; ++d)
    c[d] = d < P.rank ? (int)((a & ((uint64_t(1) << P.thi[d]) - 1)) >> P.tlo[d]) : 0;
}

}  // namespace sv
