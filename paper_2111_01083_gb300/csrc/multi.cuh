// Multi-cell launches of the batched operator.
//
// A batch of cells runs its per-cell phases (point and strength preparation,
// far-field formation, weights, evaluation, the NUFFT stages) as one launch
// per phase over all cells instead of one launch per cell and phase.  Each
// per-cell kernel is written as a body taking its block index explicitly and
// an argument struct; the single-cell kernel calls it with blockIdx, the
// multi-cell kernel with the block of the cell's own grid that its flat
// block index maps to (prefix table `off` of the cells' block counts, their
// grids in `dims`).
//
// While a Recorder is installed (g_rec, batch code only) the launchers
// record (phase, multi-cell kernel, grid, arguments) instead of launching;
// launches of equal (phase, kernel) across the cells become one launch, and
// phases run in increasing order, which keeps each cell's own order.
#pragma once
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

namespace pfmm {

// phases of a cell's execute, in order
enum Phase {
  PH_ZERO = 0,  // memsets of status, coefficients, NUFFT scratch, outputs
  PH_PTS,       // point preparation (sources, targets)
  PH_NET,       // net strengths (projection to zero net charge)
  PH_Q,         // strengths and moments
  PH_FORM,      // far-field formation
  PH_W,         // lattice weights
  PH_EVAL,      // evaluation (writes the outputs)
  PH_FORM2,     // modified Stokes: the Laplace family
  PH_W2,
  PH_EVAL2,     // (adds to the outputs)
  PH_SPREAD,    // NUFFT south/north: spreading
  PH_FWD,
  PH_MODES,
  PH_INV,
  PH_INTERP,    // (adds to the outputs)
  PH_COUNT
};

struct LaunchRec {
  const void* fn;  // multi-cell kernel fn(const Args* cells, const int* off, const uint3* dims, int n)
  int phase;
  int block;       // threads per block
  size_t smem;     // dynamic shared memory
  uint3 grid;      // the cell's own grid
  std::vector<unsigned char> args;
};

struct Recorder {
  std::vector<LaunchRec> recs;
};

extern thread_local Recorder* g_rec;

template <typename A>
inline void record_launch(const void* fn, int phase, dim3 grid, int block, size_t smem, const A& args) {
  LaunchRec r;
  r.fn = fn;
  r.phase = phase;
  r.block = block;
  r.smem = smem;
  r.grid = make_uint3(grid.x, grid.y, grid.z);
  r.args.resize(sizeof(A));
  std::memcpy(r.args.data(), &args, sizeof(A));
  g_rec->recs.push_back(std::move(r));
}

// Launch a single-cell kernel, or record its multi-cell twin while recording.
template <typename A>
inline cudaError_t launch_or_record(void (*single)(const A), void (*multi)(const A*, const int*, const uint3*, int),
                                    int phase, dim3 grid, int block, size_t smem, cudaStream_t st, const A& args) {
  if (grid.x == 0 || grid.y == 0 || grid.z == 0) return cudaSuccess;
  if (g_rec) {
    record_launch((const void*)multi, phase, grid, block, smem, args);
    return cudaSuccess;
  }
  single<<<grid, block, smem, st>>>(args);
  return cudaGetLastError();
}

// Status of the launches just issued; while recording nothing was launched
// (and a sticky error of unrelated earlier work, or a host without a GPU,
// must not fail the recording).
inline cudaError_t launch_status() { return g_rec ? cudaSuccess : cudaGetLastError(); }

// The block of a multi-cell launch: its cell (the last one whose first block
// is at or before it; cells with no blocks are passed over) and its index in
// that cell's grid.
struct SubBlock {
  int cell;
  uint3 bid;
};

__device__ __forceinline__ SubBlock sub_block(const int* __restrict__ off, const uint3* __restrict__ dims, int n) {
  const int b = (int)blockIdx.x;
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  const uint3 d = dims[lo];
  unsigned loc = (unsigned)(b - __ldg(off + lo));
  SubBlock s;
  s.cell = lo;
  s.bid.x = loc % d.x;
  loc /= d.x;
  s.bid.y = loc % d.y;
  s.bid.z = loc / d.y;
  return s;
}

// Single- and multi-cell kernels of a body `NAME##_body(uint3 bid, const ARGS&)`
// (non-template bodies; templates spell the two kernels out).
#define PFMM_CELL_KERNELS(NAME, ARGS, BOUNDS)                                                              \
  __global__ void BOUNDS NAME(const __grid_constant__ ARGS A) { NAME##_body(blockIdx, A); }               \
  __global__ void BOUNDS NAME##_multi(const ARGS* __restrict__ cells, const int* __restrict__ off,        \
                                      const uint3* __restrict__ dims, int n) {                             \
    const SubBlock s = sub_block(off, dims, n);                                                            \
    NAME##_body(s.bid, cells[s.cell]);                                                                     \
  }

// Memset of a range of 8-byte words (multi-cell zeroing; the single-cell
// path uses cudaMemsetAsync).
struct ZeroArgs {
  unsigned long long* p;
  long long n;
};
cudaError_t zero_or_record(void* p, size_t bytes, cudaStream_t st);

}  // namespace pfmm
