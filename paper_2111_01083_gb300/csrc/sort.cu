// Spatial sort of point sets (see sort.h).
//
//   k_sort_keys    key = (cell << 16) | Morton(bin x, bin y), value = slot
//   k_rs_hist      per 4096-slot block: histogram of one 8-bit digit
//   k_rs_scan      exclusive scan of the histograms, digit-major then block
//   k_rs_scatter   stable scatter: within a block, rank = earlier rounds +
//                  earlier warps of the round + earlier lanes of the warp
//   k_sort_gather  sorted coordinates, strengths, subtile centres, boxes
//
// LSD radix sort: each pass is stable, so equal keys keep their slot order and
// the result does not depend on scheduling.
#include <algorithm>
#include <cmath>
#include "sort.h"

namespace pfmm {

constexpr int kRsThreads = 256;
constexpr int kRsPerThread = 16;
constexpr int kRsBlock = kRsThreads * kRsPerThread;  // slots per histogram block
constexpr int kRsWarps = kRsThreads / 32;

__device__ __forceinline__ unsigned spread8(unsigned v) {
  v &= 0xFFu;
  v = (v | (v << 4)) & 0x0F0Fu;
  v = (v | (v << 2)) & 0x3333u;
  v = (v | (v << 1)) & 0x5555u;
  return v;
}

__global__ void k_sort_keys(const SortCell* __restrict__ cells, uint32_t* __restrict__ keys, int* __restrict__ vals) {
  const int c = blockIdx.y;
  const SortCell& s = cells[c];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s.n) return;
  const double x = s.xy[j], y = s.xy[(size_t)s.n + j];
  int bx = (int)floor((x - s.x0) * s.ibx), by = (int)floor((y - s.y0) * s.iby);
  bx = min(max(bx, 0), s.nbx - 1);
  by = min(max(by, 0), s.nby - 1);
  const uint32_t m = spread8((unsigned)bx) | (spread8((unsigned)by) << 1);
  keys[s.off + j] = ((uint32_t)c << 16) | m;
  vals[s.off + j] = (int)(s.off + j);
}

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                         int nblk, int* __restrict__ hist) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsBlock;
  for (int k = 0; k < kRsPerThread; ++k) {
    const int64_t e = base + k * kRsThreads + threadIdx.x;
    if (e < n) atomicAdd(&h[(keys[e] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of m ints in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_rs_scan(int* __restrict__ a, int m) {
  __shared__ int part[1024];
  const int per = (m + 1023) / 1024;
  const int lo = min(m, threadIdx.x * per), hi = min(m, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += a[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - s;  // exclusive prefix of this thread's chunk
  for (int i = lo; i < hi; ++i) {
    const int v = a[i];
    a[i] = run;
    run += v;
  }
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint32_t* __restrict__ kin, const int* __restrict__ vin,
                                                            uint32_t* __restrict__ kout, int* __restrict__ vout,
                                                            int64_t n, int shift, int nblk,
                                                            const int* __restrict__ scan) {
  __shared__ int base[256], running[256];
  __shared__ int wcnt[kRsWarps][257];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  base[t] = scan[(size_t)t * nblk + blockIdx.x];
  running[t] = 0;
  for (int w = 0; w < kRsWarps; ++w) wcnt[w][t] = 0;
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  const int64_t b0 = (int64_t)blockIdx.x * kRsBlock;
  for (int k = 0; k < kRsPerThread; ++k) {
    const int64_t e = b0 + k * kRsThreads + t;
    const bool valid = e < n;
    const uint32_t key = valid ? kin[e] : 0u;
    const int val = valid ? vin[e] : 0;
    const int d = valid ? (int)((key >> shift) & 255u) : 256;  // 256: no slot
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    if (rank == 0 && valid) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int pre = 0;
      for (int w = 0; w < warp; ++w) pre += wcnt[w][d];
      const int pos = base[d] + running[d] + pre + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    int tot = 0;
    for (int w = 0; w < kRsWarps; ++w) {
      tot += wcnt[w][t];
      wcnt[w][t] = 0;
    }
    running[t] += tot;
    __syncthreads();
  }
}

// One block per (tile of 128 sorted points, cell).  Subtile centre = centre of
// the bounding box of its 16 points (FP64), split hi/lo; relative coordinates
// use the same FP32 expression as the P2P kernels,
//   rel = (x_hi - c_hi) + (x_lo - c_lo),
// so a target that coincides with a source gives exactly zero difference.
__global__ void __launch_bounds__(kBoxTile) k_sort_gather(const SortCell* __restrict__ cells,
                                                          const int* __restrict__ vals) {
  const SortCell& s = cells[blockIdx.y];
  const int p0 = blockIdx.x * kBoxTile;
  if (p0 >= s.n) return;
  const int t = threadIdx.x, p = p0 + t;
  const bool valid = p < s.n;
  const int j = valid ? (int)(vals[s.off + p] - s.off) : 0;
  const double x = valid ? s.xy[j] : 0.0, y = valid ? s.xy[(size_t)s.n + j] : 0.0;
  if (valid) {
    s.perm[p] = j;
    if (s.xy_sorted) {
      s.xy_sorted[p] = x;
      s.xy_sorted[(size_t)s.n + p] = y;
    }
    for (int r = 0; r < s.nq; ++r) s.q_out[(size_t)r * s.n + p] = s.q_in[(size_t)r * s.n + j];
  }
  double xmn = valid ? x : INFINITY, xmx = valid ? x : -INFINITY;
  double ymn = valid ? y : INFINITY, ymx = valid ? y : -INFINITY;
  // subtile (16 lanes) bounding box
  for (int o = 8; o > 0; o >>= 1) {
    xmn = fmin(xmn, __shfl_xor_sync(0xffffffffu, xmn, o));
    xmx = fmax(xmx, __shfl_xor_sync(0xffffffffu, xmx, o));
    ymn = fmin(ymn, __shfl_xor_sync(0xffffffffu, ymn, o));
    ymx = fmax(ymx, __shfl_xor_sync(0xffffffffu, ymx, o));
  }
  const bool any = xmn <= xmx;  // the subtile holds at least one point
  const double cx = any ? 0.5 * (xmn + xmx) : 0.0, cy = any ? 0.5 * (ymn + ymx) : 0.0;
  const float cxh = (float)cx, cxl = (float)(cx - (double)cxh);
  const float cyh = (float)cy, cyl = (float)(cy - (double)cyh);
  if (s.rel) {
    if (valid) {
      const float xh = (float)x, xl = (float)(x - (double)xh);
      const float yh = (float)y, yl = (float)(y - (double)yh);
      s.rel[p] = make_float2(__fadd_rn(__fsub_rn(xh, cxh), __fsub_rn(xl, cxl)),
                             __fadd_rn(__fsub_rn(yh, cyh), __fsub_rn(yl, cyl)));
      s.hl[p] = make_float4(xh, xl, yh, yl);
    }
    if ((t & 15) == 0 && any) {
      s.sub[p / kSubtile] = make_float4(cxh, cxl, cyh, cyl);
      const float hx = (float)(0.5 * (xmx - xmn)) * (1.0f + 1e-6f) + 1e-30f;
      const float hy = (float)(0.5 * (ymx - ymn)) * (1.0f + 1e-6f) + 1e-30f;
      s.ext[p / kSubtile] = make_float2(hx, hy);
    }
  }
  // tile (128 points) box
  __shared__ double red[4][4];
  for (int o = 16; o > 8; o >>= 1) {
    xmn = fmin(xmn, __shfl_xor_sync(0xffffffffu, xmn, o));
    xmx = fmax(xmx, __shfl_xor_sync(0xffffffffu, xmx, o));
    ymn = fmin(ymn, __shfl_xor_sync(0xffffffffu, ymn, o));
    ymx = fmax(ymx, __shfl_xor_sync(0xffffffffu, ymx, o));
  }
  if ((t & 31) == 0) {
    red[t >> 5][0] = xmn;
    red[t >> 5][1] = xmx;
    red[t >> 5][2] = ymn;
    red[t >> 5][3] = ymx;
  }
  __syncthreads();
  if (t == 0 && s.box) {
    double a = red[0][0], b = red[0][1], c = red[0][2], d = red[0][3];
    for (int w = 1; w < kBoxTile / 32; ++w) {
      a = fmin(a, red[w][0]);
      b = fmax(b, red[w][1]);
      c = fmin(c, red[w][2]);
      d = fmax(d, red[w][3]);
    }
    const double mx = 0.5 * (a + b), my = 0.5 * (c + d);
    const float fx = (float)mx, fy = (float)my;
    // half extents rounded outward so that the FP32 box contains every point
    const float hx = (float)(0.5 * (b - a) + fabs(mx - (double)fx)) * (1.0f + 1e-6f) + 1e-30f;
    const float hy = (float)(0.5 * (d - c) + fabs(my - (double)fy)) * (1.0f + 1e-6f) + 1e-30f;
    s.box[p0 / kBoxTile] = make_float4(fx, fy, hx, hy);
  }
}

void sort_grid(const Geom& g, int n, SortCell* c) {
  const double W = g.d + std::fabs(g.xi), H = g.eta;
  const double nb = std::max(1.0, n / 8.0);
  int nbx = (int)std::lround(std::sqrt(nb * W / H));
  nbx = std::min(256, std::max(1, nbx));
  int nby = (int)std::lround(nb / nbx);
  nby = std::min(256, std::max(1, nby));
  c->x0 = -0.5 * W;
  c->y0 = -0.5 * H;
  c->ibx = nbx / W;
  c->iby = nby / H;
  c->nbx = nbx;
  c->nby = nby;
}

static inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
static inline int rs_blocks(int64_t total) { return (int)std::max<int64_t>(1, (total + kRsBlock - 1) / kRsBlock); }

size_t sort_scratch_bytes(int64_t total, int ncell) {
  (void)ncell;
  const size_t t = (size_t)std::max<int64_t>(1, total);
  return 4 * al256(t * 4) + al256((size_t)256 * rs_blocks(total) * sizeof(int));
}

int64_t radix_hist_ints(int64_t n) { return (int64_t)256 * rs_blocks(n); }

cudaError_t radix_sort_pairs(uint32_t* ka, int* va, uint32_t* kb, int* vb, int* hist, int64_t n, int bits,
                             cudaStream_t st, bool* in_b, int* nlaunch) {
  *in_b = false;
  if (n <= 0) return cudaSuccess;
  const int nblk = rs_blocks(n);
  bool b = false;
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_hist<<<nblk, kRsThreads, 0, st>>>(b ? kb : ka, n, shift, nblk, hist);
    k_rs_scan<<<1, 1024, 0, st>>>(hist, 256 * nblk);
    k_rs_scatter<<<nblk, kRsThreads, 0, st>>>(b ? kb : ka, b ? vb : va, b ? ka : kb, b ? va : vb, n, shift, nblk,
                                              hist);
    b = !b;
    if (nlaunch) *nlaunch += 3;
  }
  *in_b = b;
  return cudaGetLastError();
}

cudaError_t scan_small(int* a, int m, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  k_rs_scan<<<1, 1024, 0, st>>>(a, m);
  return cudaGetLastError();
}

cudaError_t sort_cells(const SortCell* cells, const SortCell* hcells, int ncell, int64_t total, char* scratch,
                       cudaStream_t st, int* nlaunch) {
  if (total <= 0 || ncell <= 0) return cudaSuccess;
  const size_t t = (size_t)total;
  uint32_t* ka = (uint32_t*)scratch;
  uint32_t* kb = (uint32_t*)(scratch + al256(t * 4));
  int* va = (int*)(scratch + 2 * al256(t * 4));
  int* vb = (int*)(scratch + 3 * al256(t * 4));
  int* hist = (int*)(scratch + 4 * al256(t * 4));
  int nmax = 0;
  for (int c = 0; c < ncell; ++c) nmax = std::max(nmax, hcells[c].n);
  if (nmax == 0) return cudaSuccess;
  k_sort_keys<<<dim3((nmax + 255) / 256, ncell), 256, 0, st>>>(cells, ka, va);
  int bits = 16;
  while ((1 << (bits - 16)) < ncell) ++bits;
  const int nblk = rs_blocks(total);
  int launches = 1;
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_hist<<<nblk, kRsThreads, 0, st>>>(ka, total, shift, nblk, hist);
    k_rs_scan<<<1, 1024, 0, st>>>(hist, 256 * nblk);
    k_rs_scatter<<<nblk, kRsThreads, 0, st>>>(ka, va, kb, vb, total, shift, nblk, hist);
    std::swap(ka, kb);
    std::swap(va, vb);
    launches += 3;
  }
  k_sort_gather<<<dim3((nmax + kBoxTile - 1) / kBoxTile, ncell), kBoxTile, 0, st>>>(cells, va);
  ++launches;
  if (nlaunch) *nlaunch += launches;
  return cudaGetLastError();
}

}  // namespace pfmm
