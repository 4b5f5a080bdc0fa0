// Near-image sum K^near q by a tree code with complex-variable expansions.
//
// The near field of the periodic operator is the free-space sum over the
// near images l of every source (Sec. 1, Definition of Lambda_near; Eq.
// nearfarsplit).  The paper evaluates it with a free-space FMM over the near
// block, and notes (Sec. 7) that the image cells share the unit cell's
// multipole moments.  This file does the same on the GPU: one quadtree over
// the unit cell's sources, whose image copies are the same boxes shifted by
// l (their expansions are the unit cell's, about shifted centres), and one
// over the targets (the same tree when targets = sources).
//
// Kernels (2D, z = x + i y, Delta = t - w for a source image w = s + l):
//  Laplace  u = -(1/2pi) sum q log|Delta|:  with F(z) = sum q log(z - w),
//           u = -(1/2pi) Re F and (u_x, u_y) = -(1/2pi) (Re F', -Im F').
//  Stokes   -(1/4pi)(log r I - r r^T/r^2) f, in complex form (U = u_1 + i u_2,
//           f = f_1 + i f_2): U = -(1/4pi) [f log|Delta| - f/2 - conj(conj(Delta) f / Delta)/2].
//           About a box centre c with u = t - c:
//             sum U = -(1/4pi) (L_1 + i L_2) + (1/8pi) conj(conj(u) C_1 - C_d),
//           L_k = sum f_k (log|Delta| - 1/2) (real-charge log sums),
//           C_1 = sum f / Delta and C_d = sum f conj(w - c) / Delta (Cauchy sums).
//           So four complex expansions per right-hand side (channels f_1, f_2,
//           f, f conj(w - c)); the box-relative charge of the fourth picks up
//           conj(shift) times the third when expansions move between centres.
//
// Expansions are scaled by the box radius R (largest distance of the box's
// points from its centre c): a source box carries
//   F(z) = Q log(z - c) + sum_{k=1}^{p-1} a_k (R / (z - c))^k,
//   Q = sum q_j,  a_k = -(1/k) sum q_j ((s_j - c)/R)^k,
// a target box F(z) = sum_{l<p} b_l ((z - c)/R)^l.  The translations are the
// textbook binomial re-expansions of log and of negative powers; M2M and L2L
// run in FP64, M2L in FP32 on the mixed path with FP64 accumulation.
//
// Pipeline (all on the caller's stream, nothing synchronises):
//  1 keys      key = set | root column | Morton(11 levels) of each point
//  2 sort      one radix sort of sources and targets (sort.cu)
//  3 gather    sorted coordinates (FP64 and hi/lo FP32), strengths
//  4 count     per point the range of tree levels at which it starts a box
//  5 scan      box numbering in preorder (a box's subtree is a contiguous range)
//  6 fill      box arrays: point range, level, parent, subtree end, geometry
//  7 up        one launch: leaf radii + P2M, then each box's radius + M2M by
//              whichever warp completes its last child (no waiting)
//  8 traverse  dual tree sweeps over (target box, source box, image) triples:
//              accepted -> M2L list, two leaves -> P2P list, else split
//  9 group     M2L and P2P lists grouped by target box (counting sort)
// 10 down      M2L over the flat grouped list (chunks per warp), then per
//              level L2L from the parent
// 11 leaf      per target leaf L2P, then the direct sums of neighbouring
//              leaves over the flat grouped list with hi/lo FP32 differences
// 12 fallback  if any list or the box count overran its capacity, the direct
//              sum over all pairs replaces steps 7-11 (their kernels return early)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "pfmm_impl.h"
#include "devmath.cuh"
#include "packed.cuh"
#include "sort.h"

namespace pfmm {

namespace {

constexpr int kKeyColShift = 2 * kFmmL;        // 22: Morton bits below
constexpr int kKeySetShift = kKeyColShift + 8;  // 30: root columns < 256
constexpr int kScanBlock = 4096;                // ints per block of the multi-block scan
constexpr int kLeafThreads = 128;
constexpr int kUpWarps = 4;
constexpr int kDownWarps = 4;
constexpr int kCtlWords = 64;
constexpr int kImgShift = 26;                   // list entries pack a box index and an image
constexpr int kBoxMask = (1 << kImgShift) - 1;
// control words
constexpr int C_OVERFLOW = 0, C_NNODES = 1, C_NM2L = 2, C_NP2P = 3, C_NRS = 4, C_NRT = 5, C_FRONT = 8;
constexpr int C_PAIRS = 48;  // uint64 at word 48 (8-byte aligned): directly evaluated pairs (profiling)
constexpr int C_P2PNEXT = 40;  // next chunk of the leaf direct sums (dynamic schedule)

struct BinomTable {
  double c[64][64];
};
constexpr BinomTable make_binom() {
  BinomTable t{};
  for (int n = 0; n < 64; ++n) {
    t.c[n][0] = 1.0;
    for (int k = 1; k <= n; ++k) t.c[n][k] = t.c[n - 1][k - 1] + (k <= n - 1 ? t.c[n - 1][k] : 0.0);
  }
  return t;
}
struct BinomTableF {
  float c[64][64];
};
constexpr BinomTableF make_binom_f() {
  BinomTable d = make_binom();
  BinomTableF t{};
  for (int n = 0; n < 64; ++n)
    for (int k = 0; k < 64; ++k) t.c[n][k] = (float)d.c[n][k];
  return t;
}
// binomial coefficients C(n, k), n, k < 64
__device__ const BinomTable g_binom = make_binom();
__device__ const BinomTableF g_binom_f = make_binom_f();

struct FmmArgs {
  int ns, nt, n;          // sources, targets of this execute; points sorted (ns + separate targets)
  int self;               // targets = sources (one tree)
  int nrhs, nchan, nleaf, nimg, nout, kernel;
  double theta;
  double x0, y0, s0;
  int ncol;
  double off[kMaxNear][2];
  double rot[4];
  int64_t os;
  int* ctl;
  uint32_t* key;          // sorted keys (after the sort)
  int* val;               // sorted slot -> input slot
  double2* xy;            // sorted coordinates
  float4* hl;             // sorted (x_hi, x_lo, y_hi, y_lo)
  int* perm;              // sorted position -> index within its set
  double* qd;             // [nrhs * ncomp][ns] sorted strengths (FP64)
  float* qf;              // same, FP32
  int* cnt;               // [n + 1] boxes starting at each point, then their preorder offsets
  signed char* lf;        // [n] first level at which the point starts a box (-1: none)
  int* bsum;              // block sums of the scans
  int *lo, *hi, *lev, *par, *nend, *nch, *done;
  double2* ctr;
  double* half;
  double* rad;
  float* scl;             // expansion scale box_scale(rad, half) in FP32
  float offh[kMaxNear][2], offl[kMaxNear][2];  // image offsets as FP32 hi/lo pairs
  double2* mult;          // [exp_cap][nchan][p]
  double2* loc;           // [exp_cap][nchan][p]
  int2* front;            // 2 x front_cap (A, C | image << 26)
  int2* m2l;
  int2* p2p;
  int* gcnt;              // [2 node_cap + 1] counts, then offsets (M2L lists, then P2P lists)
  int* gcur;              // [2 node_cap] scatter cursors
  int* glist;             // C | image << 26, grouped by target box
  int* gtgt;              // target box of each grouped M2L entry
  int* roots;             // [2][256] source roots, target roots
  int64_t node_cap, exp_cap, m2l_cap, p2p_cap, front_cap;
  const double* src64;    // canonical coordinates [2][ns] / [2][nt]
  const double* trg64;
  const double* qc;       // canonical strengths [nrhs][ncomp][ns]
  double* pot;
  double* grad;
  bool count_pairs;
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cpow(double2 z, int k) {
  double2 r = make_double2(1.0, 0.0);
  while (k) {
    if (k & 1) r = cmul(r, z);
    z = cmul(z, z);
    k >>= 1;
  }
  return r;
}
__device__ __forceinline__ float2 cpowf(float2 z, int k) {
  float2 r = make_float2(1.f, 0.f);
  while (k) {
    if (k & 1) r = cmulf(r, z);
    z = cmulf(z, z);
    k >>= 1;
  }
  return r;
}
__device__ __forceinline__ double2 ldcg2(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ float fpowi(float x, int k) {
  float r = 1.0f;
  while (k) {
    if (k & 1) r *= x;
    x *= x;
    k >>= 1;
  }
  return r;
}
__device__ __forceinline__ double dpowi(double x, int k) {
  double r = 1.0;
  while (k) {
    if (k & 1) r *= x;
    x *= x;
    k >>= 1;
  }
  return r;
}

__device__ __forceinline__ uint32_t spread11(uint32_t v) {
  v &= 0x7FFu;
  v = (v | (v << 8)) & 0x00FF00FFu;
  v = (v | (v << 4)) & 0x0F0F0F0Fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}
__device__ __forceinline__ uint32_t compact11(uint32_t v) {
  v &= 0x55555555u;
  v = (v | (v >> 1)) & 0x33333333u;
  v = (v | (v >> 2)) & 0x0F0F0F0Fu;
  v = (v | (v >> 4)) & 0x00FF00FFu;
  v = (v | (v >> 8)) & 0x0000FFFFu;
  return v;
}
__device__ __forceinline__ int level_shift(int l) { return 2 * (kFmmL - l); }

// first j in [lo, hi) with (key[j] >> sh) > P, resp. >= P (keys sorted)
__device__ int upper_prefix(const uint32_t* key, int lo, int hi, uint32_t P, int sh) {
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if ((key[m] >> sh) > P) hi = m;
    else lo = m + 1;
  }
  return lo;
}
__device__ int lower_prefix(const uint32_t* key, int lo, int hi, uint32_t P, int sh) {
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if ((key[m] >> sh) >= P) hi = m;
    else lo = m + 1;
  }
  return lo;
}

// box scale for the expansions: the radius, kept away from zero
__device__ __forceinline__ double box_scale(double rad, double half) { return fmax(rad, half * 1e-7); }

// ---------------------------------------------------------------------------
// 1-3: keys, gather
__global__ void k_fmm_keys(FmmArgs a, uint32_t* __restrict__ key, int* __restrict__ val) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const bool src = i < a.ns;
  const int j = src ? i : i - a.ns;
  const int m = src ? a.ns : a.nt;
  const double* xy = src ? a.src64 : a.trg64;
  const double x = xy[j], y = xy[(size_t)m + j];
  const double gx = (x - a.x0) / a.s0, gy = (y - a.y0) / a.s0;
  int col = (int)floor(gx);
  col = min(max(col, 0), a.ncol - 1);
  const double fx = gx - col;
  int ix = (int)floor(fx * (1 << kFmmL)), iy = (int)floor(gy * (1 << kFmmL));
  ix = min(max(ix, 0), (1 << kFmmL) - 1);
  iy = min(max(iy, 0), (1 << kFmmL) - 1);
  key[i] = ((uint32_t)(src ? 0 : 1) << kKeySetShift) | ((uint32_t)col << kKeyColShift) | spread11(ix) |
           (spread11(iy) << 1);
  val[i] = i;
}

__global__ void k_fmm_gather(FmmArgs a, int ncq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int slot = a.val[i];
  const bool src = slot < a.ns;
  const int j = src ? slot : slot - a.ns;
  const int m = src ? a.ns : a.nt;
  const double* xy = src ? a.src64 : a.trg64;
  const double x = xy[j], y = xy[(size_t)m + j];
  a.xy[i] = make_double2(x, y);
  const float xh = (float)x, yh = (float)y;
  a.hl[i] = make_float4(xh, (float)(x - (double)xh), yh, (float)(y - (double)yh));
  a.perm[i] = j;
  if (src)
    for (int c = 0; c < ncq; ++c) {
      const double v = a.qc[(size_t)c * a.ns + j];
      a.qd[(size_t)c * a.ns + i] = v;
      a.qf[(size_t)c * a.ns + i] = (float)v;
    }
}

// ---------------------------------------------------------------------------
// 4-6: tree
//
// Point i starts a box at level l when its level-l key prefix differs from
// that of point i - 1; once it does, it starts boxes at all finer levels.  The
// box (l, i) is in the tree when its parent holds more than nleaf points
// (then every ancestor does too), and it is a leaf when it holds at most
// nleaf points or l = kFmmL.  So the boxes point i starts are the levels
// lf .. lf + cnt - 1, and numbering boxes by (first point, level) is a
// preorder of the tree.
__global__ void k_fmm_count(FmmArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > a.n) return;
  if (i == a.n) {
    a.cnt[i] = 0;  // the scan turns this into the total
    return;
  }
  const uint32_t k = a.key[i];
  int lf = 0;
  if (i > 0) {
    const uint32_t d = k ^ a.key[i - 1];
    if (d == 0) {
      a.cnt[i] = 0;
      a.lf[i] = -1;
      return;
    }
    const int h = 31 - __clz(d);
    lf = max(0, kFmmL - (h >> 1));
  }
  if (lf > 0) {
    const int sh = level_shift(lf - 1);
    const uint32_t P = k >> sh;
    const int b0 = lower_prefix(a.key, 0, i, P, sh);
    const int b1 = upper_prefix(a.key, i, a.n, P, sh);
    if (b1 - b0 <= a.nleaf) {  // the parent is a leaf: no box starts here
      a.cnt[i] = 0;
      a.lf[i] = -1;
      return;
    }
  }
  int l = lf, end = a.n;
  for (;; ++l) {
    const int sh = level_shift(l);
    end = upper_prefix(a.key, i, end, k >> sh, sh);
    if (end - i <= a.nleaf || l == kFmmL) break;
  }
  a.cnt[i] = l - lf + 1;
  a.lf[i] = (signed char)lf;
}

// exclusive scan of a.cnt[0 .. n] (n + 1 entries) in three launches
__global__ void __launch_bounds__(1024) k_fmm_scan_reduce(const int* __restrict__ v, int m, int* __restrict__ bsum) {
  __shared__ int red[32];
  const int b0 = blockIdx.x * kScanBlock;
  int s = 0;
  for (int k = threadIdx.x; k < kScanBlock; k += 1024) {
    const int i = b0 + k;
    if (i < m) s += v[i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = red[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) bsum[blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(1024) k_fmm_scan_apply(int* __restrict__ v, int m, const int* __restrict__ bsum) {
  __shared__ int warp_tot[32];
  __shared__ int carry;
  const int b0 = blockIdx.x * kScanBlock;
  if (threadIdx.x == 0) carry = bsum[blockIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k0 = 0; k0 < kScanBlock; k0 += 1024) {
    const int i = b0 + k0 + threadIdx.x;
    const int x = i < m ? v[i] : 0;
    int inc = x;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
      int t = warp_tot[lane], ti = t;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, ti, o);
        if (lane >= o) ti += y;
      }
      warp_tot[lane] = ti - t;  // exclusive prefix of the warps
    }
    __syncthreads();
    const int base = carry;
    if (i < m) v[i] = base + warp_tot[w] + inc - x;
    __syncthreads();
    if (threadIdx.x == 1023) carry = base + warp_tot[w] + inc;
    __syncthreads();
  }
}

__global__ void k_fmm_fill(FmmArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    const int nn = a.cnt[a.n];
    a.ctl[C_NNODES] = nn;
    if (nn > a.exp_cap) atomicOr(a.ctl + C_OVERFLOW, 1);
  }
  if (i >= a.n) return;
  const int c = a.cnt[i + 1] - a.cnt[i];
  if (c == 0) return;
  const int lf = a.lf[i];
  const uint32_t k = a.key[i];
  const int set = (int)(k >> kKeySetShift);
  const int col = (int)((k >> kKeyColShift) & 255u);
  int end = a.n;
  for (int l = lf; l < lf + c; ++l) {
    const int id = a.cnt[i] + (l - lf);
    const int sh = level_shift(l);
    end = upper_prefix(a.key, i, end, k >> sh, sh);
    a.lo[id] = i;
    a.hi[id] = end;
    a.lev[id] = (l == lf + c - 1) ? (l | 0x100) : l;  // bit 8: leaf
    a.nend[id] = a.cnt[end];
    int parent = -1;
    if (l > lf) {
      parent = id - 1;
    } else if (l > 0) {
      const int psh = level_shift(l - 1);
      const int ps = lower_prefix(a.key, 0, i, k >> psh, psh);
      parent = a.cnt[ps] + (l - 1 - a.lf[ps]);
    }
    a.par[id] = parent;
    if (parent >= 0) atomicAdd(a.nch + parent, 1);
    const uint32_t mort = (k & ((1u << kKeyColShift) - 1u)) >> sh;
    const int bx = (int)compact11(mort), by = (int)compact11(mort >> 1);
    const double side = a.s0 / (double)(1 << l);
    a.ctr[id] = make_double2(a.x0 + col * a.s0 + (bx + 0.5) * side, a.y0 + (by + 0.5) * side);
    a.half[id] = 0.5 * side;
    (void)set;
  }
}

__device__ __forceinline__ bool is_leaf(const FmmArgs& a, int X) { return (a.lev[X] & 0x100) != 0; }
__device__ __forceinline__ int level_of(const FmmArgs& a, int X) { return a.lev[X] & 0xFF; }
__device__ __forceinline__ bool is_source(const FmmArgs& a, int X) { return a.lo[X] < a.ns; }

// ---------------------------------------------------------------------------
// 7: upward pass
//
// Channel charges: Laplace q_r; Stokes, per rhs, f_1, f_2, f, f conj(s - c).
// P2M of a source leaf; one warp.  The scaled offsets u = (s - c)/R have
// |u| <= 1, so the powers and the per-lane and per-warp sums are formed in
// FP32 (relative error ~1e-7 of sum |q|); the coefficients are stored FP64.
template <int KER>
__device__ __forceinline__ float2 channel_charge_f(const FmmArgs& a, int ch, int j, double2 s, double2 c) {
  if (KER == PFMM_LAPLACE) return make_float2(a.qf[(size_t)ch * a.ns + j], 0.f);
  const int r = ch >> 2, k = ch & 3;
  const float f1 = a.qf[((size_t)r * 2) * a.ns + j], f2 = a.qf[((size_t)r * 2 + 1) * a.ns + j];
  if (k == 0) return make_float2(f1, 0.f);
  if (k == 1) return make_float2(f2, 0.f);
  if (k == 2) return make_float2(f1, f2);
  const float dx = (float)(s.x - c.x), dy = (float)(s.y - c.y);  // f conj(s - c)
  return make_float2(f1 * dx + f2 * dy, f2 * dx - f1 * dy);
}

template <int KER>
__device__ __forceinline__ double2 channel_charge_d(const FmmArgs& a, int ch, int j, double2 s, double2 c) {
  if (KER == PFMM_LAPLACE) return make_double2(a.qd[(size_t)ch * a.ns + j], 0.0);
  const int r = ch >> 2, k = ch & 3;
  const double f1 = a.qd[((size_t)r * 2) * a.ns + j], f2 = a.qd[((size_t)r * 2 + 1) * a.ns + j];
  if (k == 0) return make_double2(f1, 0.0);
  if (k == 1) return make_double2(f2, 0.0);
  if (k == 2) return make_double2(f1, f2);
  const double dx = s.x - c.x, dy = s.y - c.y;  // f conj(s - c)
  return make_double2(f1 * dx + f2 * dy, f2 * dx - f1 * dy);
}

template <int P, int KER>
__device__ void p2m(const FmmArgs& a, int X, double R, int lane) {
  const int lo = a.lo[X], hi = a.hi[X];
  const double2 c = a.ctr[X];
  const double iR = 1.0 / R;
  for (int ch = 0; ch < a.nchan; ++ch) {
    // the box charge Q (coefficient 0) in FP64 from the FP64 strengths: its
    // Q log|z - c| term is the bulk of the far potential of the box, and an
    // FP32 rounding of Q would put a smooth error of that size on every target
    float2 acc[P];
    double2 q0 = make_double2(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < P; ++k) acc[k] = make_float2(0.f, 0.f);
    for (int j = lo + lane; j < hi; j += 32) {
      const double2 s = a.xy[j];
      const float2 u = make_float2((float)((s.x - c.x) * iR), (float)((s.y - c.y) * iR));
      const float2 q = channel_charge_f<KER>(a, ch, j, s, c);
      const double2 qd = channel_charge_d<KER>(a, ch, j, s, c);
      q0.x += qd.x;
      q0.y += qd.y;
      float2 pw = u;
#pragma unroll
      for (int k = 1; k < P; ++k) {
        const float2 t = cmulf(q, pw);
        acc[k].x += t.x;
        acc[k].y += t.y;
        pw = cmulf(pw, u);
      }
    }
    double2 mine = make_double2(0.0, 0.0);
    for (int o = 16; o > 0; o >>= 1) {
      q0.x += __shfl_xor_sync(0xffffffffu, q0.x, o);
      q0.y += __shfl_xor_sync(0xffffffffu, q0.y, o);
    }
    if (lane == 0) mine = q0;
#pragma unroll
    for (int k = 1; k < P; ++k) {
      float2 v = acc[k];
      for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
      }
      if (lane == k) mine = make_double2((double)v.x, (double)v.y);
    }
    if (lane < P) {
      if (lane > 0) mine = make_double2(-mine.x / lane, -mine.y / lane);
      a.mult[((size_t)X * a.nchan + ch) * P + lane] = mine;
    }
  }
}

// radius of a leaf from its points; one warp
__device__ double leaf_radius(const FmmArgs& a, int X, int lane) {
  const int lo = a.lo[X], hi = a.hi[X];
  const double2 c = a.ctr[X];
  double r2 = 0.0;
  for (int j = lo + lane; j < hi; j += 32) {
    const double2 s = a.xy[j];
    r2 = fmax(r2, (s.x - c.x) * (s.x - c.x) + (s.y - c.y) * (s.y - c.y));
  }
  for (int o = 16; o > 0; o >>= 1) r2 = fmax(r2, __shfl_xor_sync(0xffffffffu, r2, o));
  return sqrt(r2) * (1.0 + 1e-12);
}

// radius of an inner box from its children (an upper bound), and M2M; one
// warp.  Children are read with L2 loads: other warps wrote them before their
// fence.  Coefficients 1 .. p-1 are translated in FP32 (|w| + rho <= 1, so
// the re-expansion is well conditioned); the box charge Q (coefficient 0)
// is summed in FP64.
template <int P, int KER>
__device__ void m2m(const FmmArgs& a, int X, int lane, float2* sT, float2* sW) {
  const double2 cX = a.ctr[X];
  const int end = a.nend[X];
  double r = 0.0;
  for (int C = X + 1; C < end; C = a.nend[C]) {
    const double2 cc = a.ctr[C];
    r = fmax(r, hypot(cc.x - cX.x, cc.y - cX.y) + __ldcg(a.rad + C));
  }
  r *= (1.0 + 1e-12);
  const double R = box_scale(r, a.half[X]);
  if (lane == 0) {
    a.rad[X] = r;
    a.scl[X] = (float)R;
  }
  if (!is_source(a, X)) return;
  const float Rf = (float)R;
  const int G = KER == PFMM_STOKES ? 4 : 1;
  for (int g0 = 0; g0 < a.nchan; g0 += G) {
    float2 acc[4];
    double2 accQ[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      acc[q] = make_float2(0.f, 0.f);
      accQ[q] = make_double2(0.0, 0.0);
    }
    for (int C = X + 1; C < end; C = a.nend[C]) {
      const double2 cc = a.ctr[C];
      const double2 z1 = make_double2(cc.x - cX.x, cc.y - cX.y);
      const float2 w = make_float2((float)z1.x / Rf, (float)z1.y / Rf);
      const float rho = __ldcg(a.scl + C) / Rf;
      __syncwarp();
      if (lane < P) sW[lane] = cpowf(w, lane);
      const float rk = fpowi(rho, lane < P ? lane : 0);
      float2 prevF = make_float2(0.f, 0.f);
      double2 prevQ = make_double2(0.0, 0.0);
      for (int q = 0; q < G; ++q) {
        const double2* mc = a.mult + ((size_t)C * a.nchan + g0 + q) * P;
        const double2 ak = lane < P ? ldcg2(mc + lane) : make_double2(0.0, 0.0);
        __syncwarp();
        if (lane < P) sT[lane] = make_float2((float)ak.x * rk, (float)ak.y * rk);
        __syncwarp();
        if (lane == 0) {
          double2 sq = ak;
          if (KER == PFMM_STOKES && q == 3) {
            // f conj(s - c_X) = f conj(s - c_C) + conj(z1) f
            sq.x += z1.x * prevQ.x + z1.y * prevQ.y;
            sq.y += z1.x * prevQ.y - z1.y * prevQ.x;
          }
          prevQ = sq;
          accQ[q].x += sq.x;
          accQ[q].y += sq.y;
        } else if (lane < P) {
          const float2 Qc = sT[0];
          float2 sv = make_float2(0.f, 0.f);
          for (int k = 1; k <= lane; ++k) {
            const float b = g_binom_f.c[lane - 1][k - 1];
            const float2 t = cmulf(sT[k], sW[lane - k]);
            sv.x += b * t.x;
            sv.y += b * t.y;
          }
          const float2 wl = sW[lane];
          const float il = 1.0f / (float)lane;
          sv.x -= (Qc.x * wl.x - Qc.y * wl.y) * il;
          sv.y -= (Qc.x * wl.y + Qc.y * wl.x) * il;
          if (KER == PFMM_STOKES && q == 3) {
            const float2 t = cmulf(make_float2((float)z1.x, -(float)z1.y), prevF);
            sv.x += t.x;
            sv.y += t.y;
          }
          prevF = sv;
          acc[q].x += sv.x;
          acc[q].y += sv.y;
        }
      }
    }
    if (lane < P)
      for (int q = 0; q < G; ++q)
        a.mult[((size_t)X * a.nchan + g0 + q) * P + lane] =
            lane == 0 ? accQ[q] : make_double2((double)acc[q].x, (double)acc[q].y);
  }
}

template <int P, int KER>
__global__ void __launch_bounds__(32 * kUpWarps) k_fmm_up(FmmArgs a) {
  if (a.ctl[C_OVERFLOW]) return;
  __shared__ float2 shT[kUpWarps][kFmmMaxP], shW[kUpWarps][kFmmMaxP];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nn = a.ctl[C_NNODES];
  const int nw = gridDim.x * kUpWarps;
  for (int X = blockIdx.x * kUpWarps + wib; X < nn; X += nw) {
    if (!is_leaf(a, X)) continue;
    const double r = leaf_radius(a, X, lane);
    if (lane == 0) {
      a.rad[X] = r;
      a.scl[X] = (float)box_scale(r, a.half[X]);
    }
    if (is_source(a, X)) p2m<P, KER>(a, X, box_scale(r, a.half[X]), lane);
    int cur = X;
    for (;;) {
      // every lane's writes of this box (radius, expansion) before lane 0's
      // signal to the parent: warp barrier, then a device-scope fence
      __syncwarp();
      __threadfence();
      const int parent = a.par[cur];
      if (parent < 0) break;
      int old = 0;
      if (lane == 0) old = atomicAdd(a.done + parent, 1);
      old = __shfl_sync(0xffffffffu, old, 0);
      if (old != a.nch[parent] - 1) break;  // another child's warp finishes the parent
      __threadfence();
      m2m<P, KER>(a, parent, lane, shT[wib], shW[wib]);
      cur = parent;
    }
  }
}

// ---------------------------------------------------------------------------
// 8: traversal
__global__ void k_fmm_roots(FmmArgs a) {
  if (threadIdx.x != 0 || a.ctl[C_OVERFLOW]) return;
  const int nn = a.ctl[C_NNODES];
  int ns = 0, nt = 0;
  for (int r = 0; r < nn; r = a.nend[r]) {
    if (is_source(a, r)) {
      if (ns < 256) a.roots[ns++] = r;
    } else if (nt < 256) {
      a.roots[256 + nt++] = r;
    }
  }
  if (a.self) {
    for (int k = 0; k < ns; ++k) a.roots[256 + k] = a.roots[k];
    nt = ns;
  }
  a.ctl[C_NRS] = ns;
  a.ctl[C_NRT] = nt;
  const long long tot = (long long)ns * nt * a.nimg;
  if (tot > a.front_cap) atomicOr(a.ctl + C_OVERFLOW, 2);
  a.ctl[C_FRONT] = (int)(tot < a.front_cap ? tot : a.front_cap);
}

__global__ void k_fmm_init(FmmArgs a) {
  if (a.ctl[C_OVERFLOW]) return;
  const int ns = a.ctl[C_NRS], nt = a.ctl[C_NRT];
  const int tot = a.ctl[C_FRONT];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
    const int img = e % a.nimg, C = (e / a.nimg) % ns, A = e / (a.nimg * ns);
    a.front[e] = make_int2(a.roots[256 + A], a.roots[C] | (img << kImgShift));
  }
  (void)nt;
}

__device__ __forceinline__ int append(int* counter, int n, int64_t cap, int* ctl, int bit) {
  const int b = atomicAdd(counter, n);
  if ((int64_t)b + n > cap) {
    atomicOr(ctl + C_OVERFLOW, bit);
    return -1;
  }
  return b;
}

__global__ void k_fmm_traverse(FmmArgs a, int it) {
  if (a.ctl[C_OVERFLOW]) return;
  const int n = a.ctl[C_FRONT + it];
  const int2* fin = a.front + (size_t)(it & 1) * a.front_cap;
  int2* fout = a.front + (size_t)((it + 1) & 1) * a.front_cap;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int2 pr = fin[e];
    const int A = pr.x, C = pr.y & kBoxMask, img = pr.y >> kImgShift;
    const double2 cA = a.ctr[A], cC = a.ctr[C];
    const double dx = cC.x + a.off[img][0] - cA.x, dy = cC.y + a.off[img][1] - cA.y;
    const double D = sqrt(dx * dx + dy * dy);
    const double rA = a.rad[A], rC = a.rad[C];
    const bool la = is_leaf(a, A), lc = is_leaf(a, C);
    if (rA + rC <= a.theta * D) {
      const int b = append(a.ctl + C_NM2L, 1, a.m2l_cap, a.ctl, 4);
      if (b >= 0) a.m2l[b] = pr;
    } else if (la && lc) {
      const int b = append(a.ctl + C_NP2P, 1, a.p2p_cap, a.ctl, 8);
      if (b >= 0) a.p2p[b] = pr;
    } else {
      int ca[4], cc[4], na = 0, nc = 0;
      if (la) ca[na++] = A;
      else
        for (int x = A + 1; x < a.nend[A] && na < 4; x = a.nend[x]) ca[na++] = x;
      if (lc) cc[nc++] = C;
      else
        for (int x = C + 1; x < a.nend[C] && nc < 4; x = a.nend[x]) cc[nc++] = x;
      const int b = append(a.ctl + C_FRONT + it + 1, na * nc, a.front_cap, a.ctl, 16);
      if (b >= 0)
        for (int i = 0; i < na; ++i)
          for (int j = 0; j < nc; ++j) fout[b + i * nc + j] = make_int2(ca[i], cc[j] | (img << kImgShift));
    }
  }
}

__global__ void k_fmm_traverse_check(FmmArgs a) {
  if (threadIdx.x == 0 && a.ctl[C_FRONT + kFmmIter] > 0) atomicOr(a.ctl + C_OVERFLOW, 32);
}

// ---------------------------------------------------------------------------
// 9: grouping by target box
__global__ void k_fmm_hist(FmmArgs a) {
  if (a.ctl[C_OVERFLOW]) return;
  const int nm = a.ctl[C_NM2L], np = a.ctl[C_NP2P];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nm + np; e += gridDim.x * blockDim.x) {
    if (e < nm) atomicAdd(a.gcnt + a.m2l[e].x, 1);
    else atomicAdd(a.gcnt + a.node_cap + a.p2p[e - nm].x, 1);
  }
}

__global__ void k_fmm_scatter(FmmArgs a) {
  if (a.ctl[C_OVERFLOW]) return;
  const int nm = a.ctl[C_NM2L], np = a.ctl[C_NP2P];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nm + np; e += gridDim.x * blockDim.x) {
    const int2 v = e < nm ? a.m2l[e] : a.p2p[e - nm];
    const int64_t slot = (e < nm ? 0 : a.node_cap) + v.x;
    const int pos = a.gcnt[slot] + atomicAdd(a.gcur + slot, 1);
    a.glist[pos] = v.y;
    a.gtgt[pos] = v.x;
  }
}

// Sort each target box's M2L and P2P segments by their entries (C | image,
// unique within a segment), one warp per segment, rank by counting in shared
// memory.  The scatter fills segments in atomic order; sorted, the chunks of
// the M2L pass and the warps' shares of the leaf pass see the same entries
// in the same order on every execute, so their FP32 partial sums repeat.
// Segments longer than kSegMax keep the scatter's order.
constexpr int kSegMax = 256;
constexpr int kSortWarps = 4;

__global__ void __launch_bounds__(32 * kSortWarps) k_fmm_sortseg(FmmArgs a) {
  if (a.ctl[C_OVERFLOW]) return;
  __shared__ int sk[kSortWarps][kSegMax];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nn = a.ctl[C_NNODES];
  const int nw = gridDim.x * kSortWarps;
  for (int idx = blockIdx.x * kSortWarps + wib; idx < 2 * nn; idx += nw) {
    const int X = idx >> 1;
    const int64_t base = (idx & 1) ? a.node_cap : 0;
    const int b = a.gcnt[base + X], e = a.gcnt[base + X + 1], n = e - b;
    if (n <= 1 || n > kSegMax) continue;
    __syncwarp();
    for (int i = lane; i < n; i += 32) sk[wib][i] = a.glist[b + i];
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      const int key = sk[wib][i];
      int rank = 0;
      for (int j = 0; j < n; ++j) rank += sk[wib][j] < key;
      a.glist[b + rank] = key;
    }
  }
}

// ---------------------------------------------------------------------------
// 10: downward pass.
// (a) M2L over the flat list grouped by target box: each warp takes
// kM2LChunk consecutive entries, lane l holds local coefficient l (FP32
// arithmetic, FP64 partial sums) and adds its partial sums to the box's local
// expansion (zeroed before) with FP64 atomics whenever the target box changes
// and at the end of its chunk.  Boxes with long lists are spread over many
// warps, so the pass is not bound by one warp walking one box's list.
constexpr int kM2LChunk = 8;

template <int P, int KER>
__device__ __forceinline__ void m2l_flush(const FmmArgs& a, int X, int g0, int G, int lane, const float2* acc) {
  if (lane >= P) return;
  for (int q = 0; q < G; ++q) {
    double2* d = a.loc + ((size_t)X * a.nchan + g0 + q) * P + lane;
    atomicAdd(&d->x, (double)acc[q].x);
    atomicAdd(&d->y, (double)acc[q].y);
  }
}

// The entry's geometry is FP32 except the difference of the FP64 box centres
// (z0 = c_C + l - c_X, |z0| >= (r_X + r_C) / theta, so its FP32 rounding is
// relative); the chunk's partial sums are FP32 (at most kM2LChunk terms) and
// are added to the FP64 expansion by the flush.  (FP64 arithmetic here made
// the pass FP64-pipe bound on this part, whose FP64 rate is ~1/74 of FP32.)
template <int P, int KER>
__global__ void __launch_bounds__(32 * kDownWarps) k_fmm_m2l(FmmArgs a) {
  if (a.ctl[C_OVERFLOW]) return;
  __shared__ float2 shT[kDownWarps][kFmmMaxP];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float2* sT = shT[wib];
  const int nm = a.ctl[C_NM2L];
  const int G = KER == PFMM_STOKES ? 4 : 1;
  const int nw = gridDim.x * kDownWarps;
  const int pl = lane < P ? lane : 0;
  for (int e0 = (blockIdx.x * kDownWarps + wib) * kM2LChunk; e0 < nm; e0 += nw * kM2LChunk) {
    const int e1 = min(nm, e0 + kM2LChunk);
    for (int g0 = 0; g0 < a.nchan; g0 += G) {
      float2 acc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);
      int cur = a.gtgt[e0];
      double2 cX = a.ctr[cur];
      float RX = a.scl[cur];
      for (int e = e0; e < e1; ++e) {
        const int X = a.gtgt[e];
        if (X != cur) {
          m2l_flush<P, KER>(a, cur, g0, G, lane, acc);
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);
          cur = X;
          cX = a.ctr[X];
          RX = a.scl[X];
        }
        const int ci = a.glist[e];
        const int C = ci & kBoxMask, img = ci >> kImgShift;
        const double2 cC = a.ctr[C];
        const float zx = (float)(cC.x + a.off[img][0] - cX.x), zy = (float)(cC.y + a.off[img][1] - cX.y);
        const float RC = a.scl[C];
        const float z2 = zx * zx + zy * zy;
        const float iz2 = 1.0f / z2;
        // rho_M = -R_C / z0, rho_L = R_X / z0
        const float2 rM = make_float2(-RC * zx * iz2, RC * zy * iz2);
        const float2 rL = make_float2(RX * zx * iz2, -RX * zy * iz2);
        const float2 pM = cpowf(rM, pl);
        const float2 pL = cpowf(rL, pl);
        const float lgz = 0.5f * logf(z2);
        float2 prev = make_float2(0.f, 0.f);
        for (int q = 0; q < G; ++q) {
          const double2 ak = lane < P ? a.mult[((size_t)C * a.nchan + g0 + q) * P + lane] : make_double2(0.0, 0.0);
          __syncwarp();
          if (lane < P) sT[lane] = cmulf(make_float2((float)ak.x, (float)ak.y), pM);
          __syncwarp();
          const float2 Q = sT[0];
          float2 sv = make_float2(0.f, 0.f);
          if (lane < P) {
#pragma unroll 4
            for (int k = 1; k < P; ++k) {
              const float b = g_binom_f.c[k + lane - 1][lane];
              sv.x += b * sT[k].x;
              sv.y += b * sT[k].y;
            }
            if (lane == 0) {
              // Q log(z - c_C) about c_X: Q log(-z0) + ...; only its real part is
              // used.  Stokes log channels carry the Stokeslet's -f/2 in their constant.
              const float c0 = (KER == PFMM_STOKES && q < 2) ? lgz - 0.5f : lgz;
              sv.x += Q.x * c0;
              sv.y += Q.y * c0;
            } else {
              const float il = 1.0f / (float)lane;
              sv = cmulf(pL, make_float2(sv.x - Q.x * il, sv.y - Q.y * il));
            }
          }
          if (KER == PFMM_STOKES && q == 3) {
            // f conj(w - c_X) = f conj(s - c_C) + conj(z0) f
            const float2 t = cmulf(make_float2(zx, -zy), prev);
            sv.x += t.x;
            sv.y += t.y;
          }
          prev = sv;
          acc[q].x += sv.x;
          acc[q].y += sv.y;
        }
      }
      m2l_flush<P, KER>(a, cur, g0, G, lane, acc);
    }
  }
}

// (b) L2L, one level per launch (parents are final when their level is):
// one warp per target box of the level adds the translated parent expansion
// to its own.  Coefficients 1 .. p-1 in FP32 (|w| + rho <= 1); the constant
// term, the bulk of the potential, keeps b_0 of the parent in FP64.
template <int P, int KER>
__global__ void __launch_bounds__(32 * kDownWarps) k_fmm_l2l(FmmArgs a, int level) {
  if (a.ctl[C_OVERFLOW]) return;
  __shared__ float2 shB[kDownWarps][kFmmMaxP], shW[kDownWarps][kFmmMaxP];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float2* sB = shB[wib];
  float2* sW = shW[wib];
  const int nn = a.ctl[C_NNODES];
  const int nw = gridDim.x * kDownWarps;
  const int G = KER == PFMM_STOKES ? 4 : 1;
  for (int X = blockIdx.x * kDownWarps + wib; X < nn; X += nw) {
    if (level_of(a, X) != level) continue;
    if (a.self ? !is_source(a, X) : is_source(a, X)) continue;
    const int parent = a.par[X];
    if (parent < 0) continue;
    const double2 cX = a.ctr[X], cP = a.ctr[parent];
    const float RP = a.scl[parent];
    const double2 z2 = make_double2(cX.x - cP.x, cX.y - cP.y);
    const float2 w = make_float2((float)z2.x / RP, (float)z2.y / RP);
    const float rm = fpowi(a.scl[X] / RP, lane < P ? lane : 0);
    __syncwarp();
    if (lane < P) sW[lane] = cpowf(w, lane);
    for (int g0 = 0; g0 < a.nchan; g0 += G) {
      float2 prevF = make_float2(0.f, 0.f);
      double2 prevD = make_double2(0.0, 0.0);
      for (int q = 0; q < G; ++q) {
        const double2 b = lane < P ? a.loc[((size_t)parent * a.nchan + g0 + q) * P + lane] : make_double2(0.0, 0.0);
        __syncwarp();
        if (lane < P) sB[lane] = lane == 0 ? make_float2(0.f, 0.f) : make_float2((float)b.x, (float)b.y);
        __syncwarp();
        float2 sv = make_float2(0.f, 0.f);
        if (lane < P) {
          for (int l = max(lane, 1); l < P; ++l) {
            const float bc = g_binom_f.c[l][lane];
            const float2 t = cmulf(sB[l], sW[l - lane]);
            sv.x += bc * t.x;
            sv.y += bc * t.y;
          }
          sv.x *= rm;
          sv.y *= rm;
        }
        double2 dv = make_double2(0.0, 0.0);
        if (lane == 0) dv = make_double2(b.x + (double)sv.x, b.y + (double)sv.y);
        if (KER == PFMM_STOKES && q == 3) {
          // f conj(w - c_X) = f conj(w - c_P) - conj(z2) f
          if (lane == 0) {
            dv.x -= z2.x * prevD.x + z2.y * prevD.y;
            dv.y -= z2.x * prevD.y - z2.y * prevD.x;
          } else {
            const float2 t = cmulf(make_float2((float)z2.x, -(float)z2.y), prevF);
            sv.x -= t.x;
            sv.y -= t.y;
          }
        }
        prevF = sv;
        prevD = dv;
        if (lane < P) {
          double2* d = a.loc + ((size_t)X * a.nchan + g0 + q) * P + lane;
          if (lane == 0) {
            d->x += dv.x;
            d->y += dv.y;
          } else {
            d->x += (double)sv.x;
            d->y += (double)sv.y;
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// 11: target leaves: L2P (one writer per target), then the direct sums of
// neighbouring leaves over the flat grouped list (FP64 atomics).
constexpr int kLeafWarps = 4;
// output scalings (multiplications: an FP64 division costs tens of FP64
// operations, and FP64 runs at 1/64 of the FP32 rate on this GPU)
constexpr double kInv2Pi = 0.15915494309189535;   // 1 / (2 pi)
constexpr double kInv4Pi = 0.079577471545947673;  // 1 / (4 pi)
constexpr double kInv8Pi = 0.039788735772973836;  // 1 / (8 pi)
constexpr double kLn2_4Pi = 0.055158900038162900; // ln 2 / (4 pi)

// (h + l) - (oh + ol) as an unevaluated FP32 pair (two-sum of the high
// parts, low parts added to its error): the image-shifted target coordinate
// with ~2^-47 relative precision, no FP64 arithmetic.
__device__ __forceinline__ void shift_hl(float h, float l, float oh, float ol, float& sh, float& sl) {
  const float sm = h - oh;
  const float bb = sm - h;
  const float err = (h - (sm - bb)) + (-oh - bb);
  sh = sm;
  sl = err + (l - ol);
}

// compensated FP32 sum (Kahan): value() = s - c
struct KSumF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return dm::f2d(s) - dm::f2d(c); }
};

// L2P: one thread per target of a target leaf (block per leaf,
// grid-stride), the local expansion evaluated and added to the outputs (the
// far field wrote them before; this is their only writer at this point).
template <int P, int KER>
__global__ void __launch_bounds__(32 * kLeafWarps) k_fmm_l2p(FmmArgs a) {
  if (a.ctl[C_OVERFLOW]) return;
  __shared__ float2 s_b[4][kFmmMaxP];
  __shared__ double s_b0[4];
  const int nn = a.ctl[C_NNODES];
  const int tid = threadIdx.x;
  const int G = KER == PFMM_STOKES ? 4 : 1;
  for (int X = blockIdx.x; X < nn; X += gridDim.x) {
    if (!is_leaf(a, X) || (a.self ? !is_source(a, X) : is_source(a, X))) continue;
    const int lo = a.lo[X], hi = a.hi[X];
    const double2 cX = a.ctr[X];
    const double RX = box_scale(a.rad[X], a.half[X]);
    const double iRX = 1.0 / RX;
    const float iRXf = (float)iRX;
    for (int r = 0; r < a.nrhs; ++r) {
      __syncthreads();
      if (tid < G * P) {
        const int q = tid / P, k = tid % P;
        const double2 b = a.loc[((size_t)X * a.nchan + r * G + q) * P + k];
        s_b[q][k] = make_float2((float)b.x, (float)b.y);
        if (k == 0) s_b0[q] = b.x;
      }
      __syncthreads();
      for (int t = lo + tid; t < hi; t += blockDim.x) {
        const double2 tq = a.xy[t];
        // FP32 Horner for sum_{l>=1} b_l u^l and its derivative (|u| <= 1,
        // decaying terms); the constant b_0 (the bulk of the potential) in FP64
        const float2 u = make_float2((float)((tq.x - cX.x) * iRX), (float)((tq.y - cX.y) * iRX));
        double2 F[4], D[4];
        for (int q = 0; q < G; ++q) {
          float2 f = s_b[q][P - 1], d = make_float2(0.f, 0.f);
          for (int l = P - 2; l >= 1; --l) {
            d = cmulf(d, u);
            d.x += f.x;
            d.y += f.y;
            f = cmulf(f, u);
            f.x += s_b[q][l].x;
            f.y += s_b[q][l].y;
          }
          const float2 fu = cmulf(f, u);
          const float2 du = cmulf(d, u);
          F[q] = make_double2(s_b0[q] + dm::f2d(fu.x), dm::f2d(fu.y));
          D[q] = make_double2(dm::f2d((f.x + du.x) * iRXf), dm::f2d((f.y + du.y) * iRXf));
        }
        const int o = a.perm[t];
        const double* R = a.rot;
        if (KER == PFMM_LAPLACE) {
          const double o0 = -F[0].x * kInv2Pi, o1 = -D[0].x * kInv2Pi, o2 = D[0].y * kInv2Pi;
          if (a.pot) a.pot[(size_t)r * a.os + o] += o0;
          if (a.grad) {
            a.grad[((size_t)r * 2) * a.os + o] += R[0] * o1 + R[2] * o2;
            a.grad[((size_t)r * 2 + 1) * a.os + o] += R[1] * o1 + R[3] * o2;
          }
        } else {
          const double2 du = make_double2(tq.x - cX.x, tq.y - cX.y);
          // conj(u) C_1 - C_d
          const double2 wv = make_double2(du.x * D[2].x + du.y * D[2].y - D[3].x,
                                          du.x * D[2].y - du.y * D[2].x - D[3].y);
          const double o0 = -F[0].x * kInv4Pi + wv.x * kInv8Pi;
          const double o1 = -F[1].x * kInv4Pi - wv.y * kInv8Pi;
          a.pot[((size_t)r * 2) * a.os + o] += R[0] * o0 + R[2] * o1;
          a.pot[((size_t)r * 2 + 1) * a.os + o] += R[1] * o0 + R[3] * o1;
        }
      }
    }
  }
}

// Direct sums of neighbouring leaves over the flat P2P list grouped by
// target leaf: each warp takes chunks of kP2PChunk consecutive entries from a
// counter (so a leaf with a long list is spread over many warps, and the
// uneven chunks balance dynamically), lane l sums targets l and l + 32 of
// the entry's target leaf as the two halves of packed FP32 operations
// (leaves with more targets take several passes), sources staged 32 at a
// time in the warp's slice of shared memory and read once per lane for both
// targets.  Partial sums over each 32-source block are FP32, added with
// compensation, and go to the outputs with FP64 atomics at each change of
// target leaf and at the end of the chunk.
constexpr int kP2PChunk = 4;

template <int KER>
__device__ __forceinline__ void p2p_flush(const FmmArgs& a, int X, int t0, int r, int lane, const KSumF (*acc)[3]) {
  const int hi = a.hi[X];
  const double* R = a.rot;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int t = t0 + lane + 32 * k;
    if (t >= hi) continue;
    const int o = a.perm[t];
    if (KER == PFMM_LAPLACE) {
      const double o0 = -acc[k][0].value() * kLn2_4Pi;
      const double o1 = -acc[k][1].value() * kInv2Pi, o2 = -acc[k][2].value() * kInv2Pi;
      if (a.pot) atomicAdd(a.pot + (size_t)r * a.os + o, o0);
      if (a.grad) {
        atomicAdd(a.grad + ((size_t)r * 2) * a.os + o, R[0] * o1 + R[2] * o2);
        atomicAdd(a.grad + ((size_t)r * 2 + 1) * a.os + o, R[1] * o1 + R[3] * o2);
      }
    } else {
      const double o0 = -acc[k][0].value() * kInv4Pi, o1 = -acc[k][1].value() * kInv4Pi;
      atomicAdd(a.pot + ((size_t)r * 2) * a.os + o, R[0] * o0 + R[2] * o1);
      atomicAdd(a.pot + ((size_t)r * 2 + 1) * a.os + o, R[1] * o0 + R[3] * o1);
    }
  }
}

__device__ __forceinline__ float lg2_mufu(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rcp_mufu(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <int P, int KER>
__global__ void __launch_bounds__(32 * kLeafWarps) k_fmm_p2p(FmmArgs a) {
  if (a.ctl[C_OVERFLOW]) return;
  __shared__ float4 s_hl[kLeafWarps][32];
  __shared__ float s_q[kLeafWarps][2][32];
  __shared__ unsigned long long s_pairs;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int ncomp = KER == PFMM_STOKES ? 2 : 1;
  const int64_t pb = a.gcnt[a.node_cap], pe = a.gcnt[2 * a.node_cap];  // the P2P part of the grouped list
  const int np = (int)(pe - pb);
  if (threadIdx.x == 0) s_pairs = 0;
  __syncthreads();
  unsigned long long my_pairs = 0;
  for (;;) {
    int ck = 0;
    if (lane == 0) ck = atomicAdd(a.ctl + C_P2PNEXT, 1);
    const int c0e = __shfl_sync(0xffffffffu, ck, 0) * kP2PChunk;
    if (c0e >= np) break;
    const int c1e = min(np, c0e + kP2PChunk);
    for (int r = 0; r < a.nrhs; ++r) {
      // the chunk's entries, in order; a leaf with more than 64 targets is
      // summed in passes of 64 (t0), each pass over the chunk's entries of it
      int e = c0e;
      while (e < c1e) {
        const int X = a.gtgt[pb + e];
        int ee = e + 1;
        while (ee < c1e && a.gtgt[pb + ee] == X) ++ee;
        const int lo = a.lo[X], hi = a.hi[X];
        for (int t0 = lo; t0 < hi; t0 += 64) {
          float4 thl[2];
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int t = t0 + lane + 32 * k;
            thl[k] = t < hi ? a.hl[t] : make_float4(0.f, 0.f, 0.f, 0.f);
          }
          KSumF acc[2][3];
          for (int j = e; j < ee; ++j) {
            const int ci = a.glist[pb + j];
            const int C = ci & kBoxMask, img = ci >> kImgShift;
            const int clo = a.lo[C], chi = a.hi[C];
            if (a.count_pairs && r == 0 && lane == 0)
              my_pairs += (unsigned long long)(min(hi, t0 + 64) - t0) * (unsigned long long)(chi - clo);
            // the two targets shifted by the image, packed: .x target t0 + lane, .y t0 + lane + 32
            float2 txh, txl, tyh, tyl;
            shift_hl(thl[0].x, thl[0].y, a.offh[img][0], a.offl[img][0], txh.x, txl.x);
            shift_hl(thl[1].x, thl[1].y, a.offh[img][0], a.offl[img][0], txh.y, txl.y);
            shift_hl(thl[0].z, thl[0].w, a.offh[img][1], a.offl[img][1], tyh.x, tyl.x);
            shift_hl(thl[1].z, thl[1].w, a.offh[img][1], a.offl[img][1], tyh.y, tyl.y);
            for (int cs = clo; cs < chi; cs += 32) {
              __syncwarp();
              const int jj0 = cs + lane;
              if (jj0 < chi) {
                s_hl[wib][lane] = a.hl[jj0];
                for (int c = 0; c < ncomp; ++c) s_q[wib][c][lane] = a.qf[((size_t)r * ncomp + c) * a.ns + jj0];
              }
              __syncwarp();
              const int m = min(32, chi - cs);
              float2 f0 = f2(0.f), f1 = f2(0.f), f2v = f2(0.f);
              for (int jj = 0; jj < m; ++jj) {
                const float4 sp = s_hl[wib][jj];
                const float2 dx = add2(add2(txh, f2(-sp.x)), add2(txl, f2(-sp.y)));
                const float2 dy = add2(add2(tyh, f2(-sp.z)), add2(tyl, f2(-sp.w)));
                float2 r2 = fma2(dx, dx, mul2(dy, dy));
                // a zero distance (the target itself) contributes nothing
                const float mx = r2.x > 0.f ? 1.f : 0.f, my = r2.y > 0.f ? 1.f : 0.f;
                r2 = make_float2(r2.x > 0.f ? r2.x : 1.f, r2.y > 0.f ? r2.y : 1.f);
                const float2 lg = make_float2(lg2_mufu(r2.x), lg2_mufu(r2.y));
                const float2 inv = make_float2(rcp_mufu(r2.x), rcp_mufu(r2.y));
                const float q0 = s_q[wib][0][jj];
                const float2 qm = make_float2(q0 * mx, q0 * my);
                if (KER == PFMM_LAPLACE) {
                  f0 = fma2(qm, lg, f0);
                  const float2 qi = mul2(qm, inv);
                  f1 = fma2(qi, dx, f1);
                  f2v = fma2(qi, dy, f2v);
                } else {
                  // -(1/4pi)[f log r - d (d.f)/r^2]; log r = (ln 2 / 2) log2 r^2
                  const float q1 = s_q[wib][1][jj];
                  const float2 q1m = make_float2(q1 * mx, q1 * my);
                  const float2 rf = mul2(fma2(dx, qm, mul2(dy, q1m)), inv);
                  const float2 lgh = mul2(lg, f2(0.34657359f));
                  f0 = fma2(qm, lgh, fma2(make_float2(-dx.x, -dx.y), rf, f0));
                  f1 = fma2(q1m, lgh, fma2(make_float2(-dy.x, -dy.y), rf, f1));
                }
              }
              acc[0][0].add(f0.x);
              acc[1][0].add(f0.y);
              acc[0][1].add(f1.x);
              acc[1][1].add(f1.y);
              if (KER == PFMM_LAPLACE) {
                acc[0][2].add(f2v.x);
                acc[1][2].add(f2v.y);
              }
            }
          }
          p2p_flush<KER>(a, X, t0, r, lane, acc);
        }
        e = ee;
      }
    }
  }
  if (a.count_pairs && lane == 0 && my_pairs) atomicAdd(&s_pairs, my_pairs);
  __syncthreads();
  if (a.count_pairs && threadIdx.x == 0 && s_pairs) atomicAdd((unsigned long long*)(a.ctl + C_PAIRS), s_pairs);
}

// ---------------------------------------------------------------------------
// 12: direct fallback over all (target, source, image) pairs, only after an
// overflow of a capacity (the FMM kernels above then did nothing)
template <int KER>
__global__ void __launch_bounds__(kLeafThreads) k_fmm_fallback(FmmArgs a) {
  if (!a.ctl[C_OVERFLOW]) return;
  __shared__ float4 s_hl[kLeafThreads];
  __shared__ float s_q[2][kLeafThreads];
  const int ncomp = KER == PFMM_STOKES ? 2 : 1;
  const int tbase = a.self ? 0 : a.ns;
  const int ntg = a.self ? a.ns : a.nt;
  for (int t0 = blockIdx.x * kLeafThreads; t0 < ntg; t0 += gridDim.x * kLeafThreads) {
    const int t = tbase + t0 + threadIdx.x;
    const bool valid = t0 + threadIdx.x < ntg;
    const double2 tp = valid ? a.xy[t] : make_double2(0.0, 0.0);
    for (int r = 0; r < a.nrhs; ++r) {
      double out0 = 0.0, out1 = 0.0, out2 = 0.0;
      for (int img = 0; img < a.nimg; ++img) {
        const double sx = tp.x - a.off[img][0], sy = tp.y - a.off[img][1];
        const float txh = (float)sx, txl = (float)(sx - (double)txh);
        const float tyh = (float)sy, tyl = (float)(sy - (double)tyh);
        for (int c0 = 0; c0 < a.ns; c0 += kLeafThreads) {
          __syncthreads();
          const int j = c0 + threadIdx.x;
          if (j < a.ns) {
            s_hl[threadIdx.x] = a.hl[j];
            for (int c = 0; c < ncomp; ++c) s_q[c][threadIdx.x] = a.qf[((size_t)r * ncomp + c) * a.ns + j];
          }
          __syncthreads();
          const int m = min(kLeafThreads, a.ns - c0);
          float f0 = 0.f, f1 = 0.f, f2 = 0.f;
          if (valid)
            for (int jj = 0; jj < m; ++jj) {
              const float4 s = s_hl[jj];
              const float dx = (txh - s.x) + (txl - s.y);
              const float dy = (tyh - s.z) + (tyl - s.w);
              const float r2 = dx * dx + dy * dy;
              if (r2 > 0.f) {
                const float lg = __log2f(r2), inv = __fdividef(1.0f, r2);
                if (KER == PFMM_LAPLACE) {
                  const float qq = s_q[0][jj];
                  f0 += qq * lg;
                  f1 += qq * dx * inv;
                  f2 += qq * dy * inv;
                } else {
                  const float g1 = s_q[0][jj], g2 = s_q[1][jj];
                  const float rf = (dx * g1 + dy * g2) * inv;
                  f0 += g1 * lg * 0.34657359f - dx * rf;
                  f1 += g2 * lg * 0.34657359f - dy * rf;
                }
              }
            }
          if (KER == PFMM_LAPLACE) {
            out0 += -dm::f2d(f0) * kLn2_4Pi;
            out1 += -dm::f2d(f1) * kInv2Pi;
            out2 += -dm::f2d(f2) * kInv2Pi;
          } else {
            out0 += -dm::f2d(f0) * kInv4Pi;
            out1 += -dm::f2d(f1) * kInv4Pi;
          }
        }
      }
      if (valid) {
        const int o = a.perm[t];
        const double* R = a.rot;
        if (KER == PFMM_LAPLACE) {
          if (a.pot) a.pot[(size_t)r * a.os + o] += out0;
          if (a.grad) {
            a.grad[((size_t)r * 2) * a.os + o] += R[0] * out1 + R[2] * out2;
            a.grad[((size_t)r * 2 + 1) * a.os + o] += R[1] * out1 + R[3] * out2;
          }
        } else {
          a.pot[((size_t)r * 2) * a.os + o] += R[0] * out0 + R[2] * out1;
          a.pot[((size_t)r * 2 + 1) * a.os + o] += R[1] * out0 + R[3] * out1;
        }
      }
    }
  }
}

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

cudaError_t scan_inplace(int* v, int m, int* bsum, cudaStream_t st, int* nl) {
  const int nb = cdiv(m, kScanBlock);
  k_fmm_scan_reduce<<<nb, 1024, 0, st>>>(v, m, bsum);
  cudaError_t e = scan_small(bsum, nb, st);
  if (e != cudaSuccess) return e;
  k_fmm_scan_apply<<<nb, 1024, 0, st>>>(v, m, bsum);
  *nl += 3;
  return cudaGetLastError();
}

template <int P, int KER>
cudaError_t run_expansions(const FmmArgs& a, int grid, cudaStream_t st, int* nl) {
  k_fmm_up<P, KER><<<grid, 32 * kUpWarps, 0, st>>>(a);
  ++*nl;
  return cudaGetLastError();
}

// Downward pass on st_tree, then the leaf kernels (which add into the
// outputs) on st, after st_tree's work through `join` when the streams differ.
template <int P, int KER>
cudaError_t run_down(const FmmArgs& a, int grid, cudaStream_t st_tree, int* nl, cudaEvent_t mid, cudaStream_t st,
                     cudaEvent_t join) {
  cudaError_t e = cudaMemsetAsync(a.loc, 0, (size_t)a.exp_cap * a.nchan * P * sizeof(double2), st_tree);
  if (e != cudaSuccess) return e;
  k_fmm_m2l<P, KER><<<grid, 32 * kDownWarps, 0, st_tree>>>(a);
  for (int l = 1; l <= kFmmL; ++l) k_fmm_l2l<P, KER><<<grid, 32 * kDownWarps, 0, st_tree>>>(a, l);
  if (mid) record_event(mid, st_tree);
  if (st_tree != st) {
    e = cudaEventRecord(join, st_tree);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, join, 0);
    if (e != cudaSuccess) return e;
  }
  k_fmm_l2p<P, KER><<<grid, 32 * kLeafWarps, 0, st>>>(a);
  k_fmm_p2p<P, KER><<<grid, 32 * kLeafWarps, 0, st>>>(a);
  *nl += kFmmL + 3;
  return cudaGetLastError();
}

#define PFMM_FMM_P_DISPATCH(FN, P, KER, ...)                                              \
  (KER == PFMM_LAPLACE                                                                    \
       ? (P <= 12 ? FN<12, PFMM_LAPLACE>(__VA_ARGS__)                                     \
                  : P <= 16 ? FN<16, PFMM_LAPLACE>(__VA_ARGS__)                           \
                            : P <= 20 ? FN<20, PFMM_LAPLACE>(__VA_ARGS__)                 \
                                      : P <= 24 ? FN<24, PFMM_LAPLACE>(__VA_ARGS__)       \
                                                : FN<32, PFMM_LAPLACE>(__VA_ARGS__))      \
       : (P <= 12 ? FN<12, PFMM_STOKES>(__VA_ARGS__)                                      \
                  : P <= 16 ? FN<16, PFMM_STOKES>(__VA_ARGS__)                            \
                            : P <= 20 ? FN<20, PFMM_STOKES>(__VA_ARGS__)                  \
                                      : P <= 24 ? FN<24, PFMM_STOKES>(__VA_ARGS__)        \
                                                : FN<32, PFMM_STOKES>(__VA_ARGS__)))

}  // namespace

// Expansion orders compiled: 12, 16, 20, 24, 32 (the plan rounds p up).
static int round_p(int p) { return p <= 12 ? 12 : p <= 16 ? 16 : p <= 20 ? 20 : p <= 24 ? 24 : 32; }

void fmm_setup(pfmm_plan* p) {
  FmmPlan& F = p->fmm;
  F = FmmPlan{};
  const pfmm_opts& o = p->opts;
  const bool capable = (o.kernel == PFMM_LAPLACE || o.kernel == PFMM_STOKES) && o.precision == PFMM_MIXED &&
                       !(o.flags & PFMM_DETERMINISTIC);
  bool on = false;
  if (o.flags & PFMM_NEAR_FMM) on = capable;
  else if (!(o.flags & PFMM_NEAR_DIRECT))
    on = capable && (double)p->ns_max * (double)p->nt_max * p->geom.nimg >= 2e9;
  F.on = on ? 1 : 0;
  F.theta = 0.5;
  // truncation error of one accepted interaction ~ theta^p relative to the
  // source box's charge: p from the requested tolerance
  int pp = o.near_order ? o.near_order : (int)std::ceil(std::log(o.tol * 0.1) / std::log(F.theta));
  F.p = round_p(std::max(8, std::min(kFmmMaxP, pp)));
  F.nleaf = o.near_leaf ? o.near_leaf : 128;
  const Geom& g = p->geom;
  const double W = g.d + std::fabs(g.xi), H = g.eta;
  int ncol = (int)std::ceil(W / H - 1e-9);
  ncol = std::max(1, std::min(256, ncol));
  F.s0 = std::max(H, W / ncol) * (1.0 + 1e-9);
  F.ncol = ncol;
  F.x0 = -0.5 * ncol * F.s0;
  F.y0 = -0.5 * F.s0;
  F.nchan = (o.kernel == PFMM_STOKES ? 4 : 1) * o.nrhs;
  if (!on) return;
  const int64_t n = p->ns_max + p->nt_max;
  F.npts = n;
  // every inner box holds more than nleaf points and the boxes of one level
  // partition the points: at most n / (nleaf + 1) inner boxes per level, each
  // with at most 4 children
  F.node_cap = 2 * 256 + 4 * (int64_t)(kFmmL + 1) * (n / (F.nleaf + 1) + 2);
  // boxes with expansions and list lengths: several times what uniform and
  // strongly clustered inputs produce (about 3 n / nleaf boxes, 30-60 M2L and
  // 9-20 direct leaf pairs per target box); beyond them the direct fallback runs
  F.exp_cap = std::min<int64_t>(F.node_cap, 8 * n / F.nleaf + 4096);
  F.m2l_cap = 64 * F.exp_cap;
  F.p2p_cap = 32 * F.exp_cap;
  F.front_cap = 48 * F.exp_cap + (int64_t)4 * 256 * 27;
  size_t off = 0;
  auto take = [&](size_t b) { size_t r = off; off = al256(off + std::max<size_t>(b, 1)); return r; };
  const size_t N = (size_t)n, NC = (size_t)F.node_cap;
  const int ncq = o.nrhs * p->ncomp;
  F.o_ctl = take(kCtlWords * sizeof(int));
  F.o_key = take(N * 4);
  F.o_val = take(N * 4);
  F.o_key2 = take(N * 4);
  F.o_val2 = take(N * 4);
  F.o_hist = take((size_t)radix_hist_ints(n) * 4);
  F.o_xy = take(N * sizeof(double2));
  F.o_hl = take(N * sizeof(float4));
  F.o_perm = take(N * 4);
  F.o_qd = take((size_t)ncq * p->ns_max * 8);
  F.o_qf = take((size_t)ncq * p->ns_max * 4);
  F.o_cnt = take((N + 1) * 4);
  F.o_lf = take(N);
  F.o_bsum = take((size_t)(cdiv(2 * (int64_t)NC + 1, kScanBlock) + cdiv(n + 1, kScanBlock) + 8) * 4);
  F.o_lo = take(NC * 4);
  F.o_hi = take(NC * 4);
  F.o_lev = take(NC * 4);
  F.o_par = take(NC * 4);
  F.o_nend = take(NC * 4);
  F.o_nch = take(NC * 4);
  F.o_done = take(NC * 4);
  F.o_ctr = take(NC * sizeof(double2));
  F.o_half = take(NC * 8);
  F.o_rad = take(NC * 8);
  F.o_scl = take(NC * 4);
  F.o_mult = take((size_t)F.exp_cap * F.nchan * F.p * sizeof(double2));
  F.o_loc = take((size_t)F.exp_cap * F.nchan * F.p * sizeof(double2));
  F.o_front = take((size_t)2 * F.front_cap * sizeof(int2));
  F.o_m2l = take((size_t)F.m2l_cap * sizeof(int2));
  F.o_p2p = take((size_t)F.p2p_cap * sizeof(int2));
  F.o_gcnt = take((2 * NC + 1) * 4);
  F.o_gcur = take(2 * NC * 4);
  F.o_glist = take((size_t)(F.m2l_cap + F.p2p_cap) * sizeof(int));
  F.o_gtgt = take((size_t)(F.m2l_cap + F.p2p_cap) * sizeof(int));
  F.o_roots = take(512 * 4);
  F.bytes = off;
}

cudaError_t launch_fmm_near(const pfmm_plan* p, char* ws, int64_t ns, int64_t nt, bool self, double* pot, double* grad,
                            cudaStream_t st_main, cudaStream_t st_tree, cudaEvent_t join) {
  // every phase before the leaf kernels on `st` (= st_tree when given)
  cudaStream_t st = (st_tree && join) ? st_tree : st_main;
  const FmmPlan& F = p->fmm;
  const Layout& L = p->lay;
  char* base = ws + L.fmm;
  g_launches = 0;
  if (nt == 0 || ns == 0) return cudaSuccess;
  FmmArgs a{};
  a.ns = (int)ns;
  a.nt = (int)nt;
  a.self = self ? 1 : 0;
  a.n = (int)(ns + (self ? 0 : nt));
  a.nrhs = p->opts.nrhs;
  a.nchan = F.nchan;
  a.nleaf = F.nleaf;
  a.nimg = p->geom.nimg;
  a.nout = p->nout;
  a.kernel = p->opts.kernel;
  a.theta = F.theta;
  a.x0 = F.x0;
  a.y0 = F.y0;
  a.s0 = F.s0;
  a.ncol = F.ncol;
  for (int i = 0; i < a.nimg; ++i)
    for (int k = 0; k < 2; ++k) {
      a.off[i][k] = p->geom.off[i][k];
      a.offh[i][k] = (float)a.off[i][k];
      a.offl[i][k] = (float)(a.off[i][k] - (double)a.offh[i][k]);
    }
  for (int k = 0; k < 4; ++k) a.rot[k] = p->geom.rot[k];
  a.os = p->o_stride;
  a.ctl = (int*)(base + F.o_ctl);
  a.key = (uint32_t*)(base + F.o_key);
  a.val = (int*)(base + F.o_val);
  a.xy = (double2*)(base + F.o_xy);
  a.hl = (float4*)(base + F.o_hl);
  a.perm = (int*)(base + F.o_perm);
  a.qd = (double*)(base + F.o_qd);
  a.qf = (float*)(base + F.o_qf);
  a.cnt = (int*)(base + F.o_cnt);
  a.lf = (signed char*)(base + F.o_lf);
  a.bsum = (int*)(base + F.o_bsum);
  a.lo = (int*)(base + F.o_lo);
  a.hi = (int*)(base + F.o_hi);
  a.lev = (int*)(base + F.o_lev);
  a.par = (int*)(base + F.o_par);
  a.nend = (int*)(base + F.o_nend);
  a.nch = (int*)(base + F.o_nch);
  a.done = (int*)(base + F.o_done);
  a.ctr = (double2*)(base + F.o_ctr);
  a.half = (double*)(base + F.o_half);
  a.rad = (double*)(base + F.o_rad);
  a.scl = (float*)(base + F.o_scl);
  a.mult = (double2*)(base + F.o_mult);
  a.loc = (double2*)(base + F.o_loc);
  a.front = (int2*)(base + F.o_front);
  a.m2l = (int2*)(base + F.o_m2l);
  a.p2p = (int2*)(base + F.o_p2p);
  a.gcnt = (int*)(base + F.o_gcnt);
  a.gcur = (int*)(base + F.o_gcur);
  a.glist = (int*)(base + F.o_glist);
  a.gtgt = (int*)(base + F.o_gtgt);
  a.roots = (int*)(base + F.o_roots);
  a.node_cap = F.node_cap;
  a.exp_cap = F.exp_cap;
  a.m2l_cap = F.m2l_cap;
  a.p2p_cap = F.p2p_cap;
  a.front_cap = F.front_cap;
  a.src64 = (const double*)(ws + L.src64);
  a.trg64 = (const double*)(ws + L.trg64);
  a.qc = (const double*)(ws + L.qc);
  a.pot = pot;
  a.grad = grad;
  a.count_pairs = p->prof;
  const int K = p->opts.kernel;
  const int ncq = a.nrhs * p->ncomp;
  int nl = 0;
  cudaError_t e;
  // control words, child counters, completion counters, group counts and cursors
  e = cudaMemsetAsync(a.ctl, 0, kCtlWords * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.nch, 0, (size_t)F.node_cap * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.done, 0, (size_t)F.node_cap * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.gcnt, 0, (2 * (size_t)F.node_cap + 1) * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.gcur, 0, 2 * (size_t)F.node_cap * 4, st);
  if (e != cudaSuccess) return e;
  // 1-3 keys, sort, gather
  uint32_t* k2 = (uint32_t*)(base + F.o_key2);
  int* v2 = (int*)(base + F.o_val2);
  k_fmm_keys<<<cdiv(a.n, 256), 256, 0, st>>>(a, a.key, a.val);
  ++nl;
  bool in_b = false;
  e = radix_sort_pairs(a.key, a.val, k2, v2, (int*)(base + F.o_hist), a.n, self ? 30 : 31, st, &in_b, &nl);
  if (e != cudaSuccess) return e;
  if (in_b) {
    a.key = k2;
    a.val = v2;
  }
  k_fmm_gather<<<cdiv(a.n, 256), 256, 0, st>>>(a, ncq);
  ++nl;
  // 4-6 tree
  k_fmm_count<<<cdiv(a.n + 1, 256), 256, 0, st>>>(a);
  ++nl;
  e = scan_inplace(a.cnt, a.n + 1, a.bsum, st, &nl);
  if (e != cudaSuccess) return e;
  k_fmm_fill<<<cdiv(a.n, 256), 256, 0, st>>>(a);
  ++nl;
  auto rec = [&](int i) { if (p->prof) record_event(p->ev[i], st); };
  rec(4);
  // 7 up
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = 8 * sms;
  e = PFMM_FMM_P_DISPATCH(run_expansions, F.p, K, a, grid, st, &nl);
  if (e != cudaSuccess) return e;
  rec(5);
  // 8 traversal
  k_fmm_roots<<<1, 32, 0, st>>>(a);
  k_fmm_init<<<grid, 256, 0, st>>>(a);
  nl += 2;
  for (int it = 0; it < kFmmIter; ++it) k_fmm_traverse<<<grid, 256, 0, st>>>(a, it);
  k_fmm_traverse_check<<<1, 32, 0, st>>>(a);
  nl += kFmmIter + 1;
  // 9 group
  k_fmm_hist<<<grid, 256, 0, st>>>(a);
  ++nl;
  e = scan_inplace(a.gcnt, 2 * (int)F.node_cap + 1, a.bsum + cdiv(a.n + 1, kScanBlock) + 4, st, &nl);
  if (e != cudaSuccess) return e;
  k_fmm_scatter<<<grid, 256, 0, st>>>(a);
  k_fmm_sortseg<<<grid, 32 * kSortWarps, 0, st>>>(a);
  nl += 2;
  rec(6);
  // 10-11 down, leaves
  e = PFMM_FMM_P_DISPATCH(run_down, F.p, K, a, grid, st, &nl, p->prof ? p->ev[7] : nullptr, st_main, join);
  if (e != cudaSuccess) return e;
  // 12 fallback (returns at once unless a capacity overflowed)
  if (K == PFMM_LAPLACE) k_fmm_fallback<PFMM_LAPLACE><<<grid, kLeafThreads, 0, st_main>>>(a);
  else k_fmm_fallback<PFMM_STOKES><<<grid, kLeafThreads, 0, st_main>>>(a);
  ++nl;
  g_launches = nl;
  return cudaGetLastError();
}

// Statistics of the last execute's tree code (tracing; synchronises `st`):
// out[0] boxes, [1] M2L entries, [2] P2P entries, [3] directly evaluated
// pairs (counted while profiling), [4] overflow bits (0: none).
cudaError_t fmm_stats(const pfmm_plan* p, const char* ws, cudaStream_t st, int64_t out[5]) {
  int h[kCtlWords];
  cudaError_t e = cudaMemcpyAsync(h, ws + p->lay.fmm + p->fmm.o_ctl, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  out[0] = h[C_NNODES];
  out[1] = h[C_NM2L];
  out[2] = h[C_NP2P];
  unsigned long long pairs = 0;
  std::memcpy(&pairs, h + C_PAIRS, sizeof pairs);
  out[3] = (int64_t)pairs;
  out[4] = h[C_OVERFLOW];
  return cudaSuccess;
}

}  // namespace pfmm
