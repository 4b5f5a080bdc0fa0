// Batched execution: many independent cells (own lattice, parameter beta,
// tolerance and point count) in one call on one stream.
//
// Each cell keeps its own plan and a private region of the workspace; the
// inputs and outputs are concatenated structure-of-arrays with per-cell
// offsets.  On the mixed path the per-cell phases (memsets, point and
// strength preparation, far-field formation, weights and evaluation, the
// NUFFT stages) run as one launch per phase over all cells (multi.cuh): the
// cells' launches are recorded once per set of buffers and merged by
// (phase, kernel), with per-cell argument tables in the workspace.  The
// FP64 path launches them per cell.  The near-image P2P, which carries almost all the work
// and the N^2 imbalance between cells, runs as one persistent kernel per
// near-block shape over a global list of (cell, target block, source range,
// rhs group) items sorted by decreasing cost and pulled from an atomic
// counter.  Descriptors and item lists are uploaded by the first execute on a
// given set of buffers; later executes on the same buffers issue only
// memsets and kernel launches, so they can be captured in a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pfmm_impl.h"
#include "p2p.h"
#include "multi.cuh"

using namespace pfmm;

struct pfmm_batch {
  int ncell = 0, kernel = 0, precision = 0, nrhs = 1;
  bool self = true;
  std::vector<pfmm_plan*> plans;
  std::vector<int64_t> soff, toff;
  int64_t NS = 0, NT = 0;
  std::vector<size_t> wsoff;
  size_t off_cells = 0, off_items = 0, off_counter = 0, total = 0;
  struct Group {
    int nimg, nr;
    size_t first;
    int n, grid;
  };
  std::vector<Group> groups;
  std::vector<P2PItem> items;
  std::vector<P2PArgs> hcells;
  // mixed path: spatial sort of every cell's sources (and modified Helmholtz
  // targets) in one radix sort over the concatenated slots
  std::vector<SortCell> hsort;
  int64_t sort_total = 0;
  size_t off_sort = 0, off_sortscr = 0;
  const void* last[7] = {};
  int p2p_chunk = 4096;
  // tracing (pfmm_batch_profile_*)
  bool prof = false, timed = false, counting = false;
  bool count_pairs = true;  // profiling mode 1 counts evaluated pairs, mode 2 records events only
  cudaEvent_t ev[3] = {};
  int nlaunch = 0;
  // per-cell phases fan out over kFan streams (fork/join with events), so the
  // many small per-cell kernels overlap; under stream capture this becomes
  // kFan parallel branches of the graph
  static constexpr int kFan = 8;
  cudaStream_t fan[kFan] = {};
  cudaEvent_t fork = nullptr, join[kFan] = {};
  bool fan_ready = false;
  // mixed path: multi-cell launches of the per-cell phases, in phase order;
  // argument tables at off_multi (multi_bytes reserved at creation)
  struct MGroup {
    const void* fn;
    int phase, block, n, nblocks;
    size_t smem, argsz;
    size_t o_args, o_off, o_dims;  // offsets within the multi region
  };
  std::vector<MGroup> mgroups;
  std::vector<unsigned char> mblob;  // host copy of the tables (kept for the async upload)
  size_t off_multi = 0, multi_bytes = 0;
};

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// Record the per-cell phases of every cell (mixed path) with the given
// buffers: nothing is launched.
static pfmm_status record_cells(pfmm_batch* b, char* ws, const double* src, const double* q, const double* tr,
                                double* pot, double* grad, Recorder* rec) {
  for (int c = 0; c < b->ncell; ++c) {
    pfmm_plan* p = b->plans[c];
    p->s_stride = b->NS;
    p->t_stride = b->NT;
    p->o_stride = b->NT;
  }
  g_rec = rec;
  pfmm_status s = PFMM_OK;
  for (int c = 0; c < b->ncell && s == PFMM_OK; ++c) {
    int64_t ns = b->soff[c + 1] - b->soff[c], nt = b->toff[c + 1] - b->toff[c];
    s = execute_cell(b->plans[c], ws + b->wsoff[c], ns, src + b->soff[c], q + b->soff[c], nt, tr + b->toff[c],
                     pot + b->toff[c], grad ? grad + b->toff[c] : nullptr, (cudaStream_t)0, b->self, false, false);
  }
  g_rec = nullptr;
  return s;
}

// Merge the recorded launches by (phase, kernel), in phase order, and lay out
// their tables (arguments, first blocks, grids) in `blob`; returns its size.
static size_t build_groups(const Recorder& rec, std::vector<pfmm_batch::MGroup>* groups,
                           std::vector<unsigned char>* blob) {
  groups->clear();
  std::vector<std::vector<const LaunchRec*>> members;
  for (int ph = 0; ph < PH_COUNT; ++ph) {
    const size_t first = groups->size();
    for (const LaunchRec& r : rec.recs) {
      if (r.phase != ph) continue;
      size_t k = first;
      while (k < groups->size() && (*groups)[k].fn != r.fn) ++k;
      if (k == groups->size()) {
        pfmm_batch::MGroup g{};
        g.fn = r.fn;
        g.phase = ph;
        g.argsz = r.args.size();
        groups->push_back(g);
        members.emplace_back();
      }
      members[k].push_back(&r);
    }
  }
  size_t off = 0;
  for (size_t k = 0; k < groups->size(); ++k) {
    pfmm_batch::MGroup& g = (*groups)[k];
    g.n = (int)members[k].size();
    g.o_args = off;
    off = al256(off + g.argsz * g.n);
    g.o_off = off;
    off = al256(off + sizeof(int) * g.n);
    g.o_dims = off;
    off = al256(off + sizeof(uint3) * g.n);
  }
  if (blob) {
    blob->assign(off, 0);
    for (size_t k = 0; k < groups->size(); ++k) {
      pfmm_batch::MGroup& g = (*groups)[k];
      int nb = 0;
      for (int i = 0; i < g.n; ++i) {
        const LaunchRec& r = *members[k][i];
        std::memcpy(blob->data() + g.o_args + g.argsz * i, r.args.data(), g.argsz);
        std::memcpy(blob->data() + g.o_off + sizeof(int) * i, &nb, sizeof(int));
        std::memcpy(blob->data() + g.o_dims + sizeof(uint3) * i, &r.grid, sizeof(uint3));
        nb += (int)(r.grid.x * r.grid.y * r.grid.z);
        g.block = std::max(g.block, r.block);
        g.smem = std::max(g.smem, r.smem);
      }
      g.nblocks = nb;
    }
  }
  return off;
}

extern "C" {

pfmm_status pfmm_batch_create(const pfmm_opts* cells, int ncell, const int64_t* src_off, const int64_t* trg_off,
                              int p2p_chunk, pfmm_batch** out) {
  if (!cells || !src_off || !out || ncell < 1) return set_error(PFMM_ERR_INVALID_ARG, "bad batch arguments");
  *out = nullptr;
  const pfmm_opts& c0 = cells[0];
  for (int c = 0; c < ncell; ++c) {
    if (cells[c].kernel != c0.kernel || cells[c].precision != c0.precision || cells[c].nrhs != c0.nrhs)
      return set_error(PFMM_ERR_INVALID_ARG, "batch cells must share kernel, precision and nrhs (cell %d)", c);
    if (cells[c].flags & (PFMM_FAR_ONLY | PFMM_NEAR_ONLY))
      return set_error(PFMM_ERR_INVALID_ARG, "batch cells compute the full operator (cell %d)", c);
    if (cells[c].flags & PFMM_SINGLY_PERIODIC)
      return set_error(PFMM_ERR_INVALID_ARG, "batch cells are doubly periodic (cell %d)", c);
    if (cells[c].flags & PFMM_DETERMINISTIC)
      return set_error(PFMM_ERR_INVALID_ARG, "DETERMINISTIC is for single-cell calls (cell %d)", c);
    if (src_off[c + 1] < src_off[c] || (trg_off && trg_off[c + 1] < trg_off[c]))
      return set_error(PFMM_ERR_INVALID_ARG, "offsets must be non-decreasing (cell %d)", c);
  }
  if (src_off[0] != 0 || (trg_off && trg_off[0] != 0)) return set_error(PFMM_ERR_INVALID_ARG, "offsets start at 0");
  if (p2p_chunk != 0 && (p2p_chunk < 128 || p2p_chunk % 128))
    return set_error(PFMM_ERR_INVALID_ARG, "p2p_chunk must be 0 or a positive multiple of 128");
  if (ncell > 32768) return set_error(PFMM_ERR_INVALID_ARG, "at most 32768 cells per batch");
  pfmm_batch* b = new pfmm_batch();
  b->ncell = ncell;
  b->kernel = c0.kernel;
  b->precision = c0.precision;
  b->nrhs = c0.nrhs;
  b->self = trg_off == nullptr;
  b->p2p_chunk = p2p_chunk ? p2p_chunk : 4096;
  b->soff.assign(src_off, src_off + ncell + 1);
  b->toff = b->self ? b->soff : std::vector<int64_t>(trg_off, trg_off + ncell + 1);
  b->NS = b->soff[ncell];
  b->NT = b->toff[ncell];
  size_t off = 0;
  for (int c = 0; c < ncell; ++c) {
    int64_t ns = b->soff[c + 1] - b->soff[c], nt = b->toff[c + 1] - b->toff[c];
    pfmm_plan* p = nullptr;
    // the near field of a batch is the batched P2P (or the per-cell direct
    // P2P on the FP64 path): plans without the tree code's workspace
    pfmm_opts oc = cells[c];
    oc.flags = (oc.flags & ~(unsigned)PFMM_NEAR_FMM) | PFMM_NEAR_DIRECT;
    pfmm_status s = pfmm_plan_create(&oc, ns, nt, &p);
    if (s != PFMM_OK) {
      for (auto* q : b->plans) pfmm_plan_destroy(q);
      delete b;
      return s;
    }
    b->plans.push_back(p);
    b->wsoff.push_back(off);
    off = al256(off + p->lay.total);
  }
  // P2P work items (mixed precision: one persistent kernel per near-block shape)
  const int tpb = p2p_targets_per_block(b->kernel);
  // rhs per item: 8 for modified Helmholtz (one Bessel evaluation serves 8 rhs), else up to 4
  const int nr = (b->kernel == PFMM_MODHELM && b->nrhs % 8 == 0) ? 8
                 : (b->nrhs % 4 == 0 ? 4 : (b->nrhs % 2 == 0 ? 2 : 1));
  for (int nimg : {9, 15}) {
    pfmm_batch::Group g{nimg, nr, b->items.size(), 0, 0};
    std::vector<std::pair<double, P2PItem>> v;
    for (int c = 0; c < ncell; ++c) {
      const pfmm_plan* p = b->plans[c];
      if (p->geom.nimg != nimg) continue;
      int ns = (int)(b->soff[c + 1] - b->soff[c]), nt = (int)(b->toff[c + 1] - b->toff[c]);
      for (int bx = 0; bx * tpb < nt; ++bx)
        for (int j0 = 0; j0 < ns; j0 += b->p2p_chunk)
          for (int r0 = 0; r0 < b->nrhs; r0 += nr) {
            int j1 = std::min(ns, j0 + b->p2p_chunk);
            double cost = (double)std::min(tpb, nt - bx * tpb) * (j1 - j0) + 2000.0;
            v.push_back({cost, P2PItem{c, bx, j0, j1, r0}});
          }
    }
    std::stable_sort(v.begin(), v.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    for (auto& e : v) b->items.push_back(e.second);
    g.n = (int)v.size();
    if (g.n > 0) b->groups.push_back(g);
  }
  if (b->precision == PFMM_MIXED) {
    const bool sort_t = !b->self;
    b->hsort.resize((size_t)ncell * (sort_t ? 2 : 1));
    b->sort_total = b->NS + (sort_t ? b->NT : 0);
    b->off_sort = off;
    off = al256(off + sizeof(SortCell) * b->hsort.size());
    b->off_sortscr = off;
    off = al256(off + sort_scratch_bytes(b->sort_total, (int)b->hsort.size()));
  }
  if (b->precision == PFMM_MIXED) {
    // size of the multi-cell launch tables: a recording with placeholder
    // addresses (the tables' sizes do not depend on them)
    Recorder rec;
    char* fake = reinterpret_cast<char*>(uintptr_t(1) << 20);
    double* fd = reinterpret_cast<double*>(fake);
    pfmm_status s = record_cells(b, fake, fd, fd, fd, fd, fd, &rec);
    if (s != PFMM_OK) {
      pfmm_batch_destroy(b);
      return s;
    }
    std::vector<pfmm_batch::MGroup> groups;
    b->multi_bytes = build_groups(rec, &groups, nullptr);
    b->off_multi = off;
    off = al256(off + b->multi_bytes);
  }
  b->off_cells = off;
  off = al256(off + sizeof(P2PArgs) * ncell);
  b->off_items = off;
  off = al256(off + sizeof(P2PItem) * std::max<size_t>(1, b->items.size()));
  b->off_counter = off;
  off = al256(off + 256);
  b->total = off;
  b->hcells.resize(ncell);
  *out = b;
  return PFMM_OK;
}

pfmm_status pfmm_batch_workspace_size(const pfmm_batch* b, size_t* bytes) {
  if (!b || !bytes) return set_error(PFMM_ERR_INVALID_ARG, "NULL argument");
  *bytes = b->total;
  return PFMM_OK;
}

void pfmm_batch_destroy(pfmm_batch* b) {
  if (!b) return;
  for (auto* p : b->plans) pfmm_plan_destroy(p);
  if (b->prof)
    for (auto& e : b->ev) cudaEventDestroy(e);
  if (b->fan_ready) {
    for (int k = 0; k < pfmm_batch::kFan; ++k) {
      cudaStreamDestroy(b->fan[k]);
      cudaEventDestroy(b->join[k]);
    }
    cudaEventDestroy(b->fork);
  }
  delete b;
}

// Streams and events of the per-cell fan-out, created at the first execute
// (on the current device) and reused; nothing is created while capturing.
static cudaError_t fan_setup(pfmm_batch* b) {
  if (b->fan_ready) return cudaSuccess;
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int k = 0; k < pfmm_batch::kFan && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->fan[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) b->fan_ready = true;
  return e;
}

pfmm_status pfmm_batch_profile_enable(pfmm_batch* b, int on) {
  if (!b) return set_error(PFMM_ERR_INVALID_ARG, "NULL batch");
  if (on < 0 || on > 2) return set_error(PFMM_ERR_INVALID_ARG, "profiling mode must be 0, 1 or 2");
  if (on) b->count_pairs = on == 1;
  if (on && !b->prof) {
    for (auto& e : b->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return set_error(PFMM_ERR_CUDA, "cudaEventCreate failed");
    b->prof = true;
    b->timed = false;
  } else if (!on && b->prof) {
    for (auto& e : b->ev) cudaEventDestroy(e);
    b->prof = false;
    b->timed = false;
  }
  return PFMM_OK;
}

pfmm_status pfmm_batch_profile_read(pfmm_batch* b, float* ms, int n, int* nlaunch, double* pairs) {
  if (!b || !ms || n < 2) return set_error(PFMM_ERR_INVALID_ARG, "NULL batch or output, or n < 2");
  if (!b->prof || !b->timed) return set_error(PFMM_ERR_INVALID_ARG, "no profiled batch execute yet");
  if (cudaEventSynchronize(b->ev[2]) != cudaSuccess) return set_error(PFMM_ERR_CUDA, "event synchronize failed");
  if (cudaEventElapsedTime(ms, b->ev[0], b->ev[1]) != cudaSuccess ||
      cudaEventElapsedTime(ms + 1, b->ev[1], b->ev[2]) != cudaSuccess)
    return set_error(PFMM_ERR_CUDA, "cudaEventElapsedTime failed");
  if (nlaunch) *nlaunch = b->nlaunch;
  if (pairs) {
    // sum the per-cell counters (modified Helmholtz mixed), else the nominal count
    double tot = 0.0;
    for (int c = 0; c < b->ncell; ++c) {
      const pfmm_plan* p = b->plans[c];
      const double ns = (double)(b->soff[c + 1] - b->soff[c]), nt = (double)(b->toff[c + 1] - b->toff[c]);
      if (b->kernel == PFMM_MODHELM && b->precision == PFMM_MIXED) {
        unsigned long long w = 0;
        if (cudaMemcpy(&w, (const char*)b->last[0] + b->wsoff[c] + p->lay.work, sizeof w, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
          return set_error(PFMM_ERR_CUDA, "read pair count");
        tot += (double)w;
      } else {
        tot += ns * nt * p->geom.nimg;
      }
    }
    *pairs = tot;
  }
  return PFMM_OK;
}

pfmm_status pfmm_batch_execute(pfmm_batch* b, void* workspace, size_t ws_bytes, const double* src, const double* q,
                               const double* trg, double* pot, double* grad, void* stream) {
  if (!b) return set_error(PFMM_ERR_INVALID_ARG, "NULL batch");
  if (!workspace || ws_bytes < b->total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return set_error(PFMM_ERR_WORKSPACE, "workspace NULL, misaligned or smaller than %zu bytes", b->total);
  if (!src || !q || !pot) return set_error(PFMM_ERR_INVALID_ARG, "NULL sources, strengths or potential");
  if (!b->self && !trg) return set_error(PFMM_ERR_INVALID_ARG, "NULL targets");
  if ((b->kernel == PFMM_STOKES || b->kernel == PFMM_MSTOKES) && grad)
    return set_error(PFMM_ERR_INVALID_ARG, "grad must be NULL for the Stokes kernels");
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  const double* tr = b->self ? src : trg;
  const bool mixed = b->precision == PFMM_MIXED;
  // per-cell strides: the caller's arrays are concatenated over cells
  for (int c = 0; c < b->ncell; ++c) {
    pfmm_plan* p = b->plans[c];
    p->s_stride = b->NS;
    p->t_stride = b->NT;
    p->o_stride = b->NT;
  }
  const void* cur[7] = {workspace, src, q, tr, pot, grad, (const void*)(uintptr_t)b->p2p_chunk};
  const bool upload = std::memcmp(cur, b->last, sizeof cur) != 0;
  cudaError_t e = cudaSuccess;
  if (upload) {
    for (int c = 0; c < b->ncell; ++c) {
      pfmm_plan* p = b->plans[c];
      char* wc = ws + b->wsoff[c];
      e = upload_tables(p, wc, st);
      if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, "upload tables: %s", cudaGetErrorString(e));
      int64_t ns = b->soff[c + 1] - b->soff[c], nt = b->toff[c + 1] - b->toff[c];
      fill_p2p_args(p, wc, ns, nt, b->self, pot + b->toff[c], grad ? grad + b->toff[c] : nullptr, &b->hcells[c]);
      set_work_counter(p, wc, b->counting, &b->hcells[c]);
      if (mixed) {
        SortCell two[2];
        const int k = fill_sort_cells(p, wc, ns, nt, b->self, b->soff[c], b->NS + b->toff[c], two);
        b->hsort[c] = two[0];
        if (k > 1) b->hsort[b->ncell + c] = two[1];
      }
    }
    if (mixed)
      e = cudaMemcpyAsync(ws + b->off_sort, b->hsort.data(), sizeof(SortCell) * b->hsort.size(),
                          cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, "upload sort descriptors: %s", cudaGetErrorString(e));
    e = cudaMemcpyAsync(ws + b->off_cells, b->hcells.data(), sizeof(P2PArgs) * b->ncell, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !b->items.empty())
      e = cudaMemcpyAsync(ws + b->off_items, b->items.data(), sizeof(P2PItem) * b->items.size(),
                          cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, "upload descriptors: %s", cudaGetErrorString(e));
    for (auto& g : b->groups) g.grid = p2p_batch_grid(b->kernel, g.nimg, g.nr, grad != nullptr);
    if (mixed) {
      // the per-cell phases with these buffers, merged into multi-cell launches
      Recorder rec;
      pfmm_status s = record_cells(b, ws, src, q, tr, pot, grad, &rec);
      if (s != PFMM_OK) return s;
      const size_t need = build_groups(rec, &b->mgroups, &b->mblob);
      if (need > b->multi_bytes)
        return set_error(PFMM_ERR_INTERNAL, "multi-cell launch tables need %zu bytes, %zu reserved", need,
                         b->multi_bytes);
      if (need) e = cudaMemcpyAsync(ws + b->off_multi, b->mblob.data(), need, cudaMemcpyHostToDevice, st);
      for (auto& g : b->mgroups)
        if (e == cudaSuccess && g.smem > 48 * 1024)
          e = cudaFuncSetAttribute(g.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
      if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, "multi-cell tables: %s", cudaGetErrorString(e));
    }
    std::memcpy(b->last, cur, sizeof cur);
  }
  e = cudaMemsetAsync(ws + b->off_counter, 0, 256, st);
  if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusActive;
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  // Phase events: plain records on an eager execute; under stream capture
  // they become external event-record nodes, so each replay of the graph
  // records them and pfmm_batch_profile_read times the replayed phases.
  const bool rec = b->prof;
  auto record = [&](cudaEvent_t ev) {
    return capturing ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal) : cudaEventRecord(ev, st);
  };
  // Evaluated-pair counters in the P2P descriptors only while profiling in
  // mode 1.  They are switched on an eager execute only (the switch uploads
  // descriptors); a capture keeps the state of the last eager execute.
  const bool count = b->prof && b->count_pairs && !capturing;
  if (mixed && b->kernel == PFMM_MODHELM && !capturing && count != b->counting) {
    for (int c = 0; c < b->ncell; ++c) set_work_counter(b->plans[c], ws + b->wsoff[c], count, &b->hcells[c]);
    e = cudaMemcpyAsync(ws + b->off_cells, b->hcells.data(), sizeof(P2PArgs) * b->ncell, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, "upload descriptors: %s", cudaGetErrorString(e));
    b->counting = count;
  }
  if (rec && (e = record(b->ev[0])) != cudaSuccess) return set_error(PFMM_ERR_CUDA, "event record: %s", cudaGetErrorString(e));
  b->nlaunch = 0;
  if (mixed) {
    // per-cell phases: one launch per (phase, kernel) over all cells
    for (const auto& g : b->mgroups) {
      const void* pa = ws + b->off_multi + g.o_args;
      const void* po = ws + b->off_multi + g.o_off;
      const void* pd = ws + b->off_multi + g.o_dims;
      int n = g.n;
      void* params[] = {(void*)&pa, (void*)&po, (void*)&pd, (void*)&n};
      e = cudaLaunchKernel(g.fn, dim3(g.nblocks), dim3(g.block), params, g.smem, st);
      if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, "multi-cell launch (phase %d): %s", g.phase,
                                             cudaGetErrorString(e));
      ++b->nlaunch;
    }
  }
  // FP64 path: per-cell phases, cell c on fan stream c % kFan, forked from
  // and joined back into the caller's stream
  const bool fan = !mixed && b->ncell > 1 &&
                   (b->fan_ready || (cap == cudaStreamCaptureStatusNone && fan_setup(b) == cudaSuccess));
  if (fan) {
    e = cudaEventRecord(b->fork, st);
    for (int k = 0; k < pfmm_batch::kFan && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->fan[k], b->fork, 0);
    if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, "fork: %s", cudaGetErrorString(e));
  }
  for (int c = 0; c < b->ncell && !mixed; ++c) {
    int64_t ns = b->soff[c + 1] - b->soff[c], nt = b->toff[c + 1] - b->toff[c];
    cudaStream_t sc = fan ? b->fan[c % pfmm_batch::kFan] : st;
    pfmm_status s = execute_cell(b->plans[c], ws + b->wsoff[c], ns, src + b->soff[c], q + b->soff[c], nt,
                                 tr + b->toff[c], pot + b->toff[c], grad ? grad + b->toff[c] : nullptr, sc, b->self,
                                 false, !mixed);
    if (s != PFMM_OK) return s;
    b->nlaunch += b->plans[c]->nlaunch;
  }
  if (fan) {
    for (int k = 0; k < pfmm_batch::kFan && e == cudaSuccess; ++k) {
      e = cudaEventRecord(b->join[k], b->fan[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->join[k], 0);
    }
    if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, "join: %s", cudaGetErrorString(e));
  }
  if (rec && (e = record(b->ev[1])) != cudaSuccess) return set_error(PFMM_ERR_CUDA, "event record: %s", cudaGetErrorString(e));
  if (mixed) {
    int nl = 0;
    e = sort_cells((const SortCell*)(ws + b->off_sort), b->hsort.data(), (int)b->hsort.size(), b->sort_total,
                   ws + b->off_sortscr, st, &nl);
    if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, "spatial sort: %s", cudaGetErrorString(e));
    b->nlaunch += nl;
    int gi = 0;
    for (auto& g : b->groups) {
      e = launch_p2p_batch(b->kernel, g.nimg, g.nr, grad != nullptr, (const P2PArgs*)(ws + b->off_cells),
                           (const P2PItem*)(ws + b->off_items) + g.first, g.n, (int*)(ws + b->off_counter) + gi,
                           g.grid, st);
      if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, "batched p2p: %s", cudaGetErrorString(e));
      ++gi;
      ++b->nlaunch;
    }
  }
  if (rec) {
    if ((e = record(b->ev[2])) != cudaSuccess) return set_error(PFMM_ERR_CUDA, "event record: %s", cudaGetErrorString(e));
    b->timed = true;
  }
  return PFMM_OK;
}

pfmm_status pfmm_batch_get_status(pfmm_batch* b, void* workspace, void* stream) {
  if (!b || !workspace) return set_error(PFMM_ERR_INVALID_ARG, "NULL argument");
  pfmm_status worst = PFMM_OK;
  for (int c = 0; c < b->ncell; ++c) {
    pfmm_status s = pfmm_get_status(b->plans[c], (char*)workspace + b->wsoff[c], stream);
    if (s != PFMM_OK && worst == PFMM_OK) worst = s;
  }
  return worst;
}

}  // extern "C"
