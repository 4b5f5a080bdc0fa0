/*
 * pfmm.h -- C ABI of the GB300 periodizing-operator library.
 *
 * Computes, for sources s_j with strengths q_j in a doubly periodic unit cell
 * spanned by lattice vectors e1, e2, the periodic field at targets t_l
 *
 *     u(t_l) = sum_j K^(p)(t_l, s_j) q_j = (K^near q)(t_l) + (P2 q)(t_l)
 *
 * (Pei, Askham, Greengard & Jiang, "Periodic Fast Multipole Method",
 * arXiv 2111.01083: Sec. 1, Eq. psum and Eq. nearfarsplit).  P2 is the
 * periodizing operator of Definition "peropdef", applied through the
 * low-rank plane-wave factorizations of its south/north/west/east parts
 * (Eq. ksplitting2; Theorems south_thm, west_thm, south_thm_lap,
 * west_thm_lap, south_thm_s, west_thm_s), either directly (Sec. 6, O(r N)) or
 * through Gauss-Legendre anterpolation + 1D NUFFTs (Sec. 6, Eqs. fastanterp,
 * fastinterp).  K^near is the direct sum over the (2 m0 + 1) x 3 near images
 * (Definition of Lambda_near in Sec. 1), self pairs excluded.
 *
 * Green's functions (Sec. 1, Sec. 5.2): Laplace (1/2pi) log(1/r); modified
 * Helmholtz (1/2pi) K0(beta r); Stokeslet -(1/4pi)(log r I - r r^T / r^2).
 * Results are u = sum G q (the sign of the paper's Eq. govpde is not used).
 *
 * Conventions for every entry point below:
 *  - All array arguments of pfmm_execute / pfmm_execute_adjoint are DEVICE
 *    pointers to caller-owned memory (double precision, structure of arrays,
 *    component-major).  The library never allocates or frees device memory;
 *    it uses only the caller's workspace.  pfmm_execute_host takes HOST
 *    pointers and stages them through the workspace.
 *  - Everything is enqueued on the caller's CUDA stream (passed as void*,
 *    a cudaStream_t; NULL = legacy default stream).  Nothing synchronises
 *    except pfmm_get_status and pfmm_execute_host.  A plan that uses the
 *    near-field tree code creates one stream and two events (no device
 *    memory) at its first execute outside stream capture; its tree phases run
 *    there beside the far field, forked from and joined back into the
 *    caller's stream (under capture: parallel branches of the graph).
 *  - Return value: PFMM_OK (0) or an error code; pfmm_last_error() gives a
 *    thread-local message.  Argument errors are detected on the host before
 *    anything is launched.  Conditions only visible on the device
 *    (non-finite input, net charge / net force not zero, a bounded wait that
 *    ran out) are written to a status word in the workspace and reported by
 *    pfmm_get_status.
 *  - Lattice vectors may have any orientation; they are reduced and rotated
 *    to the paper's canonical form e1 = (d, 0), e2 = (xi, eta), d >= |e2|,
 *    eta > 0 (Sec. 1).  Points may lie anywhere; they are wrapped into the
 *    cell.  Vector inputs/outputs (forces, gradients, velocities) are in the
 *    caller's frame.
 *  - Laplace potentials and Stokes velocities are defined up to an additive
 *    constant (per rhs, per component).  The library's constant is fixed but
 *    arbitrary; compare modulo a constant.  Laplace and Stokes require zero
 *    net charge / net force per rhs (Eq. chargeneutral).
 *  - Plans are not thread-safe; different plans may run concurrently on
 *    different streams with different workspaces.
 */
#ifndef PFMM_H
#define PFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* MSTOKES: the modified Stokeslet (Eq. msgreen), u = G f with
 * G = (grad grad^T - Lap I) G_MB, G_MB = -(1/(2 pi beta^2))(K0(beta r) - log(1/r)),
 * the fundamental solution of (beta^2 - Lap) u + grad p = 0, div u = 0
 * (beta > 0; no net-force condition).  Forces and velocities are laid out as
 * for STOKES.  Far field by Theorems south_thm_ms / west_thm_ms (direct and
 * NUFFT paths), periodic sum in the paper's order (image rows).  Single cells
 * and batches; the adjoint for the strengths (the operator is symmetric); not
 * singly periodic. */
typedef enum { PFMM_LAPLACE = 0, PFMM_MODHELM = 1, PFMM_STOKES = 2, PFMM_MSTOKES = 3 } pfmm_kernel;

/* FP64: every step in double precision.
 * MIXED: plane-wave generation, spreading, FFT, interpolation and the P2P
 * pair terms in FP32 (P2P coordinates as hi/lo float pairs so that
 * differences are exact to FP32 rounding), with FP64/compensated
 * accumulation of the coefficient sums and of the per-target totals; lattice
 * weights, quadrature nodes and compatibility moments in FP64. */
typedef enum { PFMM_FP64 = 0, PFMM_MIXED = 1 } pfmm_precision;

/* Far-field south/north application: DIRECT = L (D (R q)) (Sec. 6);
 * NUFFT = GL anterpolation + ES-kernel NUFFT (Sec. 6, Eqs. fastanterp and
 * fastinterp), for all four kernels.  AUTO picks NUFFT when M >= 64 and the
 * fine grid (power of two >= 2 (2M + 1)) has at most 8192 points.  For the
 * singly periodic operator the path applies to its west/east parts (see
 * PFMM_SINGLY_PERIODIC). */
typedef enum { PFMM_PATH_AUTO = 0, PFMM_PATH_DIRECT = 1, PFMM_PATH_NUFFT = 2 } pfmm_path;

/* flags */
enum {
  PFMM_FAR_ONLY = 1,   /* output P2 q only (no near-image sum)            */
  PFMM_NEAR_ONLY = 2,  /* output K^near q only                            */
  PFMM_NO_GRAD = 4,    /* scalar kernels: skip the gradient even if given */
  PFMM_PROJECT_NEUTRAL = 8, /* Laplace/Stokes: subtract the mean strength (force) per rhs
                               before use, i.e. apply the operator to the zero-net part */
  PFMM_SINGLY_PERIODIC = 16, /* P1: periodic along e1 only.  e2 spans the strip: points
                               are wrapped along e1 and must lie within |y| < eta/2 across
                               it (eta = |e1 x e2| / |e1|); others set the status
                               PFMM_ERR_INVALID_ARG.  Near images m e1, |m| <= 1; the far
                               images through the west/east factorization restricted to
                               the image row n = 0 (Theorems west_thm, west_thm_lap,
                               west_thm_s), no south/north parts; single-cell calls
                               only (not in a batch).  The NUFFT path (Sec. 6.1 with x
                               and y exchanged, for strips with eta >> d) takes the
                               west/east sums through GL lines in x, a type-1 transform
                               in y and ES interpolation onto the quadrature nodes; AUTO
                               picks it when at least 128 nodes qualify. */
  PFMM_WE_ROTATED = 32,    /* west/east plane waves decay along e2-perp instead of e1
                               (App. A, Eq. k0west2): the near block is 3 x 3 images
                               (m0 = 1) for every parallelogram, at the price of more
                               west/east quadrature nodes on strongly skewed cells */
  PFMM_WE_AXIS = 64,       /* west/east plane waves decay along e1; m0 = 1 unless the
                               canonical skew |xi| > 3d/8, then m0 = 2 (15 images).
                               Neither flag (default): rotated exactly when the axis
                               direction would need m0 = 2.  Both: PFMM_ERR_INVALID_ARG.
                               The singly periodic operator always uses the axis. */
  PFMM_NEAR_DIRECT = 128,  /* near-image sum by the direct P2P over all pairs            */
  PFMM_NEAR_FMM = 256,     /* near-image sum by the tree code (the paper evaluates the
                               near field with an FMM, Sec. 7): one quadtree of the unit
                               cell's sources, its image copies shifted by l (sharing the
                               unit cell's expansions), one of the targets; complex
                               multipole/local expansions of p terms, boxes expanded when
                               r_t + r_s <= theta |c_t - c_s - l| (theta = 1/2), neighbouring
                               leaves summed directly.  Laplace and Stokes, mixed precision.
                               Neither flag (default): the tree code when the kernel and
                               precision allow it and ns * nt * images >= 2e9, else the
                               direct P2P.  Both: PFMM_ERR_INVALID_ARG.  The FMM flag with
                               another kernel or FP64 selects the direct P2P. */
  PFMM_DETERMINISTIC = 512 /* bit-identical results for identical inputs: every cross-block
                               sum (moments, coefficient formation) goes through per-block
                               partials added in a fixed order instead of atomics, the P2P
                               gives each output one addition, the far field takes the
                               direct path and the near field the direct P2P (with NUFFT or
                               NEAR_FMM: PFMM_ERR_INVALID_ARG).  Single-cell calls only (a
                               batch refuses it).  Not in the paper. */
};

typedef enum {
  PFMM_OK = 0,
  PFMM_ERR_INVALID_ARG = 1,
  PFMM_ERR_LATTICE = 2,     /* degenerate lattice vectors                         */
  PFMM_ERR_NOT_NEUTRAL = 3, /* |sum q| > 1e-8 sum|q| for Laplace/Stokes (device)  */
  PFMM_ERR_TOLERANCE = 4,   /* tol outside [1e-14, 1e-2]                          */
  PFMM_ERR_WORKSPACE = 5,   /* workspace NULL, too small or misaligned            */
  PFMM_ERR_CUDA = 6,        /* a CUDA runtime call failed                         */
  PFMM_ERR_NONFINITE = 7,   /* NaN/Inf in coordinates or strengths (device)       */
  PFMM_ERR_TIMEOUT = 8,     /* a bounded device wait gave up (device)             */
  PFMM_ERR_INTERNAL = 9
} pfmm_status;

typedef struct {
  double e1[2], e2[2];  /* lattice vectors (any orientation, not collinear)     */
  int kernel;           /* pfmm_kernel                                          */
  double beta;          /* > 0 for PFMM_MODHELM and PFMM_MSTOKES, ignored otherwise */
  double tol;           /* requested precision eps, in [1e-14, 1e-2]            */
  int precision;        /* pfmm_precision                                       */
  int path;             /* pfmm_path                                            */
  int nufft_w;          /* ES kernel width (2..16); 0 = ceil(log10(1/tol)) + 2  */
  int n_gl;             /* GL interpolation lines (4..32); 0 = 8 (tol>=1e-7), else 16 */
  int nrhs;             /* number of right-hand sides (>= 1)                    */
  unsigned flags;       /* OR of PFMM_FAR_ONLY, PFMM_NEAR_ONLY, PFMM_NO_GRAD,
                           PFMM_PROJECT_NEUTRAL, PFMM_SINGLY_PERIODIC,
                           PFMM_WE_ROTATED, PFMM_WE_AXIS, PFMM_NEAR_DIRECT,
                           PFMM_NEAR_FMM, PFMM_DETERMINISTIC (see the enum above) */
  int near_order;       /* tree-code expansion terms p (8..32, rounded up to 12, 16, 20,
                           24 or 32); 0 = from tol: theta^p <= tol / 10 */
  int near_leaf;        /* tree code: a box with more points is split (8..1024); 0 = 128 */
} pfmm_opts;

/* Parameters chosen by a plan (read-only; for inspection and tests). */
typedef struct {
  double d, xi, eta;    /* canonical cell                                       */
  double rot[4];        /* canonical = rot * input, row-major 2x2               */
  int m0;               /* near block is (2 m0 + 1) x 3 images                  */
  int M;                /* south/north modes m = 1..M kept (Eq. mpk0s, pruned)  */
  int mode0;            /* 1 if the m = 0 mode is used (Laplace/Stokes, or modhelm when not negligible) */
  int Nq;               /* west/east quadrature nodes                           */
  int path;             /* PFMM_PATH_DIRECT or PFMM_PATH_NUFFT after AUTO        */
  int n_gl, nf, nufft_w;/* NUFFT: GL lines, fine grid size, ES width           */
  double es_beta;       /* ES kernel shape parameter                            */
  int nlaunch;          /* kernels launched by the last pfmm_execute on this plan */
  int64_t npairs;       /* near-image pairs of the last execute: ns * nt * (2 m0 + 1) * 3 */
  int we_rotated;       /* 1 if the west/east plane waves decay along e2-perp   */
  double we_dir[2];     /* (cos, sin) of that direction's rotation: canonical
                           (x, y) -> (cos x - sin y, sin x + cos y); (1, 0) on the axis */
  int near_fmm;         /* 1 if the near-image sum runs through the tree code      */
  int near_order;       /* its expansion terms p                                    */
  int near_leaf;        /* its leaf size                                            */
  double near_theta;    /* its acceptance parameter                                 */
  int p1_nufft_nodes;   /* singly periodic operator on the NUFFT path: west/east nodes
                           whose sums go through the transforms (the others, lambda below
                           (w/2 + 2) pi / eta, stay direct); 0 otherwise                 */
} pfmm_plan_desc;

typedef struct pfmm_plan pfmm_plan;

/* Build a plan: canonical cell (Sec. 1), m0, modes M (Eq. mpk0s), west/east
 * quadrature nodes and weights (own composite Gauss-Legendre rule; the
 * paper's GGQ tables are not printed), NUFFT sizes.  Host only, no GPU work.
 * ns_max/nt_max bound the sizes later passed to pfmm_execute.
 * Errors: PFMM_ERR_INVALID_ARG (NULL, nrhs < 1, sizes < 0, beta <= 0 for
 * MODHELM, bad enum), PFMM_ERR_LATTICE, PFMM_ERR_TOLERANCE. */
pfmm_status pfmm_plan_create(const pfmm_opts* opts, int64_t ns_max, int64_t nt_max,
                             pfmm_plan** out);

/* Bytes of device workspace pfmm_execute needs (256-byte aligned pointer). */
pfmm_status pfmm_workspace_size(const pfmm_plan* plan, size_t* bytes);

/* Bytes of device workspace pfmm_execute_host needs (adds staging space). */
pfmm_status pfmm_workspace_size_host(const pfmm_plan* plan, size_t* bytes);

pfmm_status pfmm_plan_describe(const pfmm_plan* plan, pfmm_plan_desc* out);

/* Apply the periodic operator.
 *   src  [2][ns]      source coordinates (x row then y row)
 *   q    [nrhs][ns]   strengths (Laplace, modhelm) or
 *        [nrhs][2][ns] forces (Stokes, modified Stokes)
 *   trg  [2][nt]      target coordinates; may be the same pointer as src with
 *                     nt == ns (targets = sources; self pairs are skipped,
 *                     and so is any pair at exactly zero distance)
 *   pot  [nrhs][nt]   potential (Laplace, modhelm) or
 *        [nrhs][2][nt] velocity (Stokes, modified Stokes); may be NULL for
 *                     scalar kernels
 *   grad [nrhs][2][nt] gradient of the potential (scalar kernels) or NULL;
 *                     must be NULL for Stokes and modified Stokes
 * Outputs are overwritten.  ns, nt >= 0 and <= the plan's maxima. */
pfmm_status pfmm_execute(pfmm_plan* plan, void* workspace, size_t ws_bytes, int64_t ns,
                         const double* src, const double* q, int64_t nt, const double* trg,
                         double* pot, double* grad, void* stream);

/* Same operation with HOST arrays: stages inputs into the workspace
 * (cudaMemcpyAsync), runs pfmm_execute, copies outputs back and synchronises
 * the stream.  Workspace from pfmm_workspace_size_host.  src == trg (same
 * host pointer, ns == nt) means targets = sources. */
pfmm_status pfmm_execute_host(pfmm_plan* plan, void* workspace, size_t ws_bytes, int64_t ns,
                              const double* src, const double* q, int64_t nt, const double* trg,
                              double* pot, double* grad, void* stream);

/* ---- Batched execution (many independent cells in one call) ----
 * Cell c has its own lattice, beta and tolerance (opts[c]); all cells share
 * kernel, precision and nrhs, and compute the full operator.  Sources of
 * cell c are columns src_off[c] .. src_off[c+1]-1 of the concatenated arrays
 * src [2][NS], q [nrhs][NS] (Stokes [nrhs][2][NS]); targets likewise with
 * trg_off (NULL: targets = sources).  Outputs pot [nrhs][NT] (Stokes
 * [nrhs][2][NT]) and grad [nrhs][2][NT].  On the mixed path the per-cell
 * phases (preparation, far field) of all cells run as one launch per phase
 * and kernel (the FP64 path launches them per cell); the near-image P2P of
 * all cells runs as one persistent kernel per near-block shape over a
 * cost-sorted list of (cell, target block, source range of p2p_chunk
 * sources, rhs group) items (p2p_chunk 0 = 4096; else a multiple of 128).
 * pfmm_batch_create is host-only: it sizes the workspace, including the
 * per-cell argument tables of those launches.  The first execute on a given
 * set of buffers uploads descriptors and tables (cudaMemcpyAsync); later
 * executes on the same buffers issue only memsets and kernels and may be
 * captured in a CUDA graph.  The paper treats one cell at a time; batching
 * is a library feature.  Errors as for the single-cell calls. */
typedef struct pfmm_batch pfmm_batch;
pfmm_status pfmm_batch_create(const pfmm_opts* opts, int ncell, const int64_t* src_off,
                              const int64_t* trg_off, int p2p_chunk, pfmm_batch** out);
pfmm_status pfmm_batch_workspace_size(const pfmm_batch* batch, size_t* bytes);
pfmm_status pfmm_batch_execute(pfmm_batch* batch, void* workspace, size_t ws_bytes, const double* src,
                               const double* q, const double* trg, double* pot, double* grad, void* stream);
/* Synchronise and return the first device status error of any cell (see pfmm_get_status). */
pfmm_status pfmm_batch_get_status(pfmm_batch* batch, void* workspace, void* stream);
/* Phase timing of batch executes with CUDA events (library tracing, not in
 * the paper).  on = 0 off; 1 events and evaluated-pair counting; 2 events
 * only.  While enabled, each execute records three events on its stream; an
 * execute captured into a CUDA graph records them as external event nodes
 * (cudaEventRecordExternal), so that every replay of the graph records them.
 * Pair counting (mode 1) adds atomics to the P2P and is switched by eager
 * executes only: a capture keeps the counting state of the last eager
 * execute on the same buffers.  pfmm_batch_profile_read waits for the events
 * and writes ms[0] = the per-cell phases (preparation and far field of every
 * cell), ms[1] = the batched near-image P2P (n >= 2), of the last execute or
 * replay, *nlaunch (may be NULL) = kernels launched by the last execute and
 * *pairs (may be NULL) = near-image pairs evaluated by the last counted
 * execute (see pfmm_profile_pairs).  Switching profiling off destroys the
 * events: do not switch it off while a graph captured with it on may still
 * be replayed.
 * Errors: PFMM_ERR_INVALID_ARG (NULL batch, bad mode, n < 2, no timed
 * execute yet), PFMM_ERR_CUDA. */
pfmm_status pfmm_batch_profile_enable(pfmm_batch* batch, int on);
pfmm_status pfmm_batch_profile_read(pfmm_batch* batch, float* ms, int n, int* nlaunch, double* pairs);
void pfmm_batch_destroy(pfmm_batch* batch);

/* The same operation as pfmm_execute for callers that cannot allocate device
 * memory (for example a C host program that is handed device pointers by
 * another component and has no device allocator, or a caller that must not
 * call cudaMalloc/cudaFree between launches because they synchronise the
 * device).  The paper has no counterpart: this is a library convenience.
 * Scratch comes from a 32 MiB array compiled into the library (held on every
 * GPU that loads the library until the process exits) instead of a
 * workspace argument; plans whose pfmm_workspace_size exceeds 32 MiB are
 * rejected with PFMM_ERR_WORKSPACE.  Nothing is allocated.  The first call
 * on each device looks up the array's device address (make it before any
 * stream capture).  All calls on one device share the array: calls that
 * overlap on the GPU race and must be serialised by the caller.  Arguments,
 * outputs and host-side errors otherwise as pfmm_execute (device pointers).
 * Conditions only visible on the device go to the array's status word:
 * read them with pfmm_get_status(plan, NULL, stream) before the next call
 * (which clears the word).  The cached address belongs to the device's
 * context: do not use the library across cudaDeviceReset. */
pfmm_status pfmm_execute_static(pfmm_plan* plan, int64_t ns, const double* src, const double* q, int64_t nt,
                                const double* trg, double* pot, double* grad, void* stream);

/* Adjoint (reverse-mode derivative) of pfmm_execute for the potential output.
 * Given g = dL/dpot [nrhs][nt] (device), computes, each only if its pointer is
 * non-NULL:
 *   dq   [nrhs][ns]   dL/dq_j     = sum_l g_l K(t_l, s_j)      (= (P^T g)_j = (P g)_j:
 *                     the periodic operator is symmetric since the far lattice is
 *                     symmetric and G is even; computed by the same kernels with the
 *                     roles of sources and targets swapped)
 *   dsrc [2][ns]      dL/ds_j     = sum_r q_rj grad psi_r(s_j), psi_r = field of the
 *                     charges g_r placed at the targets (scalar kernels only)
 *   dtrg [2][nt]      dL/dt_l     = sum_r g_rl grad u_r(t_l); needs grad_fwd
 *                     [nrhs][2][nt], the gradient output of the forward call.
 *                     With targets = sources, dtrg == dsrc (same pointer) returns
 *                     the sum of both roles in that one array.
 * Laplace/Stokes potentials are defined up to a constant, so only the
 * mean-free part of g matters; g is projected to zero mean per rhs (and
 * component) before use.  Stokes and modified Stokes: dq only (g is [nrhs][2][nt],
 * dq [nrhs][2][ns]; modified Stokes uses g as given: its velocity has no free constant).
 * The plan must admit the swapped sizes: nt <= ns_max and ns <= nt_max
 * (automatic when targets = sources).  src, q, trg as in the forward call.
 * Nothing is stored between the forward and the adjoint: the plane-wave
 * factors are recomputed.  Not in the paper (it applies the operator only). */
pfmm_status pfmm_execute_adjoint(pfmm_plan* plan, void* workspace, size_t ws_bytes, int64_t ns,
                                 const double* src, const double* q, int64_t nt, const double* trg,
                                 const double* g, const double* grad_fwd, double* dq, double* dsrc,
                                 double* dtrg, void* stream);

/* Pressure of the periodic Stokeslet sum (the Stokes kernel of Sec. 5 and
 * its lattice sum, Eq. psum): for the Stokeslet u = (1/4pi)(-log r I +
 * r r^T / r^2) f the pressure is p = (1/2pi) f . r / r^2 = -f . grad G_L with
 * G_L = -(1/2pi) log r, so the periodic pressure is
 *   p(t) = -(d/dx phi[f_x] + d/dy phi[f_y])(t),
 * phi[c] the periodic Laplace potential of charges c (zero net force makes
 * both Laplace sums converge).  It is computed by the Laplace operator of
 * `plan`, which must be a PFMM_LAPLACE plan on the same lattice with an even
 * nrhs = 2 * (Stokes rhs).  f [nrhs/2][2][ns] (input frame) is read as nrhs
 * charge vectors; pres [nrhs/2][nt].  The gradient lives in the plan's
 * workspace.  Errors: as pfmm_execute; PFMM_ERR_INVALID_ARG if the plan is not
 * Laplace or nrhs is odd; PFMM_ERR_NOT_NEUTRAL via pfmm_get_status. */
pfmm_status pfmm_stokes_pressure(pfmm_plan* plan, void* workspace, size_t ws_bytes, int64_t ns, const double* src,
                                 const double* f, int64_t nt, const double* trg, double* pres, void* stream);

/* Synchronise the stream and read the device status word written by the
 * last execute on this workspace; returns it (PFMM_OK, PFMM_ERR_NONFINITE,
 * PFMM_ERR_NOT_NEUTRAL, PFMM_ERR_TIMEOUT, or PFMM_ERR_INVALID_ARG for points
 * outside a singly periodic strip) and clears it.  workspace == NULL reads
 * the status word of pfmm_execute_static's scratch array on the current
 * device.  Errors: PFMM_ERR_INVALID_ARG (NULL plan), PFMM_ERR_CUDA. */
pfmm_status pfmm_get_status(pfmm_plan* plan, void* workspace, void* stream);

/* Per-phase GPU timing (tracing).  When enabled (on != 0), pfmm_execute
 * records CUDA events on the caller's stream around its phases; the events
 * are created here (no device memory).  pfmm_profile_read waits for the last
 * recorded event and returns milliseconds per phase in ms[0..n-1] (n <= 8):
 * [0] prep (wrap, convert, moments), [1] far field (periodizing operator),
 * [2] near-image sum; when the tree code ran, [3..7] split [2] into tree
 * construction, upward pass (P2M, M2M), traversal and list grouping,
 * downward pass (M2L, L2L) and leaves (L2P + direct sums), else they are 0.
 * Errors: PFMM_ERR_INVALID_ARG, PFMM_ERR_CUDA. */
pfmm_status pfmm_profile_enable(pfmm_plan* plan, int on);
pfmm_status pfmm_profile_read(pfmm_plan* plan, float* ms, int n);
/* Near-image pairs (target, source, image) the P2P evaluated in the last
 * profiled execute on `workspace`: ns * nt * images, except for the mixed
 * modified Helmholtz kernel, which skips (target block, source tile, image)
 * triples beyond beta r = x_c (x_c from the tolerance: every skipped term
 * below tol/10 / (images * ns_max), between 10 and 50) and counts what it
 * evaluates, and for the
 * tree code, which counts the pairs of neighbouring leaves it sums directly.  Synchronises
 * `stream`.  Errors: PFMM_ERR_INVALID_ARG (NULL, profiling off), PFMM_ERR_CUDA. */
pfmm_status pfmm_profile_pairs(pfmm_plan* plan, const void* workspace, void* stream, double* pairs);

/* Statistics of the tree code in the last execute on `workspace` (tracing;
 * synchronises `stream`): out[0] tree boxes (sources and targets), out[1]
 * M2L interactions, out[2] leaf pairs summed directly (list entries), out[3]
 * (target, source) point pairs summed directly (counted only while profiling
 * is on, else 0), out[4] overflow bits (0 = none; otherwise a capacity ran
 * out and the direct sum replaced the tree code).  Errors:
 * PFMM_ERR_INVALID_ARG (NULL, or the plan does not use the tree code),
 * PFMM_ERR_CUDA. */
pfmm_status pfmm_near_stats(pfmm_plan* plan, const void* workspace, void* stream, int64_t out[5]);

const char* pfmm_last_error(void);
void pfmm_plan_destroy(pfmm_plan* plan);

/* Library version string (for logs). */
const char* pfmm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PFMM_H */
