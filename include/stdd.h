/*
 * stdd.h -- C ABI of the GB300 overlapping source-transfer DDM solver for
 * 2-D TM FDFD (arXiv 2509.20801).
 *
 * The library solves A e = b (Eq. 4) for the stretched-coordinate PML
 * Helmholtz operator of Eq. 9 discretised on the 5-point stencil of Eq. 2,
 * with flexible GMRES(m) right-preconditioned by one Jacobi sweep of the
 * paper's PML-based overlapping source-transfer iteration (Algorithm 1):
 *
 *     M^-1 v = sum_i E_i A_i^-1 R_i^I v,
 *
 * where A_i is the operator of strip i closed by its own PML (Sec. 2.3,
 * Fig. 3), factored once by a nested-dissection multifrontal LU (Sec. 2.4,
 * Eqs. 22-23) and applied by batched forward/back substitution, R_i^I keeps
 * the strip's own (non-overlapping) columns, and E_i zero-extends the full
 * local field (Eq. 21).  Krylov vectors, residuals, Arnoldi and Givens are
 * FP64 complex; the factors are complex128 or complex64 (set_precision).
 *
 * Conventions used by every entry point
 *   - Grid: nx x ny nodes, PML included.  Node (i, j), i along x, j along y,
 *     has flat index g = i*ny + j.  Field is zero outside the grid.
 *   - Complex vectors are interleaved doubles (re, im): a field is 2*nx*ny
 *     doubles, nrhs fields are stored one after another.
 *   - Pointers marked "is_device" are device pointers on the context's GPU
 *     when the flag is 1 and host pointers when it is 0.  Inputs are copied
 *     (the caller may free them on return); outputs are written into
 *     caller-owned buffers and are complete when the call returns.
 *   - Every call returns a status; on failure stdd_last_error() describes it.
 *     No C++ exception crosses this boundary.  Calls on one context must not
 *     overlap (a context is used by one thread at a time).
 *   - Time convention e^{-i w t}: the PML stretch is s = 1 + i sigma/(w eps0)
 *     (Eq. 10) and a unit point source b_s = -1/(dx dy) gives a field close to
 *     (i/4) H0^(1)(k r).
 */
#ifndef STDD_H
#define STDD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stdd_ctx stdd_ctx;

typedef enum {
  STDD_OK = 0,
  STDD_EINVAL = 1,      /* bad argument or configuration                 */
  STDD_ESTATE = 2,      /* call out of order (e.g. solve before factor)   */
  STDD_ENOMEM = 3,      /* device or host allocation failed               */
  STDD_ECUDA = 4,       /* a CUDA runtime call failed                     */
  STDD_EPIVOT = 5,      /* zero or non-finite pivot in a front            */
  STDD_EBREAKDOWN = 6,  /* Krylov breakdown or non-finite residual        */
  STDD_ENOCONV = 7,     /* maxit reached before rtol (x_out still written) */
  STDD_ETIMEOUT = 8     /* a bounded device wait gave up                  */
} stdd_status;

enum {
  STDD_PREC_FP64 = 0,     /* complex128 factors and substitutions           */
  STDD_PREC_C64 = 1,      /* complex64 factors and substitutions, FP32 math */
  STDD_PREC_C64_BF16 = 2, /* complex64, large-front updates on the tensor
                             cores with BF16 inputs, FP32 accumulation     */
  STDD_PREC_C64_FP16 = 3  /* same with FP16 inputs (power-of-two scaling per
                             64 x 128 tile keeps them in range)            */
};

enum {
  STDD_X0_ZERO = 0,   /* x0 = 0                                            */
  STDD_X0_USER = 1,   /* x0 given by the caller                            */
  STDD_X0_LEARNED = 2 /* x0 from the network attached by
                         stdd_set_learned_guess, scaled to the minimal
                         residual; zero guess where it does not help       */
};

/* Create a context on CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t to run on (NULL: the context creates its own stream).  Every
 * kernel of the context is launched on that stream. */
stdd_status stdd_create(stdd_ctx **out, int device, void *cuda_stream);
void stdd_destroy(stdd_ctx *ctx);

/* Grid of nx x ny nodes with steps dx, dy (same length unit as the
 * wavelength), Eq. 2.  Invalidates the factors. */
stdd_status stdd_set_grid(stdd_ctx *ctx, int nx, int ny, double dx, double dy);

/* Node permittivity epsbar (Eq. 3; real, nx*ny doubles, index g).
 * Requires set_grid.  Copied.  Invalidates the factors. */
stdd_status stdd_set_permittivity(stdd_ctx *ctx, const double *eps_node, int is_device);

/* Free-space wavelength; k0 = 2 pi / wavelength (Eq. 1).  Invalidates the
 * factors. */
stdd_status stdd_set_frequency(stdd_ctx *ctx, double wavelength);

/* Global PML: npml = {x0, x1, y0, y1} cells at the four sides, polynomial
 * order m and normal-incidence reflection R0 (Eqs. 10-13).  sigma/(w eps0)
 * = (m+1)(-ln R0)/(2 k0 d) (rho/d)^m with d = L*delta; node u = 1..L of a
 * PML sits at depth rho = (u - 1/2) delta and half node u + 1/2 at u delta
 * from the interface.  Invalidates the factors. */
stdd_status stdd_set_pml(stdd_ctx *ctx, const int npml[4], int order_m, double R0);

/* Strip decomposition along x (Sec. 2.3, Fig. 3).  nsub strips own the node
 * columns [c_k, c_{k+1}); x_cuts holds c_0 = 0 < c_1 < ... < c_nsub = nx
 * (nsub+1 ints) or NULL for equal widths (remainder to the first strips).
 * Each strip's local box extends `overlap` physical columns and then an
 * `interface_pml`-cell PML into each neighbour; the global x-PML stays with
 * the end strips and the y-PML with every strip.  overlap + interface_pml
 * must not exceed a neighbour's width.  Invalidates the factors. */
stdd_status stdd_set_decomposition(stdd_ctx *ctx, int nsub, const int *x_cuts, int overlap,
                                   int interface_pml);

/* Two-dimensional (checkerboard) decomposition: the strip construction of
 * Sec. 2.3 applied along x (px parts, x_cuts as above) and, independently,
 * along y (py parts, y_cuts: c_0 = 0 < ... < c_py = ny, or NULL for equal
 * heights).  Box k = kx * py + ky owns the columns of x-part kx and the rows
 * of y-part ky; its local box extends `overlap` nodes and then an
 * `interface_pml`-cell PML past every side that has a neighbour, in x and in
 * y, and keeps the global PML on the domain's sides; Dirichlet outside.  The
 * preconditioner keeps its definition, M^-1 v = sum_k E_k A_k^-1 R_k^I v,
 * summed over boxes (a node is covered by at most 9 local boxes).
 * overlap + interface_pml must not exceed a neighbouring part's width or
 * height.  py = 1 is stdd_set_decomposition.  With py > 1 only the additive
 * order and full-space FGMRES apply (the other orders, band space and the
 * Richardson mode return STDD_EINVAL).  Invalidates the factors.  (The paper
 * partitions into x-strips only.) */
stdd_status stdd_set_decomposition_2d(stdd_ctx *ctx, int px, const int *x_cuts, int py, const int *y_cuts,
                                      int overlap, int interface_pml);

/* Extents of box (or strip) k: out[0..7] = owned columns [c0, c1), owned
 * rows [r0, r1), local box columns [x0, x1), local box rows [y0, y1).  The
 * box's local fields (stdd_local_solve) are (x1 - x0) * (y1 - y0) complex
 * values, local node (i - x0) * (y1 - y0) + (j - y0). */
stdd_status stdd_box_info(const stdd_ctx *ctx, int box, int out[8]);

/* One of STDD_PREC_*.  Invalidates the factors.  The Krylov iteration,
 * residuals and the returned fields are FP64 in every mode. */
stdd_status stdd_set_precision(stdd_ctx *ctx, int mode);

/* nrhs right-hand sides b (Eq. 4), nrhs * 2*nx*ny doubles.  Copied.  Does
 * not invalidate the factors (the matrix is unchanged). */
stdd_status stdd_set_sources(stdd_ctx *ctx, int nrhs, const double *b_interleaved, int is_device);

/* Preprocessing of Algorithm 1: nested-dissection symbolic analysis of each
 * strip shape (host) and numeric multifrontal LU of every strip's A_i
 * (device, batched over strips and fronts), A_i = P^T L U Q^T (Eq. 22). */
stdd_status stdd_factor(stdd_ctx *ctx);

typedef struct {
  int restart;            /* GMRES restart length m (>= 1)                   */
  int maxit;              /* total inner iterations (or sweeps) allowed     */
  double rtol;            /* stop at ||b - A x|| / ||b|| <= rtol             */
  int x0_mode;            /* STDD_X0_ZERO, STDD_X0_USER or STDD_X0_LEARNED   */
  const double *x0;       /* initial guesses (nrhs fields) if USER          */
  int x0_is_device;
  int paper_richardson;   /* 1: run Algorithm 1 itself (Richardson form,
                             stop when sum_i ||e_i^F|| < rtol * ||e^(0)||,
                             Eq. 20) instead of FGMRES                       */
} stdd_solve_opts;

/* Solve every right-hand side; x_out receives nrhs fields.  Returns
 * STDD_ENOCONV if some right-hand side did not reach rtol within maxit (its
 * last iterate is still written). */
stdd_status stdd_solve(stdd_ctx *ctx, const stdd_solve_opts *opts, double *x_out, int is_device);

/* Relative residual history of right-hand side `rhs` of the last solve:
 * entry 0 is the initial true residual, entry k the estimate after inner
 * iteration k (FGMRES) or the true residual after sweep k (Richardson).
 * Copies min(cap, n) values into out (host) and stores n in *n_out. */
stdd_status stdd_residual_history(stdd_ctx *ctx, int rhs, double *out, int cap, int *n_out);

const char *stdd_last_error(const stdd_ctx *ctx);

/* ---------------------------------------------------------------------
 * Operator-level entry points (each one step of the hot path).  All take
 * single complex vectors.
 * ------------------------------------------------------------------- */

/* y = A x, the global stretched 5-point operator (Eqs. 2, 9).  Needs grid,
 * permittivity, frequency and PML. */
stdd_status stdd_apply_operator(stdd_ctx *ctx, const double *x, double *y, int is_device);

/* z = M^-1 v = sum_i E_i A_i^-1 R_i^I v: restriction to owned columns,
 * batched multifrontal forward/back substitution in every strip, and
 * synthesis of the full local fields (Algorithm 1 sweep, Eq. 21).  Needs
 * stdd_factor. */
stdd_status stdd_apply_preconditioner(stdd_ctx *ctx, const double *v, double *z, int is_device);

/* z = A_k^-1 t for strip (or box) k alone; t and z are local fields of
 * (x1 - x0) * ny complex values, local index (i - x0)*ny + j (a box:
 * (x1 - x0) * (y1 - y0) values, see stdd_box_info). */
stdd_status stdd_local_solve(stdd_ctx *ctx, int strip, const double *t, double *z, int is_device);

/* Columns of strip k: owned [c0, c1), local box [x0, x1). */
stdd_status stdd_strip_info(const stdd_ctx *ctx, int strip, int *c0, int *c1, int *x0, int *x1);

typedef struct {
  long long nfronts;          /* fronts over all strips                     */
  int depth;                  /* levels of the deepest elimination tree     */
  int max_pivots;             /* largest separator / leaf pivot block       */
  int max_border;             /* largest front border                       */
  long long factor_entries;   /* complex entries stored in L and U          */
  double factor_flops;        /* real flops the factorization executes (the
                                 Gauss-Jordan sweep: sum p n^2 complex
                                 multiply-adds over fronts)                 */
  double solve_flops;         /* real flops of one M^-1 application         */
  long long local_dofs;       /* sum of local box sizes                     */
  long long device_bytes;     /* device memory held by the context          */
  int iterations;             /* inner iterations of the last solve (rhs 0) */
  double final_residual;      /* true relative residual (rhs 0)             */
  double min_pivot;           /* smallest |pivot| seen by the factorization */
  int reorth_passes;          /* second Gram-Schmidt passes in the last solve */
  long long raised_pivots;    /* pivots raised to the static-pivot floor    */
  double factor_flops_lu;     /* the same elimination counted as an LU
                                 factorization (Eq. 22): pivot k of a front
                                 of n updates the (n-k-1)^2 trailing block  */
} stdd_stats;

stdd_status stdd_get_stats(stdd_ctx *ctx, stdd_stats *out);

/* r = b - A x for one field and its relative norm ||r|| / ||b|| (FP64,
 * deterministic reduction).  x, b, r: 2*nx*ny doubles each; *rel_out is a
 * host double.  Needs grid, permittivity, frequency and PML. */
stdd_status stdd_residual(stdd_ctx *ctx, const double *x, const double *b, double *r, double *rel_out,
                          int is_device);

/* Same result as stdd_residual, without allocating device memory.  The
 * paper has no counterpart: this entry point exists for callers that may not
 * call cudaMalloc at the time they need a residual -- real-time loops that
 * reserve all of their device memory before they start, or host
 * applications that hand out GPU memory only through their own pool and
 * forbid libraries to allocate behind it.
 *   x, b : device pointers, 2*nx*ny doubles each (inputs);
 *   r    : device pointer, 2*nx*ny doubles (output, b - A x).  r may be the
 *          same buffer as b (each entry of b is read before it is
 *          overwritten) but must not overlap x, whose neighbouring entries
 *          other threads still read, nor overlap b only in part: both are
 *          rejected with STDD_EINVAL;
 *   *rel_out : host double, ||r|| / ||b|| (||r|| if b = 0).
 * Scratch is one fixed array compiled into the library (2*16384 + 2
 * doubles, about 256 KiB); every GPU that loads the library keeps it until
 * the process exits.  Grids above 67,108,864 nodes are rejected with
 * STDD_EINVAL.  The operator must already be set up on the context (any
 * earlier stdd_apply_operator, stdd_residual or stdd_factor call does it),
 * else STDD_ESTATE.  The first call on a device looks up the scratch
 * array's device address (cudaGetSymbolAddress), so make that first call
 * before any stream capture.  All calls share the one array: calls that
 * overlap on the GPU (other contexts, other streams, other threads) race and
 * must be serialised by the caller.  Each call writes every scratch slot it
 * reads before reading it, so nothing carries over between calls.  The call
 * synchronises the context stream to return *rel_out. */
stdd_status stdd_residual_noalloc(stdd_ctx *ctx, const double *x, const double *b, double *r,
                                  double *rel_out);

/* Phase profile: with profiling on, the context records CUDA events on its
 * stream around each phase; get_profile synchronises the stream and sums the
 * device times (ms) of the phases completed since the last reset.  Kernel
 * launches are counted whether or not profiling is on. */
typedef struct {
  double factor_ms;       /* numeric factorization (all levels)           */
  double minv_ms;         /* preconditioner applications (M^-1)           */
  int minv_calls;
  double matvec_ms;       /* global stencil products                      */
  int matvec_calls;
  double ortho_ms;        /* Gram-Schmidt passes of the Arnoldi steps      */
  int ortho_calls;
  double solve_ms;        /* whole stdd_solve calls                        */
  long long launches;     /* kernels of this library launched             */
  /* the dominant kernels, launch by launch, with their algorithmic work:
   * small-front and blocked-update eliminations (real flops of the LU
   * trailing-block updates they stand for, Eq. 22), the upward and
   * downward substitution sweeps (factor bytes read) */
  double small_ms, small_flops;
  int small_calls;
  double update_ms, update_flops;
  int update_calls;
  double up_ms, up_bytes;
  int up_calls;
  double down_ms, down_bytes;
  int down_calls;
  /* real flops the two elimination kernels execute (Gauss-Jordan: the
   * updates also cover the eliminated pivot rows and columns) */
  double small_flops_executed, update_flops_executed;
  /* persistent one-strip solves (STDD_OPT_PERSISTENT): launches, time and
   * the factor bytes they read */
  double sweep_ms, sweep_bytes;
  int sweep_calls;
} stdd_profile;

/* level 0: off; 1: phase spans (factor, M^-1, matvec, Gram-Schmidt,
 * solve); 2: also one span per launch of the dominant kernels (this
 * bypasses the CUDA graphs of the M^-1 application). */
stdd_status stdd_set_profiling(stdd_ctx *ctx, int level);

/* Execution options; none of them changes a computed value.
 *   STDD_OPT_GRAPHS   (default 1): replay captured CUDA graphs of the M^-1
 *                     application (one graph per input/output buffer pair,
 *                     captured on first use; the first use must not happen
 *                     inside the caller's own stream capture).
 *   STDD_OPT_AUTOTUNE (default 1): choose the substitution launch shapes per
 *                     tree level by timing them once per level shape.
 *   STDD_OPT_LEAF     (default 16): nested-dissection leaf size in nodes
 *                     (changes the factorization, invalidates factors).
 * and one that changes the preconditioner (not the solution):
 *   STDD_OPT_ORDER    (default 0): 0 = the additive order of Algorithm 1,
 *                     M^-1 v = sum_i E_i A_i^-1 R_i^I v, all strips at once;
 *                     1 = symmetric multiplicative order, strips one after
 *                     another forward then backward (k = 0..n-1, n-2..0),
 *                     each solving for the current residual:
 *                     z += E_k A_k^-1 R_k^I (v - A z), starting from z = 0
 *                     (the layer-by-layer transfer of the original source
 *                     transfer method, Sec. 1); 2 = red-black: the even
 *                     strips all at once, then the odd strips, each group
 *                     solving for the residual left by the previous one
 *                     (the same as solving them one by one, since a strip's
 *                     local box never reaches the owned columns of the next
 *                     strip of its colour: needs every interior strip wider
 *                     than overlap + interface PML + 1, else STDD_EINVAL
 *                     when it is applied); 3 = forward multiplicative, the
 *                     strips once, k = 0..n-1 (half the local solves of
 *                     order 1 per application; not symmetric, which flexible
 *                     GMRES does not need).  In paper_richardson mode the
 *                     stationary iteration uses the chosen order.
 * and one that changes how FGMRES works (same iterates in exact arithmetic):
 *   STDD_OPT_BAND     (default 0): 1 = band-space FGMRES.  For the additive
 *                     order, A M^-1 - I maps everything into the interface
 *                     bands (the overlap and interface-PML columns around
 *                     each interface, plus one), so with r0 = b - A x0 the
 *                     solve runs GMRES on the band system
 *                     (I + T) s = -T r0, T = A M^-1 - I, and returns
 *                     x = x0 + M^-1 (r0 + s).  Krylov vectors hold only the
 *                     band columns, and each band application of M^-1 skips
 *                     the subtrees with no band sources (going up) and the
 *                     fronts off the band (coming down).  Its residuals are
 *                     the true residuals because the local solves are exact,
 *                     so it needs FP64 factors and the additive order (else
 *                     stdd_solve returns STDD_EINVAL): complex64 local solves
 *                     leave too large an error off the bands.  It costs one
 *                     full application before the iteration (counted as the
 *                     first iteration) and one after; the residual history
 *                     ends with the true residual of the returned field.
 * and one that changes the factors (and so the preconditioner, not the
 * solution):
 *   STDD_OPT_STATIC_PIVOT (default 0): static pivoting of the front
 *                     sweeps.  k in 1..15: a pivot whose modulus is below
 *                     10^-k (2/dx^2 + 2/dy^2) is replaced by that floor
 *                     times its phase (the factors are then those of A + E,
 *                     E diagonal with one entry per raised pivot; the count
 *                     is in stdd_stats.raised_pivots); 0: off (the plain
 *                     elimination of Eq. 22).  The sweep has no pivoting,
 *                     and nested dissection eliminates each box with its
 *                     separators held fixed, i.e. as a closed cavity; near a
 *                     cavity resonance the pivot block is near-singular and
 *                     the elimination's growth, harmless in FP64, can ruin
 *                     complex64 factors (high-index guided-wave geometries).
 *                     Invalidates the factors. */
/*   STDD_OPT_UPDATE_TILE (default 0): tile edge of the blocked front
 *                     update.  0: chosen per tree level by the autotuner (the
 *                     first factorization of a level shape times the
 *                     factorization with 64 x 64 and with 32 x 32 tiles and
 *                     keeps the faster per level; cached for the process);
 *                     64 or 32: that shape on every level.  Every entry sums
 *                     its products in the same order on either shape, so
 *                     results do not change.  (With STDD_OPT_AUTOTUNE 0 and
 *                     this option 0 the shape is 64.)
 *   STDD_OPT_PERSISTENT (default -1): in the sequential orders (1 and 3,
 *                     one right-hand side at a time) each strip's solve --
 *                     residual restriction, the upward and the downward
 *                     sweep over all tree levels, the add-back -- runs as
 *                     one cooperative launch whose levels are separated by
 *                     grid-wide barriers instead of ~3 launches per level;
 *                     0: one launch per level; k = 1..8: the cooperative
 *                     grid holds k blocks per SM (at most what fits); -1: 2
 *                     for complex64 factors, 0 for complex128 ones (whose
 *                     products are FP64-bound per warp and run faster in the
 *                     per-level kernels' deeper load pipelines).  Same
 *                     arithmetic, same results.
 *   STDD_OPT_SWEEP_WAIT (default 0 = 4,194,304): polls a block spends at one
 *                     grid barrier of a persistent sweep before it gives up;
 *                     then every block returns, the call that applied the
 *                     preconditioner returns STDD_ETIMEOUT, and the context
 *                     stays usable.
 *   STDD_OPT_PIVOTING (default 0): 1 = partial pivoting restricted to each
 *                     front's pivot rows.  Before each pivot (each 32-pivot
 *                     block of a large front) the not yet eliminated pivot
 *                     row whose entry in the pivot column is largest in
 *                     modulus is swapped in; rows are never exchanged with
 *                     the front's border, so the nested-dissection order and
 *                     the fronts stay as they are (Eq. 22's P is then the
 *                     fill-reducing order times these interchanges).  It
 *                     bounds the element growth of the unpivoted sweep
 *                     inside a front, which complex64 factors of high-index
 *                     guided-wave geometries cannot afford.  Invalidates the
 *                     factors.
 *   STDD_OPT_SYMMETRIC (default 1): factor each box's operator in its
 *                     complex-symmetric form D A_i, D the diagonal of the
 *                     box's stretch products s_x s_y at the nodes (Eqs.
 *                     10-13: row u of the SC-PML operator times s_x s_y at
 *                     u is symmetric), and solve A_i x = r as D A_i x = D r.
 *                     The working matrix of the blocked Gauss-Jordan sweep
 *                     is then symmetric within the eliminated and within the
 *                     remaining rows and antisymmetric between them, so the
 *                     large-front update (most of the factorization's
 *                     arithmetic) computes one triangle and mirrors it.
 *                     Used when STDD_OPT_PIVOTING is 0 (row interchanges
 *                     break the symmetry) and the factors are not formed
 *                     with tensor-core updates (STDD_PREC_C64_BF16 /
 *                     _FP16 update whole tiles).  1: complex128 factors;
 *                     2: complex64 factors too (in single precision the
 *                     scaling by D, up to the PML's largest |s_x s_y| apart
 *                     between rows, adds element growth that the unpivoted
 *                     sweep cannot afford on resonant geometries: the
 *                     48-geometry ellipse batch then needs 192 instead of
 *                     31 red-black iterations, 4 of its 2048-wide
 *                     geometries no longer converging); 0: the factors of
 *                     A_i as assembled.  The forms agree to rounding.
 *                     Invalidates the factors.
 *   STDD_OPT_FP64_TC (default 1): complex128 factors in the symmetric form
 *                     compute the large-front update products on the BF16
 *                     tensor cores by exact splitting (the scheme of Ozaki,
 *                     Ogita, Oishi and Rump, Numer. Algorithms 59, 2012):
 *                     each real row of the pivot-column panel and each real
 *                     column of the pivot-row panel is scaled by a power of
 *                     two and cut into eight 7-bit slices (exact BF16
 *                     numbers); the 36 slice products whose orders sum to at
 *                     most 7 are accumulated exactly in FP32, combined in
 *                     64-bit integers and rounded to FP64 once, so the
 *                     product's error is bounded like an FP64 dot product's
 *                     (relative to the row's and the column's largest
 *                     entries).  0: the FP64 pipe.  The two agree to
 *                     rounding.  Invalidates the factors.
 *   STDD_OPT_SWEEP_SPLIT (default 0): how the substitution products of a
 *                     work item (a front's 16 or 32 rows) share its columns,
 *                     which are summed in fixed segments of 128 columns whose
 *                     sums are added in column order.  0: chosen per level
 *                     by the autotuner; 1, 2, 4, 8: that many warps of one
 *                     block per item; 16: one warp per (item, segment)
 *                     anywhere on the GPU, the segment sums added by a
 *                     second launch (32-row items; the FP64 pipe of one SM
 *                     no longer bounds a root-level item).  Every choice
 *                     gives the same sums in the same order: results do not
 *                     change.  Applied at the next stdd_factor. */
enum {
  STDD_OPT_GRAPHS = 1,
  STDD_OPT_AUTOTUNE = 2,
  STDD_OPT_LEAF = 3,
  STDD_OPT_ORDER = 4,
  STDD_OPT_BAND = 5,
  STDD_OPT_STATIC_PIVOT = 6,
  STDD_OPT_PIVOTING = 7,
  STDD_OPT_PERSISTENT = 8,
  STDD_OPT_SWEEP_WAIT = 9,
  STDD_OPT_UPDATE_TILE = 10,
  STDD_OPT_SYMMETRIC = 11,
  STDD_OPT_FP64_TC = 12,
  STDD_OPT_SWEEP_SPLIT = 13
};
stdd_status stdd_set_option(stdd_ctx *ctx, int option, int value);
stdd_status stdd_get_profile(stdd_ctx *ctx, stdd_profile *out, int reset);

/* Diagnostic: one tile product D = C R of the tensor-core front update
 * (tcgen05, the kernel path of STDD_PREC_C64_BF16 / _FP16) with host
 * arrays, so that a caller can check it against its own reference.  C is
 * 64 x kc complex, R kc x 128, D 64 x 128, all column-major interleaved
 * doubles (C(i, j) at 2 (j*64 + i), R(j, c) at 2 (c*kc + j), D(i, c) at
 * 2 (c*64 + i)); 1 <= kc <= 32.  The inputs are converted to float, scaled
 * by a power of two per operand (2^ea for C, 2^eb for R, with the largest
 * |component| scaled into [1, 2)), rounded to FP16 (fmt 0) or BF16 (fmt 1),
 * multiplied with FP32 accumulation through the real 2 x 2 embedding of the
 * complex product, and scaled back by 2^-(ea+eb).  STDD_ETIMEOUT if the
 * tile's bounded wait gave up.  No counterpart in the paper. */
stdd_status stdd_tc_tile_product(int device, int fmt, int kc, const double *C, const double *R, double *D);

/* Diagnostic: one 64 x 64 complex128 tile product D = C R through the
 * exact-splitting tensor-core path of STDD_OPT_FP64_TC, with host arrays:
 * C 64 x kc, R kc x 64, D 64 x 64, column-major interleaved doubles (C(i, j)
 * at 2 (j*64 + i), R(j, c) at 2 (c*kc + j), D(i, c) at 2 (c*64 + i));
 * 1 <= kc <= 32.  Each real row of the embedded C ([Re, -Im] and [Im, Re]
 * rows of complex row i) and each complex column of R is scaled by the power
 * of two just above its largest |component| and cut into eight 7-bit
 * slices; D(i, c) is exact up to the dropped slice orders (below 2^-53 of
 * the scales times 2 kc) and one rounding to FP64.  STDD_EINVAL for
 * non-finite inputs or kc out of range, STDD_ETIMEOUT if the tile's bounded
 * wait gave up.  No counterpart in the paper. */
stdd_status stdd_tc_f64_tile_product(int device, int kc, const double *C, const double *R, double *D);

/* Host-only nested-dissection analysis of one W x H box (no GPU needed).
 * First call with nodes == NULL to get *nfronts and *nnodes; then call
 * again with arrays of those sizes.  Fronts come in elimination order
 * (children before parents).  For front f: p[f] pivots and b[f] border
 * nodes, listed in nodes[off_f .. off_f + p[f] + b[f]) with off_f the
 * running sum of p + b, pivots first; a node is x*H + y.  parent[f] = -1
 * for the root; level[f] is the depth from the root. */
stdd_status stdd_nd_analyze(int W, int H, int leaf_max, int *nfronts, long long *nnodes, int *p,
                            int *b, int *parent, int *level, int *nodes);

/* ---------------------------------------------------------------------
 * Learned initial guess.  No counterpart in the paper: a convolutional
 * encoder-decoder maps (permittivity, Re b, Im b) on the grid to an initial
 * field for the Krylov iteration, which still runs to the same tolerance --
 * the zero-guess method remains both the fallback and the yardstick the
 * guess is measured against.
 *
 * Network with L levels and channels c_l = min(c0 * 2^l, cmax):
 *   encoder level l: conv3x3 + ReLU, conv3x3 + ReLU (= skip_l); the input of
 *     level 0 is the 3-channel image, of level l > 0 the 2x2 average pool of
 *     skip_{l-1};
 *   decoder level l = L-2 .. 0: nearest 2x upsampling of the level below,
 *     conv3x3 (c_{l+1} -> c_l) + ReLU, plus skip_l, conv3x3 + ReLU;
 *   output: conv3x3 (c_0 -> 2), no activation.
 * Convolutions: 3x3, stride 1, zero padding, cross-correlation
 *   out[co](y, x) = bias[co] + sum_ci sum_ky,kx w[co][ci][ky][kx] *
 *                   in[ci](y + ky - 1, x + kx - 1).
 * Parameters: one float array, layer by layer in the order above (encoder
 * 0 first conv, second conv, encoder 1 ..., decoder L-2 upsampled conv,
 * second conv, ..., decoder 0, output), each layer its weights
 * [cout][cin][3][3] then its bias [cout].
 * Images: float, NCHW, [batch][channel][H][W] row-major; H and W multiples
 * of 2^(L-1).  The solver's node (i, j) is image row j, column i.
 * Arithmetic (mode): the weights used by forward and backward passes are the
 * FP32 master weights rounded to BF16, or the FP32 weights themselves
 * (STDD_NN_FP32); activations are FP32 and rounded to BF16 only as
 * tensor-core operands (STDD_NN_TC); accumulation is FP32.
 * Loss: mean squared error over all outputs of the batch.  Optimiser: Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32 master weights.
 * ------------------------------------------------------------------- */
typedef struct stdd_nn stdd_nn;

enum {
  STDD_NN_FP32 = 0,       /* FP32 weights, CUDA-core convolutions (exact-layout
                             reference mode)                                 */
  STDD_NN_BF16 = 1,       /* BF16-rounded weights, FP32 activations, CUDA cores */
  STDD_NN_TC = 2          /* BF16 weights and activations in the convolutions
                             on the tensor cores (tcgen05), FP32 accumulation;
                             weight gradients on CUDA cores in FP32; at most
                             256 channels                                    */
};

/* Create a network on `device` (stream as in stdd_create), weights He-normal
 * from `seed` (output layer scaled by 0.1), biases zero.  levels 1..8,
 * 1 <= base_channels <= max_channels, mode one of STDD_NN_*.  A tensor-core
 * wait that times out makes the call that launched it return STDD_ECUDA. */
stdd_status stdd_nn_create(stdd_nn **out, int device, void *cuda_stream, int levels, int base_channels,
                           int max_channels, int mode, unsigned long long seed);
void stdd_nn_destroy(stdd_nn *nn);
/* Number of floats in the parameter array (-1 for NULL). */
long long stdd_nn_num_params(const stdd_nn *nn);
/* Copy the FP32 master parameters out / in (host arrays of num_params
 * floats).  set_params also resets nothing else (Adam moments are kept). */
stdd_status stdd_nn_get_params(stdd_nn *nn, float *host);
stdd_status stdd_nn_set_params(stdd_nn *nn, const float *host);
/* output[batch][2][H][W] = network(input[batch][3][H][W]); device pointers. */
stdd_status stdd_nn_forward(stdd_nn *nn, int batch, int H, int W, const float *input, float *output);
/* Loss and its gradient with respect to every parameter for one batch
 * (input, target: device pointers, target [batch][2][H][W]); *loss_out
 * (host, may be NULL) and grad_host (host, num_params floats, may be NULL)
 * receive them.  Parameters are not changed. */
stdd_status stdd_nn_gradient(stdd_nn *nn, int batch, int H, int W, const float *input, const float *target,
                             float *loss_out, float *grad_host);
/* One Adam step with learning rate lr on the batch; *loss_out (host, may be
 * NULL) receives the loss before the step. */
stdd_status stdd_nn_train_step(stdd_nn *nn, int batch, int H, int W, const float *input, const float *target,
                               float lr, float *loss_out);
/* Network images of one problem, with the normalisation the solver's
 * STDD_X0_LEARNED guess uses (device pointers; eps: nx*ny doubles, b and x:
 * 2*nx*ny doubles, node (i, j) at i*ny + j):
 *   input[3][H][W]:  (eps - 1) / 10, Re b / s, Im b / s at row j, column i;
 *   target[2][H][W]: Re x / (s * unit), Im x / (s * unit) (skipped if x is
 *                    NULL), s = max over nodes of max(|Re b|, |Im b|).
 * H >= ny and W >= nx; pixels outside the grid are zero.  The solver uses
 * unit = dx * dy. */
stdd_status stdd_nn_make_images(stdd_nn *nn, int nx, int ny, double unit, const double *eps, const double *b,
                                const double *x, int H, int W, float *input, float *target);
const char *stdd_nn_last_error(const stdd_nn *nn);

/* Attach a network (or NULL to detach) as the context's STDD_X0_LEARNED
 * guess; the network must live on the context's device and outlive its use.
 * For right-hand side b the start is built in three steps:
 *   y  = network((eps - 1) / 10, Re b / s, Im b / s) * s * dx * dy,
 *        s = max over nodes of max(|Re b|, |Im b|) (the grid is zero-padded
 *        to a multiple of 2^(L-1) for the network);
 *   x  = y + M^-1 (b - A y): one sweep of the preconditioner from y (one
 *        batched application for all right-hand sides), which removes the
 *        short-range error the network leaves and keeps its long-range
 *        field;
 *   x0 = alpha x with alpha = (A x)^H b / ||A x||^2, the factor that
 *        minimises ||b - alpha A x||.
 * If that residual is not below ||b|| (or is not finite) the zero guess is
 * used.  The sweep is not counted in the iteration count. */
stdd_status stdd_set_learned_guess(stdd_ctx *ctx, stdd_nn *nn);

/* After a solve with STDD_X0_LEARNED: for right-hand side `rhs`, the
 * relative residuals ||b - A y|| / ||b|| of the raw network field and
 * ||b - alpha A x|| / ||b|| of the start, and whether the start was used
 * (1) or replaced by zero (0).  Any output pointer may be NULL. */
stdd_status stdd_learned_guess_info(stdd_ctx *ctx, int rhs, double *raw_rel, double *scaled_rel, int *used);

#ifdef __cplusplus
}
#endif
#endif /* STDD_H */
