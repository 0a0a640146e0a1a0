/*
 * fc.h -- C-ABI of libfc, a single-GPU (GB300, sm_103a) geometric multigrid
 * solver for finite cell Stokes problems with the restricted additive (RA)
 * patch smoother of Saberi & Vogel, "A restricted additive smoother for
 * finite cell flow problems".
 *
 * Problem (paper Sec. 2): -eta lap u + grad p = f, div u = 0 in the fluid
 * Omega, embedded in the box Omega_e; the fictitious part (inside obstacles)
 * is weighted by alpha << 1 (eq. stokes_weak_fcm); no-slip on the obstacle
 * boundary is imposed weakly by the symmetric Nitsche method; equal-order
 * Q1-Q1 elements with the local L2 pressure-projection stabilisation
 * (eq. stabilization_l2) on a uniform background grid; strong Dirichlet data
 * on box faces per boundary preset.  The discrete system is L x = b
 * (Sec. 3, eq. linear_system).
 *
 * Conventions for every entry point:
 *  - Vectors are caller-owned DEVICE pointers to float64 in node-interleaved
 *    layout: node (i, j, k) with i fastest, then the d velocity components,
 *    then the pressure: x[((k*(ny+1) + j)*(nx+1) + i)*(d+1) + c].
 *  - Levels are numbered as in the paper (Sec. 3): 1 = coarsest, L = finest.
 *  - A vector of level l holds ndof(l) = (d+1) prod_k (n_k / 2^(L-l) + 1)
 *    doubles (fc_info reports it).  The library reads or writes exactly that
 *    many values at each pointer and cannot check a pointer's extent or
 *    memory space: a shorter buffer, a host pointer or another GPU's memory
 *    is an illegal access on the device.  The Python binding checks all
 *    three before it passes a pointer.
 *  - All device work is enqueued on the stream given to fc_setup and is
 *    asynchronous unless the entry point says it synchronises.
 *  - Threads: different handles are independent and may be used from
 *    different host threads at the same time (fc_smooth_noalloc excepted,
 *    see there); calls on one handle, and on a batch together with the
 *    handles it groups, must not overlap.
 *  - Errors are returned as fc_status codes; fc_last_error(h) gives a
 *    message.  No entry point aborts the process.  A handle stays valid
 *    after FC_ERR_NOT_CONVERGED and after argument errors.  A handle whose
 *    fc_setup failed answers only fc_last_error, fc_sync and fc_destroy;
 *    every other call returns FC_ERR_INVALID without touching the device.
 *  - Environment variables (read at setup or first use; unset = the
 *    defaults, which the results above are measured with).  Tuning: each
 *    changes a launch shape and so the rounding order only.
 *      FC_APPLY_TPP       lanes per patch of the float-pair apply (2..32)
 *      FC_APPLY64_TPP     lanes per 3D patch of the FP64-row apply (4..32)
 *      FC_AMR_LANES       lanes per patch / node on adaptive levels (4, 8, 16)
 *      FC_FACTOR_THREADS  threads per CTA of the dense patch factorisations
 *    Validation: FC_LDL_MIN_PIVOT (default 1e-14) is the smallest pivot the
 *    banded LDL^T of a 3D patch's velocity block accepts before the patch
 *    goes to the pivoted dense LU; a value above 1 sends every patch there
 *    (the two paths give the same rows up to rounding, which tests use).
 */
#ifndef FC_H
#define FC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fc_handle_s* fc_handle; /* opaque; owns all device memory it allocates */

typedef enum {
  FC_OK = 0,
  FC_ERR_INVALID = 1,        /* bad argument or unsupported combination */
  FC_ERR_OOM = 2,            /* device allocation failed */
  FC_ERR_CUDA = 3,           /* a CUDA call or kernel failed */
  FC_ERR_NOT_CONVERGED = 4,  /* fc_solve stopped at maxit above rtol */
  FC_ERR_SINGULAR = 5,       /* a local or coarse LU met a zero pivot */
  FC_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
  FC_WARN_FP64_FALLBACK = 100 /* informational: some patches kept in FP64 */
} fc_status;

/* Patch cache policy (Sec. 3.1.2). */
typedef enum {
  FC_CACHE_INVERSE = 0, /* store the 1+d owned rows of L_i^{-1} */
  FC_CACHE_MATRIX = 1,  /* store the block factorisation of L_i; solve per apply */
  FC_CACHE_NONE = 2     /* gather L_i from the operator, factor and solve per apply */
} fc_cache;

/* Storage/arithmetic of the cached patch rows (cache_inverse only).  The rows
 * are computed in float64 (3D Q1-Q1: banded LDL^T of the velocity block, or
 * the pivoted dense LU where that block is not positive definite) and then
 * stored in the chosen precision; in 2D, float-pair rows come from a
 * float-pair elimination and float32 / bfloat16 rows from float32 factors
 * with two refinement steps. */
typedef enum {
  FC_PREC_FP64 = 0, /* float64 rows, float64 arithmetic */
  FC_PREC_FP32 = 1, /* float32 rows, float32 accumulation */
  FC_PREC_BF16 = 2, /* bfloat16 rows, float32 accumulation */
  FC_PREC_DF64 = 3  /* rows and residual as float32 pairs (hi + lo), pair arithmetic */
} fc_prec;

/* Uniform background grid of the finest level: n cells per direction on the
 * box [lo, hi].  dim is 2 or 3; entries of n/lo/hi beyond dim are ignored. */
typedef struct {
  int dim;
  int n[3];
  double lo[3], hi[3];
} fc_grid;

/* Obstacle (fictitious region).  type 0: circle (2D) or sphere (3D) of
 * radius r[0] around c; type 1: ellipse (2D) with semi-axes r[0] along the
 * direction rot = (cos theta, sin theta) and r[1] across it.  The level set
 * is phi = max over shapes, phi > 0 inside an obstacle (Sec. 2, alpha). */
typedef struct {
  int type;
  double c[3];
  double r[3];
  double rot[2];
} fc_shape;

typedef struct {
  int nshapes;
  const fc_shape* shapes; /* host array, copied by fc_setup */
} fc_levelset;

typedef struct {
  double eta;          /* viscosity (Sec. 4: 1e-3) */
  double nitsche_beta; /* Nitsche lambda = beta * eta / h_min (default 100) */
  double omega;        /* smoother damping (Sec. 4: 0.8) */
  int nu_pre, nu_post; /* V-cycle smoothing steps */
  int quad_depth;      /* cut-cell quadtree/octree depth k */
  fc_cache cache;
  fc_prec prec;
  int fgmres_restart;  /* FGMRES(m) restart length (default 30) */
  int bc_preset;       /* 0: channel (inflow x=lo, walls y(,z)), 1: porous (walls y(,z)), 2: none */
  double ubar;         /* mean inflow speed of the channel preset (eq. cf_inflow) */
  int force_kind;      /* 0: constant force[]; 1: (f0 sin(pi x), f1 cos(pi y));
                          2: (f0 sin(pi y)[sin(pi z)], 0, 0); 3: (-f0 pi/2 sin(pi x/2), 0, 0) */
  double force[3];
  int dedup;           /* 1: patches with bit-identical blocks L_i (uncut, one alpha, away
                          from constraints) share one stored row/factor block; 0: one block
                          per patch (the paper's layout).  Same results either way. */
  int tc;              /* float32 / bfloat16 rows with dedup 1: how the V-cycle applies the
                          shared class blocks.  0: CUDA cores (float32 FMA); 1: tensor cores,
                          rows and residual rounded to TF32; 2: tensor cores, rows and residual
                          each split into two TF32 terms (three products, float32-class
                          accuracy); 3: tensor cores, rows and residual in BF16.  FP32
                          accumulation in every mode; cut patches (own blocks) always take
                          the CUDA cores.  Ignored for FP64 / float-pair rows. */
  double badcut_frac;  /* float32 / bfloat16 rows: a patch whose smallest cut-cell fluid
                          fraction over the 4^d cells its velocity nodes touch is below
                          badcut_frac gets its rows from the float-pair (FP64-class)
                          factorisation instead of float32 factors with refinement; 0 off.
                          In 3D (Q1-Q1) every patch's rows are factored in FP64 (banded
                          LDL^T, rounded for storage), so the rule only counts its patches
                          (fc_info). */
  int element;         /* 0: equal-order Q1-Q1 with the local L2 pressure projection (the
                          paper's pair, Sec. 2); 1: Q2-Q1 Taylor-Hood (cache_inverse, FP64
                          rows; 2D and 3D): Q2 velocities on the half-spaced grid of 2 n_k + 1 nodes per
                          direction, no stabilisation; patch of pressure vertex a = the Q2
                          nodes 2a-4 .. 2a+4 and the pressures a-1 .. a+1; each Q2 node is
                          written by the vertex at the lower corner of its cell, edge or face
                          (the paper's restricted write R~_i, Sec. 3.1, with an explicit owner
                          for the nodes away from the vertices).  Vectors: the velocity block
                          (Q2 node, x fastest, d components inner), then the vertex pressures. */
  int galerkin;        /* coarser-grid operators (Q1-Q1): 0 rediscretised on each grid of the
                          hierarchy with the same geometry and data (the paper's hierarchy of
                          coarser discretisations, Sec. 3); 1 Galerkin products R L P of the
                          next finer operator with the V-cycle's transfers (no quadrature on
                          the coarser grids; constrained coarse DoFs keep identity rows). */
  int amr_uniform;     /* -1: uniform grids (fc_grid.n cells on the finest level).  >= 0: adaptive
                          space-tree grids, quadtrees in 2D and octrees in 3D (Sec. 3; Q1-Q1,
                          cache_inverse, FP64 rows): fc_grid.n is the lattice of the finest
                          level's cells, the root grid is fc_grid.n / 2^(depth-1); every cell
                          is refined uniformly to level amr_uniform, a cell whose level set
                          changes sign among its 3^d sample points to level depth-1, and the
                          tree is 2:1 balanced across faces, edges and corners; a hanging
                          node is constrained to the mean of the end points of its edge or,
                          in 3D, of the four corners of its face; the coarser grids follow
                          Algorithm 1.  Vectors: the free nodes in lattice order (x fastest,
                          then y, then z), the velocity components and then p per node. */
} fc_options;

/* Fill the defaults:
 *   eta 1e-3, nitsche_beta 100, omega 0.8 (Sec. 4), nu_pre = nu_post = 2;
 *   quad_depth 4 (the 2D configurations; 3D problems use 3, set it);
 *   cache FC_CACHE_INVERSE, prec FC_PREC_FP64, fgmres_restart 30;
 *   bc_preset 0 (channel), ubar 0.3, force_kind 0 with force = 0;
 *   dedup 1 (shared class blocks; the Python binding's default too);
 *   tc 0 (CUDA cores), badcut_frac 1e-3, element 0 (Q1-Q1), galerkin 0
 *   (rediscretised coarser grids), amr_uniform -1 (uniform grids). */
fc_status fc_options_default(fc_options* o);

/* Build the hierarchy of `depth` levels (paper Sec. 3, Algorithm 1 on a
 * uniform grid: each coarser level halves n), discretise every level on the
 * GPU (cut-cell quadrature, element matrices, operator), build the patch
 * cache of every level above the coarsest (Sec. 3.1.2) and the dense coarse
 * solve (Sec. 3).  n must be divisible by 2^(depth-1).  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream).  Synchronises.
 * Errors: FC_ERR_INVALID (arguments), FC_ERR_OOM, FC_ERR_CUDA,
 * FC_ERR_SINGULAR (a local or coarse block could not be factored). */
fc_status fc_setup(fc_handle* h, const fc_grid* g, const fc_levelset* ls, double alpha, int depth,
                   const fc_options* o, void* cuda_stream);

/* b_dev <- right-hand side of the finest level: the load f(v) and the
 * lifted strong Dirichlet data (eq. stokes_disc_weak_fcm_2), b = w on
 * constrained DoFs.  b_dev holds ndof(L) doubles. */
fc_status fc_rhs(fc_handle h, double* b_dev);

/* r_dev <- b_dev - L x_dev on `level` (FP64).  Constrained DoFs have
 * identity rows. */
fc_status fc_residual(fc_handle h, int level, const double* x_dev, const double* b_dev,
                      double* r_dev);

/* y_dev <- L x_dev on `level` (FP64). */
fc_status fc_apply(fc_handle h, int level, const double* x_dev, double* y_dev);

/* `nsweeps` RA smoother sweeps on `level` (eq. iteration with eq. smoother):
 * r = b - L x over all DoFs, then for every pressure node i,
 * x[owned DoFs of node i] += omega (L_i^{-1} R_i r)[owned]; constrained DoFs
 * take b.  Uses the handle's cache policy and precision.  level >= 2
 * (the coarsest level has no patch cache; use fc_coarse_solve). */
fc_status fc_smooth(fc_handle h, int level, double* x_dev, const double* b_dev, int nsweeps);

/* As fc_smooth, but allocates nothing: the padded residual it needs lives in
 * one file-scope static device array of 16 MiB (held on every GPU that loads
 * the library until exit) instead of in handle memory.  The paper has no
 * counterpart; this is for callers that cannot allocate at call time, such
 * as a serving runtime that reserved its device memory up front, or a loop
 * that must not enter the CUDA allocator (cudaMalloc/cudaFree can
 * synchronise the device).  The caller passes x (in/out) and b as for
 * fc_smooth; the handle's operator and patch cache are used read-only.
 * The first call on a device looks up the array's address
 * (cudaGetSymbolAddress, with that device current); make that call before
 * any stream capture.  All calls share the array and it keeps the last
 * call's contents: each call clears the part it uses first.  Calls whose
 * work overlaps on the GPU race on the array.  Errors: FC_ERR_INVALID when
 * the level's padded residual exceeds 16 MiB (3D up to 64^3 cells, 2D up to
 * about 700^2 in float64) or when the current device is not the one that
 * was current at fc_setup (the array is looked up on the current device),
 * FC_ERR_CUDA. */
fc_status fc_smooth_noalloc(fc_handle h, int level, double* x_dev, const double* b_dev, int nsweeps);

/* b_coarse <- R r_fine from `level` to `level-1` (eq. restriction_op with the
 * transfer T the identity on one GPU; R = P^T, Q1 full weighting on every
 * component); constrained coarse DoFs are set to zero. */
fc_status fc_restrict(fc_handle h, int level, const double* r_fine, double* b_coarse);

/* x_fine += P e_coarse from `level-1` to `level` (P = Q1 interpolation);
 * constrained fine DoFs are left unchanged. */
fc_status fc_prolong_add(fc_handle h, int level, const double* e_coarse, double* x_fine);

/* x_dev <- L_1^{-1} b_dev on the coarsest level (direct solve, Sec. 3). */
fc_status fc_coarse_solve(fc_handle h, const double* b_dev, double* x_dev);

/* One V(nu_pre, nu_post) cycle on the finest level: x_dev is updated in
 * place (coarse levels start from zero). */
fc_status fc_vcycle(fc_handle h, double* x_dev, const double* b_dev);

/* FGMRES(restart), right-preconditioned with one V-cycle, FP64 outer
 * iteration (Sec. 4 remark on Krylov methods).  x_dev holds x0 on entry and
 * the solution on exit.  Stops when ||b - L x||_2 <= rtol ||b||_2 (checked
 * on the true residual) or after maxit preconditioner applications.
 * *iters = preconditioner applications, *relres = true relative residual.
 * Synchronises.  Returns FC_ERR_NOT_CONVERGED if rtol was not reached. */
fc_status fc_solve(fc_handle h, const double* b_dev, double* x_dev, double rtol, int maxit,
                   int* iters, double* relres);

/* Standalone geometric multigrid (the setting of the paper's experiments,
 * Sec. 4): V(nu_pre, nu_post) cycles on x_dev until ||b - L x||_2 <=
 * reduction * ||b - L x0||_2 or maxit cycles.  *iters = cycles,
 * *relred = achieved reduction.  Synchronises once per cycle.  Returns
 * FC_ERR_NOT_CONVERGED if the reduction was not reached. */
fc_status fc_gmg_solve(fc_handle h, const double* b_dev, double* x_dev, double reduction, int maxit,
                       int* iters, double* relred);

/* As fc_solve, with HOST buffers (pinned memory recommended): copies b to
 * the device, solves from x0 = x_host, copies x back.  Synchronises. */
fc_status fc_solve_host(fc_handle h, const double* b_host, double* x_host, double rtol, int maxit,
                        int* iters, double* relres);

/* Sizes of `level`: DoFs, patches (= pressure nodes) and device bytes by
 * part: [0] operator, [1] patch cache, [2] vectors/workspace, [3] coarse
 * solve, [4] setup temporaries peak; [5] is a count, not bytes: patches (all
 * levels) whose float32 factorisation with iterative refinement did not
 * converge and that were rebuilt by float-pair elimination (2D float32 /
 * bfloat16 rows), or, in 3D (FP64, float32 and bfloat16 rows, all factored
 * in FP64), whose equilibrated velocity block was not positive definite for
 * the banded LDL^T factorisation and that were built by the pivoted dense
 * LU; [6] is a count too: the algorithmic floating-point
 * operations of one patch apply on `level` with cached rows, 2 x (active
 * patch DoFs x free owned DoFs) summed over the patches (0 on level 1);
 * [7] is a count: patches (all levels) that the bad-cut rule selects
 * (fc_options.badcut_frac; float32 / bfloat16 rows only); in 2D their rows
 * came from the float-pair factorisation, in 3D from the FP64 one that
 * every patch takes.  Any pointer may be NULL. */
fc_status fc_info(fc_handle h, int level, long long* ndof, long long* npatch,
                  size_t* bytes_by_part);

/* Copy the cached rows of patch `node` on `level` to host memory (cache
 * inverse only): rows[(d+1)][nslot] in float64 whatever the storage
 * precision, nslot = 5^d d + 3^d; slot order: velocity nodes of the 5^d box
 * around the node (x fastest) with the component inner, then the pressure
 * nodes of the 3^d box; absent DoFs have zero coefficients.  Q2-Q1:
 * rows[9][171] (2D) or rows[25][2214] (3D), row d (sx + 2 sy + 4 sz) + c for
 * the owned Q2 nodes 2a + s and the last row for the pressure; slots: the
 * Q2 nodes 2a-4 .. 2a+4 (x fastest, component inner), then the vertices
 * a-1 .. a+1.  Synchronises. */
fc_status fc_patch_rows(fc_handle h, int level, long long node, double* rows_host);

/* Adaptive grids (fc_options.amr_uniform >= 0): the DoFs of the patch of
 * free node `node` on `level` (velocity DoFs of the connected nodes in
 * ascending order, then the pressures; at most 2048), at most `capacity` of
 * them, into dofs_host, and their count into *n; fc_patch_rows then gives
 * rows[d+1][n] (the velocity components and p of the node; zero rows for
 * constrained velocity DoFs) in the same order.  FC_ERR_INVALID on uniform
 * grids or a short buffer.  Synchronises. */
fc_status fc_patch_dofs(fc_handle h, int level, long long node, long long* dofs_host, int capacity, int* n);

/* Upper bound of the device bytes a handle for this problem holds at the
 * peak of fc_setup: everything it keeps, plus the largest setup temporary
 * (element matrices of a level, or the float64 build of reduced-precision
 * rows, which coexists with the converted rows), assuming that no two patches
 * share a stored block (dedup = 1 can only lower the real use) and, for the
 * 3D cache_matrix policy, that at most 1 % of the patches need dense factor
 * records (their velocity block not positive definite; 0.19 % of the 64^3
 * porous hierarchy), plus 2 % and 8 MiB for small buffers and allocator
 * rounding.  Pure host arithmetic; 0 for invalid arguments. */
size_t fc_footprint_estimate(const fc_grid* g, int depth, const fc_options* o);

/* Per-kernel device time of the patch apply, the residual and the whole
 * sweep, collected with CUDA events on the handle's stream while enabled.
 * kind: 0 patch apply (all levels), 1 residual (smoother), 2 V-cycle,
 * 3 patch-cache build, 4 patch apply on the finest level only.
 * Reading synchronises and resets the counters of that kind. */
fc_status fc_profile_enable(fc_handle h, int on);
fc_status fc_profile_read(fc_handle h, int kind, long long* launches, double* total_ms,
                          double* bytes_per_launch);

/* Number of CUDA kernels libfc has launched in this process (all handles),
 * for launch accounting around timed regions. */
fc_status fc_launch_count(long long* count);

/* Arithmetic throughput of the current GPU, for the roofline of kernels
 * bound by a pipe rather than by memory (the paper has no counterpart; its
 * CPU runs need none).  precision 0: FP64 FMA, 1: FP32 FMA.  Runs
 * independent FMA chains on every SM for one timed launch (CUDA events,
 * after a warm-up launch) and stores FLOP/s (2 per FMA) in *flop_per_s and
 * the launch's duration in *launch_ms (may be NULL).  Allocates a few bytes
 * and a stream of its own; changes no device setting.  Synchronises.
 * Errors: FC_ERR_INVALID (NULL output, other precision), FC_ERR_CUDA. */
fc_status fc_probe_fma_rate(int precision, double* flop_per_s, double* launch_ms);

/* ---- Batches: many independent problems in one set of launches --------
 *
 * A batch groups handles made by fc_setup (same dimension; cache_inverse
 * with FC_PREC_FP64, FP32 or BF16 rows; equal nu_pre, nu_post and
 * fgmres_restart) and runs their smoother sweeps, V-cycles and FGMRES
 * solves together: each phase of the paper's V-cycle (Sec. 3: RA sweeps of
 * Sec. 3.1, transfers of eq. restriction_op, coarse direct solve) is one
 * persistent launch over the patches of every problem, with levels aligned
 * at the coarsest grid, and each Arnoldi step of the solve is one CUDA
 * graph.  The batch references the handles' device data: they must
 * outlive it and must not be used by other calls while a batch call runs.
 *
 * Vectors of a batch are PACKED: one device array of float64 holding every
 * problem's finest-level vector (node-interleaved as above) back to back,
 * problem p at [offsets[p], offsets[p+1]).  All calls are asynchronous on
 * the stream given to fc_batch_create unless they say they synchronise.
 * With the same patch-apply tile (see fc_batch_tile / fc_batch_set_tile)
 * a problem's result is bit-identical alone and in any batch; different
 * tiles change only the rounding order. */
typedef struct fc_batch_s* fc_batch;

/* Build a batch of nprob handles on cuda_stream (NULL = legacy default
 * stream).  Times every patch-apply tile candidate (lanes per patch
 * {1,2,4,8,16,32} x threads per CTA {128,256,512} x CTAs per SM
 * {2,4,8,16}, at most 2048 threads per SM and 256 patches per CTA pass) on
 * the batch's finest levels and keeps the fastest.  Synchronises.  Errors:
 * FC_ERR_INVALID (no handles, a NULL handle or one given twice, mixed
 * dimensions, policies, precisions or sweep counts; DF64 rows),
 * FC_ERR_CUDA.  On error *out is still set and must be passed to
 * fc_batch_destroy. */
fc_status fc_batch_create(fc_batch* out, const fc_handle* handles, int nprob, void* cuda_stream);

/* As fc_batch_create, with the patch-apply tile given instead of timed:
 * lanes per patch tpp in {1,2,4,8,16,32}, threads in {128,256,512} with
 * threads / tpp <= 256, CTAs per SM in 1..64.  A problem's result is then
 * bit-identical in every batch built with the same tile, whatever the other
 * members (serving loops build a batch per round of in-flight requests).
 * Errors: those of fc_batch_create; FC_ERR_INVALID for a tile outside
 * these sets (*out is then NULL). */
fc_status fc_batch_create_tiled(fc_batch* out, const fc_handle* handles, int nprob, void* cuda_stream, int tpp,
                                int threads, int ctas_per_sm);

/* offsets[0..nprob] (host) of the packed finest-level vectors. */
fc_status fc_batch_offsets(fc_batch b, long long* offsets);

/* Tile picked by the autotuner, or set by fc_batch_set_tile (tests and
 * sweeps): lanes per patch in {1,2,4,8,16,32}, threads per CTA in
 * {128,256,512} with threads / lanes <= 256, CTAs per SM in 1..64
 * (persistent grid size).  FC_ERR_INVALID otherwise. */
fc_status fc_batch_tile(fc_batch b, int* lanes_per_patch, int* threads, int* ctas_per_sm);
fc_status fc_batch_set_tile(fc_batch b, int lanes_per_patch, int threads, int ctas_per_sm);

/* nsweeps RA sweeps on every problem's finest level (packed x, b);
 * problems with a single level (no smoothed level) are left unchanged. */
fc_status fc_batch_smooth(fc_batch b, double* x_dev, const double* b_dev, int nsweeps);

/* One V(nu_pre, nu_post) cycle on every problem (packed x updated in place). */
fc_status fc_batch_vcycle(fc_batch b, double* x_dev, const double* b_dev);

/* FGMRES(restart) with one V-cycle as right preconditioner, per problem,
 * with each problem's own stopping test as in fc_solve; x_dev holds x0.
 * iters[p], relres[p] (host arrays of nprob, may be NULL) as in fc_solve.
 * Synchronises once per Arnoldi step.  Returns FC_ERR_NOT_CONVERGED if any
 * problem stopped above rtol. */
fc_status fc_batch_solve(fc_batch b, const double* b_dev, double* x_dev, double rtol, int maxit, int* iters,
                         double* relres);

/* As fc_batch_solve with packed HOST buffers (pinned memory recommended):
 * b and x0 are copied in on the caller's stream, x is copied back.
 * Synchronises. */
fc_status fc_batch_solve_host(fc_batch b, const double* b_host, double* x_host, double rtol, int maxit,
                              int* iters, double* relres);

/* Problems, total packed DoFs, patches on the finest levels (of problems
 * with more than one level), deepest hierarchy.  Any pointer may be NULL. */
fc_status fc_batch_info(fc_batch b, int* nprob, long long* ndof_total, long long* npatch_finest,
                        int* levels_max);
/* Per-launch device time of the finest-level smoothing in fc_batch_smooth
 * while enabled (CUDA events on the batch stream): kind 0 patch apply,
 * 1 residual; bytes_per_launch = algorithmic bytes of one apply (stored
 * rows once, residual gathered once, x read and written).  Reading
 * synchronises and resets that kind. */
fc_status fc_batch_profile_enable(fc_batch b, int on);
fc_status fc_batch_profile_read(fc_batch b, int kind, long long* launches, double* total_ms,
                                double* bytes_per_launch);
fc_status fc_batch_sync(fc_batch b);
const char* fc_batch_last_error(fc_batch b);
fc_status fc_batch_destroy(fc_batch b);

/* Wait for all work enqueued by the handle.  Errors: FC_ERR_INVALID (NULL
 * handle), FC_ERR_CUDA (the stream reported an error). */
fc_status fc_sync(fc_handle h);

/* Message of the handle's last error ("" if none).  The string belongs to
 * the handle and stays valid until the next call on it or fc_destroy; for a
 * NULL handle a static message is returned. */
const char* fc_last_error(fc_handle h);

/* Wait for the handle's stream, release every device and host buffer it
 * holds (including the CUDA graphs and the single-problem batch of the
 * float32 V-cycle) and free the handle.  Every handle that fc_setup stored
 * into *h, also one returned with an error status, is destroyed exactly
 * once.  FC_ERR_INVALID for NULL. */
fc_status fc_destroy(fc_handle h);

#ifdef __cplusplus
}
#endif

#endif /* FC_H */
