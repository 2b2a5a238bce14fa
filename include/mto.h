/*
 * libmto -- matrix-free multigrid-preconditioned conjugate gradient (pCGMG)
 * for the multi-material plane-stress Q4 compliance problem of Luu & Banh,
 * "A novel preconditioned conjugate gradient multigrid method for
 * multi-material topology optimization" (arXiv 2301.07457).
 *
 * C ABI.  Plain pointers and sizes only.  Every array argument documents
 * whether it lives on the device ("_dev": memory of the context's CUDA
 * device) or on the host ("_host").  The caller owns every array it passes;
 * the library owns the context and everything the context allocates.
 *
 * Mesh conventions (the paper's Fig. 3 is missing; these are the library's):
 *   nelx x nely unit-square elements, element e = j*nelx + i;
 *   nodes (nelx+1) x (nely+1), node n = j*(nelx+1) + i (x fastest);
 *   DOF 2n is u_x, 2n+1 is u_y, so nodal vectors are [nely+1][nelx+1][2];
 *   design fractions are [n_phase][nely][nelx];
 *   element local nodes run counter-clockwise from the bottom-left.
 *
 * Alignment: nodal vectors on the device (f, u, v, y, r, z of the elasticity
 * calls) are read and written as (u_x, u_y) pairs and must be 16-byte aligned
 * (every cudaMalloc'd address is; an offset into one must be a whole number
 * of nodes); misaligned ones are rejected with MTO_ERR_ARG before any device
 * work.  Other device arrays need the natural alignment of their type.
 *
 * Errors: every call returns an mto_status; nothing is thrown across the ABI.
 * A CUDA failure inside a call returns MTO_ERR_CUDA and leaves the context
 * in a state where mto_destroy is still valid.
 *
 * Streams: the context runs its device work on a private stream that is
 * ordered after the caller's stream (given at creation) on entry to every
 * call, and before it on return.  mto_set_design, mto_solve, mto_run_host,
 * mto_run_host_wait and mto_last_stats synchronise (the solve polls its
 * convergence flag); mto_compliance_grad, mto_run_host_async and the
 * diagnostics only enqueue.
 *
 * Threads: a context is not thread-safe; use one context per host thread.
 *
 * Profiling: the public calls that do work open an NVTX range named after
 * the call (mto_set_design, mto_solve, ...).
 */
#ifndef MTO_H
#define MTO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mto_ctx mto_ctx; /* opaque; owned by the library */

typedef enum {
  MTO_OK = 0,
  MTO_ERR_ARG = 1,              /* invalid argument (null pointer, bad size, bad option) */
  MTO_ERR_UNSUPPORTED_MESH = 2, /* nelx or nely not divisible by 2^n_coarsen, coarsest grid too large,
                                   more than 2^30 elements */
  MTO_ERR_OOM = 3,              /* device allocation failed */
  MTO_ERR_CUDA = 4,             /* a CUDA call failed */
  MTO_ERR_NOT_CONVERGED = 5,    /* max_it reached; u holds the last iterate */
  MTO_ERR_BREAKDOWN = 6,        /* p.Kp <= 0, z.r <= 0 or a non-finite scalar in PCG */
  MTO_ERR_TIMEOUT = 7,          /* a bounded device wait gave up */
  MTO_ERR_STATE = 8             /* call out of order (e.g. solve before set_design) */
} mto_status;

/* Clamped edges (both displacement components fixed on every node of the edge). */
enum { MTO_EDGE_BOTTOM = 1, MTO_EDGE_LEFT = 2, MTO_EDGE_RIGHT = 4, MTO_EDGE_TOP = 8 };
/* Coarse operators: Galerkin P^T K P (exact), or rediscretised with the mean
 * of the four child moduli (Sec. 2.1: "obtained from discretization in the
 * mesh Omega_n"). */
enum { MTO_COARSE_GALERKIN = 0, MTO_COARSE_REDISCRETIZE = 1 };
/* FP64: every step in float64.  MIXED: V-cycle in float32 with bfloat16
 * fine moduli; outer CG vectors, K p, dot products, residual replacement and
 * the coarsest dense solve in float64. */
enum { MTO_PRECISION_FP64 = 0, MTO_PRECISION_MIXED = 1 };

typedef struct {
  double tol;       /* stop when ||f - K u||_2 <= tol * ||f||_2 (recursive residual; Alg. 2) */
  int max_it;       /* maximum PCG iterations */
  double omega;     /* damped-Jacobi weight (Sec. 2.3), 0 < omega <= 1 */
  int nu1, nu2;     /* pre- and post-smoothing sweeps of Alg. 1, each >= 1 */
  int n_coarsen;    /* number of coarsenings; the V-cycle has n_coarsen+1 grids */
  int coarse_kind;  /* MTO_COARSE_* */
  int precision;    /* MTO_PRECISION_* */
  int rr_every;     /* mixed path: replace r by f - K u every k iterations (0: never) */
  int flexible;     /* 1: flexible (Polak-Ribiere) beta, 0: Fletcher-Reeves as in Alg. 2 */
  int check_every;  /* host convergence poll interval in iterations (>= 1) */
  int gamma;        /* cycle index of Alg. 1 below the finest grid, 1..4 (1: V-cycle,
                       2: W-cycle); the finest grid calls the next one once.  At most
                       512 coarse-grid calls per cycle (MTO_ERR_ARG otherwise). */
  int concurrent_rhs; /* 1..4: right-hand sides of one mto_solve solved at the same time, each
                         with its own vectors, scalars, stream and solve graph (the design data
                         is shared); more than 1 costs one extra set of solve vectors per slot,
                         allocated on the first solve with that many right-hand sides.  The
                         results do not depend on it (bit for bit). */
} mto_solver_opts;

typedef struct {
  int iters;            /* PCG iterations performed (x updates) */
  int converged;        /* 1 if the stopping rule was met */
  double rel_res_rec;   /* recursive ||r|| / ||f|| at exit */
  double rel_res_true;  /* true ||f - K u|| / ||f|| at exit, float64 operator */
  double ms_setup;      /* device time of the last mto_set_design (ms) */
  double ms_solve;      /* device time of this mto_solve (ms), all right-hand sides */
} mto_solve_stats;

/* Fills the defaults: tol 1e-8, max_it 500, omega 0.6, nu1 = nu2 = 2,
 * n_coarsen 3, Galerkin, FP64, rr_every 25, flexible 0, check_every 4, gamma 1,
 * concurrent_rhs 2. */
void mto_default_opts(mto_solver_opts* opts);

/* Creates a context for an nelx x nely mesh with Poisson ratio nu and the
 * given clamped edges (at least one, so that K_ff is positive definite).
 * Allocates every device buffer of the level hierarchy (sizes depend only on
 * the mesh and the options).  Meshes of more than 2^30 elements are
 * rejected with MTO_ERR_UNSUPPORTED_MESH before any allocation.  device: CUDA ordinal; cuda_stream: a
 * cudaStream_t (NULL = legacy default stream).
 * Paper: Eq. 6-10 (problem statement), Alg. 1 (grid hierarchy). */
mto_status mto_create_mesh(mto_ctx** out, int nelx, int nely, double nu, unsigned fixed_edges,
                           const mto_solver_opts* opts, int device, void* cuda_stream);

/* Sets the design and builds every operator of the hierarchy on the device:
 * E_e = sum_i x_{e,i}^penal * E_phase[i] (Eq. 5), the fine Jacobi diagonal,
 * the coarse operators of every level and the coarsest dense inverse.
 * x_dev: device, float64 [n_phase][nely][nelx], finite values in [0, 1]
 * (not validated on the device).  E_phase: host, float64 [n_phase], > 0.
 * n_phase in [1, 16].  penal >= 1. */
mto_status mto_set_design(mto_ctx* ctx, int n_phase, const double* x_dev, const double* E_phase,
                          double penal);

/* Solves K u = f for n_rhs load cases by PCG (Alg. 2) preconditioned with one
 * V-cycle (Alg. 1).  f_dev: device, float64 [n_rhs][nely+1][nelx+1][2];
 * loads on clamped DOFs are ignored.  u_dev: device, same layout; in: the
 * warm start (zeros for a cold start), out: the solution, zero on clamped
 * DOFs.  stats: host, may be NULL.  Returns MTO_ERR_NOT_CONVERGED or
 * MTO_ERR_BREAKDOWN when a right-hand side failed (u then holds its last
 * iterate); stats describe the last right-hand side, with iters summed over
 * all of them. */
mto_status mto_solve(mto_ctx* ctx, int n_rhs, const double* f_dev, double* u_dev,
                     mto_solve_stats* stats);

/* Batched solves (independent problems of any mesh size in one CUDA graph).
 * One context per problem; the contexts must differ, live on one device and
 * not have kernel timing on.  Each item gives the problem's design and loads
 * (same layouts and meanings as mto_set_design / mto_solve /
 * mto_compliance_grad; E_phase is a host array, copied at creation; n_rhs <=
 * 64; compliance_dev may be NULL, then dcdx_dev must be NULL too).
 * mto_batch_create captures, per problem, set_design + one device-side PCG
 * loop per load case (cold start from u_dev as given) + compliance into one
 * branch of a graph; the device arrays named in the items are baked into it
 * and must stay valid.  mto_batch_run launches the graph once on the stream
 * given at creation (ordered after it, and it after the batch), waits for it
 * and fills stats (host [n], may be NULL: iterations summed over the
 * problem's load cases, residuals of its last one, ms_solve = device time of
 * the whole batch).  Returns the worst status over the problems.
 * mto_solve_batched is create + run + destroy in one call.  The paper solves
 * one system at a time; batching is this library's extension (Sec. 4: the
 * optimiser solves once per design update). */
typedef struct mto_batch mto_batch;
typedef struct {
  int n_phase;
  const double* x_dev;    /* device [n_phase][nely][nelx] */
  const double* E_phase;  /* host [n_phase] */
  double penal;
  int n_rhs;
  const double* f_dev;    /* device [n_rhs][nely+1][nelx+1][2] */
  double* u_dev;          /* device, same layout: warm start in, solution out */
  double* compliance_dev; /* device [n_rhs], may be NULL */
  double* dcdx_dev;       /* device [n_phase][nely][nelx], may be NULL */
} mto_batch_item;
mto_status mto_batch_create(mto_batch** out, int n, mto_ctx* const* ctxs, const mto_batch_item* items,
                            void* cuda_stream);
mto_status mto_batch_run(mto_batch* batch, mto_solve_stats* stats);
mto_status mto_batch_time(mto_batch* batch, double* ms_last_run);
/* Launch shapes for the batch as a whole: the problems run side by side, so
 * launches sized for one problem alone (one full wave of blocks per sweep)
 * hold SMs that the other problems' kernels could use.  Times the batch graph
 * with each context's own launch shapes and with one cap of 16, 8, 6, 4, 3
 * or 2 warps per SM on every sweep of every problem (two cold runs each, from
 * u = 0; the u_dev contents at the call are put back), recaptures the graph
 * with the fastest and reports its cap in *warps_per_sm (0: the contexts' own
 * shapes; may be NULL).  The contexts keep their own shapes for their own
 * solves.  The runs overwrite the items' compliance and dcdx arrays; results
 * with another shape differ from the untuned batch only in the order of the
 * reductions' partial sums.  On an error other than MTO_ERR_OOM the batch
 * must be destroyed.  Takes about 15 batch runs. */
mto_status mto_batch_tune(mto_batch* batch, int* warps_per_sm);
void mto_batch_destroy(mto_batch* batch);
mto_status mto_solve_batched(int n, mto_ctx* const* ctxs, const mto_batch_item* items,
                             mto_solve_stats* stats, void* cuda_stream);

/* Launch-shape tuner: for every level, times the marching sweep with several
 * numbers of warps per launch (hence rows per warp task) on the device and
 * keeps the fastest; results are cached for the process by (mesh size,
 * precision, operator kind, SM count).  Needs a design (mto_set_design) and
 * synchronises; later solves and batches use the chosen shapes.
 * mto_get_launch_shape returns the chosen warps per launch, or 0 for the
 * default: one full wave of the sweep kernel (its resident blocks per SM,
 * set by its register use, times the SM count); level -1 is the float64
 * outer sweeps. */
mto_status mto_autotune(mto_ctx* ctx);
mto_status mto_get_launch_shape(mto_ctx* ctx, int level, int* target_warps);
/* Sets the warps per launch of level's sweeps by hand (0: one full wave);
 * level -1 addresses the float64 outer sweeps of the finest level (K p and
 * the residuals), 0..n_coarsen the V-cycle sweeps.  target_warps <= 128 per
 * SM.  The solver's graphs are rebuilt on the next solve; results do not
 * depend on the shape beyond the order of the reductions' partial sums. */
mto_status mto_set_launch_shape(mto_ctx* ctx, int level, int target_warps);

/* Statistics of the last mto_solve (synchronises the context's stream). */
mto_status mto_last_stats(mto_ctx* ctx, mto_solve_stats* stats);

/* Compliance and sensitivities after a solve (Eq. 6; Sec. 4):
 * compliance_dev[k] = f_k . u_k (device, float64 [n_rhs]);
 * dcdx_dev[i][e] = sum_k -penal x_{e,i}^(penal-1) E_i u_{k,e}^T KE u_{k,e}
 * (device, float64 [n_phase][nely][nelx], may be NULL), using the design of
 * the last mto_set_design.  f_dev, u_dev as in mto_solve. */
mto_status mto_compliance_grad(mto_ctx* ctx, int n_rhs, const double* f_dev, const double* u_dev,
                               double* compliance_dev, double* dcdx_dev);

/* One call with host buffers: copies x and f to the device, runs
 * set_design + solve (cold start) + compliance/sensitivities, copies u, the
 * compliances and the sensitivities back.  x_host [n_phase][nely][nelx],
 * f_host/u_host [n_rhs][nely+1][nelx+1][2], compliance_host [n_rhs],
 * dcdx_host [n_phase][nely][nelx] (may be NULL).  Host arrays may be
 * pageable or pinned (pinned ones let the transfers overlap the kernels: x
 * arrives in row chunks whose moduli are formed while the next chunk is in
 * flight, f during set-up, u and dcdx while the sensitivities are formed);
 * the call synchronises.  stats->ms_setup includes the transfer of x. */
mto_status mto_run_host(mto_ctx* ctx, int n_phase, const double* x_host, const double* E_phase,
                        double penal, int n_rhs, const double* f_host, double* u_host,
                        double* compliance_host, double* dcdx_host, mto_solve_stats* stats);

/* The same call, pipelined: mto_run_host_async enqueues it and returns at
 * once; mto_run_host_wait blocks until the oldest outstanding call has
 * finished and its outputs are in the host arrays, and returns that call's
 * status and statistics (stats may be NULL).  Arguments, layouts and results
 * are those of mto_run_host, bit for bit.  At most two calls are outstanding:
 * while call k computes, call k+1's x and f travel to the device and call
 * k-1's u and sensitivities travel back, on their own streams.  For that
 * overlap the host arrays must be pinned (pageable ones work, but their
 * copies serialise with the host thread).  Every host array of a call belongs
 * to the library until the wait that returns that call: the caller neither
 * writes the inputs nor reads the outputs before then.  Errors: MTO_ERR_ARG
 * as mto_run_host; MTO_ERR_STATE for a third outstanding call, for an async
 * call while kernel timing is on, for a wait with nothing outstanding, and
 * for mto_run_host while pipelined calls are outstanding; MTO_ERR_BREAKDOWN
 * from the wait when the design's coarsest factorisation broke down.  Other
 * entry points may be called in between: their device work is ordered after
 * the outstanding calls' kernels.  mto_destroy waits for outstanding calls.
 * The paper has no counterpart: it serves optimisation loops that keep the
 * design on the host. */
mto_status mto_run_host_async(mto_ctx* ctx, int n_phase, const double* x_host, const double* E_phase,
                              double penal, int n_rhs, const double* f_host, double* u_host,
                              double* compliance_host, double* dcdx_host);
mto_status mto_run_host_wait(mto_ctx* ctx, mto_solve_stats* stats);

/* Diagnostics for per-kernel checks.
 * level: 0 = coarsest ... n_coarsen = finest (the numbering of Alg. 1).
 * Vectors are device float64 in the level's own layout [ny_l+1][nx_l+1][2]
 * with nx_l = nelx >> (n_coarsen - level).
 * mto_apply_operator: y = K_l v with v treated as zero on clamped DOFs and y
 * zero there; K_l is the operator the solver uses on that level in the
 * context's precision (float32 levels compute in float32; the finest level
 * of the mixed path offers both: use_vcycle_operator = 1 selects the
 * bfloat16/float32 smoother operator, 0 the float64 outer operator).
 * mto_apply_preconditioner: z = one V-cycle applied to r on the finest level
 * (Alg. 1 from U = 0, as inside PCG). */
mto_status mto_apply_operator(mto_ctx* ctx, int level, int use_vcycle_operator, const double* v_dev,
                              double* y_dev);
mto_status mto_apply_preconditioner(mto_ctx* ctx, const double* r_dev, double* z_dev);

/* Mesh and hierarchy facts: number of free DOFs of the coarsest grid, number
 * of levels, and the element moduli E (device float64 [nely][nelx]) of the
 * last set_design. */
mto_status mto_get_info(mto_ctx* ctx, int* n_levels, int* coarsest_free_dofs);
mto_status mto_get_moduli(mto_ctx* ctx, double* E_dev);

/* Compliance and sensitivities with no device allocation and no context.
 * The paper has no counterpart: this exists for callers that cannot allocate
 * device memory -- hosts whose memory pool owns the device's memory and
 * forbids other allocations, and
 * latency-critical loops that cannot take the device-wide synchronisation of
 * cudaMalloc/cudaFree.  Computes, for one load case on an nelx x nely mesh,
 * compliance_dev[0] = f . u and (if dcdx_dev != NULL) dcdx_dev[i][e] =
 * -penal x_{e,i}^(penal-1) E_phase[i] u_e^T KE u_e, the same values as
 * mto_compliance_grad (up to summation order for the compliance).
 * Arrays: f_dev, u_dev device float64 [nely+1][nelx+1][2]; x_dev device
 * float64 [n_phase][nely][nelx] (needed only with dcdx_dev); compliance_dev
 * device float64 [1]; dcdx_dev device float64 [n_phase][nely][nelx];
 * E_phase host [n_phase].  Work is enqueued on cuda_stream of `device`.
 * Scratch: a fixed 512 KiB device array inside the library, held on every GPU
 * that loads it until the process exits; meshes above 33,554,432 nodes are
 * rejected with MTO_ERR_UNSUPPORTED_MESH.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current.
 * Every call shares the
 * array and clears its counter at the start; calls whose work overlaps on the
 * GPU (other streams, other host threads) race and must be serialised by the
 * caller.  No cudaMalloc, cudaFree or allocating library routine is called. */
mto_status mto_compliance_grad_noalloc(int nelx, int nely, double nu, int n_phase,
                                       const double* x_dev, const double* E_phase, double penal,
                                       const double* f_dev, const double* u_dev,
                                       double* compliance_dev, double* dcdx_dev, int device,
                                       void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Scalar Poisson problem (Sec. 5.1, Table 1): -Laplace(u) = f on an
 * nelx x nely mesh of unit bilinear (Q4) elements, u = 0 on all four edges,
 * solved by the same pCGMG (Alg. 2 preconditioned by one V-cycle of Alg. 1,
 * damped Jacobi, bilinear transfers R = P^T, coarsest grid by a dense
 * inverse factored with Alg. 3).  One DOF per node; nodal vectors are
 * [nely+1][nelx+1] float64.  The constant-coefficient Q4 Laplacian is the
 * 9-point stencil (8 u_n - sum of the 8 neighbours) / 3 on every grid (its
 * Galerkin coarse operator is the same stencil).  Float64 throughout, or
 * a float32 V-cycle inside the float64 CG (precision MIXED).
 *
 * A solve is ONE kernel launch: each right-hand side is solved by one
 * thread-block cluster (cluster_ctas CTAs; 0 = chosen by mesh size, one CTA
 * up to 256 interior nodes, else about one per 256, at most 16) that runs the
 * whole PCG loop with
 * hardware cluster barriers; right-hand sides run as concurrent clusters.
 * --------------------------------------------------------------------------- */
typedef struct mto_poisson mto_poisson;
typedef struct {
  double tol;        /* stop when ||r||_2 <= tol ||f||_2 over the interior nodes */
  int max_it;        /* maximum PCG iterations */
  double omega;      /* damped-Jacobi weight, 0 < omega <= 1 */
  int nu1, nu2;      /* pre- and post-smoothing sweeps, 1..16 */
  int n_coarsen;     /* coarsenings (Sec. 5.1 coarsens down to a 2 x 2 grid) */
  int cluster_ctas;  /* 0 (automatic), 1, 2, 4, 8 or 16 CTAs per right-hand side; more than
                        one only when the finest grid has over 256 interior nodes, and at
                        most what the device can schedule */
  int precision;     /* MTO_PRECISION_FP64, or MTO_PRECISION_MIXED: the V-cycle (smoothing,
                        transfers, coarse grids) in float32, the CG vectors, K p, dot
                        products and the coarsest dense solve in float64, flexible beta */
} mto_poisson_opts;

/* Defaults: tol 1e-8, max_it 500, omega 0.6, nu1 = nu2 = 2, n_coarsen 3,
 * cluster_ctas 0, precision FP64. */
void mto_poisson_default_opts(mto_poisson_opts* opts);

/* Creates the solver for an nelx x nely mesh (both >= 2, divisible by
 * 2^n_coarsen; the coarsest grid needs at least one and at most 1,024
 * interior nodes, else MTO_ERR_UNSUPPORTED_MESH) and factors the coarsest
 * grid's matrix on the device (Alg. 3, band Cholesky, then K_0^-1).  device:
 * CUDA ordinal; cuda_stream: the caller's stream (work is ordered after it
 * on entry to every call and before it on return). */
mto_status mto_poisson_create(mto_poisson** out, int nelx, int nely, const mto_poisson_opts* opts,
                              int device, void* cuda_stream);

/* Solves K u = f for n_rhs (1..64) right-hand sides at once.
 * f_dev: device float64 [n_rhs][nely+1][nelx+1] (boundary values ignored).
 * u_dev: device, same layout: in, the warm start (zeros = cold start; its
 * boundary values are ignored); out, the solution, zero on the boundary.
 * stats: host, may be NULL (iterations summed over the right-hand sides,
 * residuals of the last one).  Synchronises.  Returns MTO_ERR_NOT_CONVERGED
 * or MTO_ERR_BREAKDOWN when a right-hand side failed (its u holds the last
 * iterate). */
mto_status mto_poisson_solve(mto_poisson* p, int n_rhs, const double* f_dev, double* u_dev,
                             mto_solve_stats* stats);

/* Diagnostics (enqueue only).  y = K v on the finest grid with v read as
 * zero on the boundary, y zero there; z = one V-cycle (Alg. 1 from U = 0)
 * applied to r.  Vectors: device float64 [nely+1][nelx+1]. */
mto_status mto_poisson_apply_operator(mto_poisson* p, const double* v_dev, double* y_dev);
mto_status mto_poisson_apply_preconditioner(mto_poisson* p, const double* r_dev, double* z_dev);

/* Number of grids, interior nodes of the coarsest grid, CTAs per cluster
 * in use, and kernels launched so far (any may be NULL). */
mto_status mto_poisson_get_info(mto_poisson* p, int* n_levels, int* coarsest_free, int* cluster_ctas,
                                long long* launches);
void mto_poisson_destroy(mto_poisson* p);

/* Measurement hooks.
 * mto_set_kernel_timing(ctx, 1) records CUDA events (on the context's stream,
 * inside the solver's CUDA graph) around two hot kernels of every PCG
 * iteration: [0] the finest-level outer sweep p = z + beta p, q = K p (float64)
 * and [1] the first finest-level damped-Jacobi sweep of the V-cycle (in the
 * V-cycle's precision).  mto_get_kernel_times returns their mean duration in
 * ms over the iterations sampled since timing was enabled (host arrays of 2).
 * mto_get_launch_count returns the number of kernels this context has
 * launched (each graph launch counts its kernel nodes).  Timing adds event
 * nodes to the graph; leave it off outside measurements. */
mto_status mto_set_kernel_timing(mto_ctx* ctx, int enable);
/* Measured issue rate of the float64 pipe on `device`: a kernel in which every
 * thread runs eight independent chains of dependent float64 fused
 * multiply-adds, eight 256-thread blocks per SM, timed with CUDA events on
 * cuda_stream (3 warm-up launches, best of 5; synchronises).  *ops_per_s =
 * FMA instructions per second, the unit in which the float64 sweeps' work is
 * counted (one add, multiply or FMA = one operation).  The paper has no
 * counterpart: it is the denominator of the float64 kernels' roofline. */
mto_status mto_measure_fp64_rate(int device, void* cuda_stream, double* ops_per_s);
mto_status mto_get_kernel_times(mto_ctx* ctx, double* ms_avg, long long* samples);
mto_status mto_get_launch_count(mto_ctx* ctx, long long* launches);

/* Device memory held by this library (contexts, their load-case workspaces,
 * batches, Poisson solvers) on all devices, in bytes, and an optional limit
 * on it (0 = none, the default).  An allocation that would pass the limit
 * fails as if the device were out of memory -- the call that needed it
 * returns MTO_ERR_OOM, or runs its load cases one after another when an extra
 * workspace does not fit -- without calling cudaMalloc.  For hosts that share
 * the GPU with other allocators, and to exercise the out-of-memory paths.
 * Thread-safe.  The paper has no counterpart. */
void mto_set_device_memory_limit(size_t bytes);
size_t mto_device_memory_in_use(void);

void mto_destroy(mto_ctx* ctx);
const char* mto_status_string(mto_status s);
/* Text of the CUDA error behind the last MTO_ERR_CUDA returned to this host
 * thread ("no error" if none). */
const char* mto_cuda_error_string(void);

#ifdef __cplusplus
}
#endif
#endif /* MTO_H */
