/*
 * sulfmg.h -- C ABI of the GB300 (sm_103a) Newton-multigrid solver for the
 * marble-sulfation system of Coco, Semplice and Serra Capizzano,
 * "A level-set multigrid technique for nonlinear diffusion in the numerical
 * simulation of marble degradation under chemical pollutants" (arXiv:1902.07029).
 *
 * One handle = one domain: a level set sampled on the nodes of a uniform grid
 * over the box [lo,hi]^dim (dim = 2 or 3) with N intervals per axis (N+1 nodes,
 * h = (hi-lo)/N, Sec. 3.3).  The library keeps the state (s, c) of every active
 * node, the multigrid hierarchy and all work arrays resident in device memory
 * and advances the state by Crank-Nicolson steps (Sec. 3.1, Eq. discTime), each
 * solved by Newton-Raphson (Sec. 3.4) with a level-set multigrid inner solver
 * (Sec. 3.5).  Every stage runs in the library's own CUDA kernels.
 *
 * Conventions
 *   - Grid arrays are (N+1)^dim values, x fastest, then y, then z.
 *   - Node types: 0 inactive, 1 inside (phi < 0), 2 ghost (Eq. ghostdef).
 *   - Host pointers are caller-owned; the library copies what it needs and
 *     never keeps them.  Device memory is owned by the library.
 *   - Every int-returning call returns SULF_OK (0) or a negative error code and
 *     records a message readable with sulf_last_error() (per thread).
 *   - Calls on one handle must not overlap; different handles are independent.
 *   - Device work is issued on the handle's stream (sulf_set_stream).  Every
 *     call returns with the handle's device work complete (also on error), so
 *     a handle may move to another stream between calls without waiting.
 */
#ifndef SULFMG_H
#define SULFMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SULF_OK 0
#define SULF_EINVAL (-1)   /* bad argument or geometry (domain on the box edge, no inside node, N not coarsest*2^k) */
#define SULF_ENOMEM (-2)   /* device or host allocation failed */
#define SULF_ENOTCONV (-3) /* Newton did not reach its tolerance within max_newton iterations, or produced NaN */
#define SULF_EGEOM (-4)    /* a finest-level ghost has no usable boundary stencil (Sec. 3.3: h too coarse) */
#define SULF_EDEVICE (-5)  /* CUDA error (no device, launch failure, ...) */

typedef struct sulf_domain* sulf_handle;

/* Model parameters of Eq. maineq with porosity phi(c) = alpha c + beta (Sec. 2);
   the paper's values are Eq. dataeq: a = 1e4, d = 0.1, m_s = 64.06,
   m_c = 100.09, alpha = 0.01, beta = 0.1.  s_ext is the Dirichlet value s_b on
   the boundary; s0, c0 the uniform initial data (Eq. BCnumtests: 0, 10, 1). */
typedef struct {
    double a, d, m_s, m_c, alpha, beta;
    double s_ext;
    double s0, c0;
} sulf_model;

/* Solver controls.
   nu1, nu2      pre- and post-relaxation sweeps (Sec. 3.5)            default 2, 2
   cycle         1 = V-cycle, 2 = W-cycle, 3 = full multigrid (Sec. 3.5's
                 transfers: the right-hand side restricted to every level,
                 the coarsest level solved, each finer level started from the
                 interpolated coarse solution with one V-cycle) as the first
                 cycle of every linear solve, V-cycles after it   default 1
   max_newton    Newton iteration cap per step                         default 20
   max_cycles    multigrid cycle cap per linear solve                  default 30
   ghost_sweeps  passes of the ghost relaxation (Eq. RelGhost) per sweep default 4
   newton_tol    Newton stops when min(|F|_inf, |dW|_inf/|W|_inf) < tol (Sec. 3.4)  default 1e-10
   lin_rtol      cycles stop when |r|_inf <= lin_rtol |F|_inf           default 1e-10
   tau_s         ghost relaxation parameter, 0 < tau_s < 1 (Eq. CFLcond)  default 0.9
   precision     0 = FP64 throughout; 1 = FP32 multigrid cycles inside FP64
                 defect correction (Newton residual, boundary rows of F and
                 the convergence tests stay FP64)                        default 0
   smoother      0 = collective (2x2 block, Eq. matrixP) red-black Gauss-Seidel,
                 1 = pointwise (Eq. matrixPclassical) red-black,
                 2 = collective lexicographic Gauss-Seidel, the paper's
                 ordering (Sec. 3.5.1): the inside nodes are visited wavefront
                 by wavefront (i+j(+k) = const, increasing), which gives the
                 box-order sweep's values exactly; one CTA per sweep, for
                 comparison with the paper, not for speed           default 0
                 (fuse_below does not apply to W-cycles, full multigrid or
                 the lexicographic smoother: every level runs as separate
                 kernels)
   graphs        1 = each multigrid cycle is captured once as a CUDA graph and
                 replayed; 0 = kernels launched one by one               default 1
   fuse_below    the first level with at most this many active nodes and all
                 coarser ones run as one single-CTA kernel per V-cycle;
                 0 = every level as separate kernels (W-cycles always are);
                 -1 = automatic: 150 for FP64, 1000 for mixed precision
                 (the fused kernel runs on one SM)                       default -1
   pdl           1 = kernels of a step are launched as programmatic dependent
                 launches (each may be scheduled while its predecessor runs and
                 waits on the device for its completion); 0 = plain stream
                 order.  Results are the same either way.                default 1
   ghost_compose 1 = the ghost_sweeps passes of one sweep's ghost relaxation
                 are applied as one precomputed affine map per ghost (the
                 passes are affine in the ghosts' values before them, their
                 right-hand sides and the inside values; built per level for
                 tau_s, ghost_sweeps and the boundary condition, and only
                 where it stays within 24 (2-D) / 27 (3-D) entries per ghost
                 on average); 0 = pass by pass.  Equal up to rounding.  default 1
   relax_occupancy 1 = the FP64 inside relaxation loads its coefficients
                 after the dependent-launch wait instead of prefetching them
                 across it, and is compiled for six resident CTAs per SM
                 instead of four: more warps hide the load latency; no effect
                 in FP32.  Same results either way.                default 0
   relax_matrix_free 1 = the FP32 red-black collective relaxation of the
                 mixed form recomputes each node's stencil coefficients from
                 (s, c) instead of reading the stored ones (same expressions:
                 fewer bytes per update, more FP32 arithmetic); 2 = the same,
                 and on 3-D levels with at least 100000 inside nodes both
                 colours of a sweep run as one kernel temporally blocked in
                 shared memory (32 x 8 x 16-node tiles streamed along z, the
                 red ring around each tile recomputed; needs even nu1 and
                 nu2); 0 = stored coefficients.  No effect in FP64 or with
                 the pointwise or lexicographic smoother.            default 1 */
typedef struct {
    int nu1, nu2, cycle, max_newton, max_cycles, ghost_sweeps;
    double newton_tol, lin_rtol, tau_s;
    int precision, smoother, graphs, fuse_below, pdl, ghost_compose, relax_occupancy, relax_matrix_free;
} sulf_solver;

/* Counters and timings of the handle. */
typedef struct {
    double t;               /* current time */
    int newton_last;        /* Newton iterations of the last step */
    int cycles_last;        /* multigrid cycles of the last step */
    long long newton_total, cycles_total, steps_total;
    double last_rho;        /* last cycle's residual reduction factor */
    double last_fnorm;      /* |F|_inf after the last Newton iteration */
    long long kernel_launches; /* kernels this handle has launched */
    int levels;             /* multigrid levels */
    long long n_inside, n_ghost; /* finest-level inside and ghost nodes (Eq. ghostdef) */
    int ghost_rows[3];      /* finest-level ghost rows: quadratic, linear, identity */
    unsigned long long device_bytes; /* device memory the handle holds */
    int loop_graph;         /* 1: the last linear solve ran its cycles as one graph
                               launch (a conditional while node with the
                               convergence test on the device); 0: one launch and
                               host test per cycle (graphs off, profiling on, or the
                               runtime refused the conditional node) */
} sulf_stats;

/* Build a domain.  levelset: host array of (N+1)^dim node values of phi
   (Omega = {phi < 0}, Sec. 3.2), copied.  box: host array {lo, hi}; the grid is
   [lo,hi]^dim.  N: intervals per axis, N = coarsest_N * 2^k with k >= 0; the
   hierarchy has k+1 levels, coarsened by injection of phi (Sec. 3.5.3).
   coarsest_N >= 2 (the paper uses 8, Sec. 4).  Classifies inside and ghost
   nodes, builds each ghost's boundary row (normal by Eq. nij, closest point on
   Gamma by bisection, weights of Eq. JssD) on every level.  The state is set to
   the default model's initial data.  Errors: SULF_EINVAL, SULF_EGEOM,
   SULF_ENOMEM, SULF_EDEVICE; *out is NULL on error. */
int sulf_create_domain(const double* levelset, int dim, const double* box, int N, int coarsest_N,
                       sulf_handle* out);

/* Set the model (Eq. maineq, Sec. 2) and reset the state to the uniform initial
   data s = s0, c = c0 on every active node (ghosts included) at t = 0. */
int sulf_set_model(sulf_handle h, const sulf_model* m);

/* Set the solver controls; NULL restores the defaults.  SULF_EINVAL on values
   out of range (tau_s must satisfy 0 < tau_s < 1, Eq. CFLcond). */
int sulf_set_solver(sulf_handle h, const sulf_solver* s);

/* Issue all device work of the handle on this cudaStream_t (NULL: the library's
   own stream). */
int sulf_set_stream(sulf_handle h, void* stream);

/* Advance nsteps Crank-Nicolson steps of size dt (Sec. 3.1), each by Newton
   (Sec. 3.4) with multigrid linear solves (Sec. 3.5).  Blocks until done.
   SULF_ENOTCONV if a step does not converge (the state is then that of the
   failed iterate). */
int sulf_step(sulf_handle h, double dt, int nsteps);

/* Copy the state to caller-owned host arrays of (N+1)^dim entries; any pointer
   may be NULL.  Inactive nodes read s = c = 0, type = 0. */
int sulf_get_state(sulf_handle h, double* s, double* c, int8_t* type);

/* Same, into caller-owned device arrays (no host round trip; synchronises). */
int sulf_get_state_device(sulf_handle h, double* s_dev, double* c_dev);

/* Replace the state from host arrays of (N+1)^dim entries (values at inactive
   nodes are ignored) and set the time to t: checkpoint/resume. */
int sulf_set_state(sulf_handle h, const double* s, const double* c, double t);

/* Same, but only the values at inside nodes are read: the ghost values (on
   which the c equation is discretised, Eq. FDc) are extrapolated from them
   with second order, as the paper prescribes for non-uniform initial data
   (Sec. 3.3, by a PDE extrapolation): the normal derivative u_n = n . grad u
   is extended outward by 64 Jacobi steps of dq/dtau + n . grad q = 0, then u
   by 64 steps of du/dtau + n . grad u = u_n (upwind toward the inside,
   dtau = h/2, n the central-difference normal of the level set). */
int sulf_set_state_extrapolated(sulf_handle h, const double* s, const double* c, double t);

/* Same, from device arrays. */
int sulf_set_state_device(sulf_handle h, const double* s_dev, const double* c_dev, double t);

/* Level-set preprocessing (Sec. 2), run before sulf_create_domain; both take
   and return host arrays of (N+1)^dim values (x fastest) and use device
   memory only for the duration of the call.

   Reinitialization toward the signed distance: `steps` explicit Euler steps
   of d phi_d / d mu = sgn(phi)(1 - |grad phi_d|), phi_d = phi at mu = 0, with
   d mu = h / dim, the smoothed sign phi / sqrt(phi^2 + h^2) and Godunov's
   first-order upwind |grad phi_d| (a missing box-edge side counts as a zero
   difference).  Information travels about h / dim per step, so 2 N steps
   reach the whole box. */
int sulf_reinit_levelset(const double* phi_in, int dim, int N, double h, int steps, double* phi_out);

/* Provisional level set of a binary mask (a scanned shape, Sec. 2): -1 where
   mask != 0 (inside), +1 elsewhere, then `steps` explicit heat steps
   phi += (1 / (4 dim)) sum_q (phi_q - phi) over the axis neighbours in the
   box.  Follow with sulf_reinit_levelset for a distance-like level set. */
int sulf_levelset_from_mask(const uint8_t* mask, int dim, int N, int steps, double* phi_out);

/* Boundary condition for s (Sec. 3.6): 0 Dirichlet s = s_b at the boundary
   points (Eq. BCs, the default); 1 Neumann ds/dn = s_b there (Eq. BCsN), the
   normal being that of the interpolated level set at B (Eq. Neumanntilde).
   s_b is the model's s_ext, or the per-ghost values of
   sulf_set_ghost_values.  With Neumann rows the ghost relaxation parameter is
   tau_s * 2 sqrt(2) h / 3 in 2-D (Eq. CFLcondN; 4 h / (3 sqrt 3) in 3-D) on a
   level of spacing h.  Rebuilds the boundary rows of every level;
   SULF_EGEOM (and the previous rows kept) if a finest-level ghost has no
   usable row for the new condition. */
int sulf_set_bc(sulf_handle h, int type);

/* Source terms of the manufactured-solution accuracy tests (Sec. 4.1): f1 and
   f2 are added to the right-hand sides of Eq. maineq and averaged over the CN
   step, i.e. F^s_p -= (f1_old[p] + f1_new[p]) / 2 on inside nodes and
   F^c_p -= (f2_old[p] + f2_new[p]) / 2 on inside and ghost nodes.  Host
   arrays of (N+1)^dim values at t_n (old) and t_{n+1} (new), copied; they
   apply to every following step until changed.  All four NULL clears them;
   a partial set is SULF_EINVAL. */
int sulf_set_sources(sulf_handle h, const double* f1_old, const double* f1_new, const double* f2_old,
                     const double* f2_new);

/* Dirichlet values s_b at the ghosts' boundary points B (Eq. BCs), one per
   finest-level ghost in the order of sulf_dbg_level_ghosts (box order of the
   ghost nodes).  Copied; they apply to every following step until changed.
   NULL restores the model's constant s_ext. */
int sulf_set_ghost_values(sulf_handle h, const double* sb);

int sulf_get_stats(sulf_handle h, sulf_stats* out);

/* Kernel timing for measurement: the library brackets launches of the
   finest-level inside relaxation (the dominant kernel) with CUDA events on its
   stream, one bracket around the two back-to-back colour launches of a sweep
   (between them the second launch's fetch of fixed data overlaps the first,
   as in the untimed pipeline).  on = 0 off; 1 the first finest-level sweep of
   every cycle (a sample that keeps the event overhead small); 2 every
   finest-level sweep.  While on, the cycles run one graph launch each (event
   nodes cannot sit in the device-side cycle loop).  sulf_kernel_time returns
   the summed device time in ms and the number of launches inside the
   brackets since the last reset (synchronises). */
int sulf_set_profiling(sulf_handle h, int on);
int sulf_kernel_time(sulf_handle h, double* ms, long long* launches);

/* The Newton residual of sulf_step's Crank-Nicolson step on the finest level
   and its max-norm, computed on caller-owned DEVICE buffers without
   allocating any device memory.  The paper has no counterpart: this entry
   point is for callers that cannot allocate device memory when they need a
   residual -- an application whose own memory manager has already reserved
   the device memory it may use, or a time-critical loop that must not take
   the device-wide synchronisation of a cudaMalloc/cudaFree.
     W_dev, Wn_dev  interleaved (s, c) per node, 2*(N+1)^dim doubles: the
                    iterate and the state at t_n (values at inactive nodes are
                    not read); 16-byte aligned
     F_dev          output, same layout and alignment; written on active nodes
                    only
     fnorm_dev      output, one double (8-byte aligned): |F|_inf over the
                    active nodes
   It evaluates the model's equations with the constant s_ext and Dirichlet
   boundary rows: the optional inputs of sulf_set_sources and
   sulf_set_ghost_values are not applied.  SULF_EINVAL after sulf_set_bc(h, 1),
   for a misaligned pointer, or when the current device is not the one the
   handle was created on; no work is queued then.
   Work is queued on the handle's stream and the call returns without waiting.
   Scratch: a static array inside the library holding 65536 partial maxima
   (512 KiB), kept by every GPU that loads the library until the process exits;
   the call fails with SULF_EINVAL when the finest level has more than
   16,777,216 active nodes.  The first call on each handle looks up the
   array's device address (cudaGetSymbolAddress) with the handle's device
   current and keeps it in the handle; make that first call before any stream
   capture.  Every call shares the array, and each call overwrites the slots it
   uses before reading them (nothing has to start at zero); calls that overlap
   on the GPU -- on different streams at the same time -- race on it. */
int sulf_newton_residual_noalloc(sulf_handle h, double dt, const double* W_dev, const double* Wn_dev, double* F_dev,
                                 double* fnorm_dev);

/* Autotuning of the solver controls that change only speed, not results
   beyond rounding order: fuse_below (the fused coarse-level threshold; only
   for V-cycles with red-black sweeps), ghost_compose, pdl,
   relax_occupancy and relax_matrix_free.  Each candidate
   is timed on this handle's own problem -- the Newton system of a CN step of
   size dt from the current state -- as a linear solve of 6 cycles (built
   once, then timed); the fused-level thresholds {0, 60, 150, 400, 1000, 3000,
   10000} are tried first, then ghost_compose and pdl at the best one, then
   relax_occupancy (FP64) or relax_matrix_free (mixed precision).  The
   fastest candidate is written into the handle's solver controls (the state
   is unchanged).  With use_cache != 0 a result found earlier in this process
   for the same problem class (dim, N, coarsest N, precision, cycle, smoother,
   nu1, nu2, boundary condition) is applied without timing.  Blocks. */
typedef struct {
    int fuse_below, ghost_compose, pdl; /* the chosen controls */
    int relax_occupancy;                /* (timed in FP64 only) */
    int relax_matrix_free;              /* (timed in mixed precision only) */
    double ms_per_cycle;                /* their time per cycle */
    double ms_per_cycle_default;        /* the defaults' (fuse_below -1, ghost_compose 1, pdl 1) */
    int candidates;                     /* candidates timed */
    int cached;                         /* 1: taken from the process cache, nothing timed */
} sulf_tune_result;
int sulf_autotune(sulf_handle h, double dt, int use_cache, sulf_tune_result* out);

/* Release the handle and its device memory. */
void sulf_destroy(sulf_handle h);

/* ---- batching: many independent domains advanced together ----
   The handles stay owned by the caller (one batch per set of handles; do not
   use them elsewhere while sulf_batch_step runs).  nstreams host workers, each
   with its own CUDA stream, take the instances largest-work-first, so the GPU
   runs several instances' kernels at once.  Results are those of advancing
   each handle alone. */
typedef struct sulf_batch_s* sulf_batch;
int sulf_batch_create(const sulf_handle* handles, int n, int nstreams, sulf_batch* out);
/* advance instance i by nsteps[i] CN steps of size dt[i]; returns the first
   failing instance's error (all instances are attempted) */
int sulf_batch_step(sulf_batch b, const double* dt, const int* nsteps);
int sulf_batch_status(sulf_batch b, int* status); /* per-instance return codes of the last step */
/* Lock-step mode for the next sulf_batch_step calls: 0 off (the default);
   1 on, each class split into chunks of at most 32 instances; m >= 2 on,
   chunks of at most m instances (chunks run on the worker streams).  Instances that share dimension, N, number of
   levels, boundary condition and the solver controls that shape a cycle
   (precision, nu1, nu2, ghost_sweeps, tau_s, tolerances, iteration caps,
   pdl, in mixed precision whether relax_matrix_free is 0), and in the step
   call dt and nsteps, form one class, provided their solver uses V-cycles (cycle
   1), the red-black smoother (smoother 0) and the composed ghost relaxation,
   and no source term or time-dependent boundary value is set.  A chunk of two
   or more advances together: every phase of the multigrid cycle of Sec. 3.5
   (a colour of the relaxation of Sec. 3.5.1, the ghost relaxation, the
   residual, the band extension and restriction of Sec. 3.5.2, the
   prolongation of Sec. 3.5.3, the coarsest solve) is one launch over all the
   chunk's instances, and an instance stops cycling (or leaves the Newton loop of Sec.
   3.4) when its own test says so, so it runs the Newton iterations and cycles
   it runs alone.  In mixed precision relax_matrix_free 1 and 2 both select
   the matrix-free FP32 relaxation (no temporally blocked sweep), and the
   coarse levels from the first
   level that every instance's fuse_below threshold fuses run as one launch
   with one CTA per instance, so results agree with stepping each instance
   alone up to rounding.  Other instances run alone as in the default mode.  The
   chunk's batched launches are counted into its instances' launch counters
   in equal shares.  Returns SULF_EINVAL for a negative mode. */
int sulf_batch_set_lockstep(sulf_batch b, int mode);
/* sulf_autotune of every instance (dt[i] its step), through the process cache:
   one timing per problem class (dim, N, precision, ...), the others take the
   result; out (may be NULL) receives one result per instance */
int sulf_batch_autotune(sulf_batch b, const double* dt, sulf_tune_result* out);
void sulf_batch_destroy(sulf_batch b);             /* the handles return to their own streams */

/* ---- serving: continuous batching of time-stepping jobs under an HBM budget ---- */
typedef struct {
    const double* levelset; /* (N+1)^dim host values, copied at submission */
    int dim, N, coarsest_N;
    double box_lo, box_hi;
    sulf_model model;
    sulf_solver solver;
    double dt;
    int nsteps;
} sulf_job;

typedef struct {
    int status;               /* the job's return code */
    double latency_ms;        /* submission to result ready */
    double queue_ms, run_ms;  /* waiting for admission / running */
    unsigned long long estimate_bytes, device_bytes;
    long long newton, cycles;
} sulf_job_result;

typedef struct {
    long long completed, failed, queued, running, max_running;
    double p50_ms, p99_ms;    /* latency percentiles of the completed jobs */
    double jobs_per_s;        /* completed jobs per second since creation */
    unsigned long long budget_bytes, peak_reserved_bytes;
} sulf_server_stats;

/* Device memory a domain of this size will hold (an upper estimate used for
   admission); 0 on invalid arguments. */
unsigned long long sulf_estimate_device_bytes(int dim, int N, int coarsest_N, int precision);

typedef struct sulf_server_s* sulf_server;
/* nworkers host workers, each with its own CUDA stream, run admitted jobs.
   A job is admitted (first come first served among the jobs that fit) when its
   estimate fits in the budget left by the running jobs; its memory returns to
   the budget when it finishes. */
int sulf_server_create(unsigned long long budget_bytes, int nworkers, sulf_server* out);
/* queue a job (the level set is copied; returns at once); SULF_ENOMEM if the
   job's estimate exceeds the whole budget */
int sulf_server_submit(sulf_server s, const sulf_job* job, long long* job_id);
int sulf_server_poll(sulf_server s, long long job_id, int* done);
/* block until the job is done, copy its state ((N+1)^dim host values each, may
   be NULL) and result, and forget the job; returns the job's return code */
int sulf_server_wait(sulf_server s, long long job_id, double* s_out, double* c_out, sulf_job_result* res);
int sulf_server_get_stats(sulf_server s, sulf_server_stats* out);
/* finish the queued and running jobs, then release the server */
void sulf_server_destroy(sulf_server s);

/* Message of the calling thread's last error ("" if none). */
const char* sulf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SULFMG_H */
