/*
 * helm.h -- C-ABI of libhelm.so: a GB300 (sm_103a) matrix-free solver for the complex
 * Helmholtz equation  (-Delta - k^2(x)) u = f  with exterior-complex-scaled absorbing layers,
 * preconditioned by a geometric multigrid cycle that approximately inverts a complex-scaled-
 * grid (CSG), complex-shifted-Laplacian (CSL), quadrant-definite (QD) or Laplacian operator,
 * inside flexible GMRES or Bi-CGSTAB.
 *
 * Method: H. bin Zubair, B. Reps, W. Vanroose, "A preconditioned iterative solver for the
 * scattering solutions of the Schroedinger equation" (arXiv 1012.4307):
 *   - model problem, eq. (2.1)-(2.2) with l1 = l2 = 0;
 *   - ECS contour (Section 3.1) and the three-point FD formula for unequal complex widths
 *     (Section 3.2);
 *   - preconditioning operators M_CSL, M_CSG, M_QD (Section 5, and eq. (4.1) for QD);
 *   - multigrid components and the cycle MG(l, A, b, u, nu1, nu2, C, gamma_f, gamma_c)
 *     (Section 4.2, Algorithm 1);
 *   - Bi-CGSTAB with one cycle per preconditioner call (Section 5) and (restarted) GMRES
 *     (Section 6).
 *
 * Conventions for every call:
 *   - Grid vectors are DEVICE pointers to n0*n1*n2 interleaved complex values (re, im), x
 *     fastest (index i + n0*(j + n1*k)), INCLUDING the Dirichlet boundary nodes.  The library
 *     never reads unknowns from, nor writes, the boundary nodes of caller vectors; callers keep
 *     them at zero.  HELM_C128 vectors are arrays of {double re, im} (16-byte aligned),
 *     HELM_C64 vectors arrays of {float re, im} (8-byte aligned).
 *   - The caller owns every vector it passes.  The library owns the workspace a handle
 *     allocates (levels, Krylov basis) from helm_create to helm_destroy.
 *   - All device work is ordered on the CUDA stream given at creation.  Calls that return
 *     statistics or a convergence decision synchronise that stream; helm_apply, mg_vcycle and
 *     helm_grad_k2 do not.
 *   - Every entry point returns a helm_status; nothing throws across the ABI.  On failure,
 *     helm_last_error() returns a message for the calling thread.  A CUDA error maps to
 *     HELM_ERR_CUDA; an argument error leaves all outputs untouched.
 *   - Handles are not thread-safe: one host thread at a time per handle.
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HELM_OK = 0,
    HELM_ERR_ARG = 1,        /* invalid argument (sizes, pointers, parameters)          */
    HELM_ERR_CUDA = 2,       /* a CUDA runtime call or kernel launch failed             */
    HELM_ERR_NOMEM = 3,      /* device or host allocation failed                        */
    HELM_ERR_NOCONV = 4,     /* iteration cap reached before the tolerance              */
    HELM_ERR_BREAKDOWN = 5,  /* Krylov breakdown (Bi-CGSTAB rho = 0, omega = 0, ...)    */
    HELM_ERR_NONFINITE = 6,  /* a residual norm became NaN or Inf                       */
    HELM_ERR_TIMEOUT = 7     /* reserved for a device-side wait that gives up; no entry */
                             /* point returns it: the library's kernels never spin-wait  */
                             /* (phases are ordered by the stream, thread-block clusters */
                             /* by hardware barriers, last-block reductions by atomics)  */
} helm_status;

typedef enum { HELM_C128 = 0, HELM_C64 = 1 } helm_prec;

/* Preconditioning operator inverted by the multigrid cycle (Section 5):
 *   CSG:     M = Z on the grid whose mesh widths are all multiplied by e^{i theta_a};
 *   CSL:     M = -Delta + (beta1 + i beta2) k^2;
 *   QD:      M = (1 - i) I + Z / |Re lambda0|   (eq. (4.1) in the table form of Section 5);
 *   LAPLACE: M = -Delta;
 *   NONE:    no preconditioner (Krylov solvers only).
 * Z = -Delta - k^2 is the Helmholtz operator of eq. (2.1), discretised on the ECS grid. */
typedef enum { HELM_PC_NONE = 0, HELM_PC_CSG = 1, HELM_PC_CSL = 2, HELM_PC_QD = 3, HELM_PC_LAPLACE = 4 } helm_pc_kind;

typedef enum { HELM_OP_A = 0, HELM_OP_M = 1 } helm_op;                   /* A = Z, M = preconditioner */
typedef enum { HELM_FGMRES = 0, HELM_BICGSTAB = 1 } helm_krylov;
typedef enum { HELM_SMOOTH_JACOBI = 0, HELM_SMOOTH_RB = 1 } helm_smoother;

/* Arithmetic of FGMRES's Arnoldi process (Gram-Schmidt inner products and updates, and the
 * product A z when the cycle is complex64).  Hessenberg matrix, Givens rotations, the true
 * residual and the solution update are IEEE FP64 either way.
 *   FP64: Krylov vectors stored as FP64; IEEE FP64 fused multiply-adds (bound by GB300's FP64
 *         units).
 *   DF:   Krylov vectors stored as float pairs (re.hi, re.lo, im.hi, im.lo) per node, 16 bytes
 *         like FP64, holding 47-48 significant bits; error-free products and sums on the FP32
 *         units (about 46 significant bits per product, 48 per sum); inner products rounded
 *         to FP64 once. */
/*   DCGS2: the DF arithmetic and storage with delayed classical Gram-Schmidt with
 *         reorthogonalisation (Swirydowicz et al. 2020): step j's single inner-product pass
 *         also reorthogonalises the vector of step j - 1, and one update pass finishes v_j and
 *         orthogonalises the new vector once; two passes over the basis per step instead of
 *         up to four.  The Hessenberg column of step j is completed, and its residual estimate
 *         known, one step later (the last column of a cycle by a closing inner product). */
typedef enum { HELM_GS_FP64 = 0, HELM_GS_DF = 1, HELM_GS_DCGS2 = 2 } helm_gs_arith;

/* Uniform real grid: n[a] nodes on [lo[a], hi[a]] per axis, boundary nodes included
 * (n - 2 unknowns per axis).  dim is 2 or 3; unused entries are ignored. */
typedef struct {
    int dim;
    int n[3];
    double lo[3], hi[3];
} helm_grid;

/* Multigrid cycle and preconditioner parameters (Section 4.2, Algorithm 1, Tables 1-4). */
typedef struct {
    helm_pc_kind kind;
    double theta_a;            /* CSG width rotation (e.g. pi/14)                     */
    double beta1, beta2;       /* CSL shift (e.g. -1, -0.5)                           */
    double re_lambda0;         /* QD: Re of the leftmost eigenvalue of Z (nonzero)    */
    int nu1, nu2;              /* pre- and post-smoothing steps (>= 0)                */
    double omega;              /* relaxation weight                                   */
    helm_smoother smoother;    /* omega-Jacobi or omega-red-black Jacobi              */
    int gamma_f, gamma_c;      /* cycle indices: (1,1) V, (1,2) F, (2,2) W            */
    int coarsest_n;            /* coarsen while some axis has more nodes than this    */
    helm_prec prec;            /* arithmetic of the cycle inside krylov_solve         */
    helm_gs_arith gs_arith;    /* arithmetic of FGMRES's Gram-Schmidt (FP64 vectors)  */
} helm_mg_params;

/* Solver statistics (host struct, filled by the solvers). */
typedef struct {
    int iterations;            /* Krylov iterations (FGMRES inner steps or Bi-CGSTAB steps) */
    int restarts;              /* FGMRES cycles started                                     */
    int status;                /* helm_status of the solve                                  */
    double rel_res;            /* final true ||f - A x||_2 / ||f||_2 in FP64                */
    double est_res;            /* last recursive / Arnoldi residual estimate (relative)     */
    double time_ms;            /* host wall time of the call                                */
    double *history;           /* optional caller array: estimate per iteration            */
    int history_len;           /* capacity of history (0 if none)                           */
    int reorthogonalizations;  /* FGMRES: Gram-Schmidt steps that needed a second pass      */
} helm_stats;

typedef struct helm_handle helm_handle;
typedef struct helm_batch helm_batch;

/* Creates a solver for Z = -Delta - k^2 on the ECS grid of Section 3.1 and the multigrid
 * hierarchy of its preconditioner (Section 4.2: rediscretisation on every coarse level, k^2
 * injected; coarsest level inverted exactly, Algorithm 1 step (0)).
 *   grid     host: geometry; every n[a] odd so that the levels nest.
 *   theta    ECS angle: beyond r0_hi[a] the contour is z = r0 + (x - r0) e^{i theta}, and the
 *            mirror image below r0_lo[a] (linear ECS, widths h e^{i theta}).  A side whose r0
 *            lies outside [lo, hi] has no layer (plain Dirichlet).
 *   r0_lo, r0_hi  host arrays of dim entries.
 *   k2       DEVICE pointer to n0*n1*n2 doubles (k^2 at the real nodes; boundary ignored).
 *            Copied; the caller may free it after the call returns.
 *   mg       host: preconditioner and cycle parameters.
 *   stream   cudaStream_t (NULL = legacy default stream) on which all work is ordered.
 *   out      receives the handle.
 * Errors: HELM_ERR_ARG (bad sizes/parameters, singular coarsest operator), HELM_ERR_NOMEM,
 * HELM_ERR_CUDA. */
helm_status helm_create(const helm_grid *grid, double theta, const double *r0_lo, const double *r0_hi,
                        const double *k2, const helm_mg_params *mg, void *stream, helm_handle **out);

void helm_destroy(helm_handle *h);

/* y = A x or y = M x on the finest grid (Section 3.2 stencil, the operators of Section 5):
 *   (M x)_p = a * sum_axes (cw x_{p-e} + cc x_p + ce x_{p+e}) + (bk k^2_p + c) x_p,
 * cw = -2/((h_{j-1}+h_j) h_{j-1}), ce = -2/((h_{j-1}+h_j) h_j), cc = -(cw + ce).
 * x, y: DEVICE vectors of precision prec; y's interior is overwritten, its boundary untouched.
 * x and y must not overlap. */
helm_status helm_apply(helm_handle *h, helm_op which, helm_prec prec, const void *x, void *y);

/* One multigrid cycle of Algorithm 1 for M x = b on the finest grid, with the handle's
 * (nu1, nu2, omega, smoother, gamma_f, gamma_c).
 *   b   DEVICE right-hand side (precision prec), unchanged.
 *   x   DEVICE initial guess on entry, cycle result on exit (precision prec).
 * b and x must not overlap. */
helm_status mg_vcycle(helm_handle *h, const void *b, void *x, helm_prec prec);

/* The preconditioner call of the outer solvers: z = one cycle of Algorithm 1 for M z = v from
 * a zero initial guess (Section 5, one cycle per preconditioner application).
 *   v   DEVICE complex128 vector (the outer solver's working precision), unchanged.
 *   z   DEVICE output of precision prec (HELM_C64: the cycle runs in complex64 on a copy of v
 *       rounded to complex64); its interior is overwritten, its boundary untouched.
 * v and z must not overlap.  Errors: HELM_ERR_ARG (null/misaligned pointers, a handle
 * without a hierarchy). */
helm_status mg_precondition(helm_handle *h, const void *v, void *z, helm_prec prec);

/* Solves A x = rhs (A = Z, FP64) to ||rhs - A x|| <= tol ||rhs||, right-preconditioned by one
 * multigrid cycle on M in the precision mg->prec (a complex64 cycle inside FP64 FGMRES, or all
 * FP64).  FGMRES(restart) (Saad's flexible GMRES; classical Gram-Schmidt with a second pass
 * whenever the first removed more than 1 - 1/sqrt(2) of the vector's norm (DGKS test);
 * complex Givens rotations; all in FP64 on the device) or Bi-CGSTAB with two cycles per
 * iteration (Section 5).
 *   rhs   DEVICE c128, unchanged.       x  DEVICE c128: initial guess in, solution out.
 *   tol   relative tolerance (> 0).     restart  FGMRES basis size (1..64; ignored by Bi-CGSTAB).
 *   maxit total iteration cap (> 0).    stats    optional host struct.
 * Returns HELM_OK when converged (confirmed by the FP64 true residual), HELM_ERR_NOCONV at the
 * cap, HELM_ERR_BREAKDOWN, HELM_ERR_NONFINITE; x holds the last iterate in every case. */
helm_status krylov_solve(helm_handle *h, helm_krylov method, const void *rhs, void *x, double tol,
                         int restart, int maxit, helm_stats *stats);

/* Adjoint solve A^T lambda = rhs (plain transpose).  The ECS FD matrix satisfies
 * (W A)^T = W A with W = prod_axes (h_{j-1} + h_j)/2 (complex dual volumes), so
 * lambda = W * A^{-1} (W^{-1} rhs) reuses the forward operator and its preconditioner.
 *   rhs DEVICE c128 (unchanged), lambda DEVICE c128 (initial guess ignored; overwritten). */
helm_status helm_solve_adjoint(helm_handle *h, const void *rhs, void *lambda, double tol, int restart,
                               int maxit, helm_stats *stats);

/* grad_p = Re(lambda_p * u_p) on interior nodes (0 on the boundary): the derivative of a real
 * loss L(u) with respect to k^2_p when A u = f and A^T lambda = conj(dL/du) (conjugate
 * Wirtinger convention), since dA/dk^2_p = -e_p e_p^T.
 *   lambda, u DEVICE c128; grad DEVICE double[n0*n1*n2]. */
helm_status helm_grad_k2(helm_handle *h, const void *lambda, const void *u, double *grad);

/* Reverse-mode step of u = A(k^2)^{-1} f for a real loss L(u) (the adjoint method; the paper
 * solves only forward problems, so this follows from eq. (2.1) with the ECS FD matrix of
 * Section 3.2): given grad_u = dL/d(conj u) as reverse-mode complex autodiff hands it (PyTorch's
 * convention), solves A^T lambda = conj(grad_u) by the weighted identity of
 * helm_solve_adjoint (FGMRES with the handle's preconditioner), then writes
 *   grad_k2[p] = Re(lambda_p u_p)   (dL/dk^2_p, since dA/dk^2_p = -e_p e_p^T), and
 *   grad_f[p]  = conj(lambda_p)     (dL/d(conj f) in the same convention),
 * both 0 on the boundary nodes.  Every conjugation and product runs on the device.
 *   grad_u  DEVICE c128, unchanged.      u  DEVICE c128 (the forward solution; unused and may be
 *                                           null when grad_k2 is null).
 *   grad_k2 DEVICE double[n0*n1*n2] or null;  grad_f DEVICE c128 or null (not both null; neither
 *           may overlap grad_u or u).
 *   tol, restart, maxit, stats  as for krylov_solve (the adjoint solve).
 * Synchronises the handle's stream.  Returns the adjoint solve's status (the gradients are
 * written for HELM_OK and HELM_ERR_NOCONV); HELM_ERR_ARG for bad pointers. */
helm_status helm_backward(helm_handle *h, const void *grad_u, const void *u, double *grad_k2, void *grad_f,
                          double tol, int restart, int maxit, helm_stats *stats);

/* Stand-alone multigrid on M x = b from x = 0 (Section 5, "mg-conv"): repeats cycles until
 * ||b - M x|| <= tol ||b|| or maxcyc cycles; returns the cycle count and the geometric mean of
 * the residual reduction over the last five cycles.
 *   b DEVICE (precision prec), x DEVICE (precision prec, overwritten). */
helm_status helm_mg_conv(helm_handle *h, const void *b, void *x, helm_prec prec, double tol, int maxcyc,
                         int *ncycles, double *factor);

/* Allocation-free helm_mg_conv (the paper has no counterpart; this is a library facility).
 * helm_mg_conv allocates a work area with cudaMalloc the first time it runs on a handle.
 * Some callers cannot allow that at the point of the call: a service that sizes its device
 * memory once at start-up (a fixed pool, or memory promised to other tenants of the GPU) and
 * forbids any later growth, or a latency-bound loop that cannot afford the device-wide
 * synchronisation that cudaMalloc and cudaFree may cause.  This entry point computes exactly
 * what helm_mg_conv computes, with the same kernels, but takes its work vectors from one fixed
 * device array of HELM_NOALLOC_SCRATCH_BYTES that the library holds on every GPU that loads it
 * until the process exits; it calls no cudaMalloc, cudaFree, cudaMallocHost or other
 * allocating routine.
 *   - Limit: the grid's nodes n0*n1*n2 must satisfy 32 * nodes + a few KB <= 16 MiB, i.e.
 *     at most about 523,000 nodes (513 x 513 in 2D, 65 x 65 x 65 in 3D); larger grids are
 *     rejected with HELM_ERR_ARG and nothing runs.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it for the life of the
 *     process; make that first call before any stream capture begins.  After a
 *     cudaDeviceReset the kept address is stale, as every handle's memory is: create new
 *     handles and do not call this entry point again in that process.
 *   - Every call shares the one array and it keeps the previous call's contents (the entry
 *     point clears what must start at zero).  Calls that overlap on the GPU (different
 *     streams, threads or handles) race on it: serialise them.
 *   - Each cycle's residual norm is read back to the host (the stream is synchronised after
 *     every cycle), as in helm_mg_conv.
 * Arguments, results and errors are those of helm_mg_conv. */
#define HELM_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
helm_status helm_mg_conv_noalloc(helm_handle *h, const void *b, void *x, helm_prec prec, double tol, int maxcyc,
                                 int *ncycles, double *factor);

/* Re(lambda0) for the QD preconditioner (helm_mg_params.re_lambda0; Section 5: lambda0 is the
 * eigenvalue of Z = -Delta - k^2 with the smallest real part).  Host computation, no device
 * work and no handle.  The two modes are the closing remark of Section 6:
 *   HELM_LAMBDA0_AXES   the one-dimensional counterpart: for every axis a, the smallest real
 *                       part over the eigenvalues of the 1D operator -d^2/dz^2 - k2_axis[a] on
 *                       that axis's ECS contour (Sections 3.1-3.2, interior nodes, Dirichlet
 *                       ends), summed over the axes.  Exact for a separable field
 *                       k^2(x) = sum_a k2_axis[a](x_a), whose discrete Z is the Kronecker sum of
 *                       the 1D operators; otherwise an estimate from the profiles given.
 *                       Eigenvalues by a complex-symmetric tridiagonal QR iteration, O(n^2).
 *   HELM_LAMBDA0_MAX_K2 minus the largest k^2 of that separable field over the interior nodes
 *                       (the rough estimate for piecewise-constant wavenumbers).
 *   grid, theta, r0_lo, r0_hi  as for helm_create (the same ECS contour per axis).
 *   k2_axis     host: dim arrays of n[a] doubles (values at the real nodes; boundary entries are
 *               ignored).
 *   re_lambda0  host output.
 * Errors: HELM_ERR_ARG (null pointers, bad grid or mode), HELM_ERR_NONFINITE (non-finite k2),
 * HELM_ERR_NOCONV (the eigenvalue iteration did not converge). */
typedef enum { HELM_LAMBDA0_AXES = 0, HELM_LAMBDA0_MAX_K2 = 1 } helm_lambda0_mode;
helm_status helm_qd_lambda0(const helm_grid *grid, double theta, const double *r0_lo, const double *r0_hi,
                            const double *const *k2_axis, int mode, double *re_lambda0);

/* Number of levels and nodes per axis of level l (host query). */
helm_status helm_levels(const helm_handle *h, int *nlev);
helm_status helm_level_shape(const helm_handle *h, int level, int n[3]);

/* ---- batched solves: many independent problems (energies, right-hand sides, grid sizes) ----
 * The paper solves one problem at a time; batching is a library facility.
 * helm_create_batch builds one handle and one non-blocking CUDA stream per problem (all with
 * the same mg parameters).  helm_solve_batch solves every problem with FGMRES as krylov_solve
 * does, concurrently, with one of the engines below; the batch's work starts after, and is
 * joined back into, the stream given at creation.  Each problem's result equals that of
 * krylov_solve on its handle (with the handle's tuning).
 *   grids, theta, r0 (2*dim per problem: lo then hi), k2 (device pointers): arrays of nprob.
 *   rhs, x: arrays of nprob DEVICE c128 pointers.  stats: nprob host structs (optional).
 * Returns the worst status over the problems. */
/* Engines of helm_solve_batch.
 *   HELM_BATCH_LOCKSTEP  every problem advances its FGMRES steps in step with the others and every
 *                        phase of a step is ONE launch over all problems: a temporally blocked pre-
 *                        and post-smoothing launch per level shape above the coarse tail (covering
 *                        every problem with a level of that shape), one thread-block-cluster launch
 *                        for all problems' coarse tails, and one launch each for A z, the inner-
 *                        product pass, its reduction, the Givens rotations and the update pass; the
 *                        step is a replayed CUDA graph.  Requires 2D grids, a complex64 V(2,2)
 *                        omega-Jacobi cycle with the delayed-CGS2 Arnoldi (HELM_GS_DCGS2), a common
 *                        coarse tail (same coarsest levels), restart <= 63.  It installs on every
 *                        problem's handle the cycle tuning it runs (cluster tail depth, tiles), so
 *                        that krylov_solve on that handle gives the same result bit for bit.
 *   HELM_BATCH_STREAMS   one stream per problem, steps interleaved by one host thread.
 *   HELM_BATCH_AUTO      lockstep when the configuration allows it, else streams (default).
 * helm_batch_set_engine: HELM_ERR_ARG for an unknown engine.  A solve with HELM_BATCH_LOCKSTEP on
 * a batch it cannot run fails with HELM_ERR_ARG and the reason.  helm_batch_get_engine returns
 * the engine of the last solve (HELM_BATCH_AUTO before any). */
typedef enum { HELM_BATCH_AUTO = 0, HELM_BATCH_LOCKSTEP = 1, HELM_BATCH_STREAMS = 2 } helm_batch_engine;
helm_status helm_batch_set_engine(helm_batch *b, int engine);
helm_status helm_batch_get_engine(const helm_batch *b, int *last);

helm_status helm_create_batch(int nprob, const helm_grid *grids, const double *theta, const double *r0,
                              const double *const *k2, const helm_mg_params *mg, void *stream,
                              helm_batch **out);
helm_status helm_solve_batch(helm_batch *b, const void *const *rhs, void *const *x, double tol, int restart,
                             int maxit, helm_stats *stats);
void helm_destroy_batch(helm_batch *b);
/* The handle of problem i (owned by the batch, valid until helm_destroy_batch), e.g. for
 * helm_set_tuning or a single solve.  Errors: HELM_ERR_ARG (null pointers, i out of range). */
helm_status helm_batch_handle(helm_batch *b, int i, helm_handle **out);

/* ---- launch timing (diagnostics; no counterpart in the paper, which reports cputime only) ----
 * helm_profile(h, 1) resets and enables per-launch timing: every kernel launch of the handle's
 * drivers is bracketed by two CUDA events on the handle's stream and tagged with its class
 * and its algorithmic DRAM bytes and flops (each operand touched once).  helm_profile(h, 0)
 * disables it.  helm_profile_read synchronises the stream and returns, per class, the number
 * of launches, the summed event time (ms), and the summed algorithmic bytes and flops, and
 * (bytes_pass, may be null) the bytes of the same work counted pass by pass: every smoothing
 * sweep, residual and grid transfer as its own pass over its operands, as separate launches
 * would move them (larger than the algorithmic bytes only for the temporally blocked kernels,
 * which do several passes per launch); the host arrays hold ncls entries
 * (ncls <= HELM_K_NCLASS).  Timed launches run eagerly (no CUDA graphs, no side stream), one
 * event pair each, so their sum exceeds a graph-replayed solve's time; and every timed launch
 * does its full work (the FGMRES steps queued behind a converged one, which an untimed solve
 * skips on the device, run in full). */
typedef enum {
    HELM_K_APPLY = 0,         /* FP64 operator apply (A z, true residual)                */
    HELM_K_SMOOTH_FINE = 1,   /* smoothing sweeps on the finest level (blocked kernels:  */
                              /* with their residual, restriction and prolongation)      */
    HELM_K_SMOOTH_COARSE = 2, /* the same on the coarser levels                          */
    HELM_K_RESTRICT = 3,      /* residual + full-weighting restriction                   */
    HELM_K_PROLONG = 4,       /* bi/trilinear prolongation + correction                  */
    HELM_K_COARSE = 5,        /* exact coarsest solve                                    */
    HELM_K_MDOT = 6,          /* Gram-Schmidt pass 1: h = V^H w                          */
    HELM_K_UPDATE_MDOT = 7,   /* Gram-Schmidt pass 2: w -= V h, h' = V^H w               */
    HELM_K_UPDATE_NORM = 8,   /* Gram-Schmidt pass 3: w -= V h', ||w||                   */
    HELM_K_VECTOR = 9,        /* other vector kernels (reductions, scaling, casts, x += Z y) */
    HELM_K_SMALL = 10,        /* single-warp kernels (Givens, back substitution, scalars) */
    HELM_K_NCLASS = 11
} helm_kernel_class;

helm_status helm_profile(helm_handle *h, int enable);
helm_status helm_profile_read(helm_handle *h, int ncls, int *launches, double *ms, double *bytes, double *flops,
                              double *bytes_pass);

/* ---- cycle tuning (kernel choices; no counterpart in the paper) ----
 * The arithmetic of Algorithm 1 is fixed by helm_mg_params; these choices only pick which
 * kernels carry it out, and every choice gives the same cycle up to FP32 rounding order.
 *   tail_levels    the coarsest levels (>= 2, or 0 for none) fused into one single-block
 *                  shared-memory launch; -1 = as many as fit (at most 4 levels, each with at
 *                  most 4096 unknowns, all in 200 KB of shared memory).  Values above what
 *                  fits are clamped.
 *   level_tile[l]  level l (0 = finest) of a 2D complex64 V(2,2) omega-Jacobi cycle runs its
 *                  two pre-sweeps + residual + full weighting, and its prolongation + two
 *                  post-sweeps, as two temporally blocked launches with tile shape
 *                  HELM_TILE_* (coarse nodes per block, or the register wavefront), or as
 *                  separate sweep / residual /
 *                  transfer launches (HELM_TILE_NONE).  Ignored where it does not apply (other
 *                  smoothers, complex128 cycles, 3D, levels inside the tail, grids the tile
 *                  does not fit: those use the separate launches).
 * Default: tail_levels = -1, HELM_TILE_32x8 on every level, cluster_levels = 0 (16 blocks, cluster_halo 3). */
#define HELM_MAX_LEVELS 16
typedef enum {
    HELM_TILE_NONE = -1,
    HELM_TILE_32x8 = 0,
    HELM_TILE_16x16 = 1,
    HELM_TILE_16x8 = 2,
    HELM_TILE_64x4 = 3,
    HELM_TILE_WAVE = 4, /* register wavefront: one warp per strip of 13 coarse columns and 8 coarse
                           rows, the sweeps pipelined down the rows, no shared memory */
    HELM_TILE_8x8 = 5,  /* small tiles: more blocks and fewer passes per phase on the small levels */
    HELM_TILE_COUNT = 6
} helm_tile;
typedef struct {
    int tail_levels;
    int level_tile[HELM_MAX_LEVELS];
    int cluster_levels;  /* 2D complex64: the coarsest levels (>= 2, 0 = off) in one launch of a
                            thread-block cluster, every level in distributed shared memory;
                            takes precedence over tail_levels; clamped to what fits (200 KB per
                            block, at most 6 levels) */
    int cluster_ctas;    /* blocks (SMs) of that cluster: 8 or 16 */
    int cluster_halo;    /* rows each block of the cluster keeps beyond its slab of every level:
                            1 = one halo row, a cluster barrier after every sweep and transfer;
                            3 = three rows, recomputed locally, so that a level's way down and its
                            way up each need one barrier (V-cycles of omega-Jacobi with at most two
                            sweeps each way from a zero guess, where the levels fit; otherwise the
                            one-row form runs).  Same results either way. */
} helm_tuning;

/* Sets / reads the handle's tuning (host struct).  Setting drops the handle's captured CUDA
 * graphs (they are re-captured on next use) and, when the tuning selects a cluster tail not
 * used before on this handle, allocates that tail's initial shared-memory image (every
 * block's, at most 3.2 MB; freed by helm_destroy) and fills it with one kernel on the handle's
 * stream.  Errors: HELM_ERR_ARG (null pointers, a tile index out of range, tail_levels < -1 or
 * == 1, cluster_levels < 0 or == 1, cluster_ctas not 8 or 16). */
helm_status helm_set_tuning(helm_handle *h, const helm_tuning *t);
helm_status helm_get_tuning(const helm_handle *h, helm_tuning *t);

/* Autotuner: times reps preconditioner applications (one cycle from zero on a fixed seeded
 * complex128 vector, Section 5's preconditioner call) of precision prec for candidate
 * tunings with CUDA events on the handle's stream, greedily level by level from the finest
 * (each level's tile choice, then the tail depth), installs the fastest, and returns it in
 * *best and its time per application (ms) in *best_ms (may be null).  Allocates two
 * temporary vectors, and the cluster-tail images of the candidates it times (kept with the
 * handle, as helm_set_tuning does); synchronises the stream.  Errors: HELM_ERR_ARG (bad arguments, a handle
 * without a hierarchy), HELM_ERR_NOMEM, HELM_ERR_CUDA. */
helm_status helm_autotune(helm_handle *h, helm_prec prec, int reps, helm_tuning *best, double *best_ms);

/* Message describing the last failure on the calling thread ("" if none). */
const char *helm_last_error(void);

/* Library version string. */
const char *helm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HELM_H */
