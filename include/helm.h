/*
 * helm.h - C ABI of the GB300 recursive moving-PML sweeping preconditioner.
 *
 * Liu & Ying, "Recursive Sweeping Preconditioner for the 3D Helmholtz
 * Equation" (arXiv 1502.07266).  The library solves the PML-padded
 * 7-point discretisation of Section 2 (Eq. system),
 *     A u = f,
 * with GMRES right-preconditioned by the recursive sweep of Section 4
 * (Algorithm 5 setup, Algorithm 6 apply, each quasi-2D problem solved by
 * one inner sweep, Algorithm 4, over quasi-1D problems factored by a block
 * LDU along x1, run from both ends of x1 and meeting in the middle: the same
 * inverse with two independent elimination chains).
 *
 * Grid and layout.  n interior points per axis, b PML layers on every face,
 * N = n + 2b nodes per axis, h = 1/(n+1); node g sits at (g - b + 1) h and
 * zero Dirichlet walls sit at g = -1 and g = N.  A 3D field is N*N*N values
 * with x fastest: index = i + N*(j + N*k) (the paper's column-major order,
 * Section 3).  A batch of nrhs fields is [nrhs][N^3].  Complex arrays are
 * interleaved (re, im): "c64" is float pairs, "c128" double pairs.
 *
 * Pointers.  Every array argument is a DEVICE pointer owned by the caller,
 * unless stated; the library never frees caller memory.  `stream` is a
 * cudaStream_t (NULL = legacy default stream).  All work is enqueued on it;
 * calls that return results to host arrays synchronise it before returning.
 *
 * Errors.  Functions return HELM_OK (0) on success, a negative code on
 * error, or HELM_ENOCONV (positive) when GMRES stopped at maxit (outputs
 * are still written).  No exception or abort crosses the ABI.  A handle is
 * not thread-safe: serialise calls on one handle.
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HELM_OK        0
#define HELM_ENOCONV   1   /* GMRES hit maxit before tol (outputs written)      */
#define HELM_EINVAL   -1   /* bad argument (sizes, null pointer, c <= 0 ...)    */
#define HELM_ENOMEM   -2   /* device allocation failed                          */
#define HELM_ECUDA    -3   /* a CUDA runtime call or kernel launch failed        */
#define HELM_ETIMEOUT -4   /* a bounded device wait expired (error flag set)     */
#define HELM_ENOTSUP  -5   /* valid but unsupported here (block size > 64 ...)   */

/* Problems in one batch handle or batched launch. */
#define HELM_MAX_BATCH 8

/* Storage of the quasi-1D factors T_i = S_i^{-1} (the precision pattern).  The
 * setup computes every T_i in complex FP32 and runs its elimination chains on
 * those values; only the copy the sweep reads is stored in the chosen form.
 * The reduced forms keep one power-of-two scale 2^e per block, chosen so that
 * the largest scaled real or imaginary part lies in [2^14, 2^15), and the
 * sweep accumulates in FP32.  GMRES keeps its FP64 true residual, Arnoldi
 * coefficients and solution, so every form reaches the same tolerance; the
 * reduced forms change the preconditioner by about their rounding error. */
#define HELM_FP32        0  /* complex FP32 factors (8 bytes per entry)                 */
#define HELM_FP16        1  /* FP16 re/im, relative rounding 2^-11 (4 bytes per entry) */
#define HELM_SPLIT_FP16  2  /* FP16 hi + lo pairs per part, about 2^-22 (8 bytes)      */

typedef struct helm_ctx* helm_handle;

typedef struct {
    int    precision;    /* HELM_FP32 (default), HELM_FP16 or HELM_SPLIT_FP16       */
    int    b_aux;        /* auxiliary (moving) PML width; 0 = b  (Sec. 4.2, mod. 2) */
    int    restart;      /* GMRES restart length; 0 = 30                           */
    int    maxit;        /* GMRES iteration cap per RHS; 0 = 300                   */
    double pml_C;        /* the PML constant C of Section 2; 0 = 10                */
    int    rhs_per_cta;  /* right-hand sides per sweep cluster: 0 or 1 (one each);
                            larger values are reserved: helm_setup returns
                            HELM_ENOTSUP                                            */
    int    schedule;     /* sweep order: HELM_ONE_FRONT (Algorithms 4 and 6 as
                            printed, the default) or HELM_TWO_FRONT (Section 4.2's
                            third modification, in both loops as in Section 5:
                            fronts from both faces meeting in a centre block with
                            a moving PML on both sides; changes M; dense form
                            only, and needs n - 1 >= 2d)                          */
    int    apply_form;   /* how each quasi-1D solve is applied: HELM_CHAIN (the
                            default) or HELM_DENSE (see below)                      */
    int    debug_unmet_wait; /* test hook, 0 in normal use: 1 makes the first wait
                            of a HELM_DENSE apply wait for an arrival that never
                            comes, so that its bounded wait expires and the call
                            reports HELM_ETIMEOUT through helm_status           */
    long long wait_cycles; /* bound of every device-side wait of a HELM_DENSE
                            apply, in SM clock cycles; 0 = 4e9 (about 2 s)       */
    int    dense_clusters; /* HELM_DENSE: clusters of 8 CTAs in the apply launch;
                            0 = as many as the GPU holds at once (at most 16);
                            larger values are clamped to that                   */
    int    reserved_;    /* 0                                                     */
} helm_opts;

#define HELM_ONE_FRONT   0
#define HELM_TWO_FRONT   1

/* Apply forms.  Both apply the same preconditioner M of Algorithm 6 (equal up
 * to rounding); they differ in what the setup stores and how a quasi-1D solve
 * |T~_{M'}| of Algorithm 4 runs.
 *   HELM_CHAIN  stores the twisted block factors T_i (k x k per x-block) and
 *               runs each solve as N dependent block substitution steps, one
 *               right-hand side per two-CTA cluster.
 *   HELM_DENSE  stores, for every quasi-1D problem, the restricted operator
 *               R_out H~^{-1} R_in^T that Algorithm 4 applies (an alternative
 *               Section 6 points to: the quasi-1D solve as a whole rather than
 *               a sequential substitution), computed in the setup from the
 *               factors, which are then released; each solve is one complex
 *               matrix product over all right-hand sides.  Precision selects
 *               the stored form and the product:
 *                 HELM_FP32        complex FP32 operators, FP32 SIMT products;
 *                 HELM_SPLIT_FP16  FP16 hi + lo operators (one power-of-two scale
 *                                  per row), inputs split the same way, three
 *                                  tcgen05 tensor-core products with FP32
 *                                  accumulation (about 2^-22 relative);
 *                 HELM_FP16        FP16 hi operators, inputs hi + lo, two products.
 *               Storage is about (d (b+d) N)^2 complex entries per problem
 *               (about 151 GB at n = 127, b = 6, d = 1 in FP32 or split FP16).
 *               helm_apply_slab and helm_autotune return HELM_ENOTSUP. */
#define HELM_CHAIN       0
#define HELM_DENSE       1

/* Fill *opts with the defaults above. */
void helm_default_opts(helm_opts* opts);

/*
 * helm_setup - Algorithm 5: coefficients and every quasi-1D factorisation
 * (with opts->apply_form = HELM_DENSE, followed by the restricted operators).
 *   c      device, N^3 floats, velocity on the padded grid (> 0, finite).
 *          Read during the call only.
 *   omega  angular frequency (> 0).
 *   n, b, d  interior points, PML layers, layers per auxiliary problem
 *          (the first modification of Section 4.2); n >= 1, b >= 1, d >= 1.
 *   opts   NULL for defaults.
 *   out    receives the handle (owns the factors, coefficient tables and
 *          work space; release with helm_destroy).
 * The quasi-1D block size (window lines x window layers) must be <= 64.
 * Errors: HELM_EINVAL, HELM_ENOTSUP, HELM_ENOMEM, HELM_ECUDA.
 */
int helm_setup(const float* c, double omega, int n, int b, int d,
               const helm_opts* opts, void* stream, helm_handle* out);

/*
 * helm_setup_batch - one handle over several problems (the batching pattern):
 * problem p has its own velocity c (device, N_p^3 floats, padded grid), omega,
 * n, b, d and a fixed number nrhs of right-hand sides; all share opts.  Each
 * problem is set up as by helm_setup (the handle owns one sub-handle per
 * problem; helm_destroy releases all).  HELM_MAX_BATCH problems at most.
 * Vectors passed with a batch handle are the problems' vectors back to back,
 * [nrhs_0][N_0^3] then [nrhs_1][N_1^3] ..., and the nrhs argument must be the
 * sum of the problems' nrhs (HELM_EINVAL otherwise); host arrays (iters,
 * relres) follow the same order.  With a batch handle:
 *   helm_apply_precond   one sweep launch over every problem (helm_apply_batch);
 *   helm_solve           the problems' solves run concurrently (helm_solve_batch);
 *   helm_matvec, helm_solve_adjoint, helm_velocity_gradient (grad is
 *   [N_0^3][N_1^3]... doubles), helm_status, helm_autotune (each problem tuned
 *   for its own nrhs; *stages_out gets problem 0's choice), helm_enable_timing,
 *   helm_get_stats / helm_reset_stats (sums), helm_factor_bytes and
 *   helm_launch_count (sums) act on every problem;
 *   helm_apply_slab and helm_apply_precond_noalloc return HELM_ENOTSUP and
 *   helm_grid_size, helm_num_blocks, helm_slab_layers return -1.
 * A batch handle may not appear in the arrays of helm_apply_batch or
 * helm_solve_batch (HELM_EINVAL).  The paper runs one problem at a time; this
 * is a serving pattern of the library.
 */
typedef struct {
    const float* c;      /* device, N^3 velocity on the padded grid (> 0)       */
    double omega;        /* angular frequency (> 0)                             */
    int    n, b, d;      /* as for helm_setup                                    */
    int    nrhs;         /* right-hand sides of this problem in every call (>= 1) */
} helm_problem;
int helm_setup_batch(int nprob, const helm_problem* probs, const helm_opts* opts, void* stream,
                     helm_handle* out);

/*
 * helm_apply_precond - Algorithm 6: z = M r, the recursive sweep.
 *   r  device c64 [nrhs][N^3], input;  z  device c64 [nrhs][N^3], output
 *   (r and z must not overlap).  Each RHS is independent (a result does not
 *   depend on the other right-hand sides of the call).  The handle's work
 *   space (nrhs * N^2 * window layers * 8 bytes, plus 4 bytes per RHS) is
 *   allocated on first use and when nrhs grows; otherwise the call only
 *   enqueues a counter reset and one kernel launch.
 */
int helm_apply_precond(helm_handle h, const void* r, void* z, int nrhs, void* stream);

/*
 * helm_apply_slab - Algorithm 4 on one quasi-2D auxiliary problem: v = H_M^{-1} g
 * approximated by the inner sweep (the operator |[T_M]| before restriction).
 *   M  outer block index, 0 <= M < helm_num_blocks(h).
 *   g, v  device c64 [nrhs][Lz][N][N] with Lz = helm_slab_layers(h, M): the
 *   slab window's layers, x fastest.  Used to check one slab at full size.
 */
int helm_apply_slab(helm_handle h, int M, const void* g, void* v, int nrhs, void* stream);

/*
 * helm_matvec - y = A x with the operator of Eq. (system).
 *   fp64 = 0: x, y device c64 [nrhs][N^3];  fp64 = 1: x, y device c128.
 */
int helm_matvec(helm_handle h, const void* x, void* y, int nrhs, int fp64, void* stream);

/*
 * helm_solve - GMRES(restart), right-preconditioned by helm_apply_precond,
 * every RHS independently; Arnoldi inner products in compensated FP32 (Dot2)
 * summed in FP64, Hessenberg and Givens in FP64; the solution accumulates in
 * FP64 and the stopping test uses the true FP64 residual ||f - A u|| / ||f||
 * <= tol at the end of each cycle (Section 5 uses GMRES with a
 * relative-residual tolerance).  Each iteration of a cycle runs as a CUDA
 * graph (captured on first use per handle, right-hand-side count, tol and
 * timing setting; the convergence test and the mask of finished right-hand
 * sides stay on the device); the host reads one count per iteration.
 *   f       device c64 [nrhs][N^3] (zero in the PML padding by convention).
 *   u       device c64 [nrhs][N^3] output (initial guess 0).
 *   iters   host int[nrhs] or NULL: Arnoldi steps per RHS.
 *   relres  host double[nrhs] or NULL: final true relative residual.
 * Returns HELM_ENOCONV if some RHS did not reach tol within maxit, or if its
 * residual became non-finite (relres then holds the non-finite value).
 */
int helm_solve(helm_handle h, const void* f, void* u, int nrhs, double tol,
               int* iters, double* relres, void* stream);

/*
 * Batching (uneven problems).  Each problem has its own handle from helm_setup
 * (its own n, b, d, omega, velocity).  HELM_MAX_BATCH problems at most.
 *
 * helm_apply_batch - one preconditioner launch over the problems: problem p
 *   applies z[p] = M_p r[p] to nrhs[p] right-hand sides (device c64
 *   [nrhs[p]][N_p^3] each); every problem's right-hand sides run concurrently
 *   in the same persistent kernel.  All handles must share one precision and
 *   one apply form (HELM_ENOTSUP otherwise); HELM_DENSE problems are applied
 *   one after another (each launch spans the GPU).
 * helm_solve_batch - helm_solve for every problem, the problems' solves running
 *   concurrently (one host thread and one internal stream each); waits for
 *   `stream` first and returns when every solve has finished.  With HELM_DENSE
 *   handles the solves run one after another on `stream` instead (each dense
 *   apply occupies the whole GPU).  iters and relres
 *   are host arrays of sum(nrhs) entries, problem by problem.  Returns the first
 *   error code, else HELM_ENOCONV if any right-hand side missed tol, else HELM_OK.
 */
int helm_apply_batch(const helm_handle* hs, const void* const* r, void* const* z, const int* nrhs,
                     int nprob, void* stream);
int helm_solve_batch(const helm_handle* hs, const void* const* f, void* const* u, const int* nrhs,
                     int nprob, double tol, int* iters, double* relres, void* stream);

/*
 * helm_autotune - choose the depth of the sweep kernel's shared-memory factor
 * ring (2..8 stages, whatever fits) by timing one slab's inner sweep for
 * nrhs right-hand sides on `stream` with each candidate; keeps the fastest.
 * Allocates a temporary work vector.  *stages_out (host, may be NULL)
 * receives the choice.  Results are unchanged (the ring depth only affects
 * timing).
 */
int helm_autotune(helm_handle h, int nrhs, int* stages_out, void* stream);

/*
 * helm_tune - the setup-level autotuner: among candidate (d, apply form,
 * precision, sweep schedule, b_aux) configurations it measures the time to
 * solution and names the fastest.  d, the layers per auxiliary problem
 * (Section 4.2's first modification), the auxiliary PML width b_aux (its
 * second) and the schedule (one front, or its third: two fronts) change the
 * preconditioner M itself, hence both the GMRES iterations and the cost of an
 * apply; the form and precision change the apply's cost and memory.
 * For each candidate: helm_setup with base opts (NULL: defaults) and the
 * candidate's fields, then helm_solve of the sample right-hand sides f
 * (device c64 [nrhs][N^3]) to tol, both timed with CUDA events on `stream`,
 * then helm_destroy.  A candidate whose setup fails (block size > 64,
 * HELM_ENOMEM for a preconditioner that does not fit, ...) or whose solve does
 * not converge is recorded with that status and skipped.
 *   score = setup_weight * setup_ms + solve_ms (setup_weight = 0: solve time
 *   only, for a handle that serves many solves).
 *   results  host, ncand entries (may be NULL): each candidate's outcome.
 *   best     host, receives the index of the lowest score (-1 if none passed).
 * Returns HELM_OK when at least one candidate passed, else HELM_ENOCONV or the
 * first failure's code; HELM_EINVAL for bad arguments.
 */
typedef struct {
    int d, apply_form, precision;
    int schedule;        /* HELM_ONE_FRONT (0) or HELM_TWO_FRONT               */
    int b_aux;           /* auxiliary PML width; 0 = b                         */
} helm_candidate;

typedef struct {
    helm_candidate cand;
    int status;          /* HELM_OK, or the setup's / solve's error code     */
    int iters_max;       /* GMRES iterations of the slowest right-hand side  */
    double relres_max;   /* largest FP64 relative residual                   */
    double setup_ms, solve_ms, score;
    size_t stored_bytes; /* factors or restricted operators (helm_factor_bytes) */
} helm_tune_result;

int helm_tune(const float* c, double omega, int n, int b, const helm_opts* base, const helm_candidate* cands,
              int ncand, const void* f, int nrhs, double tol, double setup_weight, helm_tune_result* results,
              int* best, void* stream);

/*
 * helm_solve_adjoint - solve A^T lambda = g with the forward factors.  Because
 * s_d depends on x_d only, A = D A_sym with D = diag(s(x1) s(x2) s(x3)) and
 * A_sym complex symmetric (Eq. system), so A^T = D^{-1} A D and
 * lambda = D^{-1} A^{-1} (D g): a helm_solve of D g, rescaled.
 *   g, lambda  device c64 [nrhs][N^3] (distinct).  iters / relres as for
 *   helm_solve, reported for the scaled system A (D lambda) = D g.
 */
int helm_solve_adjoint(helm_handle h, const void* g, void* lambda, int nrhs, double tol,
                       int* iters, double* relres, void* stream);

/*
 * helm_velocity_gradient - the pointwise velocity gradient of a loss L(u)
 * with A(c) u_r = f_r, given the adjoint fields A^T lambda_r = conj(dL/du_r):
 *   grad[idx] = sum_r Re(lambda_r[idx] u_r[idx]) * 2 omega^2 / c[idx]^3
 * (d kappa / dc = -2 omega^2 / c^3 for kappa = omega^2 / c^2).
 *   lambda, u  device c64 [nrhs][N^3];  grad  device double [N^3] (overwritten).
 */
int helm_velocity_gradient(helm_handle h, const void* lambda, const void* u, int nrhs,
                           double* grad, void* stream);

/*
 * helm_update_velocity - local factor update (Section 6, "Conclusion and Future
 * Work": a velocity change on a subdomain touches only the quasi-1D problems
 * whose windows meet it, so only those are refactored).
 *   c_new  device, N^3 floats, the new velocity on the padded grid; it must
 *          equal the handle's current velocity outside the box (not checked).
 *   box    node ranges of the padded grid, half-open: x in [box[0], box[1]),
 *          y in [box[2], box[3]), z in [box[4], box[5]); 0 <= lo < hi <= N.
 *   nprob_out  NULL or receives the number of quasi-1D problems rebuilt.
 * Recomputes kappa everywhere (N^3, cheap), then refactors (chain form) or
 * rebuilds the restricted operators (dense form) of the problems (M, M') with
 * M's z-window and M''s y-window meeting the box (helm_affected_problems);
 * every quasi-1D problem spans all of x.  The result equals a fresh
 * helm_setup with c_new, bit for bit.  Blocking (synchronises the stream).
 * Errors: HELM_EINVAL (box; or c_new <= 0 / non-finite somewhere, found after
 * kappa was recomputed: the handle then holds that velocity's coefficients
 * and its old factors, and is usable again after a call with a valid c_new),
 * HELM_ENOTSUP (batch handles), HELM_ENOMEM, HELM_ECUDA.
 */
int helm_update_velocity(helm_handle h, const float* c_new, const int* box, int* nprob_out, void* stream);

/*
 * helm_affected_problems - host only, no handle: the quasi-1D problems a
 * velocity change in `box` (as above) touches on the grid (n, b, d, b_aux;
 * b_aux = 0 means b) and sweep schedule: out[0..3] = first and last slab M, first and last line
 * block M' (inclusive, windows meeting the box's z and y ranges), or -1 when
 * none.  Returns HELM_OK or HELM_EINVAL.
 */
int helm_affected_problems(int n, int b, int d, int b_aux, int schedule, const int* box, int* out);

/*
 * helm_status - synchronise `stream` and report a bounded device wait that
 * expired in an earlier asynchronous call on this handle (HELM_ETIMEOUT),
 * or HELM_OK.  helm_apply_precond, helm_apply_slab and helm_matvec only
 * enqueue work; helm_setup and helm_solve check this themselves.
 */
int helm_status(helm_handle h, void* stream);

/*
 * helm_apply_precond_noalloc - the same preconditioner apply as
 * helm_apply_precond, for callers that must not allocate device memory during
 * the call: code running inside a captured stream or under a fixed memory
 * budget (an embedding application that owns the device's memory pool, a
 * real-time loop that forbids allocator calls, a process that pre-reserves
 * all memory at start-up).  helm_apply_precond allocates its per-right-hand-
 * side slab work space on first use; this entry point instead uses one
 * fixed array compiled into the library (HELM_NOALLOC_SCRATCH_BYTES, held by
 * every GPU that loads the library until the process exits) and makes no
 * cudaMalloc or cudaFree call.  The paper has no counterpart: this is a
 * deployment option of this library.
 *   r, z, nrhs, stream  as for helm_apply_precond; z receives the same values.
 *   Work space needed: nrhs * N^2 * (window layers) * 8 bytes, N = n + 2b,
 *   plus 4 bytes per right-hand side (rounded up to 8) for the kernel's
 *   per-cluster pacing counters; a request beyond HELM_NOALLOC_SCRATCH_BYTES
 *   returns HELM_EINVAL and launches nothing (e.g. n = 127, b = 6 fits 15
 *   right-hand sides per call).
 * Every call looks up the array's device address (cudaGetSymbolAddress, no
 * allocation) with the current device, which must be the handle's device
 * (HELM_EINVAL otherwise).  The first call on a device may also load the
 * library's device code there, so make one call before any stream capture.
 * Every call on a device shares the one array and keeps the last call's
 * contents; nothing in it needs to start at zero (each call writes every slab
 * entry before reading it, and the call enqueues a reset of the per-cluster
 * pacing counters before its launch).  Calls that may overlap on the GPU
 * (different streams, or different handles on one device) race: serialise
 * them.
 */
#define HELM_NOALLOC_SCRATCH_BYTES (16u << 20)
int helm_apply_precond_noalloc(helm_handle h, const void* r, void* z, int nrhs, void* stream);

/* Sizes: nodes per axis N, swept-axis blocks B, layers of slab M's window. */
int helm_grid_size(helm_handle h);
int helm_num_blocks(helm_handle h);
int helm_slab_layers(helm_handle h, int M);

/*
 * Kernel timing (opt-in).  With timing on, the library records CUDA events on
 * the call's stream around every sweep (preconditioner) and stencil launch;
 * helm_get_stats waits for the recorded events and returns the accumulated
 * counts and device milliseconds of completed launches.
 */
typedef struct {
    long long sweep_launches;   /* preconditioner applies (one launch each)   */
    double    sweep_ms;         /* their summed device time                   */
    long long stencil_launches; /* matvec and residual launches               */
    double    stencil_ms;
    long long rhs_applied;      /* right-hand sides carried by those applies  */
} helm_stats;

int  helm_enable_timing(helm_handle h, int on);
int  helm_get_stats(helm_handle h, helm_stats* out);
void helm_reset_stats(helm_handle h);

/* Bytes of device memory held by the stored preconditioner: the quasi-1D
 * factors (HELM_CHAIN) or the restricted operators and their scales
 * (HELM_DENSE). */
size_t helm_factor_bytes(helm_handle h);

/*
 * helm_dense_operator - read back one stored restricted operator of a
 * HELM_DENSE handle (the map |T~_{M'}| of Algorithm 4 uses for slab M, line
 * block M'), decoded to complex FP32.
 *   dir    0: the operator of (M, M') (it serves both passes of Algorithm 4,
 *          except at the boundary line blocks, where it is the forward pass);
 *          1 with M' = 0 (or M' = B-1 with HELM_TWO_FRONT): the backward pass
 *          of that boundary line block.
 *   n_out, n_in  host, may be NULL: its size.
 *   rects  host int[13] or NULL: {nrect, in rect, out rect 0, out rect 1},
 *          each rect {first line (global y), lines, first z row of the slab
 *          window, z rows} over every x.  Output entries run rect by rect
 *          with x fastest, then the z row, then the line; input entries (one
 *          rect) with the z row fastest, then the line, then x.
 *   G      device c64 [n_out][n_in] or NULL (sizes only).
 * Returns HELM_ENOTSUP for a HELM_CHAIN or batch handle.
 */
int helm_dense_operator(helm_handle h, int M, int Mp, int dir, int* n_out, int* n_in, int* rects, void* G,
                        void* stream);

/* Number of kernels this handle has launched since it was created. */
long long helm_launch_count(helm_handle h);

/* Release everything the handle owns.  NULL is accepted. */
void helm_destroy(helm_handle h);

/* Static description of an error code. */
const char* helm_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* HELM_H */
