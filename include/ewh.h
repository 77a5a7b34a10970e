/*
 * ewh.h -- C ABI of the GB300 El-WaveHoltz library (libewh.so).
 *
 * El-WaveHoltz (Appelo, Garcia, Alvarez Loya, Runborg) finds the time-harmonic
 * solution v of the elastic (Navier) equation rho w^2 v + div T(v) = f
 * (Section 2.2, eq. elastic-frequency) by applying the WaveHoltz operator
 *     Pi u0 = (2/T) int_0^T (cos wt - 1/4) u(t) dt,   T = 2 pi / w
 * (Section 3, eq. el_WHI_OP) inside a Krylov solve of the symmetric positive
 * definite system M (I - S) v = M Pi 0 (Section 4.5, eq. amat_sym), where
 * u(t) solves rho u_tt = div T(u) - f cos wt (Section 2.1, eq. elastic-time)
 * with u(0) = u0, u_t(0) = 0 and S is Pi with f = 0.
 *
 * Discretisation (Section 4.1 and 4.3): nodes of a Cartesian grid (or, through
 * ewh_create_mapped, of a curvilinear 2D grid), an energy-conserving symmetric
 * L_h (order 2: compact; order 4: fourth-order summation-by-parts) with
 * diagonal mass M, the time-corrected explicit
 * leapfrog of eq. (elastic-time-explicit-corrected) with the Taylor start, and
 * the trapezoidal rule for the filter integral (eq. qoper).
 *
 * Conventions shared by every entry point
 *   - Grid: n[a] nodes along axis a *including* both boundary nodes, spacing h.
 *   - Sides (bc[6] = x-, x+, y-, y+, z-, z+): EWH_BC_DIRICHLET fixes the
 *     boundary nodes to zero (they are not unknowns); EWH_BC_FREE makes the side
 *     traction free (its boundary nodes are unknowns).
 *   - Media rho, lambda, mu: one double per node of the full grid, C order
 *     [z][y][x] (x fastest).  Forcing: [nrhs][dim][z][y][x] on the full grid.
 *   - Solution-space vectors (v_in, v_out, b, x0, ...): double precision,
 *     [nrhs][dim][z][y][x] over the UNKNOWN nodes only (Dirichlet boundary
 *     nodes removed), x fastest.  Device pointers unless stated otherwise.
 *   - Every call returns an ewh_status; nothing throws across the ABI.  A
 *     failing call leaves a message retrievable with ewh_last_error().
 *     Asynchronous CUDA errors surface as EWH_ECUDA at the next call.
 *   - Calls on one context are not thread safe; distinct contexts are
 *     independent.
 */
#ifndef EWH_H
#define EWH_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ewh_ctx ewh_ctx; /* opaque, owned by the library */

typedef enum {
  EWH_OK = 0,
  EWH_EINVAL = 1,      /* invalid argument (sizes, media, omega, ...) */
  EWH_ENOMEM = 2,      /* device or host allocation failed */
  EWH_ECUDA = 3,       /* a CUDA call failed */
  EWH_ENOTCONV = 4,    /* Krylov solve hit maxit before tol */
  EWH_EBREAKDOWN = 5,  /* CG found (p, (I-S)p)_M <= 0: system not definite */
  EWH_ETIMEOUT = 6     /* a bounded device-side wait gave up */
} ewh_status;

enum { EWH_BC_DIRICHLET = 0, EWH_BC_FREE = 1 };

/* Arithmetic of the wave solves.  Krylov vectors, inner products and
 * residual norms are always FP64. */
enum {
  EWH_FP64 = 0,          /* FP64 stencil, state and filter */
  EWH_FP32_STENCIL = 1   /* FP32 stencil, state and filter; FP64 Krylov.  The
                            solve replaces the recursive residual by the FP64
                            true residual each time it has fallen tenfold, stops
                            on the FP64 residual, and continues with the FP64
                            operator if the FP32 one loses definiteness. */
};

typedef struct {
  int dim;        /* 2 or 3 */
  int n[3];       /* nodes per axis including the two boundary nodes (>= 4;
                     >= 8 for order 4; each axis is stored padded to a
                     multiple of 32 plus 12, and one padded component must
                     hold fewer than 2^31 nodes) */
  double h;       /* grid spacing (> 0) */
  int order;      /* 2 or 4 */
  int bc[6];      /* EWH_BC_DIRICHLET or EWH_BC_FREE per side */
  int precision;  /* EWH_FP64 or EWH_FP32_STENCIL */
  double cfl;     /* dt_CFL = cfl h / sqrt(max (lambda + (dim+1) mu) / rho);
                     0 selects 0.5.  Must be in (0, 1). */
  int periods;    /* K >= 1: filter over K periods (eq. many_periods_filter) */
  int corrected;  /* 1: time-corrected scheme (Section 4.3, default);
                     0: standard leapfrog (converges to the w~ problem) */
  int nt;         /* time steps per period; 0 = ceil(T / dt_CFL), at least 5 */
  int implicit;   /* 0: explicit leapfrog (above).  1: the implicit scheme of
                     Section 4.4 (eq. ImplicitScheme; with corrected = 1 the
                     modified alpha = cos(w dt)(2 + w^2 dt^2) and start, so
                     the fixed point is the w problem; with 0, the w~ =
                     2 sin(w dt/2)/(dt sqrt(cos w dt)) problem).  Needs
                     precision EWH_FP64 and an explicit nt >= 5 (no CFL
                     limit); each level solves with I + (dt^2/2) M^{-1} K by
                     CG in the M inner product on the device.  Not for
                     batches. */
} ewh_grid_desc;

/* Scalars of a created problem. */
typedef struct {
  int nt;              /* steps per period */
  int periods;
  double dt;           /* T / nt */
  double omega;
  double omega_tilde;  /* 2 sin(w dt / 2) / dt */
  double kt;           /* c dt^2, c = (w~/w)^2 if corrected else 1 */
  long long nodes;     /* unknown nodes per component */
  long long n_unknowns;/* dim * nodes (one right-hand side) */
  int nrhs;
  int nu[3];           /* unknown nodes per axis */
  int kernel_variant[2]; /* step-kernel variant picked by the autotuner for the
                            FP64 / FP32 wave solves (-1 = not picked yet; it is
                            picked on the first solve of that precision) */
  int resident[10];    /* when the FP32 wave solve runs on chip (2D, order 4),
                          one cooperative launch per group of right-hand sides:
                          its partition -- CTA shape index, CTAs along x and y
                          per rhs, interior block width, first block width,
                          block height (nodes), threads per CTA, register node
                          pairs per thread, rhs per launch, launches; CTA
                          (cx, cy) of a rhs owns x from X0 = cx ? first +
                          (cx-1) width : 0 and y from cy height.  All -1
                          otherwise. */
} ewh_problem_info;

typedef struct {
  int iters;           /* Krylov iterations (max over right-hand sides) */
  int s_applies;       /* S applications of the working precision */
  int s_applies_fp64;  /* FP64 S applications used for residual checks */
  double rel_res;      /* final ||b - (I-S)x||_M / ||b||_M, max over rhs,
                          recomputed with an FP64 S apply */
  double seconds;      /* wall time of the solve (device work included) */
  int status;          /* ewh_status of the solve */
  int minres_iters;    /* of iters, those of MINRES continuing after CG met
                          (p, A p)_M <= 0 on the FP64 operator (0 otherwise) */
} ewh_solve_info;

/* Create a problem (Section 2.1 data, Section 4 discretisation).
 *   desc       grid, boundary conditions, order, precision, cfl, periods.
 *   rho,lambda,mu  host or device pointers, one double per full-grid node;
 *              copied.  Requires rho > 0, mu > 0, lambda > -2 mu / dim, finite.
 *   omega      angular frequency w > 0 (T = 2 pi / w).
 *   forcing    host or device pointer [nrhs][dim][full grid] or NULL (f = 0);
 *              copied.  The wave equation uses -f cos(wt).
 *   nrhs       >= 1 right-hand sides that share medium and w.
 *   cuda_stream  the caller's cudaStream_t (NULL = legacy default stream);
 *              work is ordered after prior work on it, and the stream waits
 *              for the library's work before each call returns.
 *   out        receives the context (NULL on failure).
 * Errors: EWH_EINVAL (bad sizes, media, omega, unstable cfl, order 4 on an
 * axis with fewer than 8 nodes), EWH_ENOMEM, EWH_ECUDA. */
ewh_status ewh_create(const ewh_grid_desc* desc, const double* rho, const double* lambda,
                      const double* mu, double omega, const double* forcing, int nrhs,
                      void* cuda_stream, ewh_ctx** out);

/* Create a problem on a curvilinear 2D grid (Section 4.1, curvilinear form).
 * The nodes are the image of (q, r) = (i h, j h), i < n[0], j < n[1], under a
 * smooth mapping: x, y (host or device, one double per node, i fastest; copied)
 * are its coordinates there.  The metric terms x_q, x_r, y_q, y_r come from the
 * order-4 SBP derivative in q and r, J = x_q y_r - x_r y_q; the operator is the
 * energy form with physical derivatives q_x D_q + r_x D_r (and y alike), the
 * mass rho J H h^2, and dt uses max (lambda + 3 mu)/rho (|grad q|^2 + |grad r|^2)/2.
 * Boundary conditions apply to the sides of the (q, r) square; a free side is
 * traction-free on the curved physical boundary it maps to.  The other
 * arguments are as for ewh_create; the identity mapping gives the Cartesian
 * problem.  Requires dim 2 and order 4 (else EWH_EINVAL) and J > 0 at every
 * node (EWH_EINVAL naming the first node where it fails); EWH_ECUDA when no
 * device is present (the metric terms are computed on the device).  Mapped
 * contexts always use the per-level two-kernel step and cannot join a batch. */
ewh_status ewh_create_mapped(const ewh_grid_desc* desc, const double* x, const double* y,
                             const double* rho, const double* lambda, const double* mu,
                             double omega, const double* forcing, int nrhs, void* cuda_stream,
                             ewh_ctx** out);

/* Fill *info with the problem's scalars. */
ewh_status ewh_get_info(const ewh_ctx* ctx, ewh_problem_info* info);

/* v_out = S v_in (Section 3: Pi with f = 0; eq. qoper): nt*periods leapfrog
 * steps from u(0) = v_in, u_t(0) = 0 with the trapezoid accumulation.
 * Device FP64 vectors of nrhs * n_unknowns; v_in and v_out may alias.
 * Computed in the context's precision. */
ewh_status ewh_apply_S(ewh_ctx* ctx, const double* v_in, double* v_out);

/* Same as ewh_apply_S but always in FP64, whatever the context precision. */
ewh_status ewh_apply_S_fp64(ewh_ctx* ctx, const double* v_in, double* v_out);

/* b_out = Pi 0 (eq. amat_non_sym right-hand side): the forced solve from rest.
 * Device FP64, nrhs * n_unknowns, context precision. */
ewh_status ewh_apply_Pi0(ewh_ctx* ctx, double* b_out);

/* out = M^{-1} K u = -M^{-1} L_h u (the spatial operator of Section 4.1 alone,
 * FP64).  Device FP64 vectors of nrhs * n_unknowns. */
ewh_status ewh_apply_minvK(ewh_ctx* ctx, const double* u, double* out);

/* out[r] = (x_r, y_r)_M, the M inner product per right-hand side (FP64,
 * deterministic order).  x, y device FP64; out host array of nrhs doubles. */
ewh_status ewh_mdot(ewh_ctx* ctx, const double* x, const double* y, double* out);

/* Solve M (I - S) v = M Pi 0 (eq. amat_sym) by CG in the M inner product,
 * independently for every right-hand side.
 *   tol        stop when ||b - (I-S)x||_M <= tol ||b||_M (b = Pi 0).
 *   maxit      iteration cap (working-precision CG iterations in total).
 *   x0_or_null initial guess (FP64, host or device) or NULL for zero.
 *   v_out      solution (FP64, host or device), nrhs * n_unknowns.
 *   info       optional; filled on return.
 * Returns EWH_OK, EWH_ENOTCONV (best iterate in v_out), EWH_EBREAKDOWN
 * (last iterate in v_out), or an error.  When CG meets (p, A p)_M <= 0 on
 * the FP64 operator (M(I - S) indefinite, or numerically so next to a
 * resonance) the solve continues from the current iterate with MINRES (the
 * Section 4.4 remark), counted in info.minres_iters; EWH_EBREAKDOWN means
 * that MINRES broke down too.  The iterations run under device control: one graph launch runs a window
 * of up to EWH_CG_POLL (environment, default 32; 1 = the host polls after
 * every iteration) iterations, a device kernel ending the window when the
 * host must act (residual replacement, breakdown, iteration limit); the
 * iterates equal those of the host-polled loop. */
ewh_status ewh_solve(ewh_ctx* ctx, double tol, int maxit, const double* x0_or_null,
                     double* v_out, ewh_solve_info* info);

/* Same problem and stopping rule as ewh_solve, by the conjugate residual
 * method in the M inner product (Section 4.5, remark on conjugate residual:
 * the residual norm is non-increasing, which the paper prefers for sweeps over
 * w).  One S apply per iteration (on the residual); in the FP32-stencil
 * precision the residual is replaced by the FP64 true residual each time it
 * has fallen tenfold, restarting the directions from it. */
ewh_status ewh_solve_cr(ewh_ctx* ctx, double tol, int maxit, const double* x0_or_null, double* v_out,
                        ewh_solve_info* info);

/* MINRES on (I - S) v = b in the M inner product (Section 4.4, the remark on
 * the implicit scheme: when few quadrature points push the discrete filter
 * transfer function above 1 near a resonance, M(I - S) can be indefinite
 * and MINRES replaces CG).  Same arguments, layout, ownership and status
 * codes as ewh_solve; the residual is minimised in the M-norm, so it never
 * increases.  One S apply per iteration; the recursive residual is replaced
 * by the FP64 true residual when it reaches tol (FP32 stencil: also each time
 * it has fallen tenfold), restarting the recurrence from the current iterate.
 * EWH_EBREAKDOWN if the Lanczos tridiagonal turns singular. */
ewh_status ewh_solve_minres(ewh_ctx* ctx, double tol, int maxit, const double* x0_or_null, double* v_out,
                            ewh_solve_info* info);

/* Copy up to cap entries of the last solve's residual history (relative
 * M-norm of the recursive residual after each iteration, max over rhs) to the
 * host array out; returns the number of entries available via *count. */
ewh_status ewh_residual_history(const ewh_ctx* ctx, double* out, int cap, int* count);

/* Number of kernel launches the library has issued on this context
 * (including launches inside graphs), for accounting. */
long long ewh_kernel_launches(const ewh_ctx* ctx);

/* Device-time accounting of the leapfrog steps.  Every wave solve (S or Pi 0
 * apply) launched by the host is bracketed by CUDA events on the context's
 * stream; the elapsed times are accumulated per precision.  The S applies of
 * CG iterations under device control (a window of iterations in one graph
 * launch, see ewh_solve) are counted apart, untimed.  Index 0 = FP64,
 * 1 = FP32. */
typedef struct {
  double wave_ms[2];     /* device milliseconds spent in event-timed wave solves */
  long long steps[2];    /* leapfrog steps (time levels) those solves covered */
  long long waves[2];    /* number of event-timed wave solves */
  long long launches;    /* kernel launches issued (as ewh_kernel_launches) */
  long long grid_wait_timeouts; /* on-chip wave solves whose grid-barrier wait
                                   gave up (see ewh_set_grid_wait) */
  long long loop_steps[2];  /* leapfrog steps of the wave solves run inside
                               device-controlled CG windows (not timed) */
  long long loop_waves[2];  /* number of those wave solves */
} ewh_stats;

/* Fill *out (synchronises the context's stream first). */
ewh_status ewh_get_stats(ewh_ctx* ctx, ewh_stats* out);

/* Zero the accumulated statistics (the launch counter included). */
ewh_status ewh_reset_stats(ewh_ctx* ctx);

/* Bound of each device-side wait of the FP32 order-4 step kernels (no
 * counterpart in the paper): the grid barrier of the on-chip wave solve (2D,
 * every time level in one cooperative launch per group of right-hand sides,
 * CTAs meeting once per level) and the mbarrier waits of the marching kernels
 * (2D y-march, 3D z-march) for their bulk-tensor copies.  Every wait is
 * bounded: after ns nanoseconds (default 1e9; the grid barrier also after 2^22
 * polls) the waiting CTA gives up (the on-chip solve raises an error flag and
 * every CTA leaves at its next barrier; a marching CTA waits, bounded, for its
 * copies in flight and returns), and the launch fills its remaining
 * accumulator nodes with NaN (so ewh_apply_S returns NaN and a solve sees an
 * FP32 breakdown and continues with the FP64 operator).  ns = 0 makes every
 * wait give up at once: a way to exercise that path without a hung GPU.  The
 * count of give-ups is in ewh_stats.grid_wait_timeouts.  Takes effect for the
 * next launch (the stream is synchronised first); a no-op on contexts that
 * run none of these kernels.  Errors: EWH_EINVAL (ns < 0), EWH_ECUDA. */
ewh_status ewh_set_grid_wait(ewh_ctx* ctx, long long ns);

/* ---- Batches: many independent problems advanced together ----------------
 *
 * Shots at different sources, frequencies and grid sizes are independent
 * El-WaveHoltz problems.  A batch advances all of them together: one CG
 * iteration of every unconverged member is one CUDA graph in which each member
 * is a parallel branch (its pack, its nt*periods leapfrog launches, its FP64
 * Krylov updates), so small members fill the GPU together and the whole
 * iteration costs one launch.  Converged members drop out of the graph.
 * Members must share dim, order and precision; sizes, media, frequencies and
 * right-hand-side counts may differ. */
typedef struct ewh_batch ewh_batch;

typedef struct {
  ewh_grid_desc desc;     /* as for ewh_create */
  const double* rho;      /* host or device, full grid */
  const double* lambda;
  const double* mu;
  double omega;
  const double* forcing;  /* [nrhs][dim][full grid], required for solves */
  int nrhs;
} ewh_problem;

/* Create a batch of nprob >= 1 problems (each is validated as by ewh_create). */
ewh_status ewh_batch_create(const ewh_problem* probs, int nprob, void* cuda_stream, ewh_batch** out);

/* v_out[k] = S v_in[k] for every member k (device FP64 vectors, member layout). */
ewh_status ewh_batch_apply_S(ewh_batch* b, const double* const* v_in, double* const* v_out);

/* Solve every member as ewh_solve does (same tolerance and stopping rule);
 * v_out[k] receives member k's solution (host or device FP64), infos[k] its
 * statistics (optional).  Returns EWH_OK when every member converged, else the
 * first failing member's status (the others are still solved).  A window of
 * iterations of every unconverged member is one graph launch (a device-side
 * loop per member, concurrent; one after another when a member runs the
 * on-chip solve, whose cooperative launch needs all its CTAs resident). */
ewh_status ewh_batch_solve(ewh_batch* b, double tol, int maxit, double* const* v_out, ewh_solve_info* infos);

/* The context of member k (owned by the batch; use for ewh_get_info). */
ewh_status ewh_batch_member(ewh_batch* b, int k, ewh_ctx** ctx);

/* Kernel launches issued by the batch (all members, graphs included). */
long long ewh_batch_kernel_launches(const ewh_batch* b);

/* Message of the batch's last failing call. */
const char* ewh_batch_last_error(const ewh_batch* b);

/* Release the batch and its member contexts (NULL is ignored). */
void ewh_batch_destroy(ewh_batch* b);

/* Allocation-free weighted inner products (no counterpart in the paper; a
 * convenience for callers that must not allocate device memory).
 *
 * Some callers cannot call cudaMalloc: code running while a CUDA graph is
 * being captured (allocation would break or be baked into the capture),
 * embedded or real-time hosts that reserve all device memory up front,
 * and frameworks whose own memory pool owns the device.  This entry point
 * needs no context (ewh_create allocates) and allocates nothing: its
 * per-block partial sums live in one fixed array inside libewh.so that every
 * GPU loading the library keeps until the process exits (64 KiB per device).
 *
 *   out[b] = sum_{c < ncomp} sum_{i < nodes} w[i] * x[b][c][i] * y[b][c][i]
 *
 * for b < nbatch, with x, y laid out [nbatch][ncomp][nodes] like the solver's
 * vectors and w one weight per node (e.g. the mass diagonal).  The sums are
 * deterministic (a fixed-order two-pass reduction); above 65536 entries per
 * member they use at most 64 blocks where ewh_mdot uses more, so the two
 * agree to rounding, not bit for bit.
 *   x, y, w, out  device pointers; out receives nbatch doubles.
 *   cuda_stream   the stream the two kernels run on (NULL = legacy default).
 * Limits: nbatch <= 128 (EWH_EINVAL beyond, with a message in
 * ewh_last_error(NULL)); nodes, ncomp >= 1.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The address is tied to the device's context:
 * after a cudaDeviceReset the next call looks it up again (so, again, make
 * that call outside a capture).  All calls share the one array: calls that
 * overlap on the GPU (different streams without ordering) race and may return
 * wrong sums, so order them.  Nothing needs clearing between calls: each call
 * writes every partial sum it reads.  Returns EWH_OK, EWH_EINVAL or
 * EWH_ECUDA; results are ready when the stream reaches them. */
ewh_status ewh_mdot_noalloc(const double* x, const double* y, const double* w, long long nodes, int ncomp,
                            int nbatch, double* out, void* cuda_stream);

/* Measured FMA throughput of the current GPU in floating-point operations per
 * second (no counterpart in the paper): the arithmetic roofline of step
 * kernels that are bound by the CUDA cores rather than by memory.  Every thread
 * of a grid of 8 blocks of 256 threads per SM runs 8 independent FMA chains
 * (one FMA = 2 operations) for about 50 ms; the run is timed with CUDA events
 * on cuda_stream (NULL = legacy default) and synchronised.
 *   precision  EWH_FP64 or EWH_FP32_STENCIL (FP32).
 * Errors: EWH_EINVAL (bad precision or null output, message in
 * ewh_last_error(NULL)), EWH_ECUDA. */
ewh_status ewh_fma_rate(int precision, double* flops_per_second, void* cuda_stream);

/* ---- Layers of the learned warm start --------------------------------------
 *
 * The paper has no learned component: these entry points serve the warm-start
 * form of the solver (an initial guess x0 for ewh_solve from a small
 * convolutional encoder-decoder over medium, forcing and frequency).
 * Conventions: activations NHWC, weights [Co][3][3][Ci]; tensors typed void*
 * hold bfloat16, float* hold FP32; all pointers are device pointers; the work
 * is enqueued on `stream` (NULL = legacy default stream) and nothing is
 * allocated.  Errors: EWH_EINVAL (bad sizes, message in ewh_last_error(NULL)),
 * EWH_ECUDA. */

/* y = conv3x3(x, w) + bias (zero padding, stride 1), BF16 tensor-core MMA with
 * FP32 accumulation.  y_pre (FP32, may be NULL) receives the pre-activation,
 * y_act (BF16, may be NULL) the activation (act = 1: leaky ReLU 0.1, 0: none).
 * Ci a multiple of 16, Co a multiple of 8; bias may be NULL. */
ewh_status ewh_conv3x3_fwd(const void* x, const void* w, const float* bias, float* y_pre, void* y_act, int act,
                           int N, int H, int W, int Ci, int Co, void* stream);

/* dx = gradient with respect to x of <conv3x3(x, w), dy> (FP32 out, BF16 dy).
 * w_scratch: caller buffer of 9*Ci*Co bf16 for the flipped weights.  Ci, Co
 * multiples of 16. */
ewh_status ewh_conv3x3_dgrad(const void* dy, const void* w, void* w_scratch, float* dx, int N, int H, int W, int Ci,
                             int Co, void* stream);

/* dw (FP32, overwritten) = gradient with respect to w of <conv3x3(x, w), dy>.
 * x, dy BF16.  Ci, Co multiples of 16. */
ewh_status ewh_conv3x3_wgrad(const void* x, const void* dy, float* dw, int N, int H, int W, int Ci, int Co,
                             void* stream);

/* db[c] = sum over the P pixels of dy[p][c] (FP32). */
ewh_status ewh_bias_grad(const float* dy, float* db, long long P, int C, void* stream);

/* Leaky-ReLU gradient from the FP32 pre-activation: dx = dy (pre > 0) or
 * 0.1 dy; written in FP32 (dx) and/or BF16 (dx_bf16). */
ewh_status ewh_leaky_relu_bwd(const float* pre, const float* dy, float* dx, void* dx_bf16, long long n,
                              void* stream);

/* 2x2 average pooling of BF16 NHWC x (H, W even) and its FP32 gradient. */
ewh_status ewh_avgpool2(const void* x, void* y, int N, int H, int W, int C, void* stream);
ewh_status ewh_avgpool2_bwd(const float* dy, float* dx, int N, int H, int W, int C, void* stream);

/* Nearest 2x upsampling of x [N,H,W,C] into channels [c_off, c_off+C) of
 * y [N,2H,2W,Cy] (BF16), and its FP32 gradient. */
ewh_status ewh_upsample2(const void* x, void* y, int N, int H, int W, int C, int Cy, int c_off, void* stream);
ewh_status ewh_upsample2_bwd(const float* dy, float* dx, int N, int H, int W, int C, int Cy, int c_off,
                             void* stream);

/* Channel concatenation: copy BF16 x [P][C] into channels [c_off, c_off+C) of
 * y [P][Cy]; and the FP32 gradient slice dx (=, or += if accumulate) dy[.][c_off..]. */
ewh_status ewh_copy_channels(const void* x, void* y, long long P, int C, int Cy, int c_off, void* stream);
ewh_status ewh_slice_channels(const float* dy, float* dx, long long P, int C, int Cy, int c_off, int accumulate,
                              void* stream);

/* FP32 -> BF16 conversion of n values. */
ewh_status ewh_f32_to_bf16(const float* a, void* b, long long n, void* stream);

/* Per-sample scaled L2 loss of FP32 y [N][P][C] (first Cu channels) against
 * FP32 t [N][P][Cu]: loss[n] = 1/2 ||y_n - t_n||^2 / ||t_n||^2; grad = d(mean
 * loss)/dy (zero on channels >= Cu). */
ewh_status ewh_scaled_l2_loss(const float* y, const float* t, float* grad, float* loss, long long P, int C, int Cu,
                              int N, void* stream);

/* One Adam step (Kingma and Ba 2015, bias-corrected, step >= 1) on FP32
 * parameters; param_bf16 (may be NULL) receives the updated BF16 copy. */
ewh_status ewh_adam_step(float* param, const float* grad, float* m, float* v, void* param_bf16, long long n,
                         float lr, float beta1, float beta2, float eps, int step, void* stream);

/* Release every resource of the context (NULL is ignored). */
void ewh_destroy(ewh_ctx* ctx);

/* Message of the last failing call on ctx (or of the last failed create when
 * ctx is NULL).  Never NULL; owned by the library. */
const char* ewh_last_error(const ewh_ctx* ctx);

/* Static name of a status code. */
const char* ewh_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* EWH_H */
