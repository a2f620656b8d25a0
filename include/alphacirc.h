/*
 * alphacirc.h — C ABI of the GB300 alpha-circulant preconditioned Richardson
 * solver for the all-at-once Radau IIA collocation system of a linear,
 * periodic, constant-coefficient PDE  u_t = A u  (+ an optional right-hand side).
 *
 * Method: Caklovic, Speck & Frank, "A parallel-in-time collocation method using
 * diagonalization: theory and implementation for linear problems"
 * (arXiv 2103.12571).  Equation, lemma and algorithm numbers below refer to it.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Layout of every space-time vector: u[l][m][n], double, l = 0..L-1 (time
 *   step), m = 0..M-1 (collocation node), n = 0..N-1 (grid point), n fastest;
 *   in 2D n = iy * nx + ix.  This is the ordering of eq. (globalsys).
 * - "device" pointers are CUDA global-memory pointers on the device that was
 *   current at ac_setup(); "host" pointers are ordinary CPU memory.  The
 *   caller owns every pointer it passes; the plan owns its own workspace.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Every call is ordered on that stream.  Only ac_richardson_solve and
 *   ac_adjoint_solve synchronise the host (once per iteration, to read a few
 *   scalars); ac_grad_params synchronises once.
 * - Return value: AC_OK (0) or a negative AC_ERR_* code.  No exception ever
 *   crosses this boundary.  ac_status_string() names a code; ac_last_error()
 *   returns a thread-local message with detail about the last failure.
 * - Device work runs only in this library's own CUDA kernels: there is no
 *   CPU fallback.  A call that cannot run on the GPU returns an error.
 */
#ifndef ALPHACIRC_H
#define ALPHACIRC_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define AC_OK                      0
#define AC_ERR_INVALID_ARG        -1  /* bad size, null pointer, unsupported combination   */
#define AC_ERR_NOT_DIAGONALIZABLE -2  /* Q G_l^{-1} numerically defective (Lemma 2, Sec. 2.3) */
#define AC_ERR_NO_CONVERGENCE     -3  /* max_iter reached, or the residual grew 3 times      */
#define AC_ERR_INNER_BREAKDOWN    -4  /* BiCGStab breakdown / iteration cap in an inner solve */
#define AC_ERR_CUDA               -5  /* a CUDA runtime call failed (see ac_last_error)      */
#define AC_ERR_NOT_FINITE         -6  /* NaN or Inf met in a residual norm                   */

/* ---- option values ------------------------------------------------------ */
#define AC_C128 0   /* preconditioner (steps ii-iv) in complex128                     */
#define AC_C64  1   /* preconditioner in complex64; residual and update stay FP64    */

#define AC_INNER_FFT      0  /* exact spatial-FFT solve of eq. (d2)                    */
#define AC_INNER_BICGSTAB 1  /* batched BiCGStab on the stencil, relative tolerance tau */
#define AC_INNER_GMRES    2  /* batched restarted GMRES(m) on the stencil, unpreconditioned,
                                relative tolerance tau (the paper's inner solver, Sec. 4.1) */

#define AC_ALPHA_FIXED 0  /* alpha_k = alpha0 for every k                                 */
#define AC_ALPHA_PAPER 1  /* Algorithm 2: alpha_{k+1} = sqrt(gamma/m_k), m_{k+1} = 2 sqrt(m_k gamma) */
#define AC_ALPHA_MIXED 2  /* fixed alpha = sqrt(L (3 eps_p + tau)), clamped to [1e-8, 0.25] */

#define AC_STOP_RESIDUAL 0  /* ||w - C u||_2 <= tol ||w||_2                               */
#define AC_STOP_PAPER    1  /* Algorithm 2: m_k <= tol, or ||u_L^{k+1} - u_L^k||_inf <= tol */

#define AC_FORM_CORRECTION 0  /* u^{k+1} = u^k + C_alpha^{-1}(w - C u^k): FP64 residual, iterative refinement */
#define AC_FORM_PAPER      1  /* eq. (Riteration) as written: C_alpha u^{k+1} = w + (C_alpha - C) u^k,
                                 whose right-hand side differs from w only by -alpha H u_L^k in block 1;
                                 requires AC_STOP_PAPER                                                   */

#define AC_UPDATE_PLAIN 0  /* update kernel: tiles read straight from global memory (default)      */
#define AC_UPDATE_TMA   1  /* complex64 plans: persistent update kernel whose X and u tiles the copy
                              engine stages in shared memory as 2D tensor tiles (double-buffered);
                              used when u is 16-byte aligned and two CTAs' buffers fit an SM     */

#define AC_MAX_STATS 128

/* Spatial operator A = nu * Lap_h - cx * D_x - cy * D_y on the periodic box
 * [0,lx) x [0,ly) with nx (x ny) points and h = length / n per axis.  Sec. 5
 * discretises the heat equation with centred and the advection equation
 * with upwind periodic stencils, of the orders in Tables 1-2; the paper
 * prints no weights, so the standard finite-difference formulas are used
 * (the weights exact on polynomials of degree <= number of points - 1):
 *   upwind = 0: centred first and second derivatives of order 2, 4 or 6
 *               (offsets -order/2 .. order/2);
 *   upwind = 1: first derivative of order 1..5 on the offsets lo .. lo+order,
 *               lo = -(order/2 + 1) (integer division), for a positive
 *               velocity component, mirrored (w(o) -> -w(-o)) for a negative
 *               one; the Laplacian is the centred one of the order rounded
 *               up to even.
 * The stencil radius is at most 3.  dim = 1 ignores ny, ly, cy. */
typedef struct {
    int dim;          /* 1 or 2                                     */
    int nx, ny;       /* grid points per axis (prime factors 2, 3, 5, 7 only for AC_INNER_FFT) */
    double lx, ly;    /* box lengths                                */
    double nu;        /* diffusion coefficient                      */
    double cx, cy;    /* advection velocity                         */
    int order;        /* centred: 2, 4, 6; upwind: 1..5             */
    int upwind;       /* 0: centred first derivative, 1: upwind     */
} ac_problem;

/* Choice of alpha_k per iteration (Sec. 3.3). */
typedef struct {
    int mode;         /* AC_ALPHA_FIXED | AC_ALPHA_PAPER | AC_ALPHA_MIXED            */
    double alpha0;    /* FIXED: the alpha; others: ignored                            */
    double m0;        /* PAPER: estimate of ||u^(0) - u*||_inf; <= 0 selects the
                         bound T (||A||_inf max|u0|) of Sec. 3.3                      */
    double tau;       /* inner-solve relative tolerance (BiCGStab), used in gamma too */
    int max_iter;     /* outer iteration cap (<= AC_MAX_STATS)                        */
    int stop_rule;    /* AC_STOP_RESIDUAL | AC_STOP_PAPER                             */
    int inner_max_iter; /* Krylov iteration cap per system (<= 0: 4000); for GMRES the
                           Arnoldi steps over all restarts                              */
    int form;           /* AC_FORM_CORRECTION | AC_FORM_PAPER                           */
    int inner_restart;  /* GMRES restart length m, 1..32 (<= 0: 30)                     */
    int update_kernel;  /* AC_UPDATE_PLAIN | AC_UPDATE_TMA                              */
    int space_cluster;  /* 2D FFT solves of planes above 160 KB (power-of-two grids):
                           0 or -1: three passes (rows, columns with the division, rows);
                           4, 8, 16: one pass, each plane held in the shared memory of a
                           thread-block cluster of that many CTAs (AC_ERR_INVALID_ARG if
                           the cluster cannot hold a plane or does not fit on the device).
                           The three passes measured faster on this GPU.                */
} ac_alpha_schedule;

/* Per-solve record (host memory, filled by the solve calls). */
typedef struct {
    int iters;                        /* outer iterations performed                    */
    int converged;                    /* 1 if the stop rule was met                     */
    double res_rel[AC_MAX_STATS];     /* ||w - C u^(k)||_2 / ||w||_2, k = 0..iters
                                         (AC_FORM_PAPER: only k = iters, the returned iterate) */
    double alpha[AC_MAX_STATS];       /* alpha_{k+1} used in iteration k                */
    double m[AC_MAX_STATS];           /* Algorithm 2's m_k (0 for other modes)          */
    double diff_last[AC_MAX_STATS];   /* ||u_L^{(k+1)} - u_L^{(k)}||_inf                 */
    int inner_iters[AC_MAX_STATS];    /* Krylov inner solver: max iterations over systems, per k */
    int inner_failed[AC_MAX_STATS];   /* Krylov inner solver: systems that stopped above tau, per k */
    double w_norm2;                   /* ||w||_2                                         */
    double w_inf;                     /* ||w||_inf                                       */
} ac_stats;

/* Shape and tuning facts of a plan. */
typedef struct {
    int N, M, L, F;                   /* F = L/2 + 1 stored time frequencies            */
    int tile_fwd, tile_upd;           /* grid points per CTA in the time kernels        */
    int spatial_path;                 /* 0: 1D one CTA per plane, 1: 2D one CTA per plane, 2: 2D three passes,
                                         3: BiCGStab, 4: GMRES; 5: 1D mixed-radix FFT (sizes that are not
                                         powers of two), one CTA per plane, 6: 2D mixed-radix three passes,
                                         7: 2D in one pass over a thread-block cluster               */
    long long workspace_bytes;        /* device memory owned by the plan               */
    long long launches;               /* kernels launched by this plan so far          */
    int update_kernel;                /* AC_UPDATE_TMA if the TMA-staged update kernel is in use
                                         (requested and applicable), else AC_UPDATE_PLAIN   */
    int update_tile_tma;              /* grid points per tile of the TMA-staged kernel (0 if unused) */
    int space_cluster;                /* spatial path 7: CTAs per cluster (else 0)      */
} ac_plan_info;

typedef struct ac_plan ac_plan;

/* ---- plan ---------------------------------------------------------------- */

/* Builds the host tables (Radau IIA nodes and Q of eq. (collocation), stencil
 * coefficients and symbols, FFT twiddles) and allocates the device workspace
 * (F*M*N complex plus small tables) on the current CUDA device.
 * M >= 1 (<= 4), L a power of two (2..1024) with L*M small enough for the
 * shared-memory time transform, dT > 0, a supported stencil scheme (see
 * ac_problem).  precision: AC_C128 or AC_C64.  inner: AC_INNER_FFT needs
 * nx (and ny) without prime factors above 7 and a 1D plane of at most 160 KB of
 * transform values (powers of two; 100 KB for other sizes, whose Stockham
 * transforms keep two copies); AC_INNER_BICGSTAB and AC_INNER_GMRES take any
 * grid with at least 2 * radius + 1 points per axis.  Writes *out.
 * Errors: AC_ERR_INVALID_ARG for unsupported sizes or schemes, AC_ERR_CUDA. */
int ac_setup(const ac_problem* prob, int M, int L, double dT,
             const ac_alpha_schedule* sched, int precision, int inner,
             ac_plan** out);

/* Frees the plan and its device memory.  NULL is ignored. */
void ac_destroy(ac_plan* plan);

int ac_plan_get_info(const ac_plan* plan, ac_plan_info* info);

/* ---- operators (eq. (globalsys)) ---------------------------------------- */

/* Cu = C u with C = I_L (x) C_coll + E (x) H, C_coll = I - dT Q (x) A, in FP64.
 * u, Cu: device, L*M*N doubles, must not overlap. */
int ac_apply_C(ac_plan* plan, const double* u, double* Cu, void* stream);

/* out = C^T lam (FP64).  lam, out: device, L*M*N doubles. */
int ac_apply_CT(ac_plan* plan, const double* lam, double* out, void* stream);

/* v_l = dT (Q (x) I_N) b_l for l = 0..L-1: the forcing part of the right-hand
 * side of eq. (collocation) / (seq_collocation_problem), from samples
 * bnodes[l][m][n] = b(T_l + dT t_m, x_n) of the forcing at the collocation
 * nodes of step l.  Pass v as the `b` argument of the solve calls.
 * bnodes, v: device, L*M*N doubles, distinct.  FP64. */
int ac_collocation_rhs(ac_plan* plan, const double* bnodes, double* v, void* stream);

/* ---- one preconditioner solve (Lemma 1, eqs. (s1)-(s3), Algorithm 1) ---- */

/* e = C_alpha^{-1} r with C_alpha = I_L (x) C_coll + E_alpha (x) H (eq. (prec)):
 * alpha-scaling along time, length-L FFT (eq. (s1)), node mixing with the
 * eigenbasis of Q G_l^{-1} (eq. (d1)), the shifted spatial solves of eq. (d2),
 * back-mixing with G_l^{-1} S_l (eqs. (d3), (Gsubstitution)), inverse FFT and
 * un-scaling (eq. (s3)).  0 < alpha < 1.  r, e: device, L*M*N doubles; r and e
 * may be the same buffer.  Runs in the plan's precision. */
int ac_precond_solve(ac_plan* plan, double alpha, const double* r, double* e,
                     void* stream);

/* ---- Richardson iteration (eq. (Riteration), correction form) ----------- */

/* One iteration u <- u + C_alpha^{-1} (w - C u) with w = (u0 stacked over the
 * M nodes in block 1) + b.  u0: device, N doubles (may be NULL = 0); b: device,
 * L*M*N doubles or NULL; u: device, in/out.  If res_rel_out is not NULL the
 * call synchronises and stores ||w - C u_in||_2 / ||w||_2 there (with
 * ||w||_2 as computed at this call).  No host synchronisation otherwise. */
int ac_richardson_step(ac_plan* plan, double alpha, const double* u0,
                       const double* b, double* u, double* res_rel_out,
                       void* stream);

/* The same iteration on HOST arrays: u0 (N doubles, may be NULL), b (L*M*N
 * doubles or NULL) and u (L*M*N doubles, in/out) live in host memory; the
 * result equals ac_richardson_step's on device copies of them, bit for bit.
 * The call copies u (and b) to the device and the new u back in `chunks`
 * chunks of grid points (0: 8; at most 32; fewer when a chunk would hold
 * less than twice the stencil's halo), overlapping the copies with the
 * residual and update kernels (eq. (Riteration)'s w - C u and u + e work
 * point by point, apart from the halo, whose points are copied ahead of the
 * chunk that needs them).  The copies overlap only from
 * page-locked host memory (cudaHostAlloc or cudaHostRegister); pageable
 * memory works but is copied synchronously.  The first call allocates the
 * plan's device copies of the arrays (L*M*N doubles each for u and b, N for
 * u0) and two copy streams.  Returns after queueing the work, without
 * waiting, unless res_rel_out is not NULL (as for ac_richardson_step); u is
 * complete once the work queued on `stream` so far has finished (for
 * example after cudaStreamSynchronize(stream)), and must not be touched by
 * the host before that.  Errors: AC_ERR_INVALID_ARG (null plan or u,
 * chunks < 0), AC_ERR_CUDA. */
int ac_richardson_step_host(ac_plan* plan, double alpha, const double* u0,
                            const double* b, double* u, int chunks,
                            double* res_rel_out, void* stream);

/* Full solve of C u = w by Richardson iterations with the plan's alpha
 * schedule (Algorithm 1 with Algorithm 2 or a fixed/mixed rule) and stop
 * rule; stops after at most sched.max_iter iterations.  If init_u is nonzero,
 * u holds the initial iterate on entry, else u^(0) = (u0, ..., u0) (Sec. 5).
 * tol: the stop tolerance of the plan's stop rule.  stats: host, may be NULL.
 * Returns AC_ERR_NO_CONVERGENCE if the rule was not met (u then holds the
 * last iterate). */
int ac_richardson_solve(ac_plan* plan, const double* u0, const double* b,
                        double* u, int init_u, double tol, ac_stats* stats,
                        void* stream);

/* Moving window (Sec. 5.2, parallel scaling runs): n_windows consecutive
 * all-at-once solves of L steps each; window w starts from the last node of
 * window w-1 (u0 for w = 0).  u_end: device, N doubles, receives the state at
 * the end of the last window.  work: device, L*M*N doubles (the window's
 * iterate).  b is not supported here (unforced problems).  stats (host, may be
 * NULL) receives the record of the last window; iters_total (host, may be
 * NULL) the sum of the windows' iteration counts.  Returns the first failing
 * window's status. */
int ac_window_solve(ac_plan* plan, const double* u0, int n_windows, double* u_end,
                    double* work, double tol, ac_stats* stats, int* iters_total,
                    void* stream);

/* Sequential collocation stepping, the baseline of Sec. 4.2 (T_Mpar): the
 * L steps of eq. (collocation) one after another, each solved by
 * diagonalising Q = S diag(lambda) S^{-1}: z = (S^{-1} x I)(1 x u_{l-1,M} + v_l),
 * the M shifted spatial solves (I - dT lambda_m A) z_m = z_m with the plan's
 * inner solver (in parallel over m), and u_l = Re (S x I) z.  It computes the
 * same u as ac_richardson_solve (the solution of eq. (globalsys)) without
 * iterating; in complex64 plans the solves carry complex64 rounding.
 * u0: device, N doubles.  b: device, L*M*N doubles (the collocation right-hand
 * side v of ac_collocation_rhs) or NULL.  u: device, L*M*N doubles, output,
 * distinct from u0 and b.  The L steps are captured once into a CUDA graph
 * per (u0, b, u) triple and replayed on `stream`; the Krylov inner solvers'
 * per-system status is not reported here.  Not thread-safe per plan. */
int ac_sequential_solve(ac_plan* plan, const double* u0, const double* b, double* u, void* stream);

/* Outer Krylov acceleration (the coupling the paper names as future work in
 * Sec. 6): flexible GMRES(m) on C u = w, right-preconditioned by C_alpha^{-1}
 * (the same preconditioner kernels as the Richardson iteration), FP64
 * vectors, classical Gram-Schmidt with one reorthogonalisation, restarted
 * every m = restart steps (<= 0: 10; at most 32) with the true residual
 * recomputed at each restart.  alpha: the plan's fixed alpha0 for
 * AC_ALPHA_FIXED, else the correction-form rule sqrt(L (3 eps + tau)).
 * Stops when ||w - C u||_2 <= tol ||w||_2 (true residual at a restart), or
 * after the plan's max_iter preconditioned steps (AC_ERR_NO_CONVERGENCE; u
 * holds the last iterate).  u0, b, u as in ac_richardson_solve (u0 may be
 * NULL only with init_u = 1 and b given).  stats: iters = preconditioned
 * steps; res_rel[k] = GMRES residual estimate after step k, replaced by the
 * true residual at each restart; alpha[k] = alpha.  Workspace: 2m + 2
 * space-time vectors, allocated on first use and kept by the plan. */
int ac_krylov_solve(ac_plan* plan, const double* u0, const double* b, double* u, int init_u, double tol,
                    int restart, ac_stats* stats, void* stream);

/* ---- adjoint (not in the paper; derived from eq. (globalsys)) ----------- */

/* lam = C^{-T} g.  Reversing the time index turns C^T into a system of the
 * same all-at-once form with Q -> Q^T, A -> A^T and H_M -> H_M^T, which the
 * same alpha-circulant kernels solve.  g, lam: device, L*M*N doubles, distinct.
 * lam^(0) = 0.  Same schedule and stop rule as the forward solve, with g in
 * the role of w. */
int ac_adjoint_solve(ac_plan* plan, const double* g, double* lam, double tol,
                     ac_stats* stats, void* stream);

/* Gradient contractions for a loss J(u) with C(theta) u = w(u0) and
 * lam = C^{-T} dJ/du:
 *   du0[n]        = sum_m lam[0][m][n]                         (device, N doubles)
 *   dparams[0]    = dJ/dnu = dT sum_l sum_{m,j} Q_mj lam_{l,m} . Lap u_{l,j}
 *   dparams[1..2] = dJ/dcx, dJ/dcy = -dT sum ... lam . D_{x,y} u     (host, 3 doubles)
 * u, lam: device, L*M*N doubles.  du0 may be NULL.  Synchronises once. */
int ac_grad_params(ac_plan* plan, const double* u, const double* lam,
                   double* du0, double* dparams, void* stream);

/* ---- preconditioner solve without device allocation --------------------- */

/* No counterpart in the paper.  e = C_alpha^{-1} r exactly as ac_precond_solve
 * computes it (the same kernels, tiles, spatial path and tables as a plan that
 * ac_setup builds for the same problem with AC_INNER_FFT), for callers that cannot
 * allocate device memory when they need a solve -- e.g. code whose device
 * memory is entirely owned by another framework's caching allocator, or a
 * latency-critical loop that must not pay for the implicit synchronisation of
 * cudaMalloc/cudaFree.  No plan is needed and nothing is allocated: every
 * buffer and table the solve uses is carved out of one fixed 32 MiB device
 * array inside this library, which each GPU that loads the library keeps
 * until the process exits.  The small tables (twiddles, symbols, eigenbases)
 * are uploaded on every call from pageable host memory, so the host waits
 * until the work queued before the call on `stream` has finished; the
 * kernels are then queued without further waits.
 *   prob, M, L, dT: as for ac_setup (FFT inner solve, grid sizes with prime
 *     factors 2, 3, 5, 7 only, L a power of two in 2..1024, M in 1..4);
 *     precision: AC_C128 or AC_C64.
 *   alpha in (0,1).  r, e: device, L*M*N doubles (may be the same buffer).
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls on a device share the array: calls whose GPU work may
 * overlap (other streams, other host threads) race and must be ordered by the
 * caller.  Problems whose buffers do not fit in 32 MiB are rejected with
 * AC_ERR_INVALID_ARG and a message naming the size needed (ac_last_error). */
int ac_precond_solve_noalloc(const ac_problem* prob, int M, int L, double dT,
                             double alpha, int precision, const double* r,
                             double* e, void* stream);

/* ---- host-side planner (no GPU needed) ---------------------------------- */

/* Radau IIA nodes 0 < t_1 < ... < t_M = 1 (roots of P_{M-1} + P_M mapped by
 * x = 1 - 2t, Sec. 2.3).  t: host, M doubles.  1 <= M <= 8. */
int ac_radau_nodes(int M, double* t);

/* Collocation matrix q_{mi} = int_0^{t_m} c_i(s) ds of eq. (collocation).
 * Q: host, M*M doubles, row-major. */
int ac_collocation_matrix(int M, double* Q);

/* Per-frequency tables used by the kernels for a given alpha (Lemma 1 and
 * eqs. (QGL), (d1)-(d3), Algorithm 1): for f = 0..L/2,
 *   d_f = -alpha^{1/L} exp(-2 pi i f / L),  G_f = I + d_f H_M  (H_M^T if transposed),
 *   B_f = Q G_f^{-1} (Q^T G_f^{-1} if transposed) = S_f diag(mu_f) S_f^{-1},
 *   Sinv_f = S_f^{-1},  P_f = G_f^{-1} S_f.
 * Outputs (host, interleaved re/im doubles): mu [F][M][2], Sinv [F][M][M][2],
 * P [F][M][M][2]; cond: host, F doubles (condition number of S_f), may be NULL.
 * Returns AC_ERR_NOT_DIAGONALIZABLE if some cond(S_f) > 1e10. */
int ac_freq_tables(int M, int L, double alpha, int transposed,
                   double* mu, double* Sinv, double* P, double* cond);

/* Per-axis stencil taps of A on the offsets -3..3 (index offset + 3), the
 * weights of the scheme above scaled by nu / h^2 and -c / h:  A u at grid
 * point (ix, iy) = sum_o tx[o+3] u(ix+o, iy) + ty[o+3] u(ix, iy+o).
 * tx, ty: host, 7 doubles each (ty zero in 1D).  rad: host int, the largest
 * |o| with a nonzero tap of either axis (may be NULL).  Returns
 * AC_ERR_INVALID_ARG for an unsupported scheme. */
int ac_stencil_taps(const ac_problem* prob, double* tx, double* ty, int* rad);

/* The launch shape ac_setup would choose for these arguments, computed on the
 * host without a GPU: out->N, M, L, F, tile_fwd, tile_upd, spatial_path and
 * space_cluster (the other fields are zero).  sched may be NULL (only its
 * space_cluster field is read).  A requested cluster (spatial path 7) is
 * reported as planned; ac_setup falls back to the three-pass solve, or fails
 * for an explicit request, when the device cannot hold the clusters.
 * Returns AC_ERR_INVALID_ARG for arguments ac_setup would reject (sizes,
 * schemes, a grid the chosen inner solver cannot take). */
int ac_plan_shape(const ac_problem* prob, int M, int L, int precision, int inner,
                  const ac_alpha_schedule* sched, ac_plan_info* out);

/* Algorithm 2's sequence: alphas[k] = alpha_{k+1}, ms[k] = m_k (ms[0] = m0),
 * k = 0..n-1 (ms has n+1 entries). */
int ac_alpha_sequence(double m0, double gamma, int n, double* alphas, double* ms);

/* ---- instrumentation ---------------------------------------------------- */

/* Per-kernel CUDA-event timing inside the library (on the stream each kernel
 * is launched on).  on = 1 enables and zeroes the accumulators. */
int ac_profile_enable(ac_plan* plan, int on);
/* names: up to `cap` kernels; for each: accumulated milliseconds, launch count.
 * Synchronises the device.  Returns the number of kernel kinds. */
int ac_profile_read(ac_plan* plan, int cap, const char** names, double* ms,
                    long long* count);

/* FP64 FMA throughput of the current device, measured with a kernel of
 * independent register-operand FMA chains (8 per thread, 8 CTAs of 256
 * threads per SM), best of three CUDA-event timed launches.  Writes FMAs per
 * second to *fma_per_s (host).  Instrumentation for the roofline of the
 * FP64-bound kernels; no counterpart in the paper.  Allocates and frees a
 * few bytes of device memory and synchronises the stream. */
int ac_measure_fp64_fma_rate(double* fma_per_s, void* stream);

const char* ac_status_string(int status);
const char* ac_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ALPHACIRC_H */
