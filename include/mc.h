/*
 * mc.h -- C ABI of the GB300 (sm_103a) decoupled multicontinuum solver.
 *
 * Method: Vasilyeva, "Efficient decoupling schemes for multiscale
 * multicontinuum problems in fractured porous media" (arXiv 2209.01158).
 *
 *   Model (Section 2, Eq. mm, mm-bc): L pressures p_a on the unit square,
 *     c_a dp_a/dt - div(k_a grad p_a) + sum_{b != a} sigma_ab (p_a - p_b) = f_a,
 *     zero-flux boundaries.
 *   Space (Section 3.1, Eqs. app-md, app, app-mc): two-point-flux finite
 *     volumes on an nx x ny grid of square cells, h = 1/nx:
 *       M_a = diag(c_a h^2), D_a: a_ii = sum_n T_in, a_ij = -T_ij with
 *       T_ij = k_face |E|/d = k_face (harmonic mean of the two cells),
 *       Q_ab = diag(sigma_ab,i h^2) (co-located continua), F_a cell-integrated.
 *   Time (Section 3.2-3.3): coupled backward Euler (Eq. ct-mc) or the
 *     decoupled D-, L-, U-schemes (Eq. si-mc): each continuum solves
 *       (M_a/tau + D_a + sum_b Q_ab) p_a^n
 *           = M_a/tau p_a^{n-1} + F_a + sum_b Q_ab p_b^{n-1 or n}.
 *   Coarse scale (Section 4): NLMC basis (Eq. eq:basis), A_bar = R A R^T,
 *     coupled (Eq. is-nlmc) and decoupled (Eq. si-nlmc) coarse stepping.
 *
 * Every linear system is solved on the GPU by matrix-free preconditioned
 * conjugate gradients on the 5-point stencil, all continua of a step in one
 * persistent kernel launch.
 *
 * Conventions for every call:
 *   - Field arrays are nx*ny doubles, cell (i, j) at index j*nx + i (x fastest).
 *   - Host arrays passed in are copied during the call; the caller keeps them.
 *   - Outputs go to caller-provided host buffers unless stated otherwise.
 *   - Every call returns mc_status; no call throws or aborts. On failure the
 *     context keeps its previous state where stated, and mc_last_error() gives
 *     a one-line explanation.
 *   - A context is bound to the CUDA device current at mc_setup and to one
 *     stream; calls on one context must not run concurrently from two threads.
 *   - All work is queued on the context's stream; calls that return host data
 *     synchronise that stream.
 */
#ifndef MC_H
#define MC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MC_MAX_CONTINUA 4

typedef struct mc_ctx mc_ctx;
typedef struct mc_nlmc mc_nlmc;
typedef struct mc_batch mc_batch;

typedef enum {
  MC_OK = 0,
  MC_E_ARG = 1,        /* invalid argument (sizes, NULL, NaN/negative data) */
  MC_E_ALLOC = 2,      /* device or host allocation failed */
  MC_E_CUDA = 3,       /* a CUDA runtime call failed */
  MC_E_NOCONV = 4,     /* a solve hit max_iter before rtol */
  MC_E_TIMEOUT = 5,    /* a device grid barrier exceeded its spin limit */
  MC_E_STATE = 6,      /* call not valid in the current state */
  MC_E_BREAKDOWN = 7   /* PCG breakdown: (p, A p) <= 0 or not finite */
} mc_status;

typedef struct {
  int32_t nx, ny;      /* cells along x and y; h = 1/nx (square cells) */
} mc_grid;

enum { MC_PREC_FP64 = 0, MC_PREC_FP32_IR = 1, MC_PREC_BF16T_IR = 2 };
/* Preconditioners of the FP64 PCG. MC_PRECOND_TWO_LEVEL (FP64 schemes
   only) adds to Jacobi a Galerkin coarse correction on the 64 x 16 stencil
   tiles, M^-1 = D^-1 + P (P^T A P)^-1 P^T with P the tile indicators; its
   dense inverse is formed on the device at the first step (at most
   MC_TWO_LEVEL_MAX_TILES tiles per continuum, else MC_E_ARG). The coupled
   scheme takes the coarse space P = blockdiag(P_a) with the Galerkin operator
   of the coupled matrix, exchange blocks included: M^-1 = D^-1 +
   P (P^T A P)^-1 P^T, an (L nc)^2 dense inverse (L nc at most
   MC_TWO_LEVEL_MAX_COUPLED, else MC_E_ARG). It changes only the Krylov
   iteration, not the system solved. */
enum { MC_PRECOND_JACOBI = 0, MC_PRECOND_TWO_LEVEL = 1 };
#define MC_TWO_LEVEL_MAX_TILES 2048
#define MC_TWO_LEVEL_MAX_COUPLED 4096
/* Inner FP32 PCG of the IR forms: single-reduction (Chronopoulos-Gear)
   recurrences, one grid-wide reduction per iteration, or the textbook
   (Hestenes-Stiefel) recurrences with two. Both are the Jacobi PCG of
   Section 3.3's per-continuum systems in exact arithmetic. */
enum { MC_INNER_SINGLE_REDUCTION = 0, MC_INNER_TWO_REDUCTIONS = 1 };
/* Iteration of the FP64 Jacobi PCG (decoupled and coupled schemes). Both run
   CG on the symmetrically scaled system S^-1 A S^-1, S = diag(sqrt(d)), which
   is Jacobi PCG on A iterate for iterate. MC_FP64_TWO_PASS: a stencil pass and
   a pointwise pass per iteration, two grid reductions (textbook recurrences);
   MC_FP64_SINGLE_PASS: one tile pass and one grid reduction (Chronopoulos-Gear
   recurrences). */
enum { MC_FP64_TWO_PASS = 0, MC_FP64_SINGLE_PASS = 1 };
enum { MC_SCHEME_COUPLED = -1, MC_SCHEME_D = 0, MC_SCHEME_L = 1, MC_SCHEME_U = 2 };

typedef struct {
  int32_t precision;   /* MC_PREC_*: FP64 PCG, or FP32 / BF16-transmissibility
                          inner PCG inside FP64 iterative refinement */
  int32_t precond;     /* MC_PRECOND_JACOBI or MC_PRECOND_TWO_LEVEL */
  int32_t max_iter;    /* PCG iterations per solve (IR forms: cap of each inner
                          solve, further limited to 16 max(nx, ny) within
                          [2048, 16384]; an inner solve also stops when its
                          smallest residual norm fails to halve within 2048
                          iterations) */
  int32_t ir_max;      /* maximum refinement sweeps per solve (IR forms) */
  double rtol;         /* stop when ||b - A x||_2 <= rtol ||b||_2 (FP64). IR
                          forms also stop at the floor of refinement (an inner
                          solve met inner_rtol but the sweep did not halve
                          ||r||) when that floor is within 1e3 rtol ||b|| or
                          the last correction was below 100 rtol ||x||;
                          rel_residual reports what was met */
  double inner_rtol;   /* inner PCG relative residual target of each IR sweep
                          (default 1e-3) */
  int64_t spin_limit;  /* polls of a grid barrier before MC_E_TIMEOUT */
  int32_t blocks;      /* persistent CTAs (0: one per SM x occupancy) */
  int32_t threads;     /* threads per CTA of the FP64 step kernels (0: default 256; any other value is MC_E_ARG) */
  int32_t inner_form;  /* MC_INNER_* (IR forms; default single reduction) */
  int32_t fp64_form;   /* MC_FP64_* iteration of the FP64 Jacobi PCG (default
                          two passes) */
} mc_opts;

typedef struct {
  int32_t steps_done;                    /* steps completed by the call */
  int32_t status;                        /* mc_status of the device run */
  int64_t iters[MC_MAX_CONTINUA];        /* PCG iterations summed over the
                                            call's steps (coupled: iters[0]) */
  int32_t max_iters[MC_MAX_CONTINUA];    /* largest single-solve count */
  int32_t ir_sweeps;                     /* refinement sweeps summed (IR) */
  int32_t reserved;
  double rel_residual[MC_MAX_CONTINUA];  /* ||r||/||b|| of the last solve */
  double mass_defect;                    /* last step: |LHS - RHS| / scale of
                                            the scheme's mass identity */
} mc_stats;

/* Fill *o with the defaults (FP64, Jacobi, rtol 1e-12, max_iter 100000). */
mc_status mc_default_opts(mc_opts* o);

/*
 * mc_setup -- build a context: coefficients and state on the device.
 *   g          grid (nx, ny >= 1).
 *   L          number of continua, 1..MC_MAX_CONTINUA.
 *   k          L host arrays of nx*ny permeabilities (>= 0, finite).
 *   c          L values c_a > 0 (Eq. mm; M_a = c_a h^2).
 *   sigma      L*L row-major symmetric exchange coefficients per unit area
 *              (diagonal ignored), or NULL for none.
 *   sigma_cell L*(L-1)/2 host pointers, one per pair (a < b) in the order
 *              (0,1),(0,2),..,(0,L-1),(1,2),..; each NULL or nx*ny per-cell
 *              values that replace sigma[a][b] for that pair. May be NULL.
 *   tau        time step > 0.
 *   opts       NULL for defaults.
 *   stream     cudaStream_t to queue all work on (NULL: legacy default).
 * The state p starts at 0 and the sources at 0.
 * Section 3.1: T_ij, a_ij, m, q entries; Section 3.3: diagonal of
 * M_a/tau + A0_aa used by the Jacobi preconditioner.
 */
mc_status mc_setup(const mc_grid* g, int32_t L, const double* const* k,
                   const double* c, const double* sigma,
                   const double* const* sigma_cell, double tau,
                   const mc_opts* opts, void* stream, mc_ctx** out);

/* Replace opts (precision, tolerances, launch shape) of a live context. */
mc_status mc_set_opts(mc_ctx* ctx, const mc_opts* opts);

/* F_a (cell-integrated source, Eq. app-mc: F = f |cell|), host nx*ny. */
mc_status mc_set_source(mc_ctx* ctx, int32_t alpha, const double* F);

/*
 * mc_set_well -- implicit well term of continuum alpha. Section 5 drives its
 *   experiments by a well source q_w (p - p_w) in the fracture cells of two
 *   small regions; it is read here as the relaxation q_w (p_w - p) toward the
 *   well pressure (the dissipative sign) and taken implicitly in p, which
 *   adds W = q_w |cell| to the diagonal of continuum alpha's own block and
 *   W p_w to its right-hand side, in every scheme and precision form.
 *   W   host nx*ny cell-integrated well indices (>= 0, finite; 0 outside the
 *       wells), or NULL to remove the wells of alpha.
 *   pw  host nx*ny well pressures (finite); ignored when W is NULL.
 *   The arrays are copied. The NLMC coarse model built on the context takes
 *   the wells it has at build time; a batch sees the wells its contexts had
 *   when mc_batch_create ran. MC_E_ARG on a bad alpha or data.
 */
mc_status mc_set_well(mc_ctx* ctx, int32_t alpha, const double* W, const double* pw);

/* Copy L host arrays into the state p^n. */
mc_status mc_set_state(mc_ctx* ctx, const double* const* p);

/* Copy the state p^n into L host arrays. Synchronises the stream. */
mc_status mc_get_state(mc_ctx* ctx, double* const* p);

/* Device pointer of continuum alpha's state (nx*ny doubles, owned by the
 * context, valid until mc_destroy). Lets a caller keep inputs resident. */
mc_status mc_state_device(mc_ctx* ctx, int32_t alpha, double** dev);

/*
 * mc_step_decoupled -- nsteps steps of the D- (Eq. si-mc, Section 3.3),
 * L- or U-scheme (A0 lower / upper block triangular; continua solved in
 * index / reverse index order, index order = ascending permeability).
 * D-scheme: every continuum's right-hand side
 *   M_a/tau p_a^{n-1} + F_a + sum_b Q_ab p_b^{n-1}
 * is assembled in one fused pass and all L solves run concurrently.
 * Whole call is one persistent kernel launch. On MC_E_NOCONV / MC_E_BREAKDOWN
 * / MC_E_TIMEOUT the state holds the last completed step (steps_done).
 * stats may be NULL. Synchronises the stream.
 */
mc_status mc_step_decoupled(mc_ctx* ctx, int32_t scheme, int32_t nsteps,
                            mc_stats* stats);

/*
 * mc_step_coupled -- nsteps steps of backward Euler on the full coupled
 * system (M/tau + D + Q) p^n = M/tau p^{n-1} + F (Eq. ct-mc, Section 3.2),
 * one PCG over all L*nx*ny unknowns per step. Same error contract as
 * mc_step_decoupled.
 */
mc_status mc_step_coupled(mc_ctx* ctx, int32_t nsteps, mc_stats* stats);

/*
 * mc_get_coefficients -- copy the device coefficients of continuum alpha:
 * TE[j*nx+i] (face to (i+1,j), 0 on the last column), TN[j*nx+i] (face to
 * (i,j+1), 0 on the last row), diag = c h^2/tau + sum_b q_ab + sum_faces T
 * (diagonal of M_a/tau + A0_aa). Any output pointer may be NULL.
 */
mc_status mc_get_coefficients(mc_ctx* ctx, int32_t alpha, double* TE,
                              double* TN, double* diag);

/* Apply the operator of one step to L host vectors x: y_a = (M_a/tau +
 * D_a + sum_b Q_ab) x_a for the decoupled schemes (scheme >= 0), or
 * y = (M/tau + D + Q) x over all continua (MC_SCHEME_COUPLED). */
mc_status mc_apply(mc_ctx* ctx, int32_t scheme, const double* const* x,
                   double* const* y);

/* D-scheme right-hand sides of the current state into L host arrays:
 * b_a = M_a/tau p_a + F_a (+ W_a p_w,a) + sum_b Q_ab p_b. */
mc_status mc_rhs_decoupled(mc_ctx* ctx, double* const* b);

/* Bytes of device memory the context holds. */
mc_status mc_device_bytes(const mc_ctx* ctx, int64_t* bytes);

/* ---------------- NLMC coarse model (Section 4) ---------------------------
 *
 * mc_nlmc_build -- multiscale basis and coarse operator for a context whose
 * grid divides into ncx x ncy coarse blocks (nx % ncx == ny % ncy == 0).
 *   Basis (Section 4.1, Eq. eq:basis): for every coarse block K_i and
 *   continuum beta, psi^{i,beta} on K_i^+ = K_i grown by `layers` coarse
 *   layers (clipped to the domain) minimises the energy of the coupled fine
 *   operator D + Q on K_i^+ with zero Dirichlet data on the part of its
 *   boundary inside the domain (ghost at h/2, T = 2k) subject to
 *   mean_{K_j}(psi_alpha) = delta_ij delta_alpha,beta for every K_j in K_i^+.
 *   Solved by projected Jacobi-PCG in the constraint null space to a
 *   preconditioned-residual reduction basis_rtol (at most basis_max_iter
 *   iterations; MC_E_NOCONV otherwise).
 *   Coarse operator: A_bar = R (D + Q) R^T; M_bar = diag(c_a |K_i|);
 *   F_bar = block sums of the context's current sources; wells of the
 *   context (mc_set_well) enter as W_bar = diag(block sums of W) and the
 *   right-hand side block sums of W p_w (the coarse finite-volume form of
 *   Section 4.1 for piecewise-constant data); the coarse state starts as the
 *   block means of the context's current state.
 * Coarse index (alpha, i) -> alpha * ncx*ncy + i, i = J*ncx + I.
 * The context must outlive the returned object. Same as mc_nlmc_build_ex
 * with support NULL and flags 0.
 */
mc_status mc_nlmc_build(mc_ctx* ctx, int32_t ncx, int32_t ncy, int32_t layers,
                        double basis_rtol, int32_t basis_max_iter, mc_nlmc** out);

/* Conservative coarse operator: after A_bar = R (D + Q) R^T, every diagonal
 * entry is set to minus the sum of the other entries of its row, so that
 * A_bar 1 = 0 and the coarse model conserves mass like the fine finite-volume
 * one. The exact (globally oversampled) basis reproduces constants and has
 * this property; local oversampling truncates the basis functions and breaks
 * it, and with very permeable fractures the defect outweighs the coarse mass
 * term (a constant state drifts). */
#define MC_NLMC_CONSERVATIVE 1

/*
 * mc_nlmc_build_ex -- mc_nlmc_build for continua that live on part of the
 *   domain (Section 4.1: the constraint of continuum alpha averages over
 *   K_j^alpha = Omega_alpha ∩ K_j).
 *   support  NULL (every continuum covers the domain), or L host pointers,
 *            each NULL (that continuum covers the domain) or nx*ny bytes,
 *            nonzero on the cells of Omega_alpha (an embedded fracture
 *            continuum: the cells its fractures cross). Copied.
 *   flags    0 or MC_NLMC_CONSERVATIVE.
 *   With a support mask, the mean constraints, M_bar = diag(c_a |K_i^alpha|),
 *   the coarse wells and the initial coarse state (means of p_alpha) run over
 *   K_i^alpha; cells of continuum alpha outside Omega_alpha are unconstrained
 *   in every basis function. A block with no cell of Omega_alpha has no coarse
 *   unknown of continuum alpha: no basis function, zero rows and columns of
 *   A_bar, M_bar = F_bar = 0, and its entry of the coarse state is held at 0
 *   by every coarse step (mc_nlmc_active lists the unknowns that exist). The
 *   coarse layout stays L * ncx * ncy.
 */
mc_status mc_nlmc_build_ex(mc_ctx* ctx, int32_t ncx, int32_t ncy, int32_t layers,
                           double basis_rtol, int32_t basis_max_iter,
                           const uint8_t* const* support, int32_t flags, mc_nlmc** out);

/* active[k] = 1 where coarse unknown k (L * ncx * ncy, host bytes) exists,
 * 0 where its block holds no cell of that continuum's support. */
mc_status mc_nlmc_active(mc_nlmc* m, uint8_t* active);

/* nsteps coarse steps: MC_SCHEME_COUPLED (Eq. is-nlmc) or the D-, L-,
 * U-schemes of Section 4.3 (A0_bar = diagonal / lower / upper blocks of
 * A_bar), with the coarse wells implicit in every scheme (like the fine
 * ones). Each coarse solve: explicit inverse (formed once) + one residual
 * correction. stats: steps_done, status. */
mc_status mc_nlmc_step(mc_nlmc* m, int32_t scheme, int32_t nsteps, mc_stats* stats);

/* Coarse state, L * ncx * ncy doubles (host). */
mc_status mc_nlmc_set_state(mc_nlmc* m, const double* pbar);
mc_status mc_nlmc_get_state(mc_nlmc* m, double* pbar);

/* A_bar ((L Nc)^2 row-major), M_bar and F_bar (L Nc each); any may be NULL. */
mc_status mc_nlmc_get_operator(mc_nlmc* m, double* Abar, double* mbar, double* fbar);

/* psi^{block,beta} as L fine fields (L * nx * ny host doubles, zero outside
 * the oversampled region). */
mc_status mc_nlmc_get_basis(mc_nlmc* m, int32_t block, int32_t beta, double* psi);

/* info[0..4] = Nc, L, total basis PCG iterations, largest basis iteration
 * count, device bytes held. */
mc_status mc_nlmc_info(const mc_nlmc* m, int64_t* info);

void mc_nlmc_destroy(mc_nlmc* m);

/* ---------------- Batched precision form -------------------------------------
 *
 * Many independent problems (instances) of uneven grid sizes and numbers of
 * continua stepped together by the D-, L- or U-scheme of Section 3.3 in the
 * precision form (FP32 or BF16-transmissibility inner PCG inside FP64
 * iterative refinement, exactly as mc_step_decoupled with that precision).
 * Each time step of the whole batch is ONE persistent kernel launch: the
 * co-resident CTAs form teams of `team` CTAs, and each team takes instances
 * (largest first) from a shared counter and solves them with team-wide
 * barriers. The launches of one mc_batch_step call are captured into a CUDA
 * graph on first use and replayed by later calls with the same scheme,
 * nsteps and team size.
 *
 * mc_batch_create -- group n contexts (from mc_setup, all on one device)
 *   into a batch. The contexts stay owned by the caller and must outlive the
 *   batch; their sources and state are read and written through the usual
 *   calls (mc_set_source, mc_set_state, mc_get_state), which may be issued
 *   between batch calls. opts: precision MC_PREC_FP32_IR or MC_PREC_BF16T_IR
 *   (else MC_E_ARG), rtol, inner_rtol, max_iter, ir_max, spin_limit apply to
 *   every instance (the contexts' own opts are not used by the batch);
 *   opts->blocks caps the CTAs of the launch (0: all co-resident). The team
 *   size starts at a heuristic (the smallest power of two for which the
 *   largest instance's share of the work fits one team's share of the GPU).
 *   Allocates the members' FP32 work vectors if they have none.
 */
mc_status mc_batch_create(mc_ctx* const* ctxs, int32_t n, const mc_opts* opts,
                          mc_batch** out);

/* CTAs per team, 1..(CTAs of the launch); MC_E_ARG otherwise. */
mc_status mc_batch_set_team(mc_batch* b, int32_t team);

/*
 * mc_batch_step -- nsteps steps of every instance (scheme MC_SCHEME_D, _L
 *   or _U). Per instance and continuum the solve stops on the FP64 residual
 *   test ||b - A x|| <= rtol ||b|| (or the refinement floor, see mc_opts).
 *   An instance whose FP32 refinement fails (MC_E_NOCONV after ir_max
 *   sweeps; on fracture continua at 1024^2 FP32 Jacobi-PCG cannot sustain
 *   the long Krylov runs the problem needs) is put back to the start of
 *   that step inside the launch; after the batched launches the host steps
 *   it through the rest of the call with the FP64 PCG path
 *   (mc_step_decoupled, same rtol and max_iter), and it stays on that path
 *   for later calls (count in mc_batch_info). An instance that fails there
 *   too keeps the start of its failed step. A barrier timeout stops the
 *   whole call (MC_E_TIMEOUT) with every instance at the end of its last
 *   completed step. Returns the status of the first failed instance (index
 *   order); `total` (may be NULL) gets the minimum steps_done, that status,
 *   iteration and sweep counts summed over the instances (max_iters: the
 *   maximum). Synchronises.
 */
mc_status mc_batch_step(mc_batch* b, int32_t scheme, int32_t nsteps, mc_stats* total);

/* Statistics of instance i from the last mc_batch_step: steps_done, status,
 * iters, max_iters, ir_sweeps, rel_residual of the last solve (mass_defect
 * is 0). */
mc_status mc_batch_instance_stats(mc_batch* b, int32_t i, mc_stats* s);

/*
 * mc_batch_autotune -- choose the team size by timing one batched step per
 *   candidate (after one untimed step), with CUDA events; every trial step is
 *   undone, so the instances' states are unchanged. candidates: ncand team
 *   sizes, or NULL for 1, 2, 4, ... up to the CTAs of the launch. ms (may be
 *   NULL): ncand times in milliseconds (-1 when not timed). cache_path (may be
 *   NULL): a JSON file mapping a key (device, precision, scheme, CTAs, and the
 *   batch's sorted list of instance shapes) to the chosen team size; a hit
 *   skips the timing, a miss appends the result. The chosen size is kept for
 *   later mc_batch_step calls and returned in *best_team (may be NULL).
 */
mc_status mc_batch_autotune(mc_batch* b, int32_t scheme, const int32_t* candidates,
                            int32_t ncand, const char* cache_path, int32_t* best_team,
                            double* ms);

/* info[0..8] = instances, team size, teams, CTAs per launch, whether the last
 * step ran as a graph replay (1/0), whether the team size came from the tuner
 * cache (1/0), continuum cells summed over the instances, device bytes held
 * by the batch itself, instances handed to the FP64 path. */
mc_status mc_batch_info(const mc_batch* b, int64_t* info);

/* Last error text of b (or of the last failed mc_batch_create when NULL). */
const char* mc_batch_last_error(const mc_batch* b);

void mc_batch_destroy(mc_batch* b);

/*
 * mc_step_single_noalloc -- nsteps backward-Euler steps of ONE continuum,
 *   (M/tau + D) p^n = M/tau p^{n-1} + F   (no exchange; h = 1/nx),
 * for callers that cannot allocate device memory. The paper has no
 * counterpart: this is a deployment variant of mc_step_decoupled with L = 1.
 *
 * Who needs it: code that runs where a cudaMalloc is not allowed or not
 * affordable -- inside a framework whose caching allocator owns the device
 * memory, in a long-running service whose memory budget is fixed at start-up,
 * or in a latency-bound loop where cudaMalloc/cudaFree (which can synchronise
 * the device) must not appear. Such a caller owns its input and output
 * buffers and only wants the solver's own scratch to come from somewhere.
 *
 * This entry point creates no context and calls no cudaMalloc, cudaFree or
 * other allocating routine. All of its scratch (pitched copies of the fields,
 * transmissibilities, PCG vectors, partial sums, barrier words, statistics)
 * lives in one fixed device array of the library, about 6 MB, which every
 * GPU that loads the library holds until the process exits.
 *
 *   nx, ny    grid; ny * (nx rounded up to 16) must be <= 65536 cells
 *             (e.g. 256 x 256), else MC_E_ARG.
 *   k         DEVICE pointer, nx*ny permeabilities (row-major, x fastest),
 *             finite and >= 0; read only.
 *   c, tau    c > 0 (M = c h^2), time step tau > 0.
 *   F         DEVICE pointer, nx*ny cell-integrated sources; read only.
 *   p         DEVICE pointer, nx*ny state: read as p^0, overwritten with the
 *             state after the last completed step (on MC_E_NOCONV,
 *             MC_E_BREAKDOWN or MC_E_TIMEOUT: the start of the failed step).
 *   rtol, max_iter  PCG stop ||r|| <= rtol ||b|| per step, iteration cap.
 *   stream    cudaStream_t (NULL: legacy default); the call synchronises it.
 *   stats     host, may be NULL: iters[0], max_iters[0], rel_residual[0],
 *             steps_done, status, mass_defect.
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture. Every call shares the one array and starts by zeroing it, so two
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race and corrupt each other: serialise them.
 */
mc_status mc_step_single_noalloc(int32_t nx, int32_t ny, const double* k, double c,
                                 double tau, const double* F, double* p, int32_t nsteps,
                                 double rtol, int32_t max_iter, void* stream,
                                 mc_stats* stats);

/* ---------------- Lower-dimensional fracture continuum ---------------------
 *
 * A fracture continuum on its own 1-D mesh, coupled to the context's matrix
 * continua (Section 2, Eqs. mm-md and mm-tc: the matrix on the square, the
 * fracture on the segments; Section 3.1, Eqs. app-md and app-tc).
 *   Mesh: every segment is clipped to the unit square and split at the grid
 *   lines it crosses and at its crossings with the other segments; each piece
 *   iota_l (length |iota_l|) is a fracture cell hosted by the matrix cell that
 *   holds its midpoint. Pieces meeting at a point (a split point, a crossing)
 *   are coupled pairwise by T_ln = t_l t_n / sum_m t_m, t_l = kf / (|iota_l|/2)
 *   (two pieces: the two-point value kf / (d_l + d_n)); free segment ends carry
 *   no flux. Mass cf |iota_l|; exchange with matrix continuum a
 *   q_al = sigma_f[a] |iota_l| / (h/4) (Eq. app-md: sigma |E| / d with the
 *   piece as interface and d = h/4).
 *   Unknowns: the context's L matrix continua (state: mc_get_state) and P
 *   pieces in segment order, pieces along each segment from its first end.
 *   Schemes (mc_frac_step): coupled backward Euler over all matrix cells and
 *   pieces (Eq. ct-mc), or the D-, L-, U-schemes of Section 3.3 with the
 *   fracture as the last (most permeable) continuum: the matrix continua are
 *   stepped by the FP64 step kernel with the exchange as an implicit diagonal
 *   term and a right-hand side from p_f, the fracture by a one-CTA PCG on its
 *   graph.
 *
 * mc_frac_create -- attach a fracture network to ctx (FP64, Jacobi opts;
 *   nx == ny; L <= MC_MAX_CONTINUA - 1).
 *   seg      nseg * 4 host doubles (x0, y0, x1, y1) per segment, any extent.
 *   kf, cf   fracture permeability and capacity (> 0).
 *   sigma_f  L values >= 0: exchange coefficient with each matrix continuum.
 *   The matrix wells the context has now are kept (mc_set_well after create
 *   is not seen). The fracture state and sources start at 0. MC_E_ARG when no
 *   segment crosses the domain. The context must outlive the object.
 */
typedef struct mc_frac mc_frac;
mc_status mc_frac_create(mc_ctx* ctx, int32_t nseg, const double* seg, double kf, double cf,
                         const double* sigma_f, mc_frac** out);

/* info[0..4] = pieces P, junctions, graph entries, hosting matrix cells,
 * device bytes held. */
mc_status mc_frac_info(const mc_frac* f, int64_t* info);

/* Geometry of the pieces: len (P), mid (2P: x, y), host (P: j*nx + i); any
 * pointer may be NULL. */
mc_status mc_frac_pieces(const mc_frac* f, double* len, double* mid, int32_t* host);

/* Cell-integrated fracture sources per piece (P host doubles). */
mc_status mc_frac_set_source(mc_frac* f, const double* Ff);

/* Implicit fracture wells W (p_w - p) per piece (W >= 0: index x length),
 * or Wf = NULL to remove them; rebuilds the fracture coefficients. */
mc_status mc_frac_set_well(mc_frac* f, const double* Wf, const double* pwf);

/* State: pm = L host arrays of nx*ny (or NULL to leave the matrix), pf = P
 * host doubles (or NULL). */
mc_status mc_frac_set_state(mc_frac* f, const double* const* pm, const double* pf);
mc_status mc_frac_get_state(mc_frac* f, double* const* pm, double* pf);

/* nsteps steps of MC_SCHEME_COUPLED / _D / _L / _U. stats: iters[a] and
 * max_iters[a] for the matrix continua, iters[L] for the fracture (coupled:
 * iters[0]), rel_residual likewise, steps_done. On failure both the matrix
 * and the fracture state hold the start of the failed step. */
mc_status mc_frac_step(mc_frac* f, int32_t scheme, int32_t nsteps, mc_stats* stats);

void mc_frac_destroy(mc_frac* f);

/*
 * mc_fp64_fma_rate -- measurement utility (the paper has no counterpart):
 *   the FP64 fused-multiply-add throughput of the current device in
 *   TFLOP/s (2 FLOP per FMA), from a register-only kernel of independent FMA
 *   chains on every SM, timed with CUDA events on `stream` (NULL: legacy
 *   default) after one warm-up launch. It is the denominator of the FP64
 *   step kernel's roofline. Allocates and frees a small output buffer on the
 *   stream; synchronises it.
 */
mc_status mc_fp64_fma_rate(void* stream, double* tflops);

void mc_destroy(mc_ctx* ctx);

/* Last error text of ctx (or of the last failed mc_setup when ctx is NULL). */
const char* mc_last_error(const mc_ctx* ctx);
const char* mc_status_string(mc_status s);

#ifdef __cplusplus
}
#endif

#endif /* MC_H */
