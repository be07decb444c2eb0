/*
 * gea.h -- C ABI of the GB300 (sm_103a) library that advances the dry
 * compressible Euler equations with the pressure-based finite-volume scheme
 * of Girfoglio, Quaini & Rozza, "GEA: a new finite volume-based open source
 * code for the numerical simulation of atmospheric and ocean flows"
 * (arXiv 2303.10499).
 *
 * One time step is the three-step split of Section 3 on a uniform Cartesian
 * x-z grid with free-slip walls (Section 4):
 *   Step 1  continuity predictor (eq. e1_d), implicit momentum predictor
 *           (eq. step2_sd, first line) and K^{n+1/3} (eq. step1_3sd);
 *   Step 2  implicit enthalpy equation (eq. step3_sd), temperature update
 *           (eq. step3_2sd) and rho^{n+2/3} (eq. step3_3sd);
 *   Step 3  PISO correctors: momentum corrector (eq. step2_sd, second line)
 *           and the compressible pressure equation (eq. p_prime_sd) in its
 *           Helmholtz form, solved by multigrid-preconditioned conjugate
 *           gradients, then p, K and rho^{n+1} (eq. step4_4sd).
 * Every stage runs in this library's CUDA kernels on one GPU, in FP64.
 *
 * Conventions
 *  - Cell fields are nz rows of nx values, x fastest (row-major, index
 *    k*nx + i for cell (i,k) centred at ((i+1/2) dx, (k+1/2) dz)).
 *  - phix holds the mass fluxes phi_j = (rho u)_j . A_j (kg/s per unit depth)
 *    through the nx+1 x-faces of each row: nz rows of nx+1 values, face f
 *    between cells f-1 and f; phiz holds the z-face fluxes: nz+1 rows of nx
 *    values, face f between rows f-1 and f. Wall faces carry zero.
 *  - Pressure split p = p' - rho g z with g > 0 and z up (the force in the
 *    momentum equation is grad p' - g z grad rho).
 *  - All calls are ordered on the context's stream (gea_set_stream). Calls
 *    that take host buffers return after the copies are complete.
 *  - Functions return GEA_OK (0) or one of the GEA_ERR_* codes;
 *    gea_last_error() gives a message for the last failure on a context.
 *  - One context must not be used from two host threads at once. Contexts
 *    are independent; the library keeps no global mutable state.
 */
#ifndef GEA_H
#define GEA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GEA_OK = 0,
    GEA_ERR_INVAL = 1,      /* bad argument: sizes, constants, null pointers */
    GEA_ERR_NOMEM = 2,      /* device allocation failed */
    GEA_ERR_CUDA = 3,       /* a CUDA runtime call failed */
    GEA_ERR_NOCONV = 4,     /* a linear solve reached its iteration cap */
    GEA_ERR_NONFINITE = 5,  /* NaN or Inf in a residual norm */
    GEA_ERR_STATE = 6,      /* no state has been set yet */
    GEA_ERR_TIMEOUT = 7     /* a device-side wait gave up (never expected) */
};

enum { GEA_STATE_CONSERVATIVE = 0, GEA_STATE_FULL = 1 };
enum { GEA_FLAG_GRAPH = 1, GEA_FLAG_MIXED = 2, GEA_FLAG_KEEP_R0 = 4, GEA_FLAG_DEBUG_PADS = 8 };
enum { GEA_MEM_HOST = 0, GEA_MEM_DEVICE = 1 };

/* Uniform Cartesian grid: nx * nz cells on [0, lx] x [0, lz] (metres).
 * nx, nz >= 4. */
typedef struct gea_grid {
    int32_t nx, nz;
    double lx, lz;
} gea_grid;

/* Physical constants (SI) and solver settings.
 *  R, cp     gas constant and heat capacity at constant pressure (eq. p,
 *            eq. K_h); cv = cp - R.
 *  g         gravitational acceleration, > 0 (0 allowed: no gravity).
 *  p0        reference pressure of the potential temperature (Remark 2).
 *  mu, Pr    constant artificial (dynamic) viscosity and Prandtl number of
 *            Remark 1, eqs. (mom_LES), (ent_LES).
 *  dt        time step (BDF1).
 *  n_corr    number of PISO correctors (Section 3), 1..4.
 *  jac_rtol, jac_maxit   Jacobi iteration for the implicit momentum and
 *            enthalpy predictors: stops after the sweep whose residual met
 *            ||r||_2 <= jac_rtol ||b||_2.
 *  cg_rtol, cg_maxit     conjugate gradients for the pressure equation:
 *            stops when ||r||_2 <= cg_rtol ||b||_2 (recursive residual).
 *  mg_min_cells  the multigrid preconditioner coarsens by 2 in x and z
 *            while both sizes are even and >= 8. 0 (default): until the
 *            estimated Laplacian-to-diagonal ratio of the pressure operator,
 *            2 dt^2 R T (1/dx^2 + 1/dz^2) at T = 300 K, is at most 1 (the
 *            coarse levels are then nearly diagonal). > 0: until a level has
 *            at most this many cells (a value >= nx*nz gives one level).
 *  flags     GEA_FLAG_GRAPH: always run steps as a CUDA graph of per-phase
 *            kernels. By default the library picks the persistent
 *            cooperative kernel when the grid has at most 4 tiles (32 x 8
 *            cells) per block that fits on the GPU at once, where a phase is
 *            latency-bound, and the graph otherwise.
 *            GEA_FLAG_MIXED: mixed-precision step (the driver is chosen as
 *            for the FP64 step; with GEA_FLAG_GRAPH the graph). The
 *            state, the hydrostatic split p' = p + rho g z, the face forces,
 *            every right-hand side and H(u) stay FP64; each of the three
 *            linear solves becomes one defect correction: an FP64 residual
 *            r0 = b - A x_old, an FP32 solve A dx = r0 (Jacobi, or multigrid
 *            CG for the pressure) to ||r|| <= mp_rtol ||r0||, and the FP64
 *            update x = x_old + dx. The pressure solve is skipped when
 *            ||r0|| <= cg_rtol ||b||. jac_maxit and cg_maxit cap the FP32
 *            iterations; gea_stats.cg_relres is then relative to ||r0||.
 *            GEA_FLAG_KEEP_R0: keep the initial residual of the first
 *            corrector's pressure solve (GEA_FIELD_R0; CUDA-graph driver;
 *            not with GEA_FLAG_MIXED).
 *            GEA_FLAG_DEBUG_PADS: a debugging layout in place of a device
 *            memory checker (gea_debug_* below): every array gets a guard
 *            band of GEA_PAD_GUARD_BYTES bytes behind it (one more before
 *            the first), and the padding of every row, the unused tail of
 *            every array and the guard bands are filled with a NaN pattern
 *            at creation. The step results are the same as without it.
 *            Other bits must be 0.
 *  mp_rtol   relative tolerance of the FP32 solves (GEA_FLAG_MIXED only);
 *            0 selects 1e-5, otherwise 1e-7 <= mp_rtol < 1.
 *  cs        Smagorinsky constant (LES; the paper names large eddy
 *            simulation without a model): the viscosity of the momentum
 *            and enthalpy diffusion becomes mu + rho (cs Delta)^2 |S| per
 *            cell from rho^n, u^n (Delta = sqrt(dx dz), |S|^2 =
 *            2 S_ij S_ij by central differences), with face values the mean
 *            of the two cells. 0: constant mu. cs > 0 requires Pr = 1. */
typedef struct gea_constants {
    double R, cp, g, p0, mu, Pr, dt;
    int32_t n_corr;
    double jac_rtol;
    int32_t jac_maxit;
    double cg_rtol;
    int32_t cg_maxit;
    int32_t mg_min_cells;
    int32_t flags;
    double mp_rtol;
    double cs;
    uint32_t reading_flags;
} gea_constants;

/* gea_constants.reading_flags: where the paper's printed scheme admits more
 * than one reading, 0 selects the library's default and a bit selects the
 * alternative.
 *  GEA_READING_K_LAGGED  eq. step3_sd as printed: the enthalpy right-hand side
 *            b~_e = (rho^n h^n + rho^n K^{n-1} - p^{n-1}) / dt uses the kinetic
 *            energy of the previous time level, K^{n-1} = |u^{n-1}|^2 / 2 (with
 *            K^{-1} := K^0 after a conservative set_state). The default uses
 *            rho^n K^n, the consistent first-order difference of rho K (the
 *            printed K^{n-1} and p^{n-1} are then the lagged terms of the
 *            time derivative of rho h + rho K - p). The state then carries
 *            K^{n-1} (gea_state_view.Kold).
 * Not built: the printed form of eq. p_prime_sd as a pure Poisson equation
 * (its time term uses the known rho^{n+2/3}, so on the closed boxes of the
 * paper's cases it is singular and, in general, inconsistent); the library
 * solves the Helmholtz form that follows from rho^{n+1} = p^{n+1}/(R T^{n+1})
 * (eq. step4_4sd). Other bits must be 0. */
enum { GEA_READING_K_LAGGED = 1 };

/* A view of caller-owned buffers (host or device, per mem). The library
 * copies from/to them; it never keeps the pointers.
 *  CONSERVATIVE: rho, rhou, rhow, rhoe (rho e = rho (cv T + |u|^2/2 + g z)).
 *  FULL: rho, u, w, T, h, p, pp (= p'), pold (= p^{n-1}), phix, phiz, and
 *        Kold (= K^{n-1}; only with GEA_READING_K_LAGGED, otherwise ignored
 *        and may be NULL) -- the complete state carried between steps; a
 *        FULL get followed by a FULL set continues bit for bit as if the run
 *        had not been interrupted. */
typedef struct gea_state_view {
    int32_t kind;
    int32_t mem;
    double *rho, *rhou, *rhow, *rhoe;
    double *u, *w, *T, *h, *p, *pp, *pold, *phix, *phiz;
    double *Kold;
} gea_state_view;

/* Counters of the last completed step. */
typedef struct gea_stats {
    int64_t steps_done;        /* steps completed since the last set_state */
    int32_t jac_u, jac_h;      /* Jacobi sweeps: momentum (u and w together), enthalpy */
    int32_t cg_iters[4];       /* CG iterations per PISO corrector */
    double cg_relres[4];       /* final ||r|| / ||b|| per corrector */
    int32_t status;            /* GEA_OK or the first device-side error */
    int32_t mg_levels;         /* multigrid levels in use */
    int64_t launches;          /* kernel launches since the last set_state */
    int32_t driver;            /* 0: CUDA graph, 1: persistent cooperative kernel,
                                  2: mixed-precision CUDA graph,
                                  3: mixed-precision persistent kernel */
    int32_t reserved;
} gea_stats;

typedef struct gea_ctx gea_ctx;

/* Create a context for one grid and constant set on the current CUDA device:
 * validates the arguments and allocates every device buffer (state, scratch,
 * multigrid hierarchy). The context owns them; gea_destroy frees them.
 * Errors: GEA_ERR_INVAL (sizes < 4, non-positive R, cp > R, dt, lengths,
 * n_corr outside 1..4, non-positive tolerances or caps), GEA_ERR_NOMEM,
 * GEA_ERR_CUDA. */
int gea_create(const gea_grid *grid, const gea_constants *c, gea_ctx **out);

/* Order all later work of ctx on this cudaStream_t (NULL: the legacy default
 * stream). */
int gea_set_stream(gea_ctx *ctx, void *stream);

/* Load a state. CONSERVATIVE derives the rest on the device: u = (rho u)/rho,
 * T = (e - K - g z)/cv, p = rho R T (eq. p), h = cp T (eq. K_h),
 * p' = p + rho g z, p^{n-1} = p, and phi on interior faces the average of the
 * two cells' normal momentum times the face area (Section 3), and checks
 * rho and T (one synchronisation). FULL copies the fields as given (no
 * check; enqueued on the stream without waiting; host buffers must stay
 * unchanged until the stream reaches the copies).
 * Errors: GEA_ERR_INVAL (null pointers, unknown kind: the context is left
 * as it was; CONSERVATIVE: rho <= 0 or T <= 0 anywhere), GEA_ERR_CUDA. After
 * an error other than a rejected argument the context holds no state
 * (gea_step: GEA_ERR_STATE) until a later set_state succeeds. */
int gea_set_state(gea_ctx *ctx, const gea_state_view *v);

/* Advance n >= 0 steps (Section 3, Steps 1-3). Returns after the launches
 * are enqueued and the status of the finished steps has been read back,
 * i.e. it synchronises the stream once at the end. On GEA_ERR_NOCONV,
 * GEA_ERR_NONFINITE or GEA_ERR_TIMEOUT the state stays at the last completed
 * step. With the persistent driver all n steps run in one cooperative kernel
 * launch whose blocks stay resident (grid barriers between phases, solver
 * loops on the device); with the graph driver each step is one CUDA graph
 * launch (see gea_constants.flags). */
int gea_step(gea_ctx *ctx, int32_t n);

/* Enqueue n steps without waiting; gea_sync reports their status. */
int gea_step_async(gea_ctx *ctx, int32_t n);
int gea_sync(gea_ctx *ctx);

/* Copy the state out (kind/mem as in set_state; null destination pointers
 * are skipped). CONSERVATIVE is computed on the device from the state:
 * rho, rho u, rho w and rho e = rho (cv T + |u|^2/2 + g z) (Section 2.1,
 * the total energy of eq. ent). Synchronises. */
int gea_get_state(gea_ctx *ctx, gea_state_view *out);

/* Diagnostics (Remark 2): theta' = T (p0/p)^(R/cp) - theta_bar(z) per cell
 * into theta_prime (host, nz*nx, may be NULL), given the background
 * theta_bar (host, nz values); mass = sum rho V and energy = sum rho e V
 * (may be NULL). Computed on the device. */
int gea_get_diag(gea_ctx *ctx, const double *theta_bar, double *theta_prime,
                 double *mass, double *energy);

/* Counters of the last completed step. */
int gea_get_stats(gea_ctx *ctx, gea_stats *s);

/* Intermediate fields of the last step, copied to host (nz*nx doubles, or
 * face arrays as in phix/phiz for GEA_FIELD_DX/DZ):
 *  RHO1 = rho^{n+1/3}; U1, W1 = u^{n+1/3}; H1 = h^{n+1}; RHO2 = rho^{n+2/3};
 *  HX, HZ = H(u) and B = pressure right-hand side of the last corrector;
 *  DX, DZ = face coefficients D_f = dt rho2_f / rho1_f;
 *  HC, HAX, HAZ = the pressure operator of the last step,
 *      (A e)_i = c_i e_i + sum_f a_f (e_i - e_N): c (cells), a on the x-faces
 *      (nz rows of nx+1, zero on the walls) and on the z-faces (nz+1 rows);
 *  R0 = initial residual b - A p' of the first corrector's pressure solve
 *      of the last step (needs GEA_FLAG_KEEP_R0). */
enum {
    GEA_FIELD_RHO1 = 0, GEA_FIELD_U1 = 1, GEA_FIELD_W1 = 2, GEA_FIELD_H1 = 3,
    GEA_FIELD_RHO2 = 4, GEA_FIELD_HX = 5, GEA_FIELD_HZ = 6, GEA_FIELD_B = 7,
    GEA_FIELD_DX = 8, GEA_FIELD_DZ = 9, GEA_FIELD_HC = 10, GEA_FIELD_HAX = 11,
    GEA_FIELD_HAZ = 12, GEA_FIELD_R0 = 13
};

/* Use a learned pressure-correction network (include/gea_net.h) in the
 * pressure solves of this context (an extension beyond the paper). mode 1:
 * before each solve's first preconditioning, the network proposes a
 * correction e for the initial residual r, and the solve starts from
 * x + alpha e, r - alpha A e with alpha = r.e / e.A e, the step that
 * minimises the A-norm error along e (so the start is never worse); the
 * solve then runs to the same tolerance as without the network. mode 2
 * (FP64 step only): the network replaces the multigrid V-cycle as the
 * preconditioner, z = N(r), in a flexible CG truncated to one previous
 * direction (beta = -z.q_old / p_old.q_old, alpha = r.p / p.A p), which
 * stays a descent method for a nonlinear preconditioner; the stopping test
 * is unchanged. mode 3: both. mode 0: detach. The context does not own the network; it must outlive the
 * attachment, and must not be used elsewhere while this context steps.
 * Steps then run through the CUDA-graph driver. nx, nz must be multiples of
 * 8 within the network's size. Errors: GEA_ERR_INVAL, GEA_ERR_CUDA. */
struct gea_net;
int gea_attach_net(gea_ctx *ctx, struct gea_net *net, int32_t mode);

/* Tile column of the per-phase kernels with a grid reduction (the CG and
 * V-cycle steps and the Jacobi sweeps of the graph driver): each block walks
 * n tiles (32 x 8 cells each) of a column, so a launch has 1/n of the blocks
 * and of the block reductions. n = 0 (the default): 4 on grids of at least
 * 16384 tiles, else 1. The persistent kernels ignore it. The results depend
 * on n only through the order of the reduction sums. Synchronises the
 * stream; the step graphs are recorded anew. Errors: GEA_ERR_INVAL (n
 * outside 0..16). */
int gea_set_tiles_per_block(gea_ctx *ctx, int32_t n);

/* Weight omega of the Jacobi sweeps of the pressure solve's preconditioner:
 * the smoother of the multigrid V-cycle (default 0.8), or the two sweeps of
 * a one-level preconditioner (default 1, undamped). Takes effect from the
 * next step (the operator's omega/d is formed in every step's EOS phase);
 * the converged pressure does not depend on it, the CG iterations do.
 * Synchronises the stream; the step graphs are recorded anew. Errors:
 * GEA_ERR_INVAL (omega outside (0, 2)). */
int gea_set_smoother_weight(gea_ctx *ctx, double omega);

/* Tile shape of the persistent step kernels (FP64, mixed precision and the
 * ensemble launch): 0 = 32 x 8 cells (the default, and the tile of the
 * per-phase kernels of the CUDA-graph driver), 1 = 16 x 16, 2 = 64 x 4; one
 * thread per cell, 256 threads a block. Halos cost less on squarer tiles,
 * rows load in longer runs on wider ones, and the number of tiles per block
 * changes the load balance, so the fastest shape depends on the grid; the
 * tile-shape autotuner of the Python binding times the candidates on real
 * steps. The results depend on the shape only through the order of the
 * reduction sums. Members of an ensemble must share one shape. The CUDA-graph
 * driver ignores it. Synchronises the stream. Errors: GEA_ERR_INVAL (shape
 * outside 0..2), GEA_ERR_CUDA. */
enum { GEA_TILE_32x8 = 0, GEA_TILE_16x16 = 1, GEA_TILE_64x4 = 2 };
int gea_set_tile_shape(gea_ctx *ctx, int32_t shape);

/* Poll limit of the grid barriers of the persistent step kernels (and of
 * this context's share of an ensemble launch): a block that has polled the
 * barrier `polls` times without every block arriving gives up, sets
 * GEA_ERR_TIMEOUT and leaves the step at the next phase boundary, as does
 * every other block, so the launch always ends; the state stays at the last
 * completed step, and the error is sticky until the next gea_set_state.
 * polls < 0 restores the default (2^23 polls, a few seconds), which is also
 * the largest limit (larger values are taken as the default, so a wait stays
 * bounded); 0 makes every block that is not the last to arrive give up at
 * once, which tests the failure path without a hang. The CUDA-graph driver has no such waits.
 * Errors: GEA_ERR_INVAL (null ctx). */
int gea_set_wait_limit(gea_ctx *ctx, int64_t polls);

/* Phase trace of the persistent step kernels (tracing; the paper has no
 * counterpart: it measures the phases of Section 3's step, Steps 1-3 and the
 * PISO correctors, as the device runs them). trace: a caller-owned device
 * buffer of `capacity` uint64 values, 8-byte aligned, written by every step
 * launched while it is set; the library keeps the pointer, not the data.
 * With B the blocks of the persistent grid (returned in *blocks, which may
 * be null; 0 when the context steps through the CUDA graph), row 0 holds,
 * per block b, its kernel entry time at [2b] and its SM at [2b + 1]; row k
 * (1 <= k <= max_barriers) holds block b's arrival at [2(kB + b)] and its
 * release from [2(kB + b) + 1] the k-th grid barrier of the launch, in
 * ns of the GPU's global timer. Barriers past max_barriers are not
 * recorded. The grid barriers of a step separate its phases: the Jacobi
 * sweeps, the right-hand sides, the EOS update, the two phases of each CG
 * iteration, the corrections. capacity must be at least
 * 2 (max_barriers + 1) B. trace null turns the trace off (as does
 * gea_set_tile_shape). Errors: GEA_ERR_INVAL (null ctx, max_barriers < 1
 * with a buffer, a capacity too small, a misaligned buffer, a context
 * without the persistent driver). */
int gea_set_trace(gea_ctx *ctx, uint64_t *trace, int32_t max_barriers, int64_t capacity, int32_t *blocks);
int gea_get_field(gea_ctx *ctx, int32_t which, double *host);

/* Apply the pressure solve's preconditioner to r: z = M r with M one
 * V(1,1)-cycle of the Galerkin multigrid hierarchy of the last completed step
 * (the operator of eq. p_prime_sd in its Helmholtz form, as the CG of Step 3
 * uses it; two undamped Jacobi sweeps when the hierarchy has one level). r, z:
 * nz*nx doubles, host or device. Lets a caller check what CG needs of M: it
 * is linear, symmetric and positive definite. FP64 contexts only.
 * Synchronises. Errors: GEA_ERR_INVAL (null pointers, a mixed-precision
 * context), GEA_ERR_STATE (no completed step since the last set_state),
 * GEA_ERR_CUDA; the step's solver counters are kept in every case. */
int gea_apply_precond(gea_ctx *ctx, const double *r, double *z);

/* Event-timed duration (ms) of the pressure solves (all correctors) of the
 * last step launched by gea_step/gea_step_async, or -1 if unavailable. */
double gea_last_pressure_ms(gea_ctx *ctx);

/* Per-kernel timing of one step. */
typedef struct gea_kernel_time {
    char name[40];     /* kernel (stage) name */
    int32_t launches;  /* launches in the step */
    int64_t cells;     /* grid cells covered, summed over the launches that did
                          their work (a solver-loop kernel launched after its
                          loop finished returns at once and adds none) */
    double ms;         /* summed CUDA-event durations of the launches */
} gea_kernel_time;

/* Advance one step with the same kernels as gea_step, launched one by one
 * (no graph) with a CUDA event pair around each launch on the context's
 * stream, the solver loops checked from the host. Writes up to max_entries
 * per-kernel totals to out and their number to *n_entries. Synchronises. */
int gea_profile_step(gea_ctx *ctx, gea_kernel_time *out, int32_t max_entries,
                     int32_t *n_entries);

/* Total mass sum rho V and total energy sum rho (cv T + |u|^2/2 + g z) V of a
 * caller-owned state, computed without allocating any device memory. The
 * paper has no counterpart: this entry point serves callers that cannot
 * allocate device memory (their memory is owned by a framework's caching
 * allocator or a fixed arena, or they must not call cudaMalloc, which can
 * synchronise the device or fail at run time). It needs no context.
 *
 * rho, u, w, T: device arrays, nz rows of nx values (x fastest, no padding).
 * out: device array of 2 doubles, receives {mass, energy}. cp, R, g as in
 * gea_constants; lx, lz the domain size. Enqueued on `stream` (a
 * cudaStream_t; NULL for the legacy default stream); it does not wait.
 *
 * Scratch: the reduction's per-block partial sums and its arrival counter
 * live in a fixed 1 MiB file-scope device array that every GPU that loads
 * the library keeps until the process exits. Its device address is looked
 * up on the first call on each device (cudaGetSymbolAddress, with that
 * device current) and kept; make that first call before any stream capture.
 * A cudaDeviceReset of that device invalidates the kept address: do not call
 * this entry point on a device after resetting it. Every
 * call shares the array: the counter is cleared at the start of each call,
 * and calls whose kernels overlap on the GPU (on different streams or
 * threads) race on it -- order them on one stream.
 * Errors: GEA_ERR_INVAL for null pointers, non-positive sizes, or more than
 * GEA_NOALLOC_MAX_CELLS cells; GEA_ERR_CUDA if a CUDA call fails. */
#define GEA_NOALLOC_MAX_CELLS 16777216
int gea_mass_energy_noalloc(int32_t nx, int32_t nz, double lx, double lz, double cp, double R,
                            double g, const double *rho, const double *u, const double *w,
                            const double *T, double *out, void *stream);

/* Arithmetic peak probe (the paper has no counterpart): `blocks` blocks of
 * 256 threads, each thread running 8 independent fused multiply-add chains
 * of `iters` steps in FP64 (bits = 64) or FP32 (bits = 32), so one launch
 * does blocks x 256 x 8 x iters FMAs (x 2 flops). out: device array of
 * blocks x 256 values of that type (the chains' sums, which keep them from
 * being removed). Enqueued on `stream` (cudaStream_t, NULL: legacy default);
 * the caller times it with CUDA events to measure the FMA issue rate that
 * bounds the FP64 stencil and solver kernels. Errors: GEA_ERR_INVAL,
 * GEA_ERR_CUDA. */
int gea_probe_fma(int32_t bits, int32_t blocks, int32_t iters, void *out, void *stream);

/* Grid-barrier latency probe (the paper has no counterpart): one cooperative
 * launch of `blocks` blocks of 256 threads (all resident at once) that pass
 * `iters` grid barriers of the protocol the persistent step kernels use
 * (one acquire-release arrival per block on a monotone counter, acquire
 * polls until it reaches the barrier's count), with nothing between them;
 * read_status != 0 adds the read of a status word after each barrier, as
 * those kernels do. scratch: caller-owned device memory of at least 16
 * bytes, zeroed by the call; its third 32-bit word is nonzero afterwards if a
 * bounded wait (2^22 polls) gave up. Enqueued on `stream`; the caller times
 * it with CUDA events (time / iters = one barrier). Errors: GEA_ERR_INVAL
 * (blocks < 1, iters < 1, null scratch, more blocks than fit at once),
 * GEA_ERR_CUDA. */
int gea_probe_barrier(int32_t blocks, int32_t iters, int32_t read_status, void *scratch, void *stream);

/* ---- ensembles: many independent contexts advanced by one launch ----
 *
 * An ensemble runs the steps of n contexts (members, each with its own
 * grid, constants and state) in one cooperative launch. The GPU's
 * co-resident thread blocks are shared out in proportion to the members'
 * weights (default: a member's number of tiles of the members' tile shape).
 * A member whose share is one block or more runs on blocks of its own (at
 * most one per tile) with its own grid barrier and its own reductions, so
 * members never wait for one another; members whose shares are below one
 * block are packed, in member order and up to one block's worth of weight,
 * onto a block they share and on which they run one after another, each as
 * a grid of one block (if that left a larger member without a block, every
 * member gets one of its own instead). The members are all FP64 or all mixed precision
 * (GEA_FLAG_MIXED: the mixed-precision step, one launch for all of them),
 * and share one tile shape (gea_set_tile_shape). The results of a member are
 * those of its own persistent driver up to the order of the reduction sums.
 * The ensemble takes over the members' streams (gea_ensemble_set_stream
 * sets all of them); while it exists, step members only through it. Members
 * must not use GEA_FLAG_KEEP_R0 or an attached network.
 * Errors: GEA_ERR_INVAL (null or unsuitable members, FP64 and mixed members
 * together, different tile shapes, no partition of the blocks that fits),
 * GEA_ERR_STATE (a member without state, on step), GEA_ERR_NOMEM,
 * GEA_ERR_CUDA. */
typedef struct gea_ensemble gea_ensemble;
/* weights (optional, n positive values): blocks in proportion to weights[m]
 * (a member's work: tiles times the phases of its step) instead of the
 * member's tile count. */
int gea_ensemble_create(gea_ctx **members, int32_t n, const double *weights, gea_ensemble **out);
int gea_ensemble_set_stream(gea_ensemble *e, void *stream);
/* The partition gea_ensemble_create makes, computed on the host alone (no
 * device or context needed): n members of weights[m] > 0 and tiles[m] >= 1
 * tiles on `blocks` co-resident blocks. member_blocks[m] receives the blocks
 * member m runs on (1 on a shared block), member_group[m] its group (a
 * group of several members shares one block and runs them in turn; a
 * group of one member owns its blocks); *ngroups and *used_blocks (each
 * may be NULL) the number of groups and of blocks used (<= blocks).
 * Errors: GEA_ERR_INVAL (bad arguments, no partition that fits). */
int gea_ensemble_plan(const double *weights, const int64_t *tiles, int32_t n, int32_t blocks,
                      int32_t *member_blocks, int32_t *member_group, int32_t *ngroups, int32_t *used_blocks);
/* Blocks member m (0 <= m < n) runs on (1 for a member on a shared block),
 * or -1. */
int gea_ensemble_blocks(const gea_ensemble *e, int32_t m);
/* Enqueue n steps of every member (one launch); gea_sync on a member, or
 * gea_ensemble_sync, waits and reports. While every member's state is in
 * the same slot parity (always, unless members were stepped apart), the
 * launch is one CUDA graph launch: a graph holding the cooperative kernel
 * node is captured on the first call for each parity, n and set of member
 * settings the arguments carry (barrier poll limits, smoother weights), with
 * its own device copy of the members' arguments, and replayed (no host
 * staging, no synchronisation). Otherwise, or after gea_ensemble_set_graph(e, 0), the
 * arguments are staged and the kernel launched directly. Both run the same
 * kernel on the same arguments. */
int gea_ensemble_step(gea_ensemble *e, int32_t n);
/* on = 0: launch directly instead of through the captured graphs. */
int gea_ensemble_set_graph(gea_ensemble *e, int32_t on);
/* Wait for the launches; the first member error code, or GEA_OK. */
int gea_ensemble_sync(gea_ensemble *e);
void gea_ensemble_destroy(gea_ensemble *e);

/* ---- Pad checking (GEA_FLAG_DEBUG_PADS contexts) ----
 * A stand-in for a device memory checker. Every array of a context lives in
 * one device allocation as rows of a fixed pitch (the row pitch of a cell
 * array is round_up(nx + 1, 32) elements), so an index off by one in x
 * lands in a row's padding, and a row or array overrun lands in the array's
 * unused tail or the guard band behind it. With the flag, all of these
 * "pad" elements hold GEA_PAD_POISON64 (FP64 arrays) or GEA_PAD_POISON32
 * (FP32 arrays), NaN bit patterns: a kernel that writes out of bounds
 * changes a pad (found by the checks below), and one that reads out of
 * bounds draws a NaN into its results (found by the residual norms,
 * GEA_ERR_NONFINITE, and by comparison with a reference). The library's
 * kernels neither read nor write pads. */
#define GEA_PAD_GUARD_BYTES 512
#define GEA_PAD_POISON64 0x7FF4BAD0DEAD0BADull
#define GEA_PAD_POISON32 0x7FA0BAD0u

/* One array of the context's allocation: cols x rows elements in use, each
 * row `pitch` elements long, then unused elements up to `span` (the array's
 * tail and its guard band). Element (row r, column c) is at
 * ptr + (r * pitch + c) * elem_bytes. */
typedef struct gea_pad_region {
    char name[24];       /* e.g. "S0.phix", "L1.az", "F.T.cC" (F: FP32) */
    void *ptr;           /* device pointer to element (0, 0) */
    int32_t elem_bytes;  /* 8 (FP64) or 4 (FP32) */
    int32_t pitch, rows, cols;
    int64_t span;        /* elements from ptr to the next array */
} gea_pad_region;

/* Result of a pad check. */
typedef struct gea_pad_report {
    int64_t bad;          /* pad elements that no longer hold the poison */
    int32_t launch;       /* gea_debug_step: index of the first launch after
                             which a pad had changed, -1 if none */
    char kernel[40];      /* its kernel (stage) name, "" if none */
    char array[24];       /* array of the first changed pad element ("" if none):
                             gea_debug_step: the lowest one changed by that
                             launch; gea_debug_check_pads: the lowest one */
    int32_t row, col;     /* its position (row >= rows or col >= cols of the array) */
} gea_pad_report;

/* The context's arrays (up to max entries into out; their number into *n).
 * Errors: GEA_ERR_INVAL (null pointers, or a context without
 * GEA_FLAG_DEBUG_PADS). */
int gea_debug_pad_regions(gea_ctx *ctx, gea_pad_region *out, int32_t max, int32_t *n);

/* Write the poison into every pad element again. Synchronises.
 * Errors: GEA_ERR_INVAL (null ctx, no GEA_FLAG_DEBUG_PADS), GEA_ERR_CUDA. */
int gea_debug_poison(gea_ctx *ctx);

/* Count the pad elements that no longer hold the poison (a device kernel
 * over every array; rep->launch = -1). Synchronises. Errors as
 * gea_debug_poison. */
int gea_debug_check_pads(gea_ctx *ctx, gea_pad_report *rep);

/* Advance one step with the kernels of gea_profile_step, launched one by
 * one, checking every pad after every launch; rep names the first launch
 * that changed a pad, and rep->bad counts the changed pads after the step.
 * Returns the step's own status (as gea_step) when the step fails.
 * Synchronises. Errors as gea_profile_step, and as gea_debug_poison. */
int gea_debug_step(gea_ctx *ctx, gea_pad_report *rep);

const char *gea_last_error(const gea_ctx *ctx);
void gea_destroy(gea_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* GEA_H */
