/*
 * gea_oracle.c -- plain FP64 CPU oracle of one predictor-corrector time step
 * of the pressure-based finite-volume solver for the dry compressible Euler
 * equations of Girfoglio, Quaini & Rozza, "GEA: a new finite volume-based
 * open source code for the numerical simulation of atmospheric and ocean
 * flows" (arXiv 2303.10499).
 *
 * TEST INFRASTRUCTURE. This file exists only to check the CUDA library. Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load it; the library never calls it and shares no code with it.
 *
 * It is written to be read against the paper, not to be fast: one loop per
 * equation, every face sum spelled out, the paper's notation for names.
 *
 * Discretisation (uniform Cartesian x-z grid, nx * nz cells of size dx * dz,
 * cell (i,k) centred at ((i+1/2) dx, (k+1/2) dz), free-slip walls on all four
 * sides, Section 4):
 *
 *  - phi_j = (rho u)_j . A_j is the mass flux through face j (eq. e1_d), kept
 *    between steps on the nx+1 x-faces of each row and nz+1 z-faces of each
 *    column; it is zero on wall faces.
 *  - Face sums are per unit volume: sum_j (...) / V with V = dx dz.
 *  - Convected face values use the fourth-order four-point interpolation
 *    X_f = (-X_{a-1} + 7 X_a + 7 X_b - X_{b+1}) / 12 (Section 3: fourth-order
 *    divergence); Laplacian and face-normal gradients are the compact
 *    two-point second-order forms (Section 3: second-order Laplacian and
 *    gradient).
 *  - One ghost layer gives the wall conditions: wall-normal velocity odd
 *    (impenetrable, Dirichlet 0 on the wall), tangential velocity even (free
 *    slip), scalars even, and h with dh/dz = -g at the bottom and top walls,
 *    the neutral-atmosphere lapse, so that a neutral column at rest has no
 *    enthalpy diffusion flux.
 *  - Sign of the hydrostatic split: with g = +9.81 and z pointing up, the
 *    identity that turns eq. (mom) into eq. (mom_split) needs
 *    p = p' - rho g z; the force is grad p' - g z grad rho. (The printed
 *    eqs. p_split, mom_split, step2_sd, p_prime_sd and step4_4sd hold as
 *    written when their g is read as the signed vertical component -9.81.)
 *  - Pressure-gradient and gravity forces live on faces:
 *      G_f = (p'_b - p'_a)/Delta - g z_f (rho_b - rho_a)/Delta
 *    and reach cell centres as the average of the two faces in each
 *    direction (zero on wall faces). At a discretely balanced rest state G_f
 *    vanishes exactly.
 *  - Step 3's pressure equation (eq. p_prime_sd) is taken in the form that
 *    follows from the discrete continuity equation with
 *    rho^{n+1} = psi p^{n+1} (eq. step4_4sd), psi = 1/(R T^{n+1}),
 *    p^{n+1} = p' - rho^{2/3} g z and the face mass flux
 *      F_f = D_f (H_f . n - G_f),  D_f = dt rho^{2/3}_f / rho^{1/3}_f,
 *    i.e. the symmetric positive definite Helmholtz problem
 *      (psi_i/dt) p'_i + (1/V) sum_f D_f |A_f| (p'_i - p'_N)/Delta_f
 *        = (rho^n_i + psi_i rho^{2/3}_i g z_i)/dt
 *          - (1/V) sum_f D_f |A_f| [H_f . n + g z_f (rho^{2/3}_N - rho^{2/3}_i)/Delta_f].
 *  - The implicit predictors (eq. step2_sd first line, eq. step3_sd) are
 *    solved by Jacobi iteration, the pressure equation by diagonally
 *    preconditioned conjugate gradients, each to a relative 2-norm residual.
 *
 * Storage: cell fields are nz * nx arrays, index k*nx + i. phix holds
 * nz * (nx+1) x-face fluxes (index k*(nx+1) + f, face f between cells f-1
 * and f); phiz holds (nz+1) * nx z-face fluxes (index f*nx + i).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nx, nz;
    double lx, lz;
    double R, cp, g, p0, mu, Pr, dt;
    int32_t n_corr;
    double jac_rtol;
    int32_t jac_maxit;
    double cg_rtol;
    int32_t cg_maxit;
    double cs;          /* Smagorinsky constant; 0: constant viscosity mu only */
    uint32_t reading_flags;   /* ORC_READING_* bits; 0: the default readings */
} orc_cfg;

/* Reading of eq. (step3_sd): b~_e = (rho^n h^n + rho^n K^{n-1} - p^{n-1})/dt as
 * printed (K of the previous time level, K^{-1} := K^0), instead of the
 * default rho^n K^n. */
enum { ORC_READING_K_LAGGED = 1 };

/* The solution tuple of Section 3 (rho, u, h, p, p', T) plus what the
 * scheme carries between steps: the face mass fluxes phi^n, p^{n-1} and
 * K^{n-1} = |u^{n-1}|^2/2 (used by the literal reading of eq. step3_sd). */
typedef struct {
    double *rho, *u, *w, *T, *h, *p, *pp, *pold, *phix, *phiz, *Kold;
} orc_state;

typedef struct {
    int32_t jac_u, jac_w, jac_h;   /* Jacobi sweeps of the last step */
    int32_t cg_iters[4];           /* CG iterations per corrector, last step */
    double cg_relres[4];           /* final ||r||/||b|| per corrector */
    int32_t status;                /* 0 ok, 1 a solver hit its iteration cap */
} orc_stats;

/* Intermediate fields of the last step (any pointer may be NULL). */
typedef struct {
    double *rho1, *u1, *w1, *h1, *T1, *rho2, *psi;
    double *Hx, *Hz, *b;           /* from the last corrector */
    double *Dx, *Dz;               /* face coefficients, nz*(nx+1) and (nz+1)*nx */
    double *bh;                    /* right-hand side of the enthalpy equation */
} orc_dump;

enum { BC_EVEN = 0, BC_U = 1, BC_W = 2, BC_H = 3 };

/* ------------------------------------------------------------------ */
/* helpers                                                             */
/* ------------------------------------------------------------------ */

static double dxof(const orc_cfg *c) { return c->lx / c->nx; }
static double dzof(const orc_cfg *c) { return c->lz / c->nz; }

/* Cell value at (i,k) with i in [-1, nx] and k in [-1, nz]; outside the box
 * the one-layer ghost given by the wall condition of field kind bc. */
static double at(const orc_cfg *c, const double *X, int i, int k, int bc)
{
    int nx = c->nx, nz = c->nz;
    if (i < 0) {
        double v = X[k * nx + 0];
        return bc == BC_U ? -v : v;
    }
    if (i >= nx) {
        double v = X[k * nx + nx - 1];
        return bc == BC_U ? -v : v;
    }
    if (k < 0) {
        double v = X[0 * nx + i];
        if (bc == BC_W) return -v;
        if (bc == BC_H) return v + c->g * dzof(c);
        return v;
    }
    if (k >= nz) {
        double v = X[(nz - 1) * nx + i];
        if (bc == BC_W) return -v;
        if (bc == BC_H) return v - c->g * dzof(c);
        return v;
    }
    return X[k * nx + i];
}

/* Fourth-order face value between cells a and b = a+1 from the four cells
 * a-1, a, b, b+1. */
static double interp4(double xm, double xa, double xb, double xp)
{
    return (-xm + 7.0 * xa + 7.0 * xb - xp) / 12.0;
}

/* x-face f (between cells f-1 and f) of row k: phi stored by the caller. */
static double phix_at(const orc_cfg *c, const double *phix, int f, int k)
{
    return phix[k * (c->nx + 1) + f];
}
static double phiz_at(const orc_cfg *c, const double *phiz, int i, int f)
{
    return phiz[f * c->nx + i];
}

/* Convective term (1/V) sum_j phi_j X_j of cell (i,k), X_j by interp4;
 * wall faces carry no flux. */
double orc_convection_cell(const orc_cfg *c, const double *phix, const double *phiz,
                           const double *X, int bc, int i, int k)
{
    int nx = c->nx, nz = c->nz;
    double V = dxof(c) * dzof(c), s = 0.0;
    if (i + 1 < nx)  /* east face, outward +x */
        s += phix_at(c, phix, i + 1, k) *
             interp4(at(c, X, i - 1, k, bc), at(c, X, i, k, bc),
                     at(c, X, i + 1, k, bc), at(c, X, i + 2, k, bc));
    if (i > 0)       /* west face, outward -x */
        s -= phix_at(c, phix, i, k) *
             interp4(at(c, X, i - 2, k, bc), at(c, X, i - 1, k, bc),
                     at(c, X, i, k, bc), at(c, X, i + 1, k, bc));
    if (k + 1 < nz)  /* top face, outward +z */
        s += phiz_at(c, phiz, i, k + 1) *
             interp4(at(c, X, i, k - 1, bc), at(c, X, i, k, bc),
                     at(c, X, i, k + 1, bc), at(c, X, i, k + 2, bc));
    if (k > 0)       /* bottom face, outward -z */
        s -= phiz_at(c, phiz, i, k) *
             interp4(at(c, X, i, k - 2, bc), at(c, X, i, k - 1, bc),
                     at(c, X, i, k, bc), at(c, X, i, k + 1, bc));
    return s / V;
}

/* Diffusive face sum (1/V) sum_j (grad X)_j . A_j of cell (i,k) with the
 * compact face-normal gradient; wall faces through the ghost layer. */
double orc_laplacian_cell(const orc_cfg *c, const double *X, int bc, int i, int k)
{
    double dx = dxof(c), dz = dzof(c), V = dx * dz;
    double xc = at(c, X, i, k, bc);
    double s = 0.0;
    s += (at(c, X, i + 1, k, bc) - xc) / dx * dz;   /* east  |A| = dz */
    s += (at(c, X, i - 1, k, bc) - xc) / dx * dz;   /* west */
    s += (at(c, X, i, k + 1, bc) - xc) / dz * dx;   /* top   |A| = dx */
    s += (at(c, X, i, k - 1, bc) - xc) / dz * dx;   /* bottom */
    return s / V;
}

/* Strain-rate magnitude |S| = sqrt(2 S_ij S_ij) of cell (i,k) from central
 * differences of the cell velocities (ghosts by the wall rules):
 * 2 S_ij S_ij = 2 (du/dx)^2 + 2 (dw/dz)^2 + (du/dz + dw/dx)^2 in x-z. */
double orc_strain_cell(const orc_cfg *c, const double *u, const double *w, int i, int k)
{
    double dx = dxof(c), dz = dzof(c);
    double dudx = (at(c, u, i + 1, k, BC_U) - at(c, u, i - 1, k, BC_U)) / (2.0 * dx);
    double dudz = (at(c, u, i, k + 1, BC_U) - at(c, u, i, k - 1, BC_U)) / (2.0 * dz);
    double dwdx = (at(c, w, i + 1, k, BC_W) - at(c, w, i - 1, k, BC_W)) / (2.0 * dx);
    double dwdz = (at(c, w, i, k + 1, BC_W) - at(c, w, i, k - 1, BC_W)) / (2.0 * dz);
    double sh = dudz + dwdx;
    return sqrt(2.0 * dudx * dudx + 2.0 * dwdz * dwdz + sh * sh);
}

/* Effective dynamic viscosity mu + mu_t with the Smagorinsky eddy viscosity
 * mu_t = rho (cs Delta)^2 |S|, Delta = sqrt(dx dz), at every cell. */
void orc_smagorinsky(const orc_cfg *c, const double *rho, const double *u, const double *w,
                     double *mu_eff)
{
    double d2 = c->cs * c->cs * dxof(c) * dzof(c);
    for (int k = 0; k < c->nz; ++k)
        for (int i = 0; i < c->nx; ++i)
            mu_eff[k * c->nx + i] = c->mu + rho[k * c->nx + i] * d2 * orc_strain_cell(c, u, w, i, k);
}

/* Variable-coefficient diffusive face sum (1/V) sum_j mu_j (grad X)_j . A_j of
 * cell (i,k): mu_j the mean of the two cells' viscosities (a wall face takes
 * the cell's own), the compact face-normal gradient through the ghost layer. */
double orc_diffusion_cell(const orc_cfg *c, const double *mu, const double *X, int bc, int i, int k)
{
    double dx = dxof(c), dz = dzof(c), V = dx * dz;
    double xc = at(c, X, i, k, bc), mc = at(c, mu, i, k, BC_EVEN);
    double s = 0.0;
    s += 0.5 * (mc + at(c, mu, i + 1, k, BC_EVEN)) * (at(c, X, i + 1, k, bc) - xc) / dx * dz;
    s += 0.5 * (mc + at(c, mu, i - 1, k, BC_EVEN)) * (at(c, X, i - 1, k, bc) - xc) / dx * dz;
    s += 0.5 * (mc + at(c, mu, i, k + 1, BC_EVEN)) * (at(c, X, i, k + 1, bc) - xc) / dz * dx;
    s += 0.5 * (mc + at(c, mu, i, k - 1, BC_EVEN)) * (at(c, X, i, k - 1, bc) - xc) / dz * dx;
    return s / V;
}

/* The diffusion term of the transport operators: nu L(X) with constant nu,
 * or nu times the variable-coefficient sum with the viscosity field mu. */
static double diffusion(const orc_cfg *c, const double *mu, double nu, const double *X, int bc,
                        int i, int k)
{
    return mu ? nu * orc_diffusion_cell(c, mu, X, bc, i, k) : nu * orc_laplacian_cell(c, X, bc, i, k);
}

/* Coefficient of X_i in -diffusion() for an interior cell. */
static double diffusion_diag(const orc_cfg *c, const double *mu, double nu, int i, int k)
{
    double dx = dxof(c), dz = dzof(c);
    if (!mu) return nu * (2.0 / (dx * dx) + 2.0 / (dz * dz));
    double mc = at(c, mu, i, k, BC_EVEN);
    return nu * ((0.5 * (mc + at(c, mu, i + 1, k, BC_EVEN)) + 0.5 * (mc + at(c, mu, i - 1, k, BC_EVEN))) / (dx * dx)
               + (0.5 * (mc + at(c, mu, i, k + 1, BC_EVEN)) + 0.5 * (mc + at(c, mu, i, k - 1, BC_EVEN))) / (dz * dz));
}

/* Flux divergence (1/V) sum_j phi_j of cell (i,k), outward positive. */
double orc_divergence_cell(const orc_cfg *c, const double *phix, const double *phiz,
                           int i, int k)
{
    double V = dxof(c) * dzof(c);
    double s = phix_at(c, phix, i + 1, k) - phix_at(c, phix, i, k)
             + phiz_at(c, phiz, i, k + 1) - phiz_at(c, phiz, i, k);
    return s / V;
}

/* Face forces G_f = (p'_b - p'_a)/Delta - g z_f (rho_b - rho_a)/Delta on all
 * faces (zero on walls). Gx: nz*(nx+1), Gz: (nz+1)*nx. */
static void face_forces(const orc_cfg *c, const double *pp, const double *rho,
                        double *Gx, double *Gz)
{
    int nx = c->nx, nz = c->nz;
    double dx = dxof(c), dz = dzof(c), g = c->g;
    for (int k = 0; k < nz; ++k) {
        double zf = (k + 0.5) * dz;              /* x-faces sit at the row height */
        for (int f = 0; f <= nx; ++f) {
            double G = 0.0;
            if (f > 0 && f < nx) {
                int a = k * nx + f - 1, b = k * nx + f;
                G = (pp[b] - pp[a]) / dx - g * zf * (rho[b] - rho[a]) / dx;
            }
            Gx[k * (nx + 1) + f] = G;
        }
    }
    for (int f = 0; f <= nz; ++f) {
        double zf = f * dz;                      /* z-face height */
        for (int i = 0; i < nx; ++i) {
            double G = 0.0;
            if (f > 0 && f < nz) {
                int a = (f - 1) * nx + i, b = f * nx + i;
                G = (pp[b] - pp[a]) / dz - g * zf * (rho[b] - rho[a]) / dz;
            }
            Gz[f * nx + i] = G;
        }
    }
}

/* Order of the reductions (the residual norms and the CG dot products):
 * index order by default, reverse index order after orc_set_reverse_sums(1).
 * Both are correct evaluations of the same sums; the tests compare the two
 * runs to measure the round-off floor of a result without any GPU. */
static int g_reverse_sums = 0;
void orc_set_reverse_sums(int on) { g_reverse_sums = on != 0; }

static double dot(const double *x, const double *y, size_t n)
{
    double s = 0.0;
    if (g_reverse_sums)
        for (size_t q = n; q-- > 0;) s += x[q] * y[q];
    else
        for (size_t q = 0; q < n; ++q) s += x[q] * y[q];
    return s;
}

static double norm2(const double *x, size_t n) { return sqrt(dot(x, x, n)); }

/* ------------------------------------------------------------------ */
/* implicit transport solves (Step 1 momentum, Step 2 enthalpy)          */
/* ------------------------------------------------------------------ */

/* Residual of (rho1/dt) X + C(X) - diffusion(X) = b at every cell (mu NULL:
 * constant viscosity nu). */
static void transport_residual(const orc_cfg *c, const double *rho1, const double *phix,
                               const double *phiz, const double *mu, double nu, const double *X,
                               int bc, const double *b, double *r)
{
    int nx = c->nx, nz = c->nz;
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < nx; ++i) {
            int q = k * nx + i;
            double lhs = rho1[q] / c->dt * X[q]
                       + orc_convection_cell(c, phix, phiz, X, bc, i, k)
                       - diffusion(c, mu, nu, X, bc, i, k);
            r[q] = b[q] - lhs;
        }
}

/* Left-hand side (rho1/dt) X + C(X) - nu L(X) at every cell. */
void orc_transport_apply(const orc_cfg *c, const double *rho1, const double *phix,
                         const double *phiz, double nu, int bc, const double *X,
                         double *out)
{
    size_t n = (size_t)c->nx * c->nz;
    double *zero = calloc(n, sizeof(double));
    transport_residual(c, rho1, phix, phiz, NULL, nu, X, bc, zero, out);
    for (size_t q = 0; q < n; ++q) out[q] = -out[q];
    free(zero);
}

/* Jacobi iteration for (rho1/dt) X + C(X) - nu L(X) = b from the initial X.
 * The Jacobi divisor is the coefficient of X_i in the interior stencil:
 * rho1/dt + (7/12) sum_j phi_j / V + nu (2/dx^2 + 2/dz^2).
 * Every sweep computes the residual r of the current X and updates
 * X <- X + r/d; the iteration stops after the sweep whose residual met
 * ||r|| <= jac_rtol ||b||, so the returned X is one contraction beyond the
 * tolerance. Returns the number of sweeps, or -1 if jac_maxit was reached. */
static int transport_solve(const orc_cfg *c, const double *rho1, const double *phix,
                           const double *phiz, const double *mu, double nu, int bc, const double *b,
                           double *X)
{
    int nx = c->nx, nz = c->nz;
    size_t n = (size_t)nx * nz;
    double *r = malloc(n * sizeof(double));
    double bn = norm2(b, n);
    int sweeps = 0, ok = 0;
    while (sweeps < c->jac_maxit) {
        transport_residual(c, rho1, phix, phiz, mu, nu, X, bc, b, r);
        double rn = norm2(r, n);
        for (int k = 0; k < nz; ++k)
            for (int i = 0; i < nx; ++i) {
                int q = k * nx + i;
                double d = rho1[q] / c->dt
                         + 7.0 / 12.0 * orc_divergence_cell(c, phix, phiz, i, k)
                         + diffusion_diag(c, mu, nu, i, k);
                X[q] += r[q] / d;
            }
        ++sweeps;
        if (rn <= c->jac_rtol * bn) { ok = 1; break; }
    }
    free(r);
    return ok ? sweeps : -1;
}

int orc_transport_solve(const orc_cfg *c, const double *rho1, const double *phix,
                        const double *phiz, double nu, int bc, const double *b,
                        double *X)
{
    return transport_solve(c, rho1, phix, phiz, NULL, nu, bc, b, X);
}

/* ------------------------------------------------------------------ */
/* pressure (Helmholtz) problem of Step 3                              */
/* ------------------------------------------------------------------ */

/* y = A x with (A x)_i = (psi_i/dt) x_i + (1/V) sum_f D_f |A_f| (x_i - x_N)/Delta_f
 * over interior faces. Dx: nz*(nx+1), Dz: (nz+1)*nx face coefficients
 * D_f = dt rho2_f / rho1_f (zero on walls). */
void orc_helmholtz_apply(const orc_cfg *c, const double *psi, const double *Dx,
                         const double *Dz, const double *x, double *y)
{
    int nx = c->nx, nz = c->nz;
    double dx = dxof(c), dz = dzof(c), V = dx * dz;
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < nx; ++i) {
            int q = k * nx + i;
            double s = 0.0;
            if (i + 1 < nx) s += Dx[k * (nx + 1) + i + 1] * dz * (x[q] - x[q + 1]) / dx;
            if (i > 0)      s += Dx[k * (nx + 1) + i] * dz * (x[q] - x[q - 1]) / dx;
            if (k + 1 < nz) s += Dz[(k + 1) * nx + i] * dx * (x[q] - x[q + nx]) / dz;
            if (k > 0)      s += Dz[k * nx + i] * dx * (x[q] - x[q - nx]) / dz;
            y[q] = psi[q] / c->dt * x[q] + s / V;
        }
}

/* Diagonal of A. */
static void helmholtz_diag(const orc_cfg *c, const double *psi, const double *Dx,
                           const double *Dz, double *d)
{
    int nx = c->nx, nz = c->nz;
    double dx = dxof(c), dz = dzof(c), V = dx * dz;
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < nx; ++i) {
            int q = k * nx + i;
            double s = 0.0;
            if (i + 1 < nx) s += Dx[k * (nx + 1) + i + 1] * dz / dx;
            if (i > 0)      s += Dx[k * (nx + 1) + i] * dz / dx;
            if (k + 1 < nz) s += Dz[(k + 1) * nx + i] * dx / dz;
            if (k > 0)      s += Dz[k * nx + i] * dx / dz;
            d[q] = psi[q] / c->dt + s / V;
        }
}

/* Diagonally preconditioned conjugate gradients for A x = b from the initial
 * x, stopped at ||r|| <= cg_rtol ||b||. Returns iterations or -1. */
int orc_pcg(const orc_cfg *c, const double *psi, const double *Dx, const double *Dz,
            const double *b, double *x, double *relres)
{
    size_t n = (size_t)c->nx * c->nz;
    double *r = malloc(n * sizeof(double)), *z = malloc(n * sizeof(double));
    double *p = malloc(n * sizeof(double)), *q = malloc(n * sizeof(double));
    double *d = malloc(n * sizeof(double));
    helmholtz_diag(c, psi, Dx, Dz, d);
    orc_helmholtz_apply(c, psi, Dx, Dz, x, q);
    for (size_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    double bn = norm2(b, n);
    double rn = norm2(r, n);
    int it = 0, ok = 0;
    for (size_t i = 0; i < n; ++i) { z[i] = r[i] / d[i]; p[i] = z[i]; }
    double rz = dot(r, z, n);
    for (;;) {
        if (rn <= c->cg_rtol * bn || rn == 0.0) { ok = 1; break; }
        if (it >= c->cg_maxit) break;
        orc_helmholtz_apply(c, psi, Dx, Dz, p, q);
        double pq = dot(p, q, n);
        double alpha = rz / pq;
        for (size_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        for (size_t i = 0; i < n; ++i) z[i] = r[i] / d[i];
        double rz_new = dot(r, z, n);
        double beta = rz_new / rz;
        rz = rz_new;
        for (size_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        rn = norm2(r, n);
        ++it;
    }
    if (relres) *relres = bn > 0.0 ? rn / bn : 0.0;
    free(r); free(z); free(p); free(q); free(d);
    return ok ? it : -1;
}

/* ------------------------------------------------------------------ */
/* set-up from conservative variables                                  */
/* ------------------------------------------------------------------ */

/* From (rho, rho u, rho w, rho e) with e = cv T + |u|^2/2 + g z (Section 2.1):
 * u = (rho u)/rho, T = (e - K - g z)/cv, p = rho R T (eq. p), h = cp T
 * (eq. K_h), p' = p + rho g z, p^{n-1} = p, K^{n-1} = K, and phi on interior
 * faces the linear average of the two cells' normal momentum times the face
 * area (zero on walls). */
int orc_derive(const orc_cfg *c, const double *rho, const double *rhou,
               const double *rhow, const double *rhoe, orc_state *s)
{
    int nx = c->nx, nz = c->nz;
    double dx = dxof(c), dz = dzof(c), cv = c->cp - c->R;
    for (int k = 0; k < nz; ++k) {
        double z = (k + 0.5) * dz;
        for (int i = 0; i < nx; ++i) {
            int q = k * nx + i;
            if (!(rho[q] > 0.0)) return 1;
            double u = rhou[q] / rho[q], w = rhow[q] / rho[q];
            double K = 0.5 * (u * u + w * w);
            double T = (rhoe[q] / rho[q] - K - c->g * z) / cv;
            if (!(T > 0.0)) return 1;
            s->rho[q] = rho[q];
            s->u[q] = u;
            s->w[q] = w;
            s->T[q] = T;
            s->h[q] = c->cp * T;
            s->p[q] = rho[q] * c->R * T;
            s->pp[q] = s->p[q] + rho[q] * c->g * z;
            s->pold[q] = s->p[q];
            s->Kold[q] = K;
        }
    }
    for (int k = 0; k < nz; ++k)
        for (int f = 0; f <= nx; ++f) {
            double v = 0.0;
            if (f > 0 && f < nx) v = 0.5 * (rhou[k * nx + f - 1] + rhou[k * nx + f]) * dz;
            s->phix[k * (nx + 1) + f] = v;
        }
    for (int f = 0; f <= nz; ++f)
        for (int i = 0; i < nx; ++i) {
            double v = 0.0;
            if (f > 0 && f < nz) v = 0.5 * (rhow[(f - 1) * nx + i] + rhow[f * nx + i]) * dx;
            s->phiz[f * nx + i] = v;
        }
    return 0;
}

/* ------------------------------------------------------------------ */
/* one time step (Section 3, Steps 1-3, PISO correctors)               */
/* ------------------------------------------------------------------ */

static double *zalloc(size_t n) { return calloc(n, sizeof(double)); }

int orc_step(const orc_cfg *c, orc_state *s, int32_t nsteps, orc_stats *st, orc_dump *dump)
{
    int nx = c->nx, nz = c->nz;
    size_t n = (size_t)nx * nz, nfx = (size_t)nz * (nx + 1), nfz = (size_t)(nz + 1) * nx;
    double dt = c->dt, g = c->g, dx = dxof(c), dz = dzof(c);
    int status = 0;

    double *rho1 = zalloc(n), *u1 = zalloc(n), *w1 = zalloc(n), *K1 = zalloc(n);
    double *bu = zalloc(n), *bw = zalloc(n), *bh = zalloc(n), *h1 = zalloc(n);
    double *T1 = zalloc(n), *rho2 = zalloc(n), *psi = zalloc(n);
    double *Hx = zalloc(n), *Hz = zalloc(n), *b = zalloc(n);
    double *U = zalloc(n), *W = zalloc(n), *pnew = zalloc(n), *rhonew = zalloc(n);
    double *pnext = zalloc(n);
    double *Gx = zalloc(nfx), *Gz = zalloc(nfz), *Dx = zalloc(nfx), *Dz = zalloc(nfz);
    double *Fx = zalloc(nfx), *Fz = zalloc(nfz);
    /* Smagorinsky LES: the viscosity field of the step (from rho^n, u^n); the
     * constant-viscosity scheme of Remark 1 otherwise */
    double *mu_eff = c->cs > 0.0 ? zalloc(n) : NULL;
    double nu_u = mu_eff ? 1.0 : c->mu, nu_h = mu_eff ? 1.0 / c->Pr : c->mu / c->Pr;

    for (int step = 0; step < nsteps; ++step) {
        if (mu_eff) orc_smagorinsky(c, s->rho, s->u, s->w, mu_eff);
        /* ---- Step 1, eq. (e1_d): rho^{n+1/3} = rho^n - dt sum_j phi^n_j / V ---- */
        for (int k = 0; k < nz; ++k)
            for (int i = 0; i < nx; ++i)
                rho1[k * nx + i] = s->rho[k * nx + i]
                                 - dt * orc_divergence_cell(c, s->phix, s->phiz, i, k);

        /* ---- Step 1, eq. (step2_sd), predictor: implicit in u^{n+1/3}, with the
         * balanced force grad p'^n - g z grad rho^n of eq. (mom_split) explicit
         * and b_u = rho^n u^n / dt ---- */
        face_forces(c, s->pp, s->rho, Gx, Gz);
        for (int k = 0; k < nz; ++k)
            for (int i = 0; i < nx; ++i) {
                int q = k * nx + i;
                double Gcx = 0.5 * (Gx[k * (nx + 1) + i] + Gx[k * (nx + 1) + i + 1]);
                double Gcz = 0.5 * (Gz[k * nx + i] + Gz[(k + 1) * nx + i]);
                bu[q] = s->rho[q] * s->u[q] / dt - Gcx;
                bw[q] = s->rho[q] * s->w[q] / dt - Gcz;
                u1[q] = s->u[q];
                w1[q] = s->w[q];
            }
        int su = transport_solve(c, rho1, s->phix, s->phiz, mu_eff, nu_u, BC_U, bu, u1);
        int sw = transport_solve(c, rho1, s->phix, s->phiz, mu_eff, nu_u, BC_W, bw, w1);
        if (su < 0 || sw < 0) status = 1;

        /* ---- Step 1, eq. (step1_3sd): K^{n+1/3} = |u^{n+1/3}|^2 / 2 ---- */
        for (size_t q = 0; q < n; ++q) K1[q] = 0.5 * (u1[q] * u1[q] + w1[q] * w1[q]);

        /* ---- Step 2, eq. (step3_sd): enthalpy, implicit in h^{n+1}. Right-hand
         * side b~_e - rho1 K1/dt - sum_j phi_j K1_j / V + p^n/dt - rho1 g w1 with
         * b~_e = (rho^n h^n + rho^n K^n - p^{n-1})/dt, or with K^{n-1} in place
         * of K^n in the literal reading ---- */
        for (int k = 0; k < nz; ++k)
            for (int i = 0; i < nx; ++i) {
                int q = k * nx + i;
                double Kn = (c->reading_flags & ORC_READING_K_LAGGED)
                                ? s->Kold[q]
                                : 0.5 * (s->u[q] * s->u[q] + s->w[q] * s->w[q]);
                double be = (s->rho[q] * s->h[q] + s->rho[q] * Kn - s->pold[q]) / dt;
                bh[q] = be - rho1[q] * K1[q] / dt
                      - orc_convection_cell(c, s->phix, s->phiz, K1, BC_EVEN, i, k)
                      + s->p[q] / dt - rho1[q] * g * w1[q];
                h1[q] = s->h[q];
            }
        int sh = transport_solve(c, rho1, s->phix, s->phiz, mu_eff, nu_h, BC_H, bh, h1);
        if (sh < 0) status = 1;

        /* ---- Step 2, eq. (step3_2sd): T^{n+1} = T^n + (h^{n+1} - h^n)/cp;
         * eq. (step3_3sd): rho^{n+2/3} = p^n / (R T^{n+1}); psi = 1/(R T^{n+1}) ---- */
        for (size_t q = 0; q < n; ++q) {
            T1[q] = s->T[q] + (h1[q] - s->h[q]) / c->cp;
            rho2[q] = s->p[q] / (c->R * T1[q]);
            psi[q] = 1.0 / (c->R * T1[q]);
        }

        /* face coefficients D_f = dt rho2_f / rho1_f (linear face averages) */
        for (int k = 0; k < nz; ++k)
            for (int f = 0; f <= nx; ++f) {
                double D = 0.0;
                if (f > 0 && f < nx) {
                    int a = k * nx + f - 1, bb = k * nx + f;
                    D = dt * (0.5 * (rho2[a] + rho2[bb])) / (0.5 * (rho1[a] + rho1[bb]));
                }
                Dx[k * (nx + 1) + f] = D;
            }
        for (int f = 0; f <= nz; ++f)
            for (int i = 0; i < nx; ++i) {
                double D = 0.0;
                if (f > 0 && f < nz) {
                    int a = (f - 1) * nx + i, bb = f * nx + i;
                    D = dt * (0.5 * (rho2[a] + rho2[bb])) / (0.5 * (rho1[a] + rho1[bb]));
                }
                Dz[f * nx + i] = D;
            }

        memcpy(U, u1, n * sizeof(double));
        memcpy(W, w1, n * sizeof(double));
        memcpy(pnew, s->pp, n * sizeof(double));   /* p' initial guess: p'^n */

        /* ---- Step 3: PISO correctors ---- */
        for (int corr = 0; corr < c->n_corr; ++corr) {
            /* H(u) = b_u - sum_j phi^n_j u_j / V + mu sum_j (grad u)_j . A_j / V at
             * the newest velocity (definition below eq. step2_sd, second line) */
            for (int k = 0; k < nz; ++k)
                for (int i = 0; i < nx; ++i) {
                    int q = k * nx + i;
                    Hx[q] = s->rho[q] * s->u[q] / dt
                          - orc_convection_cell(c, s->phix, s->phiz, U, BC_U, i, k)
                          + diffusion(c, mu_eff, nu_u, U, BC_U, i, k);
                    Hz[q] = s->rho[q] * s->w[q] / dt
                          - orc_convection_cell(c, s->phix, s->phiz, W, BC_W, i, k)
                          + diffusion(c, mu_eff, nu_u, W, BC_W, i, k);
                }
            /* right-hand side of the pressure equation (eq. p_prime_sd, Helmholtz
             * form from continuity with rho^{n+1} = psi (p' - rho2 g z)) */
            for (int k = 0; k < nz; ++k) {
                double zc = (k + 0.5) * dz;
                for (int i = 0; i < nx; ++i) {
                    int q = k * nx + i;
                    double flux = 0.0;   /* sum_f D_f |A_f| [H_f . n + g z_f (rho2_N - rho2_i)/Delta] */
                    if (i + 1 < nx) {
                        int N = q + 1;
                        double Hf = 0.5 * (Hx[q] + Hx[N]);
                        flux += Dx[k * (nx + 1) + i + 1] * dz * (Hf + g * zc * (rho2[N] - rho2[q]) / dx);
                    }
                    if (i > 0) {
                        int N = q - 1;
                        double Hf = 0.5 * (Hx[q] + Hx[N]);
                        flux += Dx[k * (nx + 1) + i] * dz * (-Hf + g * zc * (rho2[N] - rho2[q]) / dx);
                    }
                    if (k + 1 < nz) {
                        int N = q + nx;
                        double Hf = 0.5 * (Hz[q] + Hz[N]);
                        double zf = (k + 1) * dz;
                        flux += Dz[(k + 1) * nx + i] * dx * (Hf + g * zf * (rho2[N] - rho2[q]) / dz);
                    }
                    if (k > 0) {
                        int N = q - nx;
                        double Hf = 0.5 * (Hz[q] + Hz[N]);
                        double zf = k * dz;
                        flux += Dz[k * nx + i] * dx * (-Hf + g * zf * (rho2[N] - rho2[q]) / dz);
                    }
                    b[q] = (s->rho[q] + psi[q] * rho2[q] * g * zc) / dt - flux / (dx * dz);
                }
            }
            double relres = 0.0;
            int it = orc_pcg(c, psi, Dx, Dz, b, pnew, &relres);
            if (corr < 4 && st) { st->cg_iters[corr] = it; st->cg_relres[corr] = relres; }
            if (it < 0) status = 1;

            /* correction: F_f = D_f (H_f - G_f) with G_f from p'^{n+1} and rho2;
             * u = (dt/rho1)(H - G_cell) (eq. step2_sd second line); eq. (step4_4sd) */
            face_forces(c, pnew, rho2, Gx, Gz);
            for (int k = 0; k < nz; ++k)
                for (int f = 0; f <= nx; ++f) {
                    double F = 0.0;
                    if (f > 0 && f < nx) {
                        int a = k * nx + f - 1, bb = k * nx + f;
                        F = Dx[k * (nx + 1) + f] * (0.5 * (Hx[a] + Hx[bb]) - Gx[k * (nx + 1) + f]);
                    }
                    Fx[k * (nx + 1) + f] = F;
                }
            for (int f = 0; f <= nz; ++f)
                for (int i = 0; i < nx; ++i) {
                    double F = 0.0;
                    if (f > 0 && f < nz) {
                        int a = (f - 1) * nx + i, bb = f * nx + i;
                        F = Dz[f * nx + i] * (0.5 * (Hz[a] + Hz[bb]) - Gz[f * nx + i]);
                    }
                    Fz[f * nx + i] = F;
                }
            for (int k = 0; k < nz; ++k) {
                double zc = (k + 0.5) * dz;
                for (int i = 0; i < nx; ++i) {
                    int q = k * nx + i;
                    double Gcx = 0.5 * (Gx[k * (nx + 1) + i] + Gx[k * (nx + 1) + i + 1]);
                    double Gcz = 0.5 * (Gz[k * nx + i] + Gz[(k + 1) * nx + i]);
                    U[q] = dt / rho1[q] * (Hx[q] - Gcx);
                    W[q] = dt / rho1[q] * (Hz[q] - Gcz);
                    double pn = pnew[q] - rho2[q] * g * zc;       /* p = p' - rho2 g z */
                    rhonew[q] = pn / (c->R * T1[q]);               /* rho = p/(R T) */
                    pnext[q] = pn;
                }
            }
        }

        if (dump) {
            if (dump->rho1) memcpy(dump->rho1, rho1, n * sizeof(double));
            if (dump->u1) memcpy(dump->u1, u1, n * sizeof(double));
            if (dump->w1) memcpy(dump->w1, w1, n * sizeof(double));
            if (dump->h1) memcpy(dump->h1, h1, n * sizeof(double));
            if (dump->T1) memcpy(dump->T1, T1, n * sizeof(double));
            if (dump->rho2) memcpy(dump->rho2, rho2, n * sizeof(double));
            if (dump->psi) memcpy(dump->psi, psi, n * sizeof(double));
            if (dump->Hx) memcpy(dump->Hx, Hx, n * sizeof(double));
            if (dump->Hz) memcpy(dump->Hz, Hz, n * sizeof(double));
            if (dump->b) memcpy(dump->b, b, n * sizeof(double));
            if (dump->Dx) memcpy(dump->Dx, Dx, nfx * sizeof(double));
            if (dump->Dz) memcpy(dump->Dz, Dz, nfz * sizeof(double));
            if (dump->bh) memcpy(dump->bh, bh, n * sizeof(double));
        }

        /* ---- end of step: the new state; p^{n-1} <- p^n, K^{n-1} <- K^n ---- */
        for (size_t q = 0; q < n; ++q) s->Kold[q] = 0.5 * (s->u[q] * s->u[q] + s->w[q] * s->w[q]);
        memcpy(s->pold, s->p, n * sizeof(double));
        memcpy(s->p, pnext, n * sizeof(double));
        memcpy(s->pp, pnew, n * sizeof(double));
        memcpy(s->rho, rhonew, n * sizeof(double));
        memcpy(s->u, U, n * sizeof(double));
        memcpy(s->w, W, n * sizeof(double));
        memcpy(s->T, T1, n * sizeof(double));
        memcpy(s->h, h1, n * sizeof(double));
        for (size_t q = 0; q < nfx; ++q) s->phix[q] = Fx[q] * dz;   /* phi = F |A| */
        for (size_t q = 0; q < nfz; ++q) s->phiz[q] = Fz[q] * dx;
        if (st) { st->jac_u = su; st->jac_w = sw; st->jac_h = sh; }
    }
    if (st) st->status = status;

    free(rho1); free(u1); free(w1); free(K1); free(bu); free(bw); free(bh); free(h1);
    free(T1); free(rho2); free(psi); free(Hx); free(Hz); free(b); free(U); free(W);
    free(pnew); free(rhonew); free(pnext); free(Gx); free(Gz); free(Dx); free(Dz); free(Fx); free(Fz);
    free(mu_eff);
    return status;
}

/* ------------------------------------------------------------------ */
/* diagnostics (Remark 2)                                              */
/* ------------------------------------------------------------------ */

/* theta' = T / (p/p0)^(R/cp) - theta_bar(z) (eqs. theta, theta_split), and the
 * totals of mass sum rho V and energy sum rho e V with e = cv T + K + g z. */
void orc_diagnostics(const orc_cfg *c, const orc_state *s, const double *theta_bar,
                     double *theta_prime, double *mass, double *energy)
{
    int nx = c->nx, nz = c->nz;
    double dz = dzof(c), V = dxof(c) * dz, cv = c->cp - c->R;
    double m = 0.0, e = 0.0;
    for (int k = 0; k < nz; ++k) {
        double z = (k + 0.5) * dz;
        for (int i = 0; i < nx; ++i) {
            int q = k * nx + i;
            double th = s->T[q] / pow(s->p[q] / c->p0, c->R / c->cp);
            if (theta_prime) theta_prime[q] = th - theta_bar[k];
            double K = 0.5 * (s->u[q] * s->u[q] + s->w[q] * s->w[q]);
            m += s->rho[q] * V;
            e += s->rho[q] * (cv * s->T[q] + K + c->g * z) * V;
        }
    }
    if (mass) *mass = m;
    if (energy) *energy = e;
}

/* Per-cell residual of the discrete continuity equation after a step,
 * (rho^{n+1} - rho^n)/dt + sum_j phi^{n+1}_j / V, given rho^n. */
void orc_continuity_residual(const orc_cfg *c, const double *rho_old, const orc_state *s,
                             double *res)
{
    int nx = c->nx, nz = c->nz;
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < nx; ++i) {
            int q = k * nx + i;
            res[q] = (s->rho[q] - rho_old[q]) / c->dt
                   + orc_divergence_cell(c, s->phix, s->phiz, i, k);
        }
}

/* Whole-field operator helpers used by the tests. */
void orc_convection(const orc_cfg *c, const double *phix, const double *phiz,
                    const double *X, int bc, double *out)
{
    for (int k = 0; k < c->nz; ++k)
        for (int i = 0; i < c->nx; ++i)
            out[k * c->nx + i] = orc_convection_cell(c, phix, phiz, X, bc, i, k);
}

void orc_strain(const orc_cfg *c, const double *u, const double *w, double *out)
{
    for (int k = 0; k < c->nz; ++k)
        for (int i = 0; i < c->nx; ++i) out[k * c->nx + i] = orc_strain_cell(c, u, w, i, k);
}

void orc_diffusion(const orc_cfg *c, const double *mu, const double *X, int bc, double *out)
{
    for (int k = 0; k < c->nz; ++k)
        for (int i = 0; i < c->nx; ++i) out[k * c->nx + i] = orc_diffusion_cell(c, mu, X, bc, i, k);
}

void orc_laplacian(const orc_cfg *c, const double *X, int bc, double *out)
{
    for (int k = 0; k < c->nz; ++k)
        for (int i = 0; i < c->nx; ++i)
            out[k * c->nx + i] = orc_laplacian_cell(c, X, bc, i, k);
}

void orc_face_forces(const orc_cfg *c, const double *pp, const double *rho,
                     double *Gx, double *Gz)
{
    face_forces(c, pp, rho, Gx, Gz);
}
