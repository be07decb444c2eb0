/*
 * gea_oracle3d.c -- plain FP64 CPU oracle of one predictor-corrector time
 * step of the GEA pressure-based Euler solver (Girfoglio, Quaini & Rozza,
 * arXiv 2303.10499, Section 3) on a uniform Cartesian x-y-z grid.
 *
 * TEST INFRASTRUCTURE. This file exists only to check the CUDA library. Only
 * the test suite and the benchmark's CPU legs may load it; the library never
 * calls it and shares no code with it.
 *
 * The discretisation is the two-dimensional oracle's with a third direction:
 * x and y horizontal, z up (gravity g along -z), nx * ny * nz cells of size
 * dx * dy * dz, free-slip walls on all six sides, constant viscosity mu
 * (Remark 1). Per face: fourth-order four-point convected values
 * X_f = (-X_{a-1} + 7 X_a + 7 X_b - X_{b+1})/12, compact two-point
 * Laplacian and gradients, face sums divided by V = dx dy dz. One ghost
 * layer: the wall-normal velocity component odd, the others even, scalars
 * even, h with dh/dz = -g on the bottom and top walls. Face forces
 * G_f = (p'_b - p'_a)/Delta - g z_f (rho_b - rho_a)/Delta reach cells as
 * the average of the two faces per direction (zero on walls). The pressure
 * equation is the Helmholtz form
 *   (psi_i/dt) p'_i + (1/V) sum_f D_f |A_f| (p'_i - p'_N)/Delta_f
 *     = (rho^n_i + psi_i rho2_i g z_i)/dt
 *       - (1/V) sum_f D_f |A_f| [H_f . n + g z_f (rho2_N - rho2_i)/Delta_f].
 * The predictors are solved by Jacobi (stopping after the sweep whose
 * residual met the tolerance), the pressure equation by diagonally
 * preconditioned conjugate gradients.
 *
 * Storage: cell (i,j,k) at (k*ny + j)*nx + i; x-faces (k*ny + j)*(nx+1) + f
 * (face f between cells f-1 and f), y-faces (k*(ny+1) + f)*nx + i, z-faces
 * (f*ny + j)*nx + i. Wall faces carry zero flux.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nx, ny, nz;
    double lx, ly, lz;
    double R, cp, g, p0, mu, Pr, dt;
    int32_t n_corr;
    double jac_rtol;
    int32_t jac_maxit;
    double cg_rtol;
    int32_t cg_maxit;
    double cs;          /* Smagorinsky constant; 0: constant viscosity mu only */
} o3_cfg;

typedef struct {
    double *rho, *u, *v, *w, *T, *h, *p, *pp, *pold, *phix, *phiy, *phiz;
} o3_state;

typedef struct {
    int32_t jac_u, jac_h;          /* Jacobi sweeps of the last step */
    int32_t cg_iters[4];
    double cg_relres[4];
    int32_t status;                /* 0 ok, 1 a solver hit its cap */
} o3_stats;

enum { B3_EVEN = 0, B3_U = 1, B3_V = 2, B3_W = 3, B3_H = 4 };

static double DX(const o3_cfg *c) { return c->lx / c->nx; }
static double DY(const o3_cfg *c) { return c->ly / c->ny; }
static double DZ(const o3_cfg *c) { return c->lz / c->nz; }
static size_t ncell(const o3_cfg *c) { return (size_t)c->nx * c->ny * c->nz; }
static size_t cid(const o3_cfg *c, int i, int j, int k) { return ((size_t)k * c->ny + j) * c->nx + i; }
static size_t fxid(const o3_cfg *c, int f, int j, int k) { return ((size_t)k * c->ny + j) * (c->nx + 1) + f; }
static size_t fyid(const o3_cfg *c, int i, int f, int k) { return ((size_t)k * (c->ny + 1) + f) * c->nx + i; }
static size_t fzid(const o3_cfg *c, int i, int j, int f) { return ((size_t)f * c->ny + j) * c->nx + i; }

/* Value of X at (i,j,k), at most one index one layer outside the box: the
 * ghost of wall rule bc there. */
static double at3(const o3_cfg *c, const double *X, int i, int j, int k, int bc)
{
    if (i < 0) { double v = X[cid(c, 0, j, k)]; return bc == B3_U ? -v : v; }
    if (i >= c->nx) { double v = X[cid(c, c->nx - 1, j, k)]; return bc == B3_U ? -v : v; }
    if (j < 0) { double v = X[cid(c, i, 0, k)]; return bc == B3_V ? -v : v; }
    if (j >= c->ny) { double v = X[cid(c, i, c->ny - 1, k)]; return bc == B3_V ? -v : v; }
    if (k < 0) {
        double v = X[cid(c, i, j, 0)];
        if (bc == B3_W) return -v;
        if (bc == B3_H) return v + c->g * DZ(c);
        return v;
    }
    if (k >= c->nz) {
        double v = X[cid(c, i, j, c->nz - 1)];
        if (bc == B3_W) return -v;
        if (bc == B3_H) return v - c->g * DZ(c);
        return v;
    }
    return X[cid(c, i, j, k)];
}

static double interp4(double xm, double xa, double xb, double xp)
{
    return (-xm + 7.0 * xa + 7.0 * xb - xp) / 12.0;
}

/* (1/V) sum_j phi_j X_j over the six faces of cell (i,j,k), X_j by interp4,
 * outward positive; wall faces carry no flux. */
double o3_convection_cell(const o3_cfg *c, const double *phix, const double *phiy, const double *phiz,
                          const double *X, int bc, int i, int j, int k)
{
    double V = DX(c) * DY(c) * DZ(c), s = 0.0;
    if (i + 1 < c->nx)
        s += phix[fxid(c, i + 1, j, k)] * interp4(at3(c, X, i - 1, j, k, bc), at3(c, X, i, j, k, bc),
                                                  at3(c, X, i + 1, j, k, bc), at3(c, X, i + 2, j, k, bc));
    if (i > 0)
        s -= phix[fxid(c, i, j, k)] * interp4(at3(c, X, i - 2, j, k, bc), at3(c, X, i - 1, j, k, bc),
                                              at3(c, X, i, j, k, bc), at3(c, X, i + 1, j, k, bc));
    if (j + 1 < c->ny)
        s += phiy[fyid(c, i, j + 1, k)] * interp4(at3(c, X, i, j - 1, k, bc), at3(c, X, i, j, k, bc),
                                                  at3(c, X, i, j + 1, k, bc), at3(c, X, i, j + 2, k, bc));
    if (j > 0)
        s -= phiy[fyid(c, i, j, k)] * interp4(at3(c, X, i, j - 2, k, bc), at3(c, X, i, j - 1, k, bc),
                                              at3(c, X, i, j, k, bc), at3(c, X, i, j + 1, k, bc));
    if (k + 1 < c->nz)
        s += phiz[fzid(c, i, j, k + 1)] * interp4(at3(c, X, i, j, k - 1, bc), at3(c, X, i, j, k, bc),
                                                  at3(c, X, i, j, k + 1, bc), at3(c, X, i, j, k + 2, bc));
    if (k > 0)
        s -= phiz[fzid(c, i, j, k)] * interp4(at3(c, X, i, j, k - 2, bc), at3(c, X, i, j, k - 1, bc),
                                              at3(c, X, i, j, k, bc), at3(c, X, i, j, k + 1, bc));
    return s / V;
}

/* (1/V) sum_j (grad X)_j . A_j, compact face gradients through the ghosts. */
double o3_laplacian_cell(const o3_cfg *c, const double *X, int bc, int i, int j, int k)
{
    double dx = DX(c), dy = DY(c), dz = DZ(c), xc = at3(c, X, i, j, k, bc);
    double s = (at3(c, X, i + 1, j, k, bc) - xc + at3(c, X, i - 1, j, k, bc) - xc) / (dx * dx)
             + (at3(c, X, i, j + 1, k, bc) - xc + at3(c, X, i, j - 1, k, bc) - xc) / (dy * dy)
             + (at3(c, X, i, j, k + 1, bc) - xc + at3(c, X, i, j, k - 1, bc) - xc) / (dz * dz);
    return s;
}

/* Strain-rate magnitude |S| = sqrt(2 S_ij S_ij) of cell (i,j,k) from central
 * differences of the cell velocities (ghosts by the wall rules):
 * 2 S_ij S_ij = 2 (u_x^2 + v_y^2 + w_z^2) + (u_y + v_x)^2 + (u_z + w_x)^2
 * + (v_z + w_y)^2. */
double o3_strain_cell(const o3_cfg *c, const double *u, const double *v, const double *w, int i, int j, int k)
{
    double hx = 1.0 / (2.0 * DX(c)), hy = 1.0 / (2.0 * DY(c)), hz = 1.0 / (2.0 * DZ(c));
    double ux = (at3(c, u, i + 1, j, k, B3_U) - at3(c, u, i - 1, j, k, B3_U)) * hx;
    double uy = (at3(c, u, i, j + 1, k, B3_U) - at3(c, u, i, j - 1, k, B3_U)) * hy;
    double uz = (at3(c, u, i, j, k + 1, B3_U) - at3(c, u, i, j, k - 1, B3_U)) * hz;
    double vx = (at3(c, v, i + 1, j, k, B3_V) - at3(c, v, i - 1, j, k, B3_V)) * hx;
    double vy = (at3(c, v, i, j + 1, k, B3_V) - at3(c, v, i, j - 1, k, B3_V)) * hy;
    double vz = (at3(c, v, i, j, k + 1, B3_V) - at3(c, v, i, j, k - 1, B3_V)) * hz;
    double wx = (at3(c, w, i + 1, j, k, B3_W) - at3(c, w, i - 1, j, k, B3_W)) * hx;
    double wy = (at3(c, w, i, j + 1, k, B3_W) - at3(c, w, i, j - 1, k, B3_W)) * hy;
    double wz = (at3(c, w, i, j, k + 1, B3_W) - at3(c, w, i, j, k - 1, B3_W)) * hz;
    double sxy = uy + vx, sxz = uz + wx, syz = vz + wy;
    return sqrt(2.0 * (ux * ux + vy * vy + wz * wz) + sxy * sxy + sxz * sxz + syz * syz);
}

/* Effective dynamic viscosity mu + rho (cs Delta)^2 |S| at every cell, with
 * the filter width Delta = (dx dy dz)^(1/3). */
void o3_smagorinsky(const o3_cfg *c, const double *rho, const double *u, const double *v, const double *w,
                    double *mu_eff)
{
    double delta = cbrt(DX(c) * DY(c) * DZ(c));
    double d2 = c->cs * c->cs * delta * delta;
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                size_t q = cid(c, i, j, k);
                mu_eff[q] = c->mu + rho[q] * d2 * o3_strain_cell(c, u, v, w, i, j, k);
            }
}

/* Variable-coefficient diffusive face sum (1/V) sum_j mu_j (grad X)_j . A_j of
 * cell (i,j,k): mu_j the mean of the two cells' viscosities (a wall face takes
 * the cell's own, the even ghost), compact face gradients through the ghosts. */
double o3_diffusion_cell(const o3_cfg *c, const double *mu, const double *X, int bc, int i, int j, int k)
{
    double dx = DX(c), dy = DY(c), dz = DZ(c);
    double xc = at3(c, X, i, j, k, bc), mc = at3(c, mu, i, j, k, B3_EVEN);
    double s = 0.0;
    s += 0.5 * (mc + at3(c, mu, i + 1, j, k, B3_EVEN)) * (at3(c, X, i + 1, j, k, bc) - xc) / (dx * dx);
    s += 0.5 * (mc + at3(c, mu, i - 1, j, k, B3_EVEN)) * (at3(c, X, i - 1, j, k, bc) - xc) / (dx * dx);
    s += 0.5 * (mc + at3(c, mu, i, j + 1, k, B3_EVEN)) * (at3(c, X, i, j + 1, k, bc) - xc) / (dy * dy);
    s += 0.5 * (mc + at3(c, mu, i, j - 1, k, B3_EVEN)) * (at3(c, X, i, j - 1, k, bc) - xc) / (dy * dy);
    s += 0.5 * (mc + at3(c, mu, i, j, k + 1, B3_EVEN)) * (at3(c, X, i, j, k + 1, bc) - xc) / (dz * dz);
    s += 0.5 * (mc + at3(c, mu, i, j, k - 1, B3_EVEN)) * (at3(c, X, i, j, k - 1, bc) - xc) / (dz * dz);
    return s;
}

/* The diffusion term of the transport operators: nu L(X) with constant nu,
 * or nu times the variable-coefficient sum with the viscosity field mu. */
static double diffusion3(const o3_cfg *c, const double *mu, double nu, const double *X, int bc, int i, int j,
                         int k)
{
    return mu ? nu * o3_diffusion_cell(c, mu, X, bc, i, j, k) : nu * o3_laplacian_cell(c, X, bc, i, j, k);
}

/* Coefficient of X_i in -diffusion3() (interior cell). */
static double diffusion_diag3(const o3_cfg *c, const double *mu, double nu, int i, int j, int k)
{
    double dx = DX(c), dy = DY(c), dz = DZ(c);
    if (!mu) return nu * (2.0 / (dx * dx) + 2.0 / (dy * dy) + 2.0 / (dz * dz));
    double mc = at3(c, mu, i, j, k, B3_EVEN);
    double fx = 0.5 * (mc + at3(c, mu, i + 1, j, k, B3_EVEN)) + 0.5 * (mc + at3(c, mu, i - 1, j, k, B3_EVEN));
    double fy = 0.5 * (mc + at3(c, mu, i, j + 1, k, B3_EVEN)) + 0.5 * (mc + at3(c, mu, i, j - 1, k, B3_EVEN));
    double fz = 0.5 * (mc + at3(c, mu, i, j, k + 1, B3_EVEN)) + 0.5 * (mc + at3(c, mu, i, j, k - 1, B3_EVEN));
    return nu * (fx / (dx * dx) + fy / (dy * dy) + fz / (dz * dz));
}

/* (1/V) sum_j phi_j, outward positive. */
double o3_divergence_cell(const o3_cfg *c, const double *phix, const double *phiy, const double *phiz,
                          int i, int j, int k)
{
    double V = DX(c) * DY(c) * DZ(c);
    return (phix[fxid(c, i + 1, j, k)] - phix[fxid(c, i, j, k)] + phiy[fyid(c, i, j + 1, k)] -
            phiy[fyid(c, i, j, k)] + phiz[fzid(c, i, j, k + 1)] - phiz[fzid(c, i, j, k)]) / V;
}

/* Face forces G_f = (p'_b - p'_a)/Delta - g z_f (rho_b - rho_a)/Delta on
 * interior faces, zero on walls; x- and y-faces sit at their cell's height. */
static void face_forces3(const o3_cfg *c, const double *pp, const double *rho, double *Gx, double *Gy,
                         double *Gz)
{
    int nx = c->nx, ny = c->ny, nz = c->nz;
    double dx = DX(c), dy = DY(c), dz = DZ(c), g = c->g;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int f = 0; f <= nx; ++f) {
                double G = 0.0, zf = (k + 0.5) * dz;
                if (f > 0 && f < nx) {
                    size_t a = cid(c, f - 1, j, k), b = cid(c, f, j, k);
                    G = (pp[b] - pp[a]) / dx - g * zf * (rho[b] - rho[a]) / dx;
                }
                Gx[fxid(c, f, j, k)] = G;
            }
    for (int k = 0; k < nz; ++k)
        for (int f = 0; f <= ny; ++f)
            for (int i = 0; i < nx; ++i) {
                double G = 0.0, zf = (k + 0.5) * dz;
                if (f > 0 && f < ny) {
                    size_t a = cid(c, i, f - 1, k), b = cid(c, i, f, k);
                    G = (pp[b] - pp[a]) / dy - g * zf * (rho[b] - rho[a]) / dy;
                }
                Gy[fyid(c, i, f, k)] = G;
            }
    for (int f = 0; f <= nz; ++f)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double G = 0.0, zf = f * dz;
                if (f > 0 && f < nz) {
                    size_t a = cid(c, i, j, f - 1), b = cid(c, i, j, f);
                    G = (pp[b] - pp[a]) / dz - g * zf * (rho[b] - rho[a]) / dz;
                }
                Gz[fzid(c, i, j, f)] = G;
            }
}

static double norm2(const double *x, size_t n)
{
    double s = 0.0;
    for (size_t q = 0; q < n; ++q) s += x[q] * x[q];
    return sqrt(s);
}

/* ------------------------------------------------------------------ */
/* implicit transport solves (Step 1 momentum, Step 2 enthalpy)          */
/* ------------------------------------------------------------------ */

/* r = b - [(rho1/dt) X + C(X) - nu L(X)] at every cell. */
static void transport_residual3(const o3_cfg *c, const double *rho1, const double *phix, const double *phiy,
                                const double *phiz, const double *mu, double nu, const double *X, int bc,
                                const double *b, double *r)
{
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                size_t q = cid(c, i, j, k);
                double lhs = rho1[q] / c->dt * X[q] + o3_convection_cell(c, phix, phiy, phiz, X, bc, i, j, k)
                           - diffusion3(c, mu, nu, X, bc, i, j, k);
                r[q] = b[q] - lhs;
            }
}

/* Jacobi for (rho1/dt) X + C(X) - D(X) = b from the initial X, D the
 * diffusion term (nu L(X), or nu times the variable-coefficient sum when mu
 * is given); divisor rho1/dt + (7/12) sum_j phi_j/V + the diagonal of -D;
 * stops after the sweep whose residual met ||r|| <= jac_rtol ||b||. Returns
 * sweeps or -1. */
int o3_transport_solve(const o3_cfg *c, const double *rho1, const double *phix, const double *phiy,
                       const double *phiz, const double *mu, double nu, int bc, const double *b, double *X)
{
    size_t n = ncell(c);
    double *r = malloc(n * sizeof(double));
    double bn = norm2(b, n);
    int sweeps = 0, ok = 0;
    while (sweeps < c->jac_maxit) {
        transport_residual3(c, rho1, phix, phiy, phiz, mu, nu, X, bc, b, r);
        double rn = norm2(r, n);
        for (int k = 0; k < c->nz; ++k)
            for (int j = 0; j < c->ny; ++j)
                for (int i = 0; i < c->nx; ++i) {
                    size_t q = cid(c, i, j, k);
                    double d = rho1[q] / c->dt + 7.0 / 12.0 * o3_divergence_cell(c, phix, phiy, phiz, i, j, k)
                             + diffusion_diag3(c, mu, nu, i, j, k);
                    X[q] += r[q] / d;
                }
        ++sweeps;
        if (rn <= c->jac_rtol * bn) { ok = 1; break; }
    }
    free(r);
    return ok ? sweeps : -1;
}

/* ------------------------------------------------------------------ */
/* pressure (Helmholtz) problem of Step 3                              */
/* ------------------------------------------------------------------ */

/* (A x)_i = (psi_i/dt) x_i + (1/V) sum_f D_f |A_f| (x_i - x_N)/Delta_f over
 * interior faces (Dx, Dy, Dz on the face arrays, zero on walls). */
void o3_helmholtz_apply(const o3_cfg *c, const double *psi, const double *Dx, const double *Dy,
                        const double *Dz, const double *x, double *y)
{
    double dx = DX(c), dy = DY(c), dz = DZ(c);
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                size_t q = cid(c, i, j, k);
                double s = 0.0;
                if (i + 1 < c->nx) s += Dx[fxid(c, i + 1, j, k)] * (x[q] - x[cid(c, i + 1, j, k)]) / (dx * dx);
                if (i > 0) s += Dx[fxid(c, i, j, k)] * (x[q] - x[cid(c, i - 1, j, k)]) / (dx * dx);
                if (j + 1 < c->ny) s += Dy[fyid(c, i, j + 1, k)] * (x[q] - x[cid(c, i, j + 1, k)]) / (dy * dy);
                if (j > 0) s += Dy[fyid(c, i, j, k)] * (x[q] - x[cid(c, i, j - 1, k)]) / (dy * dy);
                if (k + 1 < c->nz) s += Dz[fzid(c, i, j, k + 1)] * (x[q] - x[cid(c, i, j, k + 1)]) / (dz * dz);
                if (k > 0) s += Dz[fzid(c, i, j, k)] * (x[q] - x[cid(c, i, j, k - 1)]) / (dz * dz);
                y[q] = psi[q] / c->dt * x[q] + s;
            }
}

/* Diagonally preconditioned CG from the initial x to ||r|| <= cg_rtol ||b||.
 * Returns iterations or -1. */
int o3_pcg(const o3_cfg *c, const double *psi, const double *Dx, const double *Dy, const double *Dz,
           const double *b, double *x, double *relres)
{
    size_t n = ncell(c);
    double dx = DX(c), dy = DY(c), dz = DZ(c);
    double *r = malloc(n * sizeof(double)), *z = malloc(n * sizeof(double));
    double *p = malloc(n * sizeof(double)), *q = malloc(n * sizeof(double));
    double *d = malloc(n * sizeof(double));
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                size_t qi = cid(c, i, j, k);
                double s = psi[qi] / c->dt;
                if (i + 1 < c->nx) s += Dx[fxid(c, i + 1, j, k)] / (dx * dx);
                if (i > 0) s += Dx[fxid(c, i, j, k)] / (dx * dx);
                if (j + 1 < c->ny) s += Dy[fyid(c, i, j + 1, k)] / (dy * dy);
                if (j > 0) s += Dy[fyid(c, i, j, k)] / (dy * dy);
                if (k + 1 < c->nz) s += Dz[fzid(c, i, j, k + 1)] / (dz * dz);
                if (k > 0) s += Dz[fzid(c, i, j, k)] / (dz * dz);
                d[qi] = s;
            }
    o3_helmholtz_apply(c, psi, Dx, Dy, Dz, x, q);
    for (size_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    double bn = norm2(b, n), rn = norm2(r, n), rz = 0.0;
    int it = 0, ok = 0;
    for (size_t i = 0; i < n; ++i) { z[i] = r[i] / d[i]; p[i] = z[i]; rz += r[i] * z[i]; }
    for (;;) {
        if (rn <= c->cg_rtol * bn || rn == 0.0) { ok = 1; break; }
        if (it >= c->cg_maxit) break;
        o3_helmholtz_apply(c, psi, Dx, Dy, Dz, p, q);
        double pq = 0.0;
        for (size_t i = 0; i < n; ++i) pq += p[i] * q[i];
        double alpha = rz / pq;
        for (size_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        double rz_new = 0.0;
        for (size_t i = 0; i < n; ++i) { z[i] = r[i] / d[i]; rz_new += r[i] * z[i]; }
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
/* set-up from conservative variables and diagnostics                  */
/* ------------------------------------------------------------------ */

/* From (rho, rho u, rho v, rho w, rho e), e = cv T + |u|^2/2 + g z: u, T,
 * p = rho R T, h = cp T, p' = p + rho g z, p^{n-1} = p, and phi on interior
 * faces the average of the two cells' normal momentum times the face area.
 * Returns 1 if some cell has rho <= 0 or T <= 0. */
int o3_derive(const o3_cfg *c, const double *rho, const double *rhou, const double *rhov, const double *rhow,
              const double *rhoe, o3_state *s)
{
    int nx = c->nx, ny = c->ny, nz = c->nz;
    double dx = DX(c), dy = DY(c), dz = DZ(c), cv = c->cp - c->R;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t q = cid(c, i, j, k);
                double z = (k + 0.5) * dz;
                if (!(rho[q] > 0.0)) return 1;
                double u = rhou[q] / rho[q], v = rhov[q] / rho[q], w = rhow[q] / rho[q];
                double T = (rhoe[q] / rho[q] - 0.5 * (u * u + v * v + w * w) - c->g * z) / cv;
                if (!(T > 0.0)) return 1;
                s->rho[q] = rho[q];
                s->u[q] = u; s->v[q] = v; s->w[q] = w;
                s->T[q] = T;
                s->h[q] = c->cp * T;
                s->p[q] = rho[q] * c->R * T;
                s->pp[q] = s->p[q] + rho[q] * c->g * z;
                s->pold[q] = s->p[q];
            }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int f = 0; f <= nx; ++f)
                s->phix[fxid(c, f, j, k)] = (f > 0 && f < nx)
                    ? 0.5 * (rhou[cid(c, f - 1, j, k)] + rhou[cid(c, f, j, k)]) * dy * dz : 0.0;
    for (int k = 0; k < nz; ++k)
        for (int f = 0; f <= ny; ++f)
            for (int i = 0; i < nx; ++i)
                s->phiy[fyid(c, i, f, k)] = (f > 0 && f < ny)
                    ? 0.5 * (rhov[cid(c, i, f - 1, k)] + rhov[cid(c, i, f, k)]) * dx * dz : 0.0;
    for (int f = 0; f <= nz; ++f)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                s->phiz[fzid(c, i, j, f)] = (f > 0 && f < nz)
                    ? 0.5 * (rhow[cid(c, i, j, f - 1)] + rhow[cid(c, i, j, f)]) * dx * dy : 0.0;
    return 0;
}

/* Totals of mass sum rho V and energy sum rho (cv T + K + g z) V. */
void o3_totals(const o3_cfg *c, const o3_state *s, double *mass, double *energy)
{
    double V = DX(c) * DY(c) * DZ(c), cv = c->cp - c->R, m = 0.0, e = 0.0;
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                size_t q = cid(c, i, j, k);
                double K = 0.5 * (s->u[q] * s->u[q] + s->v[q] * s->v[q] + s->w[q] * s->w[q]);
                m += s->rho[q] * V;
                e += s->rho[q] * (cv * s->T[q] + K + c->g * (k + 0.5) * DZ(c)) * V;
            }
    if (mass) *mass = m;
    if (energy) *energy = e;
}

/* ------------------------------------------------------------------ */
/* the time step (Section 3: Steps 1-3, n_corr PISO correctors)        */
/* ------------------------------------------------------------------ */

static double *zal(size_t n) { return calloc(n, sizeof(double)); }

/* Face value D_f = dt rho2_f / rho1_f with linear face averages. */
static double dface(double dt, const double *rho1, const double *rho2, size_t a, size_t b)
{
    return dt * (0.5 * (rho2[a] + rho2[b])) / (0.5 * (rho1[a] + rho1[b]));
}

int o3_step(const o3_cfg *c, o3_state *s, int32_t nsteps, o3_stats *st)
{
    int nx = c->nx, ny = c->ny, nz = c->nz;
    size_t n = ncell(c);
    size_t nfx = (size_t)nz * ny * (nx + 1), nfy = (size_t)nz * (ny + 1) * nx, nfz = (size_t)(nz + 1) * ny * nx;
    double dt = c->dt, g = c->g, dx = DX(c), dy = DY(c), dz = DZ(c);
    int status = 0;
    double *rho1 = zal(n), *u1 = zal(n), *v1 = zal(n), *w1 = zal(n), *K1 = zal(n);
    double *bu = zal(n), *bv = zal(n), *bw = zal(n), *bh = zal(n), *h1 = zal(n);
    double *T1 = zal(n), *rho2 = zal(n), *psi = zal(n), *Hx = zal(n), *Hy = zal(n), *Hz = zal(n), *b = zal(n);
    double *U = zal(n), *Vv = zal(n), *W = zal(n), *pnew = zal(n), *rhonew = zal(n), *pnext = zal(n);
    double *Gx = zal(nfx), *Gy = zal(nfy), *Gz = zal(nfz), *Dx = zal(nfx), *Dy = zal(nfy), *Dz = zal(nfz);
    double *Fx = zal(nfx), *Fy = zal(nfy), *Fz = zal(nfz);
    int su = 0, sv = 0, sw = 0, sh = 0;
    /* LES: mu_eff from rho^n, u^n once per step; the diffusion of momentum and
     * enthalpy then takes its face means (Pr = 1: one field for both) */
    double *mu_eff = c->cs > 0.0 ? zal(n) : NULL;
    double nu_u = mu_eff ? 1.0 : c->mu, nu_h = mu_eff ? 1.0 / c->Pr : c->mu / c->Pr;

    for (int step = 0; step < nsteps; ++step) {
        if (mu_eff) o3_smagorinsky(c, s->rho, s->u, s->v, s->w, mu_eff);
        /* Step 1, eq. (e1_d): rho^{n+1/3} = rho^n - dt sum_j phi^n_j / V */
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t q = cid(c, i, j, k);
                    rho1[q] = s->rho[q] - dt * o3_divergence_cell(c, s->phix, s->phiy, s->phiz, i, j, k);
                }
        /* Step 1, eq. (step2_sd): implicit momentum predictor with the balanced
         * force of eq. (mom_split) explicit, b_u = rho^n u^n / dt - G_cell */
        face_forces3(c, s->pp, s->rho, Gx, Gy, Gz);
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t q = cid(c, i, j, k);
                    double gcx = 0.5 * (Gx[fxid(c, i, j, k)] + Gx[fxid(c, i + 1, j, k)]);
                    double gcy = 0.5 * (Gy[fyid(c, i, j, k)] + Gy[fyid(c, i, j + 1, k)]);
                    double gcz = 0.5 * (Gz[fzid(c, i, j, k)] + Gz[fzid(c, i, j, k + 1)]);
                    bu[q] = s->rho[q] * s->u[q] / dt - gcx;
                    bv[q] = s->rho[q] * s->v[q] / dt - gcy;
                    bw[q] = s->rho[q] * s->w[q] / dt - gcz;
                    u1[q] = s->u[q]; v1[q] = s->v[q]; w1[q] = s->w[q];
                }
        su = o3_transport_solve(c, rho1, s->phix, s->phiy, s->phiz, mu_eff, nu_u, B3_U, bu, u1);
        sv = o3_transport_solve(c, rho1, s->phix, s->phiy, s->phiz, mu_eff, nu_u, B3_V, bv, v1);
        sw = o3_transport_solve(c, rho1, s->phix, s->phiy, s->phiz, mu_eff, nu_u, B3_W, bw, w1);
        if (su < 0 || sv < 0 || sw < 0) status = 1;
        /* eq. (step1_3sd) */
        for (size_t q = 0; q < n; ++q) K1[q] = 0.5 * (u1[q] * u1[q] + v1[q] * v1[q] + w1[q] * w1[q]);

        /* Step 2, eq. (step3_sd): enthalpy, implicit in h^{n+1} */
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t q = cid(c, i, j, k);
                    double Kn = 0.5 * (s->u[q] * s->u[q] + s->v[q] * s->v[q] + s->w[q] * s->w[q]);
                    double be = (s->rho[q] * s->h[q] + s->rho[q] * Kn - s->pold[q]) / dt;
                    bh[q] = be - rho1[q] * K1[q] / dt
                          - o3_convection_cell(c, s->phix, s->phiy, s->phiz, K1, B3_EVEN, i, j, k)
                          + s->p[q] / dt - rho1[q] * g * w1[q];
                    h1[q] = s->h[q];
                }
        sh = o3_transport_solve(c, rho1, s->phix, s->phiy, s->phiz, mu_eff, nu_h, B3_H, bh, h1);
        if (sh < 0) status = 1;
        /* eqs. (step3_2sd), (step3_3sd) */
        for (size_t q = 0; q < n; ++q) {
            T1[q] = s->T[q] + (h1[q] - s->h[q]) / c->cp;
            rho2[q] = s->p[q] / (c->R * T1[q]);
            psi[q] = 1.0 / (c->R * T1[q]);
        }
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int f = 0; f <= nx; ++f)
                    Dx[fxid(c, f, j, k)] = (f > 0 && f < nx) ? dface(dt, rho1, rho2, cid(c, f - 1, j, k), cid(c, f, j, k)) : 0.0;
        for (int k = 0; k < nz; ++k)
            for (int f = 0; f <= ny; ++f)
                for (int i = 0; i < nx; ++i)
                    Dy[fyid(c, i, f, k)] = (f > 0 && f < ny) ? dface(dt, rho1, rho2, cid(c, i, f - 1, k), cid(c, i, f, k)) : 0.0;
        for (int f = 0; f <= nz; ++f)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i)
                    Dz[fzid(c, i, j, f)] = (f > 0 && f < nz) ? dface(dt, rho1, rho2, cid(c, i, j, f - 1), cid(c, i, j, f)) : 0.0;

        memcpy(U, u1, n * sizeof(double));
        memcpy(Vv, v1, n * sizeof(double));
        memcpy(W, w1, n * sizeof(double));
        memcpy(pnew, s->pp, n * sizeof(double));

        /* Step 3: PISO correctors */
        for (int corr = 0; corr < c->n_corr; ++corr) {
            /* H(u) = b_u - C(u) + mu L(u) at the newest velocity */
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        size_t q = cid(c, i, j, k);
                        Hx[q] = s->rho[q] * s->u[q] / dt - o3_convection_cell(c, s->phix, s->phiy, s->phiz, U, B3_U, i, j, k)
                              + diffusion3(c, mu_eff, nu_u, U, B3_U, i, j, k);
                        Hy[q] = s->rho[q] * s->v[q] / dt - o3_convection_cell(c, s->phix, s->phiy, s->phiz, Vv, B3_V, i, j, k)
                              + diffusion3(c, mu_eff, nu_u, Vv, B3_V, i, j, k);
                        Hz[q] = s->rho[q] * s->w[q] / dt - o3_convection_cell(c, s->phix, s->phiy, s->phiz, W, B3_W, i, j, k)
                              + diffusion3(c, mu_eff, nu_u, W, B3_W, i, j, k);
                    }
            /* right-hand side of the Helmholtz pressure equation */
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        size_t q = cid(c, i, j, k);
                        double zc = (k + 0.5) * dz, fl = 0.0;
                        if (i + 1 < nx) {
                            size_t N = cid(c, i + 1, j, k);
                            fl += Dx[fxid(c, i + 1, j, k)] / dx * (0.5 * (Hx[q] + Hx[N]) + g * zc * (rho2[N] - rho2[q]) / dx);
                        }
                        if (i > 0) {
                            size_t N = cid(c, i - 1, j, k);
                            fl += Dx[fxid(c, i, j, k)] / dx * (-0.5 * (Hx[q] + Hx[N]) + g * zc * (rho2[N] - rho2[q]) / dx);
                        }
                        if (j + 1 < ny) {
                            size_t N = cid(c, i, j + 1, k);
                            fl += Dy[fyid(c, i, j + 1, k)] / dy * (0.5 * (Hy[q] + Hy[N]) + g * zc * (rho2[N] - rho2[q]) / dy);
                        }
                        if (j > 0) {
                            size_t N = cid(c, i, j - 1, k);
                            fl += Dy[fyid(c, i, j, k)] / dy * (-0.5 * (Hy[q] + Hy[N]) + g * zc * (rho2[N] - rho2[q]) / dy);
                        }
                        if (k + 1 < nz) {
                            size_t N = cid(c, i, j, k + 1);
                            double zf = (k + 1) * dz;
                            fl += Dz[fzid(c, i, j, k + 1)] / dz * (0.5 * (Hz[q] + Hz[N]) + g * zf * (rho2[N] - rho2[q]) / dz);
                        }
                        if (k > 0) {
                            size_t N = cid(c, i, j, k - 1);
                            double zf = k * dz;
                            fl += Dz[fzid(c, i, j, k)] / dz * (-0.5 * (Hz[q] + Hz[N]) + g * zf * (rho2[N] - rho2[q]) / dz);
                        }
                        b[q] = (s->rho[q] + psi[q] * rho2[q] * g * zc) / dt - fl;
                    }
            double relres = 0.0;
            int it = o3_pcg(c, psi, Dx, Dy, Dz, b, pnew, &relres);
            if (corr < 4 && st) { st->cg_iters[corr] = it; st->cg_relres[corr] = relres; }
            if (it < 0) status = 1;
            /* correction: F_f = D_f (H_f - G_f); u = (dt/rho1)(H - G_cell);
             * p = p' - rho2 g z; rho = p / (R T^{n+1}) */
            face_forces3(c, pnew, rho2, Gx, Gy, Gz);
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int f = 0; f <= nx; ++f) {
                        size_t e = fxid(c, f, j, k);
                        Fx[e] = (f > 0 && f < nx)
                            ? Dx[e] * (0.5 * (Hx[cid(c, f - 1, j, k)] + Hx[cid(c, f, j, k)]) - Gx[e]) : 0.0;
                    }
            for (int k = 0; k < nz; ++k)
                for (int f = 0; f <= ny; ++f)
                    for (int i = 0; i < nx; ++i) {
                        size_t e = fyid(c, i, f, k);
                        Fy[e] = (f > 0 && f < ny)
                            ? Dy[e] * (0.5 * (Hy[cid(c, i, f - 1, k)] + Hy[cid(c, i, f, k)]) - Gy[e]) : 0.0;
                    }
            for (int f = 0; f <= nz; ++f)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        size_t e = fzid(c, i, j, f);
                        Fz[e] = (f > 0 && f < nz)
                            ? Dz[e] * (0.5 * (Hz[cid(c, i, j, f - 1)] + Hz[cid(c, i, j, f)]) - Gz[e]) : 0.0;
                    }
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        size_t q = cid(c, i, j, k);
                        double gcx = 0.5 * (Gx[fxid(c, i, j, k)] + Gx[fxid(c, i + 1, j, k)]);
                        double gcy = 0.5 * (Gy[fyid(c, i, j, k)] + Gy[fyid(c, i, j + 1, k)]);
                        double gcz = 0.5 * (Gz[fzid(c, i, j, k)] + Gz[fzid(c, i, j, k + 1)]);
                        U[q] = dt / rho1[q] * (Hx[q] - gcx);
                        Vv[q] = dt / rho1[q] * (Hy[q] - gcy);
                        W[q] = dt / rho1[q] * (Hz[q] - gcz);
                        double pn = pnew[q] - rho2[q] * g * (k + 0.5) * dz;
                        rhonew[q] = pn / (c->R * T1[q]);
                        pnext[q] = pn;
                    }
        }
        /* end of step; p^{n-1} <- p^n; phi = F |A| */
        memcpy(s->pold, s->p, n * sizeof(double));
        memcpy(s->p, pnext, n * sizeof(double));
        memcpy(s->pp, pnew, n * sizeof(double));
        memcpy(s->rho, rhonew, n * sizeof(double));
        memcpy(s->u, U, n * sizeof(double));
        memcpy(s->v, Vv, n * sizeof(double));
        memcpy(s->w, W, n * sizeof(double));
        memcpy(s->T, T1, n * sizeof(double));
        memcpy(s->h, h1, n * sizeof(double));
        for (size_t q = 0; q < nfx; ++q) s->phix[q] = Fx[q] * dy * dz;
        for (size_t q = 0; q < nfy; ++q) s->phiy[q] = Fy[q] * dx * dz;
        for (size_t q = 0; q < nfz; ++q) s->phiz[q] = Fz[q] * dx * dy;
    }
    if (st) {
        st->jac_u = su > sv ? (su > sw ? su : sw) : (sv > sw ? sv : sw);
        st->jac_h = sh;
        st->status = status;
    }
    free(rho1); free(u1); free(v1); free(w1); free(K1); free(bu); free(bv); free(bw); free(bh); free(h1);
    free(T1); free(rho2); free(psi); free(Hx); free(Hy); free(Hz); free(b); free(U); free(Vv); free(W);
    free(pnew); free(rhonew); free(pnext); free(Gx); free(Gy); free(Gz); free(Dx); free(Dy); free(Dz);
    free(Fx); free(Fy); free(Fz);
    free(mu_eff);
    return status;
}
