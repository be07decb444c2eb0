/*
 * gea3d.h -- C ABI of the three-dimensional time step (GB300, sm_103a).
 *
 * The scheme of gea.h (Section 3 of Girfoglio, Quaini & Rozza, arXiv
 * 2303.10499: continuity and implicit momentum predictor, implicit enthalpy
 * equation, EOS update, PISO correctors with the Helmholtz pressure
 * equation) on a uniform Cartesian x-y-z grid: x and y horizontal, z up,
 * free-slip walls on all six sides, constant viscosity mu (Remark 1) or a
 * Smagorinsky eddy viscosity, FP64.
 * The pressure equation is solved by conjugate gradients preconditioned by a
 * Galerkin geometric multigrid V(1,1) cycle (coarsening 2 x 2 x 2); the
 * solver loops run on the device inside a CUDA graph.
 *
 * Conventions
 *  - Cell fields are dense nz x ny x nx arrays, x fastest: cell (i,j,k)
 *    centred at ((i+1/2) dx, (j+1/2) dy, (k+1/2) dz) at index
 *    (k ny + j) nx + i.
 *  - Pressure split p = p' - rho g z (g > 0, z up), as in gea.h.
 *  - The constants are gea_constants of gea.h (reading_flags must be 0: the
 *    three-dimensional step has the default readings only). flags: 0 or GEA_FLAG_MIXED,
 *    the mixed-precision step as in gea.h (FP64 state, residuals and
 *    updates; FP32 Jacobi on the momentum and enthalpy increments and FP32
 *    multigrid CG on the pressure increment, each to mp_rtol times its
 *    initial residual; mp_rtol 0 selects 1e-5, else 1e-7 <= mp_rtol < 1;
 *    gea_stats.driver is then 2). cs > 0 turns on Smagorinsky
 *    LES: mu_eff = mu + rho^n (cs Delta)^2 |S| per cell, Delta =
 *    (dx dy dz)^(1/3), |S| = sqrt(2 S_ij S_ij) from central differences of
 *    u^n, and the diffusion of momentum and enthalpy takes the face means
 *    of mu_eff; it requires Pr = 1.
 *  - All calls are ordered on the context's stream; calls with host
 *    buffers return after the copies.
 *  - Functions return GEA_OK or a GEA_ERR_* code of gea.h.
 */
#ifndef GEA3D_H
#define GEA3D_H

#include <stdint.h>

#include "gea.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gea3d_grid {
    int32_t nx, ny, nz;     /* >= 4 each */
    double lx, ly, lz;
} gea3d_grid;

typedef struct gea3d_ctx gea3d_ctx;

/* Validate and allocate every device buffer (two state slots, scratch, the
 * multigrid hierarchy). Errors: GEA_ERR_INVAL, GEA_ERR_NOMEM, GEA_ERR_CUDA. */
int gea3d_create(const gea3d_grid *grid, const gea_constants *c, gea3d_ctx **out);
int gea3d_set_stream(gea3d_ctx *ctx, void *stream);

/* Set the state from conservative fields (rho, rho u, rho v, rho w,
 * rho e with e = cv T + |u|^2/2 + g z; host or device per mem): u, T,
 * p = rho R T, h = cp T, p' = p + rho g z, p^{n-1} = p, and the face mass
 * fluxes from the mean of the two cells' momenta. GEA_ERR_INVAL if some
 * cell has rho <= 0 or T <= 0. After an error other than a rejected argument
 * the context holds no state (gea3d_step: GEA_ERR_STATE) until a later call
 * succeeds. */
int gea3d_set_conservative(gea3d_ctx *ctx, const double *rho, const double *rhou, const double *rhov,
                           const double *rhow, const double *rhoe, int32_t mem);

int gea3d_step_async(gea3d_ctx *ctx, int32_t n);
int gea3d_sync(gea3d_ctx *ctx);
int gea3d_step(gea3d_ctx *ctx, int32_t n);

/* Copy cell fields of the current state out (any pointer may be NULL). */
int gea3d_get_state(gea3d_ctx *ctx, double *rho, double *u, double *v, double *w, double *T, double *p,
                    double *pp, int32_t mem);

/* Diagnostics of the current state (Remark 2), computed on the device:
 * theta' = T (p0/p)^(R/cp) - theta_bar(z) per cell into theta_prime (host or
 * device, nz*ny*nx, x fastest; may be NULL) given the background theta_bar
 * (host or device, nz values); mass = sum rho V and energy = sum rho e V with
 * e = cv T + |u|^2/2 + g z (Section 2.1) (each may be NULL). Synchronises.
 * Errors: GEA_ERR_INVAL (null ctx, theta_prime without theta_bar),
 * GEA_ERR_STATE (no state), GEA_ERR_CUDA. */
int gea3d_get_diag(gea3d_ctx *ctx, const double *theta_bar, double *theta_prime, double *mass, double *energy);

/* Counters of the last completed step (driver 0: CUDA graph). */
int gea3d_get_stats(gea3d_ctx *ctx, gea_stats *s);

/* Advance one step with the kernels of gea3d_step launched one by one (no
 * graph), a CUDA event pair around each launch on the context's stream and
 * the solver loops checked from the host; up to max_entries per-kernel
 * totals (gea_kernel_time of gea.h, cells = the cells of the level each
 * launch covers) go to out and their number to *n_entries. Synchronises. */
int gea3d_profile_step(gea3d_ctx *ctx, gea_kernel_time *out, int32_t max_entries, int32_t *n_entries);

const char *gea3d_last_error(const gea3d_ctx *ctx);
void gea3d_destroy(gea3d_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* GEA3D_H */
