// gea_kernels.cu -- per-phase CUDA kernels (sm_103a, FP64) of one time step
// of the GEA pressure-based Euler solver (Girfoglio, Quaini & Rozza, arXiv
// 2303.10499, Section 3) and their host-side launchers: the graph path, one
// kernel per phase (the phase bodies are the tile functions of
// gea_tiles.cuh, one tile per block), with the solver loops as conditional
// WHILE nodes of a CUDA graph. The same kernels also serve the per-kernel
// profiled step. Reductions are deterministic: block partials, added in a
// fixed order by the last block to arrive. Kernels inside a device-side
// loop return early (uniformly across the grid) once the loop has converged
// or failed.
#include "gea_internal.cuh"
#include "gea_tiles.cuh"

#include <math.h>

namespace gea {

namespace {

using namespace tiles;

__device__ __forceinline__ bool loop_over(const Scal *sc, int which)
{
    return sc->status || sc->done[which];
}

__global__ void k_derive(Geom G, Phys F, const double *__restrict__ rho,
                         const double *__restrict__ rhou, const double *__restrict__ rhow,
                         const double *__restrict__ rhoe, State S, Scal *sc)
{
    int i, k;
    if (!cell_of(G, blockIdx.x, blockIdx.y, i, k)) return;
    const int q = cidx(G, i, k);
    const double cv = F.cp - F.R;
    const double z = (k + 0.5) * G.dz;
    const double r = rho[q];
    const double u = rhou[q] / r, w = rhow[q] / r;
    const double K = 0.5 * (u * u + w * w);
    const double T = (rhoe[q] / r - K - F.g * z) / cv;
    if (!(r > 0.0) || !(T > 0.0)) atomicAdd(&sc->bad_cells, 1);
    S.rho[q] = r;
    S.u[q] = u;
    S.w[q] = w;
    S.T[q] = T;
    S.h[q] = F.cp * T;
    const double p = r * F.R * T;
    S.p[q] = p;
    S.pp[q] = p + r * F.g * z;
    S.pold[q] = p;
    S.Kold[q] = K;   // K^{-1} := K^0
    S.phix[k * G.P + i] = i > 0 ? 0.5 * (rhou[q - 1] + rhou[q]) * G.dz : 0.0;
    if (i == G.nx - 1) S.phix[k * G.P + G.nx] = 0.0;
    S.phiz[k * G.P + i] = k > 0 ? 0.5 * (rhow[q - G.P] + rhow[q]) * G.dx : 0.0;
    if (k == G.nz - 1) S.phiz[G.nz * G.P + i] = 0.0;
}

// Conservative variables of a state (Section 2.1), the inverse of k_derive:
// rho, rho u, rho w and rho e with the total energy e = cv T + |u|^2/2 + g z.
__global__ void k_conserve(Geom G, Phys F, State S, double *__restrict__ rho, double *__restrict__ rhou,
                           double *__restrict__ rhow, double *__restrict__ rhoe)
{
    int i, k;
    if (!cell_of(G, blockIdx.x, blockIdx.y, i, k)) return;
    const int q = cidx(G, i, k);
    const double z = (k + 0.5) * G.dz;
    const double r = S.rho[q], u = S.u[q], w = S.w[q];
    const double K = 0.5 * (u * u + w * w);
    rho[q] = r;
    rhou[q] = r * u;
    rhow[q] = r * w;
    rhoe[q] = r * ((F.cp - F.R) * S.T[q] + K + F.g * z);
}

// ---- Step 1 ----

__global__ void k_les(StepArgs a)
{
    if (a.sc->status) return;
    __shared__ double sm[2 * kT1];
    ph_les(a, sm, blockIdx.x, blockIdx.y);
}

__global__ void k_pred_setup(StepArgs a)
{
    if (a.sc->status) return;
    __shared__ double red[2 * NTHREADS];
    double acc[2] = {0.0, 0.0}, tot[2];
    ph_pred(a, blockIdx.x, blockIdx.y, acc);
    if (grid_sum<2>(acc, red, a.partials, &a.sc->counters[CNT_PRED], tot)) fin_pred(a.sc, tot);
}

// Sweeps run in pairs (X_a -> X_b -> X_a) so that the loop ends in X_a. The
// second sweep of a pair whose first sweep met the tolerance copies X_b back
// instead: the iteration stops after that sweep.
__global__ void k_mom_jacobi(StepArgs a, const double *uin, const double *win, double *uout,
                             double *wout, int second)
{
    if (a.sc->status) return;
    if (second && a.sc->done[LOOP_MOM]) {
        block_tiles(a.G, [&](int bx, int bz) {
            ph_copy(a.G, uin, uout, bx, bz);
            ph_copy(a.G, win, wout, bx, bz);
        });
        return;
    }
    __shared__ double sm[2 * kT2];
    __shared__ double red[2 * NTHREADS];
    double acc[2] = {0.0, 0.0}, tot[2];
    block_tiles(a.G, [&](int bx, int bz) { ph_mom(a, uin, win, uout, wout, sm, bx, bz, acc); });
    if (grid_sum<2>(acc, red, a.partials, &a.sc->counters[CNT_MOM], tot)) fin_mom(a.sc, tot, a.jac_rtol2);
}

// ---- Step 2 ----

__global__ void k_enth_rhs(StepArgs a)
{
    if (a.sc->status) return;
    __shared__ double sm[2 * kT2];
    __shared__ double red[NTHREADS];
    double acc[1] = {0.0}, tot[1];
    ph_enth_rhs(a, a.ua, a.wa, a.ha, sm, blockIdx.x, blockIdx.y, acc);
    if (grid_sum<1>(acc, red, a.partials, &a.sc->counters[CNT_ENTH_RHS], tot)) fin_enth_rhs(a.sc, tot);
}

__global__ void k_enth_jacobi(StepArgs a, const double *hin, double *hout, int second)
{
    if (a.sc->status) return;
    if (second && a.sc->done[LOOP_ENTH]) {
        block_tiles(a.G, [&](int bx, int bz) { ph_copy(a.G, hin, hout, bx, bz); });
        return;
    }
    __shared__ double sm[kT2];
    __shared__ double red[NTHREADS];
    double acc[1] = {0.0}, tot[1];
    block_tiles(a.G, [&](int bx, int bz) { ph_enth(a, hin, hout, sm, bx, bz, acc); });
    if (grid_sum<1>(acc, red, a.partials, &a.sc->counters[CNT_ENTH], tot)) fin_enth(a.sc, tot, a.jac_rtol2);
}

__global__ void k_eos_coef(StepArgs a, Level L)
{
    if (a.sc->status) return;
    __shared__ double sm[2 * kT1 + BZ * (BX + 1) + (BZ + 1) * BX];
    ph_eos(a, L, a.ha, sm, blockIdx.x, blockIdx.y);
}

__global__ void k_mg_coarsen(Level f, Level c, double omega)
{
    ph_coarsen(f, c, omega, blockIdx.x, blockIdx.y);
}

// ---- Step 3 ----

__global__ void k_H(StepArgs a, const double *U, const double *W)
{
    if (a.sc->status) return;
    __shared__ double sm[2 * kT2];
    ph_H(a, U, W, sm, blockIdx.x, blockIdx.y);
}

__global__ void k_helm_rhs(StepArgs a, Level L, const double *xin, double *xout, int corr)
{
    if (a.sc->status) return;
    __shared__ double sm[4 * kT1];
    __shared__ double red[2 * NTHREADS];
    double acc[2] = {0.0, 0.0}, tot[2];
    ph_helm_rhs(a, L, xin, xout, sm, blockIdx.x, blockIdx.y, acc);
    if (grid_sum<2>(acc, red, a.partials, &a.sc->counters[CNT_HELM], tot))
        fin_helm(a.sc, tot, a.cg_rtol2, corr);
}

__global__ void k_mg_down(Level f, Level c, double omega, Scal *sc)
{
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double sm[kT1 + BZ * BX];
    ph_mg_down(f, c, omega, sm, blockIdx.x, blockIdx.y);
}

__global__ void k_mg_coarse_sweep(Level L, const double *ein, double *eout, int first, Scal *sc)
{
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double sm[kT1];
    ph_mg_coarse(L, ein, eout, first, sm, blockIdx.x, blockIdx.y);
}

__global__ void k_mg_up(Level f, const double *ec, int Pc, double *out, int finest, StepArgs a)
{
    if (loop_over(a.sc, LOOP_CG)) return;
    __shared__ double sm[kT1];
    __shared__ double red[NTHREADS];
    double acc[1] = {0.0}, tot[1];
    // the finest level's residual alternates between two buffers
    const double *res = finest ? res_of(f, a.sc->cg_it) : f.r;
    block_tiles(f.G, [&](int bx, int bz) { ph_mg_up(f, res, ec, Pc, out, sm, bx, bz, acc); });
    if (!finest) return;
    if (grid_sum<1>(acc, red, a.partials, &a.sc->counters[CNT_RZ], tot)) fin_rz(a.sc, tot);
}

__global__ void k_mg_single(Level f, double *out, StepArgs a)
{
    if (loop_over(a.sc, LOOP_CG)) return;
    __shared__ double sm[kT1];
    __shared__ double red[NTHREADS];
    double acc[1] = {0.0}, tot[1];
    block_tiles(f.G, [&](int bx, int bz) { ph_mg_single(f, out, sm, bx, bz, acc); });
    if (grid_sum<1>(acc, red, a.partials, &a.sc->counters[CNT_RZ], tot)) fin_rz(a.sc, tot);
}

// The directions alternate between p0 and p1 by iteration parity: iteration
// it reads p[it & 1] and writes p[(it + 1) & 1].
__global__ void k_cg_pspmv(StepArgs a, Level L)
{
    Scal *sc = a.sc;
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double sm[kT1];
    __shared__ double red[NTHREADS];
    const int it = sc->cg_it;
    const double *pold = (it & 1) ? a.p1 : a.p0;
    double *pnew = (it & 1) ? a.p0 : a.p1;
    double acc[1] = {0.0}, tot[1];
    block_tiles(L.G, [&](int bx, int bz) { ph_pspmv<double>(L, pold, pnew, a.q, sc->beta, sm, bx, bz, acc); });
    if (grid_sum<1>(acc, red, a.partials, &sc->counters[CNT_PQ], tot)) fin_pq(sc, tot);
}

__global__ void k_cg_update_single(StepArgs a, Level L, double *x)
{
    Scal *sc = a.sc;
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double sm[2 * kT1];
    __shared__ double red[2 * NTHREADS];
    const int it = sc->cg_it;
    const double *p = (it & 1) ? a.p0 : a.p1;
    double acc[2] = {0.0, 0.0}, tot[2];
    block_tiles(L.G, [&](int bx, int bz) {
        ph_update_single<double>(L, a.q, res_of(L, it), res_of(L, it + 1), x, p, sc->alpha, sm, bx, bz, acc);
    });
    if (grid_sum<2>(acc, red, a.partials, &sc->counters[CNT_UPD], tot)) {
        const double t0[1] = {tot[0]}, t1[1] = {tot[1]};
        fin_update(sc, t0, a.cg_rtol2);
        fin_rz(sc, t1);
    }
}

__global__ void k_cg_update_down(StepArgs a, Level f, Level c, double *x)
{
    Scal *sc = a.sc;
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double sm[2 * kT1 + BZ * BX];
    __shared__ double red[NTHREADS];
    const int it = sc->cg_it;
    const double *p = (it & 1) ? a.p0 : a.p1;
    double acc[1] = {0.0}, tot[1];
    block_tiles(f.G, [&](int bx, int bz) {
        ph_update_down<double>(f, c, a.q, res_of(f, it), res_of(f, it + 1), x, p, sc->alpha, a.F.omega, sm,
                               bx, bz, acc);
    });
    if (grid_sum<1>(acc, red, a.partials, &sc->counters[CNT_UPD], tot)) fin_update(sc, tot, a.cg_rtol2);
}

__global__ void k_correct(StepArgs a)
{
    if (a.sc->status) return;
    __shared__ double sm[2 * kT1 + BZ * (BX + 1) + (BZ + 1) * BX];
    ph_correct(a, sm, blockIdx.x, blockIdx.y);
}

// ---- loop control and step bookkeeping (one thread) ----

__global__ void k_loop_ctl(Scal *sc, cudaGraphConditionalHandle h, int graph, int which,
                           int maxtrips, int body_launches)
{
    const int trips = ++sc->trips[which];
    const int done = sc->done[which];
    sc->launches += body_launches;
    if (!done && !sc->status && trips >= maxtrips) sc->status = GEA_ERR_NOCONV;
    if (graph) cudaGraphSetConditional(h, (done || sc->status || trips >= maxtrips) ? 0u : 1u);
}

// Before a gated loop: run it only while it is not finished.
__global__ void k_loop_gate(Scal *sc, cudaGraphConditionalHandle h, int which)
{
    cudaGraphSetConditional(h, (sc->done[which] || sc->status) ? 0u : 1u);
}

__global__ void k_step_begin(Scal *sc)
{
    sc->u1_slot = sc->h1_slot = 0;
    for (int c = 0; c < 4; ++c) { sc->cg_iters[c] = 0; sc->cg_relres[c] = 0.0; }
    sc->sweeps[0] = sc->sweeps[1] = 0;
}

__global__ void k_step_end(Scal *sc, int fixed_launches)
{
    sc->launches += fixed_launches;
    if (sc->status) {
        sc->last_status = sc->status;
        return;
    }
    sc->steps_done += 1;
    sc->last_sweeps[0] = sc->sweeps[0];
    sc->last_sweeps[1] = sc->sweeps[1];
    for (int c = 0; c < 4; ++c) {
        sc->last_cg_iters[c] = sc->cg_iters[c];
        sc->last_cg_relres[c] = sc->cg_relres[c];
    }
    sc->last_status = 0;
}

// ---- diagnostics (Remark 2) ----

__global__ void k_diag(Geom G, Phys F, State S, const double *__restrict__ thbar,
                       double *__restrict__ th, Scal *sc, double *partials)
{
    __shared__ double red[2 * NTHREADS];
    int i, k;
    const bool in = cell_of(G, blockIdx.x, blockIdx.y, i, k);
    double v[2] = {0.0, 0.0};
    if (in) {
        const int q = cidx(G, i, k);
        const double z = (k + 0.5) * G.dz;
        if (th) th[q] = S.T[q] / pow(S.p[q] / F.p0, F.R / F.cp) - thbar[k];
        const double V = G.dx * G.dz;
        const double K = 0.5 * (S.u[q] * S.u[q] + S.w[q] * S.w[q]);
        v[0] = S.rho[q] * V;
        v[1] = S.rho[q] * ((F.cp - F.R) * S.T[q] + K + F.g * z) * V;
    }
    double tot[2];
    if (grid_sum<2>(v, red, partials, &sc->counters[CNT_DIAG], tot)) {
        sc->mass = tot[0];
        sc->energy = tot[1];
    }
}

inline dim3 grid_of(const Geom &G) { return dim3((G.nx + BX - 1) / BX, (G.nz + BZ - 1) / BZ); }
const dim3 kBlock(BX, BZ);

}  // namespace

int max_blocks(const Geom &G)
{
    dim3 g = grid_of(G);
    return (int)(g.x * g.y);
}

void launch_derive(const Geom &G, const Phys &F, const double *rho, const double *rhou,
                   const double *rhow, const double *rhoe, const State &S, Scal *sc,
                   cudaStream_t st)
{
    k_derive<<<grid_of(G), kBlock, 0, st>>>(G, F, rho, rhou, rhow, rhoe, S, sc);
}

void launch_conserve(const Geom &G, const Phys &F, const State &S, double *rho, double *rhou, double *rhow,
                     double *rhoe, cudaStream_t st)
{
    k_conserve<<<grid_of(G), kBlock, 0, st>>>(G, F, S, rho, rhou, rhow, rhoe);
}

// Launch with an optional trace bracket.
#define TRACED(tr, name, cells, launch)                         \
    do {                                                        \
        if (tr) (tr)->begin(name, (long long)(cells), st);      \
        launch;                                                 \
        if (tr) (tr)->end(st);                                  \
    } while (0)

inline long long ncell(const Geom &G) { return (long long)G.nx * G.nz; }

void launch_les(const StepArgs &a, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "les", ncell(a.G), (k_les<<<grid_of(a.G), kBlock, 0, st>>>(a)));
}

void launch_pred_setup(const StepArgs &a, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "pred_setup", ncell(a.G), (k_pred_setup<<<grid_of(a.G), kBlock, 0, st>>>(a)));
}

void launch_mom_jacobi(const StepArgs &a, const double *uin, const double *win, double *uout,
                       double *wout, int second, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "mom_jacobi", ncell(a.G),
           (k_mom_jacobi<<<grid_tiles(a.G, a.tiles_per_block), kBlock, 0, st>>>(a, uin, win, uout, wout, second)));
}

void launch_enth_rhs(const StepArgs &a, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "enth_rhs", ncell(a.G), (k_enth_rhs<<<grid_of(a.G), kBlock, 0, st>>>(a)));
}

void launch_enth_jacobi(const StepArgs &a, const double *hin, double *hout, int second,
                        cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "enth_jacobi", ncell(a.G),
           (k_enth_jacobi<<<grid_tiles(a.G, a.tiles_per_block), kBlock, 0, st>>>(a, hin, hout, second)));
}

void launch_eos_coef(const StepArgs &a, const Level &L0, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "eos_coef", ncell(a.G), (k_eos_coef<<<grid_of(a.G), kBlock, 0, st>>>(a, L0)));
}

void launch_mg_coarsen(const Level &f, const Level &c, double omega, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "mg_coarsen", ncell(c.G), (k_mg_coarsen<<<grid_of(c.G), kBlock, 0, st>>>(f, c, omega)));
}

void launch_H(const StepArgs &a, const double *U, const double *W, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "H", ncell(a.G), (k_H<<<grid_of(a.G), kBlock, 0, st>>>(a, U, W)));
}

void launch_helm_rhs(const StepArgs &a, const Level &L0, const double *xin, double *xout,
                     int corr, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "helm_rhs", ncell(a.G),
           (k_helm_rhs<<<grid_of(a.G), kBlock, 0, st>>>(a, L0, xin, xout, corr)));
}

// z = M^-1 r into levels[0].e2 (one V(1,1)-cycle; ncoarse sweeps on the
// coarsest level). Returns the number of kernels launched.
int launch_vcycle(const StepArgs &a, Level *L, int nlev, int ncoarse, cudaStream_t st, Tracer *tr)
{
    if (nlev == 1) {
        TRACED(tr, "mg_single", ncell(L[0].G),
               (k_mg_single<<<grid_tiles(L[0].G, a.tiles_per_block), kBlock, 0, st>>>(L[0], L[0].e2, a)));
        return 1;
    }
    int n = 0;
    for (int l = 0; l + 1 < nlev; ++l, ++n)
        TRACED(tr, "mg_down", ncell(L[l].G),
               (k_mg_down<<<grid_of(L[l].G), kBlock, 0, st>>>(L[l], L[l + 1], a.F.omega, a.sc)));
    Level &C = L[nlev - 1];
    // sweep s writes e2 when ncoarse-1-s is even, so the last sweep ends in e2
    for (int s = 0; s < ncoarse; ++s, ++n) {
        double *out = ((ncoarse - 1 - s) % 2 == 0) ? C.e2 : C.e;
        const double *in = (out == C.e2) ? C.e : C.e2;
        TRACED(tr, "mg_coarse", ncell(C.G),
               (k_mg_coarse_sweep<<<grid_of(C.G), kBlock, 0, st>>>(C, in, out, s == 0, a.sc)));
    }
    for (int l = nlev - 2; l >= 0; --l, ++n)
        TRACED(tr, "mg_up", ncell(L[l].G),
               (k_mg_up<<<grid_tiles(L[l].G, a.tiles_per_block), kBlock, 0, st>>>(L[l], L[l + 1].e2, L[l + 1].G.P, L[l].e2,
                                                             l == 0, a)));
    return n;
}

// V-cycle levels below the finest: restriction steps of levels 1..nlev-2,
// the coarsest sweeps and the prolongation steps down to the finest (which
// yields z and r.z). Returns the number of kernels launched.
static int launch_vcycle_rest(const StepArgs &a, Level *L, int nlev, int ncoarse, cudaStream_t st,
                              Tracer *tr)
{
    int n = 0;
    for (int l = 1; l + 1 < nlev; ++l, ++n)
        TRACED(tr, "mg_down", ncell(L[l].G),
               (k_mg_down<<<grid_of(L[l].G), kBlock, 0, st>>>(L[l], L[l + 1], a.F.omega, a.sc)));
    Level &C = L[nlev - 1];
    for (int s = 0; s < ncoarse; ++s, ++n) {
        double *out = ((ncoarse - 1 - s) % 2 == 0) ? C.e2 : C.e;
        const double *in = (out == C.e2) ? C.e : C.e2;
        TRACED(tr, "mg_coarse", ncell(C.G),
               (k_mg_coarse_sweep<<<grid_of(C.G), kBlock, 0, st>>>(C, in, out, s == 0, a.sc)));
    }
    for (int l = nlev - 2; l >= 0; --l, ++n)
        TRACED(tr, "mg_up", ncell(L[l].G),
               (k_mg_up<<<grid_tiles(L[l].G, a.tiles_per_block), kBlock, 0, st>>>(L[l], L[l + 1].e2, L[l + 1].G.P, L[l].e2,
                                                             l == 0, a)));
    return n;
}

// One CG iteration after the first preconditioning: p = z + beta p and q = A p;
// x, r updated together with the first step of the next V-cycle; the rest of
// the V-cycle. Returns the number of kernels launched.
int launch_cg_iter(const StepArgs &a, Level *L, int nlev, int ncoarse, double *x, cudaStream_t st,
                   Tracer *tr)
{
    TRACED(tr, "cg_pspmv", ncell(a.G), (k_cg_pspmv<<<grid_tiles(a.G, a.tiles_per_block), kBlock, 0, st>>>(a, L[0])));
    if (nlev == 1) {
        TRACED(tr, "cg_update_single", ncell(a.G),
               (k_cg_update_single<<<grid_tiles(a.G, a.tiles_per_block), kBlock, 0, st>>>(a, L[0], x)));
        return 2;
    }
    TRACED(tr, "cg_update_down", ncell(a.G),
           (k_cg_update_down<<<grid_tiles(a.G, a.tiles_per_block), kBlock, 0, st>>>(a, L[0], L[1], x)));
    return 2 + launch_vcycle_rest(a, L, nlev, ncoarse, st, tr);
}

namespace {

// graph = 1: block (0,0) also sets the IF condition of the network pass
// (run it only while the solve is not finished)
template <class R>
__global__ void k_guess_in(Geom G, const R *r, float *dense, Scal *sc, cudaGraphConditionalHandle h, int graph,
                           int body_launches)
{
    const bool over = loop_over(sc, LOOP_CG);
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        if (graph) cudaGraphSetConditional(h, over ? 0u : 1u);
        if (!over) sc->launches += body_launches;
    }
    if (over) return;
    int i, k;
    if (!cell_of(G, blockIdx.x, blockIdx.y, i, k)) return;
    dense[(size_t)k * G.nx + i] = (float)r[cidx(G, i, k)];
}

template <class R>
__global__ void k_guess_dots(LevelT<R> L, const float *e, const R *r, R *q, Scal *sc, double *partials)
{
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double sm[kT1];
    __shared__ double red[2 * NTHREADS];
    R acc[2] = {(R)0, (R)0};
    double tot[2];
    ph_guess_dots<R>(L, e, r, q, sm, blockIdx.x, blockIdx.y, acc);
    if (grid_sum<2, R>(acc, red, partials, &sc->counters[CNT_GUESS], tot)) fin_guess_dots(sc, tot);
}

template <class R>
__global__ void k_guess_apply(LevelT<R> L, const float *e, const R *q, R *r, R *x, Scal *sc, double *partials,
                              double tol2)
{
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double red[NTHREADS];
    R acc[1] = {(R)0};
    double tot[1];
    ph_guess_apply<R>(L, e, q, r, x, sc->galpha, blockIdx.x, blockIdx.y, acc);
    if (grid_sum<1, R>(acc, red, partials, &sc->counters[CNT_GUESS], tot)) fin_guess_apply(sc, tot, tol2);
}

// ---- flexible CG with a two-stage preconditioner (attach mode 2) ----
//
// z = g e + M(r - g A e): the network's correction e = N(r) with the step g
// that minimises the A-norm error along it, then one multigrid V-cycle M on
// the residual it leaves. The network alone stagnates (it cannot represent
// the residual its own step leaves), the V-cycle keeps the linear part.
// The preconditioner is nonlinear, so the one-term recurrence is written in
// the form that stays a descent method for a changing preconditioner
// (flexible CG truncated to one previous direction): beta = -(z.q_old) /
// (p_old.q_old), p = z + beta p_old, alpha = r.p / p.A p.

// A e at cell (i, k) of a tile holding e (FP64, halo 1).
__device__ __forceinline__ double fcg_ae(const Level &L, int q, int i, int k, const Tile<1> &se, int y, int x)
{
    return helm_tile<1, double>(L, q, i, k, se, y, x);
}

// The network's correction e (FP32, dense) on the tile and its halo.
__device__ __forceinline__ void fcg_load_e(Tile<1> &se, const Geom &G, const float *e, int bx, int bz)
{
    load_tile_fn<1, double>(se, G, bx, bz, [&](int, int i, int k) { return (double)e[(size_t)k * G.nx + i]; });
}

// acc += (r.e, e.A e); g = r.e / e.A e (0 unless e.A e > 0).
__global__ void k_fcg_dots(Level L, const float *e, Scal *sc, double *partials)
{
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double sm[kT1];
    __shared__ double red[2 * NTHREADS];
    const Geom &G = L.G;
    const double *r = res_of(L, sc->cg_it);
    Tile<1> &se = tile_at<1>(sm, 0);
    fcg_load_e(se, G, e, blockIdx.x, blockIdx.y);
    __syncthreads();
    double acc[2] = {0.0, 0.0}, tot[2];
    int i, k;
    if (cell_of(G, blockIdx.x, blockIdx.y, i, k)) {
        const int q = cidx(G, i, k);
        const int y = threadIdx.y + 1, x = threadIdx.x + 1;
        const double ev = se[y][x];
        acc[0] = ld(&r[q]) * ev;
        acc[1] = ev * fcg_ae(L, q, i, k, se, y, x);
    }
    if (grid_sum<2>(acc, red, partials, &sc->counters[CNT_GUESS], tot))
        sc->galpha = (tot[1] > 0.0 && isfinite(tot[0]) && isfinite(tot[1])) ? tot[0] / tot[1] : 0.0;
}

// s = r - g A e, the V-cycle's input.
__global__ void k_fcg_rest(Level L, const float *e, double *s, Scal *sc)
{
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double sm[kT1];
    const Geom &G = L.G;
    const double *r = res_of(L, sc->cg_it);
    const double g = sc->galpha;
    Tile<1> &se = tile_at<1>(sm, 0);
    fcg_load_e(se, G, e, blockIdx.x, blockIdx.y);
    __syncthreads();
    int i, k;
    if (cell_of(G, blockIdx.x, blockIdx.y, i, k)) {
        const int q = cidx(G, i, k);
        const int y = threadIdx.y + 1, x = threadIdx.x + 1;
        s[q] = fma(-g, fcg_ae(L, q, i, k, se, y, x), ld(&r[q]));
    }
}

// z = g e + z_MG (the V-cycle's output in e2), written to e2; acc += z.q_old
// (none before the first direction); beta = -z.q_old / p_old.q_old.
__global__ void k_fcg_out(Level L, const float *e, const double *q_old, Scal *sc, double *partials)
{
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double red[NTHREADS];
    const Geom &G = L.G;
    const bool first = sc->cg_it == 0;
    const double g = sc->galpha;
    double acc[1] = {0.0}, tot[1];
    int i, k;
    if (cell_of(G, blockIdx.x, blockIdx.y, i, k)) {
        const int q = cidx(G, i, k);
        const double z = fma(g, (double)e[(size_t)k * G.nx + i], L.e2[q]);
        L.e2[q] = z;
        if (!first) acc[0] = z * ld(&q_old[q]);
    }
    if (grid_sum<1>(acc, red, partials, &sc->counters[CNT_RZ], tot)) {
        sc->beta = (first || sc->pq == 0.0) ? 0.0 : -tot[0] / sc->pq;
        if (!isfinite(tot[0])) sc->status = GEA_ERR_NONFINITE;
    }
}

// r for the network (FP32, dense), from the residual of the current iteration.
__global__ void k_fcg_stage_in(Level L, float *dense, Scal *sc)
{
    if (loop_over(sc, LOOP_CG)) return;
    const Geom &G = L.G;
    int i, k;
    if (!cell_of(G, blockIdx.x, blockIdx.y, i, k)) return;
    dense[(size_t)k * G.nx + i] = (float)ld(&res_of(L, sc->cg_it)[cidx(G, i, k)]);
}

// p = z + beta p_old (on the tile and its halo), q = A p; acc += (p.q, r.p);
// alpha = r.p / p.q.
__global__ void k_fcg_pspmv(StepArgs a, Level L)
{
    Scal *sc = a.sc;
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double sm[kT1];
    __shared__ double red[2 * NTHREADS];
    const Geom &G = L.G;
    const int it = sc->cg_it;
    const double *pold = (it & 1) ? a.p1 : a.p0;
    double *pnew = (it & 1) ? a.p0 : a.p1;
    const double *r = res_of(L, it);
    const double beta = sc->beta;
    const int bx = blockIdx.x, bz = blockIdx.y;
    Tile<1> &sp = tile_at<1>(sm, 0);
    load_tile_fn<1, double>(sp, G, bx, bz, [&](int q, int, int) { return fma(beta, ld(&pold[q]), ld(&L.e2[q])); });
    __syncthreads();
    double acc[2] = {0.0, 0.0}, tot[2];
    int i, k;
    if (cell_of(G, bx, bz, i, k)) {
        const int q = cidx(G, i, k);
        const int y = threadIdx.y + 1, x = threadIdx.x + 1;
        const double pq = sp[y][x];
        const double Ap = helm_tile<1, double>(L, q, i, k, sp, y, x);
        pnew[q] = pq;
        a.q[q] = Ap;
        acc[0] = pq * Ap;
        acc[1] = ld(&r[q]) * pq;
    }
    if (grid_sum<2>(acc, red, a.partials, &sc->counters[CNT_PQ], tot)) {
        sc->pq = tot[0];
        sc->alpha = tot[0] != 0.0 ? tot[1] / tot[0] : 0.0;
        if (!isfinite(tot[0]) || !isfinite(tot[1])) sc->status = GEA_ERR_NONFINITE;
    }
}

// x += alpha p, r_new = r - alpha q (into the other residual buffer); acc += r_new^2.
__global__ void k_fcg_update(StepArgs a, Level L, double *x)
{
    Scal *sc = a.sc;
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double red[NTHREADS];
    const Geom &G = L.G;
    const int it = sc->cg_it;
    const double *p = (it & 1) ? a.p0 : a.p1;
    const double *rin = res_of(L, it);
    double *rout = res_of(L, it + 1);
    const double alpha = sc->alpha;
    double acc[1] = {0.0}, tot[1];
    int i, k;
    if (cell_of(G, blockIdx.x, blockIdx.y, i, k)) {
        const int q = cidx(G, i, k);
        x[q] = fma(alpha, ld(&p[q]), x[q]);
        const double rn = fma(-alpha, ld(&a.q[q]), ld(&rin[q]));
        rout[q] = rn;
        acc[0] = rn * rn;
    }
    if (grid_sum<1>(acc, red, a.partials, &sc->counters[CNT_UPD], tot)) fin_update(sc, tot, a.cg_rtol2);
}

}  // namespace

template <class R>
void launch_guess_in(const StepArgs &a, const LevelT<R> &L, const R *r, float *dense_r,
                     cudaGraphConditionalHandle h, bool graph, cudaStream_t st, Tracer *tr)
{
    const Geom &G = L.G;
    TRACED(tr, "guess_in", ncell(G),
           (k_guess_in<R><<<grid_of(G), kBlock, 0, st>>>(G, r, dense_r, a.sc, h, graph ? 1 : 0,
                                                          2 + gea_net_launches())));
}

template <class R>
int launch_net_guess(const StepArgs &a, const LevelT<R> &L, R *r, R *q, R *x, double tol2, gea_net *net,
                     float *dense_r, float *dense_e, cudaStream_t st, Tracer *tr)
{
    const Geom &G = L.G;
    if (tr) tr->begin("net_forward", ncell(G), st);
    const int nk = gea_net_run(net, st, 1, G.nz, G.nx, dense_r, dense_e);
    if (tr) tr->end(st);
    if (nk < 0) return -1;
    TRACED(tr, "guess_dots", ncell(G),
           (k_guess_dots<R><<<grid_of(G), kBlock, 0, st>>>(L, dense_e, r, q, a.sc, a.partials)));
    TRACED(tr, "guess_apply", ncell(G),
           (k_guess_apply<R><<<grid_of(G), kBlock, 0, st>>>(L, dense_e, q, r, x, a.sc, a.partials, tol2)));
    return 2 + nk;
}

int launch_fcg_iter(const StepArgs &a, Level *L, int nlev, int ncoarse, double *x, gea_net *net,
                    float *dense_r, float *dense_e, double *s_buf, cudaStream_t st, Tracer *tr)
{
    const Geom &G = L[0].G;
    TRACED(tr, "fcg_stage_in", ncell(G), (k_fcg_stage_in<<<grid_of(G), kBlock, 0, st>>>(L[0], dense_r, a.sc)));
    if (tr) tr->begin("net_forward", ncell(G), st);
    const int nk = gea_net_run(net, st, 1, G.nz, G.nx, dense_r, dense_e);
    if (tr) tr->end(st);
    if (nk < 0) return -1;
    TRACED(tr, "fcg_dots", ncell(G), (k_fcg_dots<<<grid_of(G), kBlock, 0, st>>>(L[0], dense_e, a.sc, a.partials)));
    TRACED(tr, "fcg_rest", ncell(G),
           (k_fcg_rest<<<grid_of(G), kBlock, 0, st>>>(L[0], dense_e, s_buf, a.sc)));
    // the V-cycle on s: a copy of the levels whose finest residual buffers
    // both name s_buf
    Level M[kMaxLevels];
    for (int l = 0; l < nlev; ++l) M[l] = L[l];
    M[0].r = M[0].r_alt = s_buf;
    const int nv = launch_vcycle(a, M, nlev, ncoarse, st, tr);
    TRACED(tr, "fcg_out", ncell(G),
           (k_fcg_out<<<grid_of(G), kBlock, 0, st>>>(L[0], dense_e, a.q, a.sc, a.partials)));
    TRACED(tr, "fcg_pspmv", ncell(G), (k_fcg_pspmv<<<grid_of(G), kBlock, 0, st>>>(a, L[0])));
    TRACED(tr, "fcg_update", ncell(G), (k_fcg_update<<<grid_of(G), kBlock, 0, st>>>(a, L[0], x)));
    return 6 + nk + nv;
}

template void launch_guess_in<double>(const StepArgs &, const LevelT<double> &, const double *, float *,
                                      cudaGraphConditionalHandle, bool, cudaStream_t, Tracer *);
template void launch_guess_in<float>(const StepArgs &, const LevelT<float> &, const float *, float *,
                                     cudaGraphConditionalHandle, bool, cudaStream_t, Tracer *);
template int launch_net_guess<double>(const StepArgs &, const LevelT<double> &, double *, double *, double *,
                                      double, gea_net *, float *, float *, cudaStream_t, Tracer *);
template int launch_net_guess<float>(const StepArgs &, const LevelT<float> &, float *, float *, float *, double,
                                     gea_net *, float *, float *, cudaStream_t, Tracer *);

void launch_correct(const StepArgs &a, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "correct", ncell(a.G), (k_correct<<<grid_of(a.G), kBlock, 0, st>>>(a)));
}

void launch_loop_ctl(Scal *sc, cudaGraphConditionalHandle h, bool graph, int which,
                     int maxtrips, int body_launches, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "loop_ctl", 1,
           (k_loop_ctl<<<1, 1, 0, st>>>(sc, h, graph ? 1 : 0, which, maxtrips, body_launches)));
}

void launch_loop_gate(Scal *sc, cudaGraphConditionalHandle h, int which, cudaStream_t st)
{
    k_loop_gate<<<1, 1, 0, st>>>(sc, h, which);
}

void launch_step_begin(Scal *sc, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "step_begin", 1, (k_step_begin<<<1, 1, 0, st>>>(sc)));
}

void launch_step_end(Scal *sc, int fixed_launches, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "step_end", 1, (k_step_end<<<1, 1, 0, st>>>(sc, fixed_launches)));
}

void launch_diag(const Geom &G, const Phys &F, const State &S, const double *theta_bar,
                 double *theta_out, Scal *sc, double *partials, cudaStream_t st)
{
    k_diag<<<grid_of(G), kBlock, 0, st>>>(G, F, S, theta_bar, theta_out, sc, partials);
}

}  // namespace gea
