// gea_mixed.cu -- per-phase kernels of the mixed-precision time step (the
// GEA pressure-based Euler scheme of Girfoglio, Quaini & Rozza, arXiv
// 2303.10499, Section 3, unchanged) and their launchers.
//
// On GB300 FP32 issues 64 times faster than FP64. The mixed path keeps
// everything that carries the hydrostatic balance or the conservation
// properties in FP64 -- the state, p' = p + rho g z, rho^{2/3}, the face
// forces, the right-hand sides, H(u), the flux correction -- and moves the
// iterative solves to FP32 by defect correction: each implicit problem
// T x = b gets one FP64 residual r0 = b - T x_old, an FP32 solve T dx = r0 to a
// relative residual of 1e-6 (Jacobi for the predictors, multigrid-
// preconditioned CG for the pressure equation) and the FP64 update
// x = x_old + dx. Increments have homogeneous wall conditions (the h ghost
// offset g dz cancels). FP32 reductions are summed per block in FP32 and
// across blocks in FP64.
#include "gea_internal.cuh"
#include "gea_tiles.cuh"

namespace gea {

namespace {

using namespace tiles;

__device__ __forceinline__ bool loop_over(const Scal *sc, int which)
{
    return sc->status || sc->done[which];
}

__global__ void k_mx_pred(StepArgs a, MixedArgs m)
{
    if (a.sc->status) return;
    __shared__ double sm[2 * kT2];
    __shared__ double red[2 * NTHREADS];
    double acc[2] = {0.0, 0.0}, tot[2];
    ph_pred_t<true>(a, m, sm, blockIdx.x, blockIdx.y, acc);
    if (grid_sum<2>(acc, red, a.partials, &a.sc->counters[CNT_PRED], tot)) fin_pred(a.sc, tot);
}

// Sweep pairs as in the FP64 path: the second sweep of a pair copies once the
// first met the tolerance.
__global__ void k_mx_mom(StepArgs a, MixedArgs m, const float *ui, const float *wi, float *uo, float *wo,
                         int second)
{
    if (a.sc->status) return;
    if (second && a.sc->done[LOOP_MOM]) {
        block_tiles(a.G, [&](int bx, int bz) {
            ph_copy(a.G, ui, uo, bx, bz);
            ph_copy(a.G, wi, wo, bx, bz);
        });
        return;
    }
    __shared__ double sm[kT2];
    __shared__ double red[2 * NTHREADS];
    float acc[2] = {0.0f, 0.0f};
    double tot[2];
    block_tiles(a.G, [&](int bx, int bz) {
        ph_sweep2<float, BC_U, BC_W>(a.G, a.F, m.T, m.dinvu, m.r0u, m.r0w, ui, wi, uo, wo, sm, bx, bz, acc);
    });
    if (grid_sum<2, float>(acc, red, a.partials, &a.sc->counters[CNT_MOM], tot)) fin_mom(a.sc, tot, m.tol2);
}

__global__ void k_mx_enth_rhs(StepArgs a, MixedArgs m)
{
    if (a.sc->status) return;
    __shared__ double sm[3 * kT2];
    __shared__ double red[NTHREADS];
    double acc[1] = {0.0}, tot[1];
    ph_enth_rhs_t<true>(a, m, nullptr, nullptr, nullptr, sm, blockIdx.x, blockIdx.y, acc);
    if (grid_sum<1>(acc, red, a.partials, &a.sc->counters[CNT_ENTH_RHS], tot)) fin_enth_rhs(a.sc, tot);
}

__global__ void k_mx_enth(StepArgs a, MixedArgs m, const float *hi, float *ho, int second)
{
    if (a.sc->status) return;
    if (second && a.sc->done[LOOP_ENTH]) {
        block_tiles(a.G, [&](int bx, int bz) { ph_copy(a.G, hi, ho, bx, bz); });
        return;
    }
    __shared__ double sm[kT2];
    __shared__ double red[NTHREADS];
    float acc[1] = {0.0f};
    double tot[1];
    block_tiles(a.G, [&](int bx, int bz) {
        ph_sweep1<float, BC_EVEN>(a.G, a.F, m.T, m.dinvh, m.r0h, (float)(a.F.mu - a.F.nuh), hi, ho, sm, bx, bz,
                                  acc);
    });
    if (grid_sum<1, float>(acc, red, a.partials, &a.sc->counters[CNT_ENTH], tot)) fin_enth(a.sc, tot, m.tol2);
}

__global__ void k_mx_eos(StepArgs a, Level L, LevelF L32, const float *dh)
{
    if (a.sc->status) return;
    __shared__ double sm[2 * kT1 + BZ * (BX + 1) + (BZ + 1) * BX];
    ph_eos_t<true>(a, L, L32, nullptr, dh, sm, blockIdx.x, blockIdx.y);
}

__global__ void k_mx_coarsen(LevelF f, LevelF c, double omega)
{
    ph_coarsen<float>(f, c, omega, blockIdx.x, blockIdx.y);
}

__global__ void k_mx_helm_rhs(StepArgs a, Level L, LevelF L32, MixedArgs m, const double *xin,
                              double *xout, int corr)
{
    if (a.sc->status) return;
    __shared__ double sm[4 * kT1];
    __shared__ double red[2 * NTHREADS];
    double acc[2] = {0.0, 0.0}, tot[2];
    ph_helm_rhs_t<true>(a, L, L32, m, xin, xout, sm, blockIdx.x, blockIdx.y, acc);
    if (grid_sum<2>(acc, red, a.partials, &a.sc->counters[CNT_HELM], tot))
        fin_helm_mixed(a.sc, tot, a.cg_rtol2, corr);
}

// ---- FP32 V-cycle and CG steps ----

__global__ void k_mx_mg_down(LevelF f, LevelF c, double omega, Scal *sc)
{
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double sm[kT1 + BZ * BX];
    ph_mg_down<float>(f, c, omega, sm, blockIdx.x, blockIdx.y);
}

__global__ void k_mx_mg_coarse(LevelF L, const float *ein, float *eout, int first, Scal *sc)
{
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double sm[kT1];
    ph_mg_coarse<float>(L, ein, eout, first, sm, blockIdx.x, blockIdx.y);
}

__global__ void k_mx_mg_up(LevelF f, const float *ec, int Pc, float *out, int finest, StepArgs a)
{
    if (loop_over(a.sc, LOOP_CG)) return;
    __shared__ double sm[kT1];
    __shared__ double red[NTHREADS];
    float acc[1] = {0.0f};
    double tot[1];
    const float *res = finest ? res_of(f, a.sc->cg_it) : f.r;
    block_tiles(f.G, [&](int bx, int bz) { ph_mg_up<float>(f, res, ec, Pc, out, sm, bx, bz, acc); });
    if (!finest) return;
    if (grid_sum<1, float>(acc, red, a.partials, &a.sc->counters[CNT_RZ], tot)) fin_rz(a.sc, tot);
}

__global__ void k_mx_mg_single(LevelF f, float *out, StepArgs a)
{
    if (loop_over(a.sc, LOOP_CG)) return;
    __shared__ double sm[kT1];
    __shared__ double red[NTHREADS];
    float acc[1] = {0.0f};
    double tot[1];
    block_tiles(f.G, [&](int bx, int bz) { ph_mg_single<float>(f, out, sm, bx, bz, acc); });
    if (grid_sum<1, float>(acc, red, a.partials, &a.sc->counters[CNT_RZ], tot)) fin_rz(a.sc, tot);
}

__global__ void k_mx_pspmv(StepArgs a, LevelF L, MixedArgs m)
{
    Scal *sc = a.sc;
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double sm[kT1];
    __shared__ double red[NTHREADS];
    const int it = sc->cg_it;
    const float *pold = (it & 1) ? m.p1 : m.p0;
    float *pnew = (it & 1) ? m.p0 : m.p1;
    float acc[1] = {0.0f};
    double tot[1];
    block_tiles(L.G, [&](int bx, int bz) { ph_pspmv<float>(L, pold, pnew, m.q, sc->beta, sm, bx, bz, acc); });
    if (grid_sum<1, float>(acc, red, a.partials, &sc->counters[CNT_PQ], tot)) fin_pq(sc, tot);
}

__global__ void k_mx_update_single(StepArgs a, LevelF L, MixedArgs m)
{
    Scal *sc = a.sc;
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double sm[kT1];
    __shared__ double red[2 * NTHREADS];
    const int it = sc->cg_it;
    const float *p = (it & 1) ? m.p0 : m.p1;
    float acc[2] = {0.0f, 0.0f};
    double tot[2];
    block_tiles(L.G, [&](int bx, int bz) {
        ph_update_single<float>(L, m.q, res_of(L, it), res_of(L, it + 1), m.x, p, sc->alpha, sm, bx, bz, acc);
    });
    if (grid_sum<2, float>(acc, red, a.partials, &sc->counters[CNT_UPD], tot)) {
        const double t0[1] = {tot[0]}, t1[1] = {tot[1]};
        fin_update(sc, t0, m.tol2);
        fin_rz(sc, t1);
    }
}

__global__ void k_mx_update_down(StepArgs a, LevelF f, LevelF c, MixedArgs m)
{
    Scal *sc = a.sc;
    if (loop_over(sc, LOOP_CG)) return;
    __shared__ double sm[kT1 + BZ * BX];
    __shared__ double red[NTHREADS];
    const int it = sc->cg_it;
    const float *p = (it & 1) ? m.p0 : m.p1;
    float acc[1] = {0.0f};
    double tot[1];
    block_tiles(f.G, [&](int bx, int bz) {
        ph_update_down<float>(f, c, m.q, res_of(f, it), res_of(f, it + 1), m.x, p, sc->alpha, a.F.omega, sm,
                              bx, bz, acc);
    });
    if (grid_sum<1, float>(acc, red, a.partials, &sc->counters[CNT_UPD], tot)) fin_update(sc, tot, m.tol2);
}

__global__ void k_mx_p_apply(StepArgs a, MixedArgs m)
{
    if (a.sc->status) return;
    ph_p_apply(a, m, blockIdx.x, blockIdx.y);
}

inline dim3 grid_of(const Geom &G) { return dim3((G.nx + BX - 1) / BX, (G.nz + BZ - 1) / BZ); }
const dim3 kBlock(BX, BZ);
inline long long ncell(const Geom &G) { return (long long)G.nx * G.nz; }

#define TRACED(tr, name, cells, launch)                         \
    do {                                                        \
        if (tr) (tr)->begin(name, (long long)(cells), st);      \
        launch;                                                 \
        if (tr) (tr)->end(st);                                  \
    } while (0)

// V-cycle of the FP32 hierarchy from level lfirst (lfirst = 0: from the
// finest residual; lfirst = 1: after ph_update_down restricted into level 1).
int vcycle32(const StepArgs &a, LevelF *L, int nlev, int ncoarse, int lfirst, cudaStream_t st, Tracer *tr)
{
    int n = 0;
    for (int l = lfirst; l + 1 < nlev; ++l, ++n)
        TRACED(tr, "mx_mg_down", ncell(L[l].G),
               (k_mx_mg_down<<<grid_of(L[l].G), kBlock, 0, st>>>(L[l], L[l + 1], a.F.omega, a.sc)));
    LevelF &C = L[nlev - 1];
    for (int s = 0; s < ncoarse; ++s, ++n) {
        float *out = ((ncoarse - 1 - s) % 2 == 0) ? C.e2 : C.e;
        const float *in = (out == C.e2) ? C.e : C.e2;
        TRACED(tr, "mx_mg_coarse", ncell(C.G),
               (k_mx_mg_coarse<<<grid_of(C.G), kBlock, 0, st>>>(C, in, out, s == 0, a.sc)));
    }
    for (int l = nlev - 2; l >= 0; --l, ++n)
        TRACED(tr, "mx_mg_up", ncell(L[l].G),
               (k_mx_mg_up<<<grid_tiles(L[l].G, a.tiles_per_block), kBlock, 0, st>>>(L[l], L[l + 1].e2, L[l + 1].G.P, L[l].e2,
                                                                l == 0, a)));
    return n;
}

}  // namespace

void launch_mx_pred(const StepArgs &a, const MixedArgs &m, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "mx_pred", ncell(a.G), (k_mx_pred<<<grid_of(a.G), kBlock, 0, st>>>(a, m)));
}

void launch_mx_mom(const StepArgs &a, const MixedArgs &m, const float *ui, const float *wi, float *uo,
                   float *wo, int second, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "mx_mom", ncell(a.G),
           (k_mx_mom<<<grid_tiles(a.G, a.tiles_per_block), kBlock, 0, st>>>(a, m, ui, wi, uo, wo, second)));
}

void launch_mx_enth_rhs(const StepArgs &a, const MixedArgs &m, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "mx_enth_rhs", ncell(a.G), (k_mx_enth_rhs<<<grid_of(a.G), kBlock, 0, st>>>(a, m)));
}

void launch_mx_enth(const StepArgs &a, const MixedArgs &m, const float *hi, float *ho, int second,
                    cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "mx_enth", ncell(a.G), (k_mx_enth<<<grid_tiles(a.G, a.tiles_per_block), kBlock, 0, st>>>(a, m, hi, ho, second)));
}

void launch_mx_eos(const StepArgs &a, const Level &L0, const LevelF &L32, const float *dh, cudaStream_t st,
                   Tracer *tr)
{
    TRACED(tr, "mx_eos", ncell(a.G), (k_mx_eos<<<grid_of(a.G), kBlock, 0, st>>>(a, L0, L32, dh)));
}

void launch_mx_coarsen(const LevelF &f, const LevelF &c, double omega, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "mx_coarsen", ncell(c.G), (k_mx_coarsen<<<grid_of(c.G), kBlock, 0, st>>>(f, c, omega)));
}

void launch_mx_helm_rhs(const StepArgs &a, const Level &L0, const LevelF &L32, const MixedArgs &m,
                        const double *xin, double *xout, int corr, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "mx_helm_rhs", ncell(a.G),
           (k_mx_helm_rhs<<<grid_of(a.G), kBlock, 0, st>>>(a, L0, L32, m, xin, xout, corr)));
}

// z = M^-1 r_0 for the FP32 solve (one V(1,1)-cycle).
int launch_mx_vcycle(const StepArgs &a, LevelF *L, int nlev, int ncoarse, cudaStream_t st, Tracer *tr)
{
    if (nlev == 1) {
        TRACED(tr, "mx_mg_single", ncell(L[0].G),
               (k_mx_mg_single<<<grid_tiles(L[0].G, a.tiles_per_block), kBlock, 0, st>>>(L[0], L[0].e2, a)));
        return 1;
    }
    return vcycle32(a, L, nlev, ncoarse, 0, st, tr);
}

// One FP32 CG iteration (see launch_cg_iter).
int launch_mx_cg_iter(const StepArgs &a, const MixedArgs &m, LevelF *L, int nlev, int ncoarse,
                      cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "mx_pspmv", ncell(a.G), (k_mx_pspmv<<<grid_tiles(a.G, a.tiles_per_block), kBlock, 0, st>>>(a, L[0], m)));
    if (nlev == 1) {
        TRACED(tr, "mx_update_single", ncell(a.G),
               (k_mx_update_single<<<grid_tiles(a.G, a.tiles_per_block), kBlock, 0, st>>>(a, L[0], m)));
        return 2;
    }
    TRACED(tr, "mx_update_down", ncell(a.G),
           (k_mx_update_down<<<grid_tiles(a.G, a.tiles_per_block), kBlock, 0, st>>>(a, L[0], L[1], m)));
    return 2 + vcycle32(a, L, nlev, ncoarse, 1, st, tr);
}

void launch_mx_p_apply(const StepArgs &a, const MixedArgs &m, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "mx_p_apply", ncell(a.G), (k_mx_p_apply<<<grid_of(a.G), kBlock, 0, st>>>(a, m)));
}

}  // namespace gea
