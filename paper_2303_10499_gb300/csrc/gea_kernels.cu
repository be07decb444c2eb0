// gea_kernels.cu -- CUDA kernels (sm_103a, FP64) of one predictor-corrector
// time step of the GEA pressure-based Euler solver (Girfoglio, Quaini &
// Rozza, arXiv 2303.10499, Section 3), and their host-side launchers.
//
// One thread per cell on 32 x 8 blocks; x is the fast index so a warp reads
// one row segment of 256 contiguous bytes. Reductions are deterministic:
// per-block partial sums, added in a fixed order by the last block.
// Kernels that run inside a device-side loop check the loop's convergence
// flag and the context's error status on entry and return early; the loop
// itself is ended by a one-thread control kernel that always runs.
#include "gea_internal.cuh"

#include <math.h>

namespace gea {

namespace {

__device__ __forceinline__ double sq(double x) { return x * x; }

// Convective term (1/V) sum_j phi_j X_j with X given by get(i,k) (which
// returns ghost values outside the box); wall faces carry no flux.
template <class Get>
__device__ __forceinline__ double conv_get(const Geom &G, const double *__restrict__ phix,
                                           const double *__restrict__ phiz, Get get, int i,
                                           int k)
{
    double s = 0.0;
    if (i + 1 < G.nx)
        s += phix[k * G.P + i + 1] * interp4(get(i - 1, k), get(i, k), get(i + 1, k), get(i + 2, k));
    if (i > 0)
        s -= phix[k * G.P + i] * interp4(get(i - 2, k), get(i - 1, k), get(i, k), get(i + 1, k));
    if (k + 1 < G.nz)
        s += phiz[(k + 1) * G.P + i] * interp4(get(i, k - 1), get(i, k), get(i, k + 1), get(i, k + 2));
    if (k > 0)
        s -= phiz[k * G.P + i] * interp4(get(i, k - 2), get(i, k - 1), get(i, k), get(i, k + 1));
    return s * G.iV;
}

__device__ __forceinline__ bool cell_of_thread(const Geom &G, int &i, int &k)
{
    i = blockIdx.x * BX + threadIdx.x;
    k = blockIdx.y * BZ + threadIdx.y;
    return i < G.nx && k < G.nz;
}

__device__ __forceinline__ bool finite2(double a) { return isfinite(a); }

// ---------------------------------------------------------------------------
// set-up from conservative variables
// ---------------------------------------------------------------------------

__global__ void k_derive(Geom G, Phys F, const double *__restrict__ rho,
                         const double *__restrict__ rhou, const double *__restrict__ rhow,
                         const double *__restrict__ rhoe, State S, Scal *sc)
{
    int i, k;
    if (!cell_of_thread(G, i, k)) return;
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
    S.phix[k * G.P + i] = i > 0 ? 0.5 * (rhou[q - 1] + rhou[q]) * G.dz : 0.0;
    if (i == G.nx - 1) S.phix[k * G.P + G.nx] = 0.0;
    S.phiz[k * G.P + i] = k > 0 ? 0.5 * (rhow[q - G.P] + rhow[q]) * G.dx : 0.0;
    if (k == G.nz - 1) S.phiz[G.nz * G.P + i] = 0.0;
}

// ---------------------------------------------------------------------------
// Step 1 (eq. e1_d and eq. step2_sd, first line)
// ---------------------------------------------------------------------------

// rho^{n+1/3} = rho^n - dt sum_j phi_j / V; right-hand sides of the implicit
// momentum predictor b = rho^n u^n / dt - G_cell^n, where G_cell is the
// average of the two face forces grad p'^n - g z grad rho^n per direction
// (zero on wall faces); the shared part of the Jacobi divisor
// rho1/dt + (7/12) sum_j phi_j / V; the initial guess u^n.
__global__ void k_pred_setup(StepArgs a)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    if (a.sc->status) return;
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    double v[2] = {0.0, 0.0};
    if (in) {
        const int q = cidx(G, i, k);
        const State &S = a.S;
        const double div = (S.phix[q + 1] - S.phix[q] + S.phiz[q + G.P] - S.phiz[q]) * G.iV;
        const double rho1 = S.rho[q] - F.dt * div;
        const double z = (k + 0.5) * G.dz;
        const double rq = S.rho[q], pq = S.pp[q];
        double gxw = 0.0, gxe = 0.0, gzs = 0.0, gzn = 0.0;
        if (i > 0) gxw = (pq - S.pp[q - 1]) * G.idx - F.g * z * (rq - S.rho[q - 1]) * G.idx;
        if (i + 1 < G.nx) gxe = (S.pp[q + 1] - pq) * G.idx - F.g * z * (S.rho[q + 1] - rq) * G.idx;
        if (k > 0) gzs = (pq - S.pp[q - G.P]) * G.idz - F.g * (k * G.dz) * (rq - S.rho[q - G.P]) * G.idz;
        if (k + 1 < G.nz)
            gzn = (S.pp[q + G.P] - pq) * G.idz - F.g * ((k + 1) * G.dz) * (S.rho[q + G.P] - rq) * G.idz;
        const double bu = rq * S.u[q] * F.idt - 0.5 * (gxw + gxe);
        const double bw = rq * S.w[q] * F.idt - 0.5 * (gzs + gzn);
        a.rho1[q] = rho1;
        a.jd[q] = rho1 * F.idt + (7.0 / 12.0) * div;
        a.bu[q] = bu;
        a.bw[q] = bw;
        a.ua[q] = S.u[q];
        a.wa[q] = S.w[q];
        v[0] = bu * bu;
        v[1] = bw * bw;
    }
    double tot[2];
    if (grid_sum<2>(v, a.partials, &a.sc->counters[CNT_PRED], tot)) {
        Scal *sc = a.sc;
        sc->bn2[0] = tot[0];
        sc->bn2[1] = tot[1];
        sc->done[LOOP_MOM] = 0;
        sc->trips[LOOP_MOM] = 0;
        sc->sweeps[0] = 0;
    }
}

// One Jacobi sweep of (rho1/dt) X + C(X) - mu L(X) = b for X = u (odd in x)
// and X = w (odd in z).
__global__ void k_mom_jacobi(StepArgs a, const double *__restrict__ uin,
                             const double *__restrict__ win, double *__restrict__ uout,
                             double *__restrict__ wout)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    if (a.sc->status) return;
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    double v[2] = {0.0, 0.0};
    if (in) {
        const int q = cidx(G, i, k);
        const double *phix = a.S.phix, *phiz = a.S.phiz;
        auto gu = [&](int ii, int kk) { return ldc<BC_U>(G, F, uin, ii, kk); };
        auto gw = [&](int ii, int kk) { return ldc<BC_W>(G, F, win, ii, kk); };
        const double r1 = a.rho1[q] * F.idt;
        const double d = a.jd[q] + F.mu * (2.0 * G.idx * G.idx + 2.0 * G.idz * G.idz);
        const double uq = uin[q], wq = win[q];
        const double ru = a.bu[q] - (r1 * uq + conv_get(G, phix, phiz, gu, i, k)
                                     - F.mu * laplacian<BC_U>(G, F, uin, i, k));
        const double rw = a.bw[q] - (r1 * wq + conv_get(G, phix, phiz, gw, i, k)
                                     - F.mu * laplacian<BC_W>(G, F, win, i, k));
        uout[q] = uq + ru / d;
        wout[q] = wq + rw / d;
        v[0] = ru * ru;
        v[1] = rw * rw;
    }
    double tot[2];
    if (grid_sum<2>(v, a.partials, &a.sc->counters[CNT_MOM], tot)) {
        Scal *sc = a.sc;
        sc->sweeps[0] += 1;
        if (!finite2(tot[0]) || !finite2(tot[1])) {
            sc->status = 5;
        } else if (tot[0] <= a.jac_rtol2 * sc->bn2[0] && tot[1] <= a.jac_rtol2 * sc->bn2[1]) {
            sc->done[LOOP_MOM] = 1;
        }
    }
}

// ---------------------------------------------------------------------------
// Step 2 (eq. step3_sd, step3_2sd, step3_3sd)
// ---------------------------------------------------------------------------

// Right-hand side of the enthalpy equation:
//   (rho^n h^n + rho^n K^n - p^{n-1})/dt - rho1 K1/dt - C(K1) + p^n/dt - rho1 g w1
// with K1 = |u^{n+1/3}|^2/2 (eq. step1_3sd); initial guess h^n.
__global__ void k_enth_rhs(StepArgs a)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    if (a.sc->status) return;
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    double v[1] = {0.0};
    if (in) {
        const int q = cidx(G, i, k);
        const State &S = a.S;
        const double *ua = a.ua, *wa = a.wa;
        auto gK = [&](int ii, int kk) {
            return 0.5 * (sq(ldc<BC_EVEN>(G, F, ua, ii, kk)) + sq(ldc<BC_EVEN>(G, F, wa, ii, kk)));
        };
        const double rq = S.rho[q];
        const double Kn = 0.5 * (S.u[q] * S.u[q] + S.w[q] * S.w[q]);
        const double K1 = 0.5 * (ua[q] * ua[q] + wa[q] * wa[q]);
        const double rho1 = a.rho1[q];
        const double be = (rq * S.h[q] + rq * Kn - S.pold[q]) * F.idt;
        const double bh = be - rho1 * K1 * F.idt - conv_get(G, S.phix, S.phiz, gK, i, k)
                          + S.p[q] * F.idt - rho1 * F.g * wa[q];
        a.bh[q] = bh;
        a.ha[q] = S.h[q];
        v[0] = bh * bh;
    }
    double tot[1];
    if (grid_sum<1>(v, a.partials, &a.sc->counters[CNT_ENTH_RHS], tot)) {
        Scal *sc = a.sc;
        sc->bn2[2] = tot[0];
        sc->done[LOOP_ENTH] = 0;
        sc->trips[LOOP_ENTH] = 0;
        sc->sweeps[1] = 0;
    }
}

// One Jacobi sweep of (rho1/dt) h + C(h) - (mu/Pr) L(h) = b_h (dh/dz = -g on
// the horizontal walls).
__global__ void k_enth_jacobi(StepArgs a, const double *__restrict__ hin, double *__restrict__ hout)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    if (a.sc->status) return;
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    double v[1] = {0.0};
    if (in) {
        const int q = cidx(G, i, k);
        auto gh = [&](int ii, int kk) { return ldc<BC_H>(G, F, hin, ii, kk); };
        const double d = a.jd[q] + F.nuh * (2.0 * G.idx * G.idx + 2.0 * G.idz * G.idz);
        const double hq = hin[q];
        const double r = a.bh[q] - (a.rho1[q] * F.idt * hq + conv_get(G, a.S.phix, a.S.phiz, gh, i, k)
                                    - F.nuh * laplacian<BC_H>(G, F, hin, i, k));
        hout[q] = hq + r / d;
        v[0] = r * r;
    }
    double tot[1];
    if (grid_sum<1>(v, a.partials, &a.sc->counters[CNT_ENTH], tot)) {
        Scal *sc = a.sc;
        sc->sweeps[1] += 1;
        if (!finite2(tot[0])) sc->status = 5;
        else if (tot[0] <= a.jac_rtol2 * sc->bn2[2]) sc->done[LOOP_ENTH] = 1;
    }
}

// T^{n+1} = T^n + (h^{n+1} - h^n)/cp; rho^{n+2/3} = p^n/(R T^{n+1});
// psi = 1/(R T^{n+1}); face coefficients D_f = dt rho2_f / rho1_f and the
// fine-level Helmholtz operator c = psi/dt, a_f = D_f |A_f| / (V Delta_f).
__global__ void k_eos_coef(StepArgs a, Level L)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    if (a.sc->status) return;
    int i, k;
    if (!cell_of_thread(G, i, k)) return;
    const int q = cidx(G, i, k);
    const State &S = a.S;
    auto rho2_at = [&](int qq) {
        const double T1 = S.T[qq] + (a.ha[qq] - S.h[qq]) / F.cp;
        return S.p[qq] / (F.R * T1);
    };
    const double T1 = S.T[q] + (a.ha[q] - S.h[q]) / F.cp;
    const double r2 = S.p[q] / (F.R * T1);
    const double psi = 1.0 / (F.R * T1);
    const double r1 = a.rho1[q];
    a.N.T[q] = T1;
    a.N.h[q] = a.ha[q];
    a.rho2[q] = r2;
    double Dw = 0.0, De = 0.0, Ds = 0.0, Dn = 0.0;
    if (i > 0) Dw = F.dt * (0.5 * (rho2_at(q - 1) + r2)) / (0.5 * (a.rho1[q - 1] + r1));
    if (i + 1 < G.nx) De = F.dt * (0.5 * (r2 + rho2_at(q + 1))) / (0.5 * (r1 + a.rho1[q + 1]));
    if (k > 0) Ds = F.dt * (0.5 * (rho2_at(q - G.P) + r2)) / (0.5 * (a.rho1[q - G.P] + r1));
    if (k + 1 < G.nz) Dn = F.dt * (0.5 * (r2 + rho2_at(q + G.P))) / (0.5 * (r1 + a.rho1[q + G.P]));
    const double ix2 = G.idx * G.idx, iz2 = G.idz * G.idz;
    const double c = psi * F.idt;
    a.Dx[k * G.P + i] = Dw;
    a.Dz[k * G.P + i] = Ds;
    L.ax[k * G.P + i] = Dw * ix2;
    L.az[k * G.P + i] = Ds * iz2;
    if (i == G.nx - 1) { a.Dx[k * G.P + G.nx] = 0.0; L.ax[k * G.P + G.nx] = 0.0; }
    if (k == G.nz - 1) { a.Dz[G.nz * G.P + i] = 0.0; L.az[G.nz * G.P + i] = 0.0; }
    L.c[q] = c;
    L.dinv[q] = 1.0 / (c + (Dw + De) * ix2 + (Ds + Dn) * iz2);
}

// ---------------------------------------------------------------------------
// multigrid hierarchy (Galerkin coarsening with piecewise-constant transfer)
// ---------------------------------------------------------------------------

__global__ void k_mg_coarsen(Level f, Level c)
{
    const Geom &G = c.G;
    int I, K;
    if (!cell_of_thread(G, I, K)) return;
    const int Pf = f.G.P;
    const int q00 = (2 * K) * Pf + 2 * I;
    const int Q = cidx(G, I, K);
    const double cc = 0.25 * (f.c[q00] + f.c[q00 + 1] + f.c[q00 + Pf] + f.c[q00 + Pf + 1]);
    const double aw = 0.25 * (f.ax[q00] + f.ax[q00 + Pf]);
    const double ae = 0.25 * (f.ax[q00 + 2] + f.ax[q00 + Pf + 2]);
    const double as = 0.25 * (f.az[q00] + f.az[q00 + 1]);
    const double an = 0.25 * (f.az[q00 + 2 * Pf] + f.az[q00 + 2 * Pf + 1]);
    c.c[Q] = cc;
    c.ax[K * G.P + I] = aw;
    c.az[K * G.P + I] = as;
    if (I == G.nx - 1) c.ax[K * G.P + G.nx] = ae;
    if (K == G.nz - 1) c.az[G.nz * G.P + I] = an;
    c.dinv[Q] = 1.0 / (cc + aw + ae + as + an);
}

// ---------------------------------------------------------------------------
// Step 3: PISO corrector (eq. step2_sd second line, eq. p_prime_sd, step4_4sd)
// ---------------------------------------------------------------------------

// H(u) = rho^n u^n/dt - C(u) + mu L(u) at the newest velocity.
__global__ void k_H(StepArgs a, const double *__restrict__ U, const double *__restrict__ W)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    if (a.sc->status) return;
    int i, k;
    if (!cell_of_thread(G, i, k)) return;
    const int q = cidx(G, i, k);
    const State &S = a.S;
    auto gu = [&](int ii, int kk) { return ldc<BC_U>(G, F, U, ii, kk); };
    auto gw = [&](int ii, int kk) { return ldc<BC_W>(G, F, W, ii, kk); };
    a.Hx[q] = S.rho[q] * S.u[q] * F.idt - conv_get(G, S.phix, S.phiz, gu, i, k)
              + F.mu * laplacian<BC_U>(G, F, U, i, k);
    a.Hz[q] = S.rho[q] * S.w[q] * F.idt - conv_get(G, S.phix, S.phiz, gw, i, k)
              + F.mu * laplacian<BC_W>(G, F, W, i, k);
}

// (A x)_i = c_i x_i + sum_f a_f (x_i - x_N); wall faces have a_f = 0 and
// their neighbours are not read.
__device__ __forceinline__ double helm_apply(const Level &L, const double *__restrict__ x, int i,
                                             int k)
{
    const Geom &G = L.G;
    const int q = cidx(G, i, k);
    const double xq = x[q];
    double s = L.c[q] * xq;
    if (i > 0) s += L.ax[k * G.P + i] * (xq - x[q - 1]);
    if (i + 1 < G.nx) s += L.ax[k * G.P + i + 1] * (xq - x[q + 1]);
    if (k > 0) s += L.az[k * G.P + i] * (xq - x[q - G.P]);
    if (k + 1 < G.nz) s += L.az[(k + 1) * G.P + i] * (xq - x[q + G.P]);
    return s;
}

// Right-hand side of the pressure equation,
//   b_i = (rho^n_i + psi_i rho2_i g z_i)/dt
//         - (1/V) sum_f D_f |A_f| [H_f . n + g z_f (rho2_N - rho2_i)/Delta_f],
// the initial residual r = b - A x (x = xin, copied to xout) and p = 0.
__global__ void k_helm_rhs(StepArgs a, Level L, const double *__restrict__ xin,
                           double *__restrict__ xout, int corr)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    if (a.sc->status) return;
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    double v[2] = {0.0, 0.0};
    if (in) {
        const int q = cidx(G, i, k);
        const double z = (k + 0.5) * G.dz;
        const double *Hx = a.Hx, *Hz = a.Hz, *r2 = a.rho2;
        const double psi = 1.0 / (F.R * a.N.T[q]);
        double flux = 0.0;
        if (i + 1 < G.nx)
            flux += a.Dx[k * G.P + i + 1] * G.dz *
                    (0.5 * (Hx[q] + Hx[q + 1]) + F.g * z * (r2[q + 1] - r2[q]) * G.idx);
        if (i > 0)
            flux += a.Dx[k * G.P + i] * G.dz *
                    (-0.5 * (Hx[q] + Hx[q - 1]) + F.g * z * (r2[q - 1] - r2[q]) * G.idx);
        if (k + 1 < G.nz)
            flux += a.Dz[(k + 1) * G.P + i] * G.dx *
                    (0.5 * (Hz[q] + Hz[q + G.P]) + F.g * ((k + 1) * G.dz) * (r2[q + G.P] - r2[q]) * G.idz);
        if (k > 0)
            flux += a.Dz[k * G.P + i] * G.dx *
                    (-0.5 * (Hz[q] + Hz[q - G.P]) + F.g * (k * G.dz) * (r2[q - G.P] - r2[q]) * G.idz);
        const double b = (a.S.rho[q] + psi * r2[q] * F.g * z) * F.idt - flux * G.iV;
        const double r = b - helm_apply(L, xin, i, k);
        a.b[q] = b;
        L.r[q] = r;
        xout[q] = xin[q];
        a.p[q] = 0.0;
        v[0] = b * b;
        v[1] = r * r;
    }
    double tot[2];
    if (grid_sum<2>(v, a.partials, &a.sc->counters[CNT_HELM], tot)) {
        Scal *sc = a.sc;
        sc->b2 = tot[0];
        sc->r2 = tot[1];
        sc->cg_it = 0;
        sc->corr = corr;
        sc->trips[LOOP_CG] = 0;
        sc->rz = 0.0;
        const int conv = tot[1] <= a.cg_rtol2 * tot[0];
        sc->done[LOOP_CG] = conv;
        sc->cg_iters[corr] = 0;
        sc->cg_relres[corr] = tot[0] > 0.0 ? sqrt(tot[1] / tot[0]) : 0.0;
        if (!finite2(tot[0]) || !finite2(tot[1])) sc->status = 5;
    }
}

// ---- V-cycle ----

// Restriction step of level l: pre-smooth one damped Jacobi sweep from zero,
// e = omega D^-1 r, and restrict the new residual r - A e by averaging the
// four fine cells of each coarse cell.
__global__ void k_mg_down(Level f, Level c, double omega, Scal *sc)
{
    if (sc->status || sc->done[LOOP_CG]) return;
    int I, K;
    if (!cell_of_thread(c.G, I, K)) return;
    const Geom &G = f.G;
    auto e_at = [&](int q) { return omega * f.dinv[q] * f.r[q]; };
    double acc = 0.0;
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int i = 2 * I + a, k = 2 * K + b;
            const int q = cidx(G, i, k);
            const double eq = e_at(q);
            double s = f.c[q] * eq;
            if (i > 0) s += f.ax[k * G.P + i] * (eq - e_at(q - 1));
            if (i + 1 < G.nx) s += f.ax[k * G.P + i + 1] * (eq - e_at(q + 1));
            if (k > 0) s += f.az[k * G.P + i] * (eq - e_at(q - G.P));
            if (k + 1 < G.nz) s += f.az[(k + 1) * G.P + i] * (eq - e_at(q + G.P));
            f.e[q] = eq;
            acc += f.r[q] - s;
        }
    c.r[cidx(c.G, I, K)] = 0.25 * acc;
}

// Coarsest level: damped Jacobi sweeps from zero (first = true starts from 0).
__global__ void k_mg_coarse_sweep(Level L, const double *__restrict__ ein, double *__restrict__ eout,
                                  int first, double omega, Scal *sc)
{
    if (sc->status || sc->done[LOOP_CG]) return;
    int i, k;
    if (!cell_of_thread(L.G, i, k)) return;
    const int q = cidx(L.G, i, k);
    if (first) {
        eout[q] = omega * L.dinv[q] * L.r[q];
    } else {
        eout[q] = ein[q] + omega * L.dinv[q] * (L.r[q] - helm_apply(L, ein, i, k));
    }
}

// Prolongation step of level l: e' = e + P e_c (piecewise constant), then
// one damped Jacobi post-smoothing sweep e'' = e' + omega D^-1 (r - A e').
// At the finest level the result is z = M^-1 r and the block sums r.z feed
// the CG coefficient beta.
__global__ void k_mg_up(Level f, const double *__restrict__ ec, int Pc, double omega,
                        double *__restrict__ out, int finest, StepArgs a)
{
    Scal *sc = a.sc;
    if (sc->status || sc->done[LOOP_CG]) return;
    const Geom &G = f.G;
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    double v[1] = {0.0};
    if (in) {
        auto ep = [&](int ii, int kk) { return f.e[cidx(G, ii, kk)] + ec[(kk >> 1) * Pc + (ii >> 1)]; };
        const int q = cidx(G, i, k);
        const double eq = ep(i, k);
        double s = f.c[q] * eq;
        if (i > 0) s += f.ax[k * G.P + i] * (eq - ep(i - 1, k));
        if (i + 1 < G.nx) s += f.ax[k * G.P + i + 1] * (eq - ep(i + 1, k));
        if (k > 0) s += f.az[k * G.P + i] * (eq - ep(i, k - 1));
        if (k + 1 < G.nz) s += f.az[(k + 1) * G.P + i] * (eq - ep(i, k + 1));
        const double z = eq + omega * f.dinv[q] * (f.r[q] - s);
        out[q] = z;
        v[0] = f.r[q] * z;
    }
    if (!finest) return;
    double tot[1];
    if (grid_sum<1>(v, a.partials, &sc->counters[CNT_RZ], tot)) {
        sc->beta = (sc->cg_it == 0 || sc->rz == 0.0) ? 0.0 : tot[0] / sc->rz;
        sc->rz = tot[0];
    }
}

// Single-level preconditioner: two damped Jacobi sweeps from zero.
__global__ void k_mg_single(Level f, double omega, double *__restrict__ out, StepArgs a)
{
    Scal *sc = a.sc;
    if (sc->status || sc->done[LOOP_CG]) return;
    const Geom &G = f.G;
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    double v[1] = {0.0};
    if (in) {
        auto e_at = [&](int q) { return omega * f.dinv[q] * f.r[q]; };
        const int q = cidx(G, i, k);
        const double eq = e_at(q);
        double s = f.c[q] * eq;
        if (i > 0) s += f.ax[k * G.P + i] * (eq - e_at(q - 1));
        if (i + 1 < G.nx) s += f.ax[k * G.P + i + 1] * (eq - e_at(q + 1));
        if (k > 0) s += f.az[k * G.P + i] * (eq - e_at(q - G.P));
        if (k + 1 < G.nz) s += f.az[(k + 1) * G.P + i] * (eq - e_at(q + G.P));
        const double z = eq + omega * f.dinv[q] * (f.r[q] - s);
        out[q] = z;
        v[0] = f.r[q] * z;
    }
    double tot[1];
    if (grid_sum<1>(v, a.partials, &sc->counters[CNT_RZ], tot)) {
        sc->beta = (sc->cg_it == 0 || sc->rz == 0.0) ? 0.0 : tot[0] / sc->rz;
        sc->rz = tot[0];
    }
}

// ---- CG vector steps ----

__global__ void k_cg_p(StepArgs a, Level L)
{
    Scal *sc = a.sc;
    if (sc->status || sc->done[LOOP_CG]) return;
    int i, k;
    if (!cell_of_thread(a.G, i, k)) return;
    const int q = cidx(a.G, i, k);
    a.p[q] = L.e2[q] + sc->beta * a.p[q];
}

__global__ void k_cg_spmv(StepArgs a, Level L)
{
    Scal *sc = a.sc;
    if (sc->status || sc->done[LOOP_CG]) return;
    int i, k;
    const bool in = cell_of_thread(a.G, i, k);
    double v[1] = {0.0};
    if (in) {
        const int q = cidx(a.G, i, k);
        const double Ap = helm_apply(L, a.p, i, k);
        a.q[q] = Ap;
        v[0] = a.p[q] * Ap;
    }
    double tot[1];
    if (grid_sum<1>(v, a.partials, &sc->counters[CNT_PQ], tot)) {
        sc->pq = tot[0];
        sc->alpha = tot[0] != 0.0 ? sc->rz / tot[0] : 0.0;
        if (!finite2(tot[0])) sc->status = 5;
    }
}

__global__ void k_cg_update(StepArgs a, Level L, double *__restrict__ x)
{
    Scal *sc = a.sc;
    if (sc->status || sc->done[LOOP_CG]) return;
    int i, k;
    const bool in = cell_of_thread(a.G, i, k);
    double v[1] = {0.0};
    if (in) {
        const int q = cidx(a.G, i, k);
        const double al = sc->alpha;
        x[q] += al * a.p[q];
        const double r = L.r[q] - al * a.q[q];
        L.r[q] = r;
        v[0] = r * r;
    }
    double tot[1];
    if (grid_sum<1>(v, a.partials, &sc->counters[CNT_UPD], tot)) {
        sc->cg_it += 1;
        sc->r2 = tot[0];
        const int c = sc->corr;
        sc->cg_iters[c] = sc->cg_it;
        sc->cg_relres[c] = sc->b2 > 0.0 ? sqrt(tot[0] / sc->b2) : 0.0;
        if (!finite2(tot[0])) sc->status = 5;
        else if (tot[0] <= a.cg_rtol2 * sc->b2) sc->done[LOOP_CG] = 1;
    }
}

// Flux and velocity correction: F_f = D_f (H_f - G_f) with
// G_f = (p'_b - p'_a)/Delta - g z_f (rho2_b - rho2_a)/Delta; u = (dt/rho1)(H - G_cell);
// p = p' - rho2 g z; rho = p / (R T^{n+1}); phi = F |A|; p^{n-1} <- p^n.
__global__ void k_correct(StepArgs a)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    if (a.sc->status) return;
    int i, k;
    if (!cell_of_thread(G, i, k)) return;
    const int q = cidx(G, i, k);
    const State &N = a.N;
    const double *x = N.pp, *r2 = a.rho2, *Hx = a.Hx, *Hz = a.Hz;
    const double z = (k + 0.5) * G.dz;
    const double xq = x[q], rq = r2[q];
    double gxw = 0.0, gxe = 0.0, gzs = 0.0, gzn = 0.0;
    if (i > 0) gxw = (xq - x[q - 1]) * G.idx - F.g * z * (rq - r2[q - 1]) * G.idx;
    if (i + 1 < G.nx) gxe = (x[q + 1] - xq) * G.idx - F.g * z * (r2[q + 1] - rq) * G.idx;
    if (k > 0) gzs = (xq - x[q - G.P]) * G.idz - F.g * (k * G.dz) * (rq - r2[q - G.P]) * G.idz;
    if (k + 1 < G.nz) gzn = (x[q + G.P] - xq) * G.idz - F.g * ((k + 1) * G.dz) * (r2[q + G.P] - rq) * G.idz;
    const double Fw = i > 0 ? a.Dx[k * G.P + i] * (0.5 * (Hx[q - 1] + Hx[q]) - gxw) : 0.0;
    const double Fs = k > 0 ? a.Dz[k * G.P + i] * (0.5 * (Hz[q - G.P] + Hz[q]) - gzs) : 0.0;
    N.phix[k * G.P + i] = Fw * G.dz;
    N.phiz[k * G.P + i] = Fs * G.dx;
    if (i == G.nx - 1) N.phix[k * G.P + G.nx] = 0.0;
    if (k == G.nz - 1) N.phiz[G.nz * G.P + i] = 0.0;
    const double r1 = a.rho1[q];
    N.u[q] = F.dt / r1 * (Hx[q] - 0.5 * (gxw + gxe));
    N.w[q] = F.dt / r1 * (Hz[q] - 0.5 * (gzs + gzn));
    const double pn = xq - rq * F.g * z;
    N.p[q] = pn;
    N.rho[q] = pn / (F.R * N.T[q]);
    N.pold[q] = a.S.p[q];
}

// ---- loop control and step bookkeeping (one thread) ----

__global__ void k_loop_ctl(Scal *sc, cudaGraphConditionalHandle h, int graph, int which,
                           int maxtrips, int body_launches)
{
    const int trips = ++sc->trips[which];
    const int done = sc->done[which];
    sc->launches += body_launches;
    if (!done && !sc->status && trips >= maxtrips) sc->status = 4;
    if (graph) cudaGraphSetConditional(h, (done || sc->status || trips >= maxtrips) ? 0u : 1u);
}

__global__ void k_step_begin(Scal *sc)
{
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
    int i, k;
    const bool in = cell_of_thread(G, i, k);
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
    if (grid_sum<2>(v, partials, &sc->counters[CNT_DIAG], tot)) {
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

// Launch with an optional trace bracket.
#define TRACED(tr, name, cells, launch)                         \
    do {                                                        \
        if (tr) (tr)->begin(name, (long long)(cells), st);      \
        launch;                                                 \
        if (tr) (tr)->end(st);                                  \
    } while (0)

inline long long ncell(const Geom &G) { return (long long)G.nx * G.nz; }

void launch_pred_setup(const StepArgs &a, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "pred_setup", ncell(a.G), (k_pred_setup<<<grid_of(a.G), kBlock, 0, st>>>(a)));
}

void launch_mom_jacobi(const StepArgs &a, const double *uin, const double *win, double *uout,
                       double *wout, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "mom_jacobi", ncell(a.G),
           (k_mom_jacobi<<<grid_of(a.G), kBlock, 0, st>>>(a, uin, win, uout, wout)));
}

void launch_enth_rhs(const StepArgs &a, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "enth_rhs", ncell(a.G), (k_enth_rhs<<<grid_of(a.G), kBlock, 0, st>>>(a)));
}

void launch_enth_jacobi(const StepArgs &a, const double *hin, double *hout, cudaStream_t st,
                        Tracer *tr)
{
    TRACED(tr, "enth_jacobi", ncell(a.G),
           (k_enth_jacobi<<<grid_of(a.G), kBlock, 0, st>>>(a, hin, hout)));
}

void launch_eos_coef(const StepArgs &a, const Level &L0, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "eos_coef", ncell(a.G), (k_eos_coef<<<grid_of(a.G), kBlock, 0, st>>>(a, L0)));
}

void launch_mg_coarsen(const Level &f, const Level &c, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "mg_coarsen", ncell(c.G), (k_mg_coarsen<<<grid_of(c.G), kBlock, 0, st>>>(f, c)));
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

// z = M^-1 r into levels[0].e2 (one V(1,1)-cycle; ncoarse sweeps, an even
// number, on the coarsest level). Returns the number of kernels launched.
int launch_vcycle(const StepArgs &a, Level *L, int nlev, int ncoarse, double omega,
                  cudaStream_t st, Tracer *tr)
{
    if (nlev == 1) {
        TRACED(tr, "mg_single", ncell(L[0].G),
               (k_mg_single<<<grid_of(L[0].G), kBlock, 0, st>>>(L[0], omega, L[0].e2, a)));
        return 1;
    }
    int n = 0;
    for (int l = 0; l + 1 < nlev; ++l, ++n)
        TRACED(tr, "mg_down", ncell(L[l].G),
               (k_mg_down<<<grid_of(L[l + 1].G), kBlock, 0, st>>>(L[l], L[l + 1], omega, a.sc)));
    Level &C = L[nlev - 1];
    // sweep s writes e2 when ncoarse-1-s is even, so the last sweep ends in e2
    for (int s = 0; s < ncoarse; ++s, ++n) {
        double *out = ((ncoarse - 1 - s) % 2 == 0) ? C.e2 : C.e;
        const double *in = (out == C.e2) ? C.e : C.e2;
        TRACED(tr, "mg_coarse", ncell(C.G),
               (k_mg_coarse_sweep<<<grid_of(C.G), kBlock, 0, st>>>(C, in, out, s == 0, omega, a.sc)));
    }
    for (int l = nlev - 2; l >= 0; --l, ++n)
        TRACED(tr, "mg_up", ncell(L[l].G),
               (k_mg_up<<<grid_of(L[l].G), kBlock, 0, st>>>(L[l], L[l + 1].e2, L[l + 1].G.P, omega,
                                                             L[l].e2, l == 0, a)));
    return n;
}

int launch_cg_iter_tail(const StepArgs &a, const Level &L0, double *x, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "cg_p", ncell(a.G), (k_cg_p<<<grid_of(a.G), kBlock, 0, st>>>(a, L0)));
    TRACED(tr, "cg_spmv", ncell(a.G), (k_cg_spmv<<<grid_of(a.G), kBlock, 0, st>>>(a, L0)));
    TRACED(tr, "cg_update", ncell(a.G), (k_cg_update<<<grid_of(a.G), kBlock, 0, st>>>(a, L0, x)));
    return 3;
}

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
