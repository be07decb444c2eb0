// gea_kernels.cu -- CUDA kernels (sm_103a, FP64) of one predictor-corrector
// time step of the GEA pressure-based Euler solver (Girfoglio, Quaini &
// Rozza, arXiv 2303.10499, Section 3), and their host-side launchers.
//
// GB300 executes FP64 at 1/64 of its FP32 rate (two FP64 lanes per SM per
// clock, about 1.2 TFLOP/s), while HBM delivers about 6.8 TB/s: every stencil
// here is FP64-issue-bound, not bandwidth-bound. The kernels are shaped to
// execute as few FP64 instructions as possible and spend loads, integer and
// shared-memory work (separate pipes) instead:
//  - one thread per cell on 32 x 8 blocks; neighbour values come from a
//    shared-memory tile with a halo, wall ghosts filled while loading, so
//    the arithmetic has no boundary branches;
//  - the implicit transport operator of Steps 1-2 is assembled once per step
//    as a 9-point stencil (Stencil9); a Jacobi sweep and the evaluation of
//    H(u) are then 9 FMAs per component;
//  - the Helmholtz operator is kept as d x - sum a x_N with omega/d stored,
//    values needed at neighbours (smoothed corrections, CG directions) are
//    computed once per tile cell;
//  - divisions are done once per step into stored reciprocals.
// Reductions are deterministic: block partials, added in a fixed order by
// the last block to arrive. Kernels inside a device-side loop return early
// (uniformly across the grid) once the loop has converged or failed.
#include "gea_internal.cuh"

#include <math.h>

namespace gea {

namespace {

__device__ __forceinline__ bool finite1(double a) { return isfinite(a); }

__device__ __forceinline__ bool cell_of_thread(const Geom &G, int &i, int &k)
{
    i = blockIdx.x * BX + threadIdx.x;
    k = blockIdx.y * BZ + threadIdx.y;
    return i < G.nx && k < G.nz;
}

template <int H>
using Tile = double[BZ + 2 * H][BX + 2 * H];

// Fill the block's (BZ+2H) x (BX+2H) shared tile of X: cells inside the box,
// the one-layer wall ghosts of rule BC, and zero elsewhere (deeper ghosts and
// corners are only ever multiplied by zero coefficients).
template <int BC, int H>
__device__ __forceinline__ void load_tile(Tile<H> &s, const Geom &G, const Phys &F,
                                          const double *__restrict__ X)
{
    const int i0 = blockIdx.x * BX - H, k0 = blockIdx.y * BZ - H;
    const int tid = threadIdx.x + threadIdx.y * BX;
    constexpr int W = BX + 2 * H, NE = (BZ + 2 * H) * (BX + 2 * H);
    for (int e = tid; e < NE; e += NTHREADS) {
        const int tk = e / W, ti = e - tk * W;
        const int i = i0 + ti, k = k0 + tk;
        const bool xin = i >= 0 && i < G.nx, zin = k >= 0 && k < G.nz;
        double v = 0.0;
        if (xin && zin) v = X[k * G.P + i];
        else if (zin && (i == -1 || i == G.nx)) v = ldc<BC>(G, F, X, i, k);
        else if (xin && (k == -1 || k == G.nz)) v = ldc<BC>(G, F, X, i, k);
        s[tk][ti] = v;
    }
}

// Same for a field given by f(q) at cell index q (no ghosts: zero outside).
template <int H, class Fn>
__device__ __forceinline__ void load_tile_fn(Tile<H> &s, const Geom &G, Fn f)
{
    const int i0 = blockIdx.x * BX - H, k0 = blockIdx.y * BZ - H;
    const int tid = threadIdx.x + threadIdx.y * BX;
    constexpr int W = BX + 2 * H, NE = (BZ + 2 * H) * (BX + 2 * H);
    for (int e = tid; e < NE; e += NTHREADS) {
        const int tk = e / W, ti = e - tk * W;
        const int i = i0 + ti, k = k0 + tk;
        s[tk][ti] = (i >= 0 && i < G.nx && k >= 0 && k < G.nz) ? f(k * G.P + i) : 0.0;
    }
}

// 9-point cross stencil sum sum_o c_o X_o at tile position (y, x).
template <int H>
__device__ __forceinline__ double apply9(const Stencil9 &T, int q, const Tile<H> &s, int y, int x)
{
    double acc = T.cC[q] * s[y][x];
    acc = fma(T.cE1[q], s[y][x + 1], acc);
    acc = fma(T.cW1[q], s[y][x - 1], acc);
    acc = fma(T.cN1[q], s[y + 1][x], acc);
    acc = fma(T.cS1[q], s[y - 1][x], acc);
    acc = fma(T.cE2[q], s[y][x + 2], acc);
    acc = fma(T.cW2[q], s[y][x - 2], acc);
    acc = fma(T.cN2[q], s[y + 2][x], acc);
    acc = fma(T.cS2[q], s[y - 2][x], acc);
    return acc;
}

// 5-point Laplacian sum (X_E + X_W - 2 X_C)/dx^2 + (X_N + X_S - 2 X_C)/dz^2.
template <int H>
__device__ __forceinline__ double lap5(const Geom &G, const Tile<H> &s, int y, int x)
{
    const double c2 = 2.0 * s[y][x];
    return (s[y][x + 1] + s[y][x - 1] - c2) * (G.idx * G.idx) + (s[y + 1][x] + s[y - 1][x] - c2) * (G.idz * G.idz);
}

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

// rho^{n+1/3} = rho^n - dt sum_j phi_j / V; the transport operator
//   T(X) = (rho1/dt) X + C(X) - mu L(X)
// as a 9-point stencil: the east face contributes f_e (-X_W1 + 7 X_C + 7 X_E1
// - X_E2) with f_e = phi_e / (12 V), the west face -f_w (-X_W2 + 7 X_W1 + 7 X_C
// - X_E1), likewise in z, and -mu L adds 2 mu (1/dx^2 + 1/dz^2) at the centre
// and -mu/dx^2, -mu/dz^2 at the nearest neighbours; the Jacobi reciprocals
// of the momentum (mu) and enthalpy (mu/Pr) diagonals; the right-hand sides
// b = rho^n u^n / dt - G_cell^n with G_cell the average of the two face forces
// grad p'^n - g z grad rho^n per direction (zero on wall faces); the initial
// guess u^n.
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
        const double pw = S.phix[q], pe = S.phix[q + 1], ps = S.phiz[q], pn = S.phiz[q + G.P];
        const double div = (pe - pw + pn - ps) * G.iV;
        const double rho1 = S.rho[q] - F.dt * div;
        const double s12 = G.iV * (1.0 / 12.0);
        const double fe = pe * s12, fw = pw * s12, fn = pn * s12, fs = ps * s12;
        const double mx = F.mu * G.idx * G.idx, mz = F.mu * G.idz * G.idz;
        const double cC = rho1 * F.idt + (7.0 / 12.0) * div + 2.0 * (mx + mz);
        a.T.cC[q] = cC;
        a.T.cE1[q] = fma(7.0, fe, fw) - mx;
        a.T.cW1[q] = -fma(7.0, fw, fe) - mx;
        a.T.cE2[q] = -fe;
        a.T.cW2[q] = fw;
        a.T.cN1[q] = fma(7.0, fn, fs) - mz;
        a.T.cS1[q] = -fma(7.0, fs, fn) - mz;
        a.T.cN2[q] = -fn;
        a.T.cS2[q] = fs;
        a.dinvu[q] = 1.0 / cC;
        a.dinvh[q] = 1.0 / (cC + 2.0 * (F.nuh - F.mu) * (G.idx * G.idx + G.idz * G.idz));
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

// One Jacobi sweep of T(X) = b for X = u (odd in x) and X = w (odd in z):
// r = b - T(X), X <- X + r / T_CC.
__global__ void k_mom_jacobi(StepArgs a, const double *__restrict__ uin,
                             const double *__restrict__ win, double *__restrict__ uout,
                             double *__restrict__ wout)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    if (a.sc->status) return;
    __shared__ Tile<2> su, sw;
    load_tile<BC_U, 2>(su, G, F, uin);
    load_tile<BC_W, 2>(sw, G, F, win);
    __syncthreads();
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    double v[2] = {0.0, 0.0};
    if (in) {
        const int q = cidx(G, i, k);
        const int y = threadIdx.y + 2, x = threadIdx.x + 2;
        const double di = a.dinvu[q];
        const double ru = a.bu[q] - apply9<2>(a.T, q, su, y, x);
        const double rw = a.bw[q] - apply9<2>(a.T, q, sw, y, x);
        uout[q] = fma(ru, di, su[y][x]);
        wout[q] = fma(rw, di, sw[y][x]);
        v[0] = ru * ru;
        v[1] = rw * rw;
    }
    double tot[2];
    if (grid_sum<2>(v, a.partials, &a.sc->counters[CNT_MOM], tot)) {
        Scal *sc = a.sc;
        sc->sweeps[0] += 1;
        if (!finite1(tot[0]) || !finite1(tot[1])) {
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
    __shared__ Tile<2> su, sw;
    load_tile<BC_U, 2>(su, G, F, a.ua);
    load_tile<BC_W, 2>(sw, G, F, a.wa);
    __syncthreads();
    // K1 in place of u (ghost velocities give the mirrored cell's K)
    {
        const int tid = threadIdx.x + threadIdx.y * BX;
        for (int e = tid; e < (BZ + 4) * (BX + 4); e += NTHREADS) {
            const int tk = e / (BX + 4), ti = e - tk * (BX + 4);
            su[tk][ti] = 0.5 * (su[tk][ti] * su[tk][ti] + sw[tk][ti] * sw[tk][ti]);
        }
    }
    __syncthreads();
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    double v[1] = {0.0};
    if (in) {
        const int q = cidx(G, i, k);
        const State &S = a.S;
        const int y = threadIdx.y + 2, x = threadIdx.x + 2;
        const Tile<2> &K = su;
        // convective sum of K1 with the four-point face values
        double c = 0.0;
        if (i + 1 < G.nx) c += S.phix[q + 1] * (7.0 * (K[y][x] + K[y][x + 1]) - (K[y][x - 1] + K[y][x + 2]));
        if (i > 0) c -= S.phix[q] * (7.0 * (K[y][x - 1] + K[y][x]) - (K[y][x - 2] + K[y][x + 1]));
        if (k + 1 < G.nz) c += S.phiz[q + G.P] * (7.0 * (K[y][x] + K[y + 1][x]) - (K[y - 1][x] + K[y + 2][x]));
        if (k > 0) c -= S.phiz[q] * (7.0 * (K[y - 1][x] + K[y][x]) - (K[y - 2][x] + K[y + 1][x]));
        c *= G.iV * (1.0 / 12.0);
        const double rq = S.rho[q];
        const double Kn = 0.5 * (S.u[q] * S.u[q] + S.w[q] * S.w[q]);
        const double rho1 = a.rho1[q];
        const double be = (rq * S.h[q] + rq * Kn - S.pold[q]) * F.idt;
        const double bh = be - rho1 * K[y][x] * F.idt - c + S.p[q] * F.idt - rho1 * F.g * sw[y][x];
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
// the horizontal walls): the momentum stencil plus (mu - mu/Pr) L(h).
__global__ void k_enth_jacobi(StepArgs a, const double *__restrict__ hin, double *__restrict__ hout,
                              int pr_differs)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    if (a.sc->status) return;
    __shared__ Tile<2> sh;
    load_tile<BC_H, 2>(sh, G, F, hin);
    __syncthreads();
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    double v[1] = {0.0};
    if (in) {
        const int q = cidx(G, i, k);
        const int y = threadIdx.y + 2, x = threadIdx.x + 2;
        double t = apply9<2>(a.T, q, sh, y, x);
        if (pr_differs) t = fma(F.mu - F.nuh, lap5<2>(G, sh, y, x), t);
        const double r = a.bh[q] - t;
        hout[q] = fma(r, a.dinvh[q], sh[y][x]);
        v[0] = r * r;
    }
    double tot[1];
    if (grid_sum<1>(v, a.partials, &a.sc->counters[CNT_ENTH], tot)) {
        Scal *sc = a.sc;
        sc->sweeps[1] += 1;
        if (!finite1(tot[0])) sc->status = 5;
        else if (tot[0] <= a.jac_rtol2 * sc->bn2[2]) sc->done[LOOP_ENTH] = 1;
    }
}

// T^{n+1} = T^n + (h^{n+1} - h^n)/cp; psi = 1/(R T^{n+1}); rho^{n+2/3} = p^n psi
// (eq. step3_3sd); face coefficients D_f = dt rho2_f / rho1_f (linear face
// averages); the fine Helmholtz operator c = psi/dt, a_f = D_f |A_f|/(V Delta_f),
// d = c + sum a_f and omega/d.
__global__ void k_eos_coef(StepArgs a, Level L)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    if (a.sc->status) return;
    __shared__ Tile<1> s2, s1;
    __shared__ double fx[BZ][BX + 1], fz[BZ + 1][BX];
    const State &S = a.S;
    const double icp = 1.0 / F.cp;
    load_tile_fn<1>(s2, G, [&](int q) {
        const double T1 = fma(a.ha[q] - S.h[q], icp, S.T[q]);
        return S.p[q] / (F.R * T1);
    });
    load_tile_fn<1>(s1, G, [&](int q) { return a.rho1[q]; });
    __syncthreads();
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int y = ty + 1, x = tx + 1;
    const double ix2 = G.idx * G.idx, iz2 = G.idz * G.idz;
    // west faces of the block's columns, plus the east face of the last column
    auto dface = [&](int ya, int xa, int yb, int xb) {
        return F.dt * (0.5 * (s2[ya][xa] + s2[yb][xb])) / (0.5 * (s1[ya][xa] + s1[yb][xb]));
    };
    if (in) {
        fx[ty][tx] = i > 0 ? dface(y, x - 1, y, x) : 0.0;
        fz[ty][tx] = k > 0 ? dface(y - 1, x, y, x) : 0.0;
        if (tx == BX - 1 || i == G.nx - 1) fx[ty][tx + 1] = i + 1 < G.nx ? dface(y, x, y, x + 1) : 0.0;
        if (ty == BZ - 1 || k == G.nz - 1) fz[ty + 1][tx] = k + 1 < G.nz ? dface(y, x, y + 1, x) : 0.0;
    }
    __syncthreads();
    if (!in) return;
    const int q = cidx(G, i, k);
    const double T1 = fma(a.ha[q] - S.h[q], icp, S.T[q]);
    const double psi = 1.0 / (F.R * T1);
    a.N.T[q] = T1;
    a.N.h[q] = a.ha[q];
    a.rho2[q] = s2[y][x];
    a.psi[q] = psi;
    const double Dw = fx[ty][tx], De = fx[ty][tx + 1], Ds = fz[ty][tx], Dn = fz[ty + 1][tx];
    a.Dx[k * G.P + i] = Dw;
    a.Dz[k * G.P + i] = Ds;
    L.ax[k * G.P + i] = Dw * ix2;
    L.az[k * G.P + i] = Ds * iz2;
    if (i == G.nx - 1) { a.Dx[k * G.P + G.nx] = 0.0; L.ax[k * G.P + G.nx] = 0.0; }
    if (k == G.nz - 1) { a.Dz[G.nz * G.P + i] = 0.0; L.az[G.nz * G.P + i] = 0.0; }
    const double c = psi * F.idt;
    const double d = c + (Dw + De) * ix2 + (Ds + Dn) * iz2;
    L.c[q] = c;
    L.d[q] = d;
    L.wd[q] = F.omega / d;
}

// ---------------------------------------------------------------------------
// multigrid hierarchy (Galerkin coarsening with piecewise-constant transfer:
// the coarse reaction term averages the four fine ones, a coarse face
// coefficient is a quarter of the sum of its two fine faces)
// ---------------------------------------------------------------------------

__global__ void k_mg_coarsen(Level f, Level c, double omega)
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
    const double d = cc + aw + ae + as + an;
    c.d[Q] = d;
    c.wd[Q] = omega / d;
}

// ---------------------------------------------------------------------------
// Step 3: PISO corrector (eq. step2_sd second line, eq. p_prime_sd, step4_4sd)
// ---------------------------------------------------------------------------

// H(u) = rho^n u^n/dt - C(u) + mu L(u) = rho^n u^n/dt + (rho1/dt) u - T(u) at the
// newest velocity.
__global__ void k_H(StepArgs a, const double *__restrict__ U, const double *__restrict__ W)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    if (a.sc->status) return;
    __shared__ Tile<2> su, sw;
    load_tile<BC_U, 2>(su, G, F, U);
    load_tile<BC_W, 2>(sw, G, F, W);
    __syncthreads();
    int i, k;
    if (!cell_of_thread(G, i, k)) return;
    const int q = cidx(G, i, k);
    const int y = threadIdx.y + 2, x = threadIdx.x + 2;
    const State &S = a.S;
    const double rdt = S.rho[q] * F.idt, r1dt = a.rho1[q] * F.idt;
    a.Hx[q] = fma(r1dt, su[y][x], fma(rdt, S.u[q], -apply9<2>(a.T, q, su, y, x)));
    a.Hz[q] = fma(r1dt, sw[y][x], fma(rdt, S.w[q], -apply9<2>(a.T, q, sw, y, x)));
}

// Right-hand side of the pressure equation,
//   b_i = (rho^n_i + psi_i rho2_i g z_i)/dt
//         - (1/V) sum_f D_f |A_f| [H_f . n + g z_f (rho2_N - rho2_i)/Delta_f],
// the initial residual r = b - A x (x = xin, copied to xout) and p0 = 0.
__global__ void k_helm_rhs(StepArgs a, Level L, const double *__restrict__ xin,
                           double *__restrict__ xout, int corr)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    if (a.sc->status) return;
    __shared__ Tile<1> sx, s2, shx, shz;
    load_tile_fn<1>(sx, G, [&](int q) { return xin[q]; });
    load_tile_fn<1>(s2, G, [&](int q) { return a.rho2[q]; });
    load_tile_fn<1>(shx, G, [&](int q) { return a.Hx[q]; });
    load_tile_fn<1>(shz, G, [&](int q) { return a.Hz[q]; });
    __syncthreads();
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    double v[2] = {0.0, 0.0};
    if (in) {
        const int q = cidx(G, i, k);
        const int y = threadIdx.y + 1, x = threadIdx.x + 1;
        const double z = (k + 0.5) * G.dz;
        const double r2q = s2[y][x];
        const double Dw = a.Dx[k * G.P + i], De = a.Dx[k * G.P + i + 1];
        const double Ds = a.Dz[k * G.P + i], Dn = a.Dz[(k + 1) * G.P + i];
        // wall faces have D = 0 and zero tile entries beyond the box
        double flux = De * G.dz * (0.5 * (shx[y][x] + shx[y][x + 1]) + F.g * z * (s2[y][x + 1] - r2q) * G.idx);
        flux += Dw * G.dz * (-0.5 * (shx[y][x] + shx[y][x - 1]) + F.g * z * (s2[y][x - 1] - r2q) * G.idx);
        flux += Dn * G.dx * (0.5 * (shz[y][x] + shz[y + 1][x]) + F.g * ((k + 1) * G.dz) * (s2[y + 1][x] - r2q) * G.idz);
        flux += Ds * G.dx * (-0.5 * (shz[y][x] + shz[y - 1][x]) + F.g * (k * G.dz) * (s2[y - 1][x] - r2q) * G.idz);
        const double b = (a.S.rho[q] + a.psi[q] * r2q * F.g * z) * F.idt - flux * G.iV;
        double ax = L.d[q] * sx[y][x];
        ax = fma(-L.ax[k * G.P + i], sx[y][x - 1], ax);
        ax = fma(-L.ax[k * G.P + i + 1], sx[y][x + 1], ax);
        ax = fma(-L.az[k * G.P + i], sx[y - 1][x], ax);
        ax = fma(-L.az[(k + 1) * G.P + i], sx[y + 1][x], ax);
        const double r = b - ax;
        a.b[q] = b;
        L.r[q] = r;
        xout[q] = sx[y][x];
        a.p0[q] = 0.0;
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
        if (!finite1(tot[0]) || !finite1(tot[1])) sc->status = 5;
    }
}

// ---- V-cycle ----

// A x at tile position (y, x) of cell (i, k): d x - sum a x_N (zero tile
// entries and zero wall coefficients beyond the box).
template <int H>
__device__ __forceinline__ double helm_tile(const Level &L, int q, int i, int k, const Tile<H> &s,
                                            int y, int x)
{
    const Geom &G = L.G;
    double t = L.d[q] * s[y][x];
    t = fma(-L.ax[k * G.P + i], s[y][x - 1], t);
    t = fma(-L.ax[k * G.P + i + 1], s[y][x + 1], t);
    t = fma(-L.az[k * G.P + i], s[y - 1][x], t);
    t = fma(-L.az[(k + 1) * G.P + i], s[y + 1][x], t);
    return t;
}

// Restriction step of a level: pre-smooth with one damped Jacobi sweep from
// zero, e = (omega/d) r, and restrict the new residual r - A e (= (1-omega) r +
// sum a e_N) by averaging the four fine cells of each coarse cell.
__global__ void k_mg_down(Level f, Level c, double omega, Scal *sc)
{
    if (sc->status || sc->done[LOOP_CG]) return;
    const Geom &G = f.G;
    __shared__ Tile<1> se;
    __shared__ double sres[BZ][BX];
    load_tile_fn<1>(se, G, [&](int q) { return f.wd[q] * f.r[q]; });
    __syncthreads();
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (in) {
        const int q = cidx(G, i, k);
        const int y = ty + 1, x = tx + 1;
        double t = (1.0 - omega) * f.r[q];
        t = fma(f.ax[k * G.P + i], se[y][x - 1], t);
        t = fma(f.ax[k * G.P + i + 1], se[y][x + 1], t);
        t = fma(f.az[k * G.P + i], se[y - 1][x], t);
        t = fma(f.az[(k + 1) * G.P + i], se[y + 1][x], t);
        f.e[q] = se[y][x];
        sres[ty][tx] = t;
    }
    __syncthreads();
    // one thread per coarse cell (the fine sizes are even, so a coarse cell's
    // four fine cells are all inside the box or all outside)
    if (tx < BX / 2 && ty < BZ / 2) {
        const int I = blockIdx.x * (BX / 2) + tx, K = blockIdx.y * (BZ / 2) + ty;
        if (I < c.G.nx && K < c.G.nz)
            c.r[cidx(c.G, I, K)] = 0.25 * ((sres[2 * ty][2 * tx] + sres[2 * ty][2 * tx + 1]) +
                                           (sres[2 * ty + 1][2 * tx] + sres[2 * ty + 1][2 * tx + 1]));
    }
}

// Coarsest level: damped Jacobi sweeps from zero (first = 1 starts from 0).
__global__ void k_mg_coarse_sweep(Level L, const double *__restrict__ ein, double *__restrict__ eout,
                                  int first, Scal *sc)
{
    if (sc->status || sc->done[LOOP_CG]) return;
    const Geom &G = L.G;
    if (first) {
        int i, k;
        if (!cell_of_thread(G, i, k)) return;
        const int q = cidx(G, i, k);
        eout[q] = L.wd[q] * L.r[q];
        return;
    }
    __shared__ Tile<1> se;
    load_tile_fn<1>(se, G, [&](int q) { return ein[q]; });
    __syncthreads();
    int i, k;
    if (!cell_of_thread(G, i, k)) return;
    const int q = cidx(G, i, k);
    const int y = threadIdx.y + 1, x = threadIdx.x + 1;
    eout[q] = fma(L.wd[q], L.r[q] - helm_tile<1>(L, q, i, k, se, y, x), se[y][x]);
}

// Prolongation step of a level: e' = e + P e_c (piecewise constant), then one
// damped Jacobi post-smoothing sweep e'' = e' + (omega/d)(r - A e'). At the
// finest level the result is z = M^-1 r and the block sums of r.z give the CG
// coefficient beta.
__global__ void k_mg_up(Level f, const double *__restrict__ ec, int Pc, double *__restrict__ out,
                        int finest, StepArgs a)
{
    Scal *sc = a.sc;
    if (sc->status || sc->done[LOOP_CG]) return;
    const Geom &G = f.G;
    __shared__ Tile<1> se;
    {
        const int i0 = blockIdx.x * BX - 1, k0 = blockIdx.y * BZ - 1;
        const int tid = threadIdx.x + threadIdx.y * BX;
        for (int e = tid; e < (BZ + 2) * (BX + 2); e += NTHREADS) {
            const int tk = e / (BX + 2), ti = e - tk * (BX + 2);
            const int ii = i0 + ti, kk = k0 + tk;
            se[tk][ti] = (ii >= 0 && ii < G.nx && kk >= 0 && kk < G.nz)
                             ? f.e[kk * G.P + ii] + ec[(kk >> 1) * Pc + (ii >> 1)]
                             : 0.0;
        }
    }
    __syncthreads();
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    double v[1] = {0.0};
    if (in) {
        const int q = cidx(G, i, k);
        const int y = threadIdx.y + 1, x = threadIdx.x + 1;
        const double rq = f.r[q];
        const double z = fma(f.wd[q], rq - helm_tile<1>(f, q, i, k, se, y, x), se[y][x]);
        out[q] = z;
        v[0] = rq * z;
    }
    if (!finest) return;
    double tot[1];
    if (grid_sum<1>(v, a.partials, &sc->counters[CNT_RZ], tot)) {
        sc->beta = (sc->cg_it == 0 || sc->rz == 0.0) ? 0.0 : tot[0] / sc->rz;
        sc->rz = tot[0];
    }
}

// Single-level preconditioner: two damped Jacobi sweeps from zero,
// z = e + (omega/d)(r - A e) with e = (omega/d) r.
__global__ void k_mg_single(Level f, double *__restrict__ out, StepArgs a)
{
    Scal *sc = a.sc;
    if (sc->status || sc->done[LOOP_CG]) return;
    const Geom &G = f.G;
    __shared__ Tile<1> se;
    load_tile_fn<1>(se, G, [&](int q) { return f.wd[q] * f.r[q]; });
    __syncthreads();
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    double v[1] = {0.0};
    if (in) {
        const int q = cidx(G, i, k);
        const int y = threadIdx.y + 1, x = threadIdx.x + 1;
        const double rq = f.r[q];
        const double z = fma(f.wd[q], rq - helm_tile<1>(f, q, i, k, se, y, x), se[y][x]);
        out[q] = z;
        v[0] = rq * z;
    }
    double tot[1];
    if (grid_sum<1>(v, a.partials, &sc->counters[CNT_RZ], tot)) {
        sc->beta = (sc->cg_it == 0 || sc->rz == 0.0) ? 0.0 : tot[0] / sc->rz;
        sc->rz = tot[0];
    }
}

// ---- CG vector steps ----

// p_new = z + beta p_old (computed once per tile cell) and q = A p_new with
// the block sums of p.q. The directions alternate between p0 and p1 by
// iteration parity: iteration it reads p[it & 1] and writes p[(it + 1) & 1].
__global__ void k_cg_pspmv(StepArgs a, Level L)
{
    Scal *sc = a.sc;
    if (sc->status || sc->done[LOOP_CG]) return;
    const Geom &G = a.G;
    const int it = sc->cg_it;
    const double beta = sc->beta;
    const double *__restrict__ pold = (it & 1) ? a.p1 : a.p0;
    double *__restrict__ pnew = (it & 1) ? a.p0 : a.p1;
    const double *__restrict__ z = L.e2;
    __shared__ Tile<1> sp;
    load_tile_fn<1>(sp, G, [&](int q) { return fma(beta, pold[q], z[q]); });
    __syncthreads();
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    double v[1] = {0.0};
    if (in) {
        const int q = cidx(G, i, k);
        const int y = threadIdx.y + 1, x = threadIdx.x + 1;
        const double pq = sp[y][x];
        const double Ap = helm_tile<1>(L, q, i, k, sp, y, x);
        pnew[q] = pq;
        a.q[q] = Ap;
        v[0] = pq * Ap;
    }
    double tot[1];
    if (grid_sum<1>(v, a.partials, &sc->counters[CNT_PQ], tot)) {
        sc->pq = tot[0];
        sc->alpha = tot[0] != 0.0 ? sc->rz / tot[0] : 0.0;
        if (!finite1(tot[0])) sc->status = 5;
    }
}

__global__ void k_cg_update(StepArgs a, Level L, double *__restrict__ x)
{
    Scal *sc = a.sc;
    if (sc->status || sc->done[LOOP_CG]) return;
    const int it = sc->cg_it;
    const double *__restrict__ p = (it & 1) ? a.p0 : a.p1;
    int i, k;
    const bool in = cell_of_thread(a.G, i, k);
    double v[1] = {0.0};
    if (in) {
        const int q = cidx(a.G, i, k);
        const double al = sc->alpha;
        x[q] = fma(al, p[q], x[q]);
        const double r = fma(-al, a.q[q], L.r[q]);
        L.r[q] = r;
        v[0] = r * r;
    }
    double tot[1];
    if (grid_sum<1>(v, a.partials, &sc->counters[CNT_UPD], tot)) {
        sc->cg_it = it + 1;
        sc->r2 = tot[0];
        const int c = sc->corr;
        sc->cg_iters[c] = it + 1;
        sc->cg_relres[c] = sc->b2 > 0.0 ? sqrt(tot[0] / sc->b2) : 0.0;
        if (!finite1(tot[0])) sc->status = 5;
        else if (tot[0] <= a.cg_rtol2 * sc->b2) sc->done[LOOP_CG] = 1;
    }
}

// Flux and velocity correction: F_f = D_f (H_f - G_f) with
// G_f = (p'_b - p'_a)/Delta - g z_f (rho2_b - rho2_a)/Delta; u = (dt/rho1)(H - G_cell);
// p = p' - rho2 g z; rho = p / (R T^{n+1}) = p psi; phi = F |A|; p^{n-1} <- p^n.
__global__ void k_correct(StepArgs a)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    if (a.sc->status) return;
    __shared__ Tile<1> sx, s2;
    __shared__ double gx[BZ][BX + 1], gz[BZ + 1][BX];
    const State &N = a.N;
    load_tile_fn<1>(sx, G, [&](int q) { return N.pp[q]; });
    load_tile_fn<1>(s2, G, [&](int q) { return a.rho2[q]; });
    __syncthreads();
    int i, k;
    const bool in = cell_of_thread(G, i, k);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int y = ty + 1, x = tx + 1;
    const double z = (k + 0.5) * G.dz;
    auto gxf = [&](int xa) {   // x-face between tile columns xa and xa+1 of row y
        return (sx[y][xa + 1] - sx[y][xa]) * G.idx - F.g * z * (s2[y][xa + 1] - s2[y][xa]) * G.idx;
    };
    auto gzf = [&](int ya, int kf) {   // z-face between tile rows ya and ya+1, face index kf
        return (sx[ya + 1][x] - sx[ya][x]) * G.idz - F.g * (kf * G.dz) * (s2[ya + 1][x] - s2[ya][x]) * G.idz;
    };
    if (in) {
        gx[ty][tx] = i > 0 ? gxf(x - 1) : 0.0;
        gz[ty][tx] = k > 0 ? gzf(y - 1, k) : 0.0;
        if (tx == BX - 1 || i == G.nx - 1) gx[ty][tx + 1] = i + 1 < G.nx ? gxf(x) : 0.0;
        if (ty == BZ - 1 || k == G.nz - 1) gz[ty + 1][tx] = k + 1 < G.nz ? gzf(y, k + 1) : 0.0;
    }
    __syncthreads();
    if (!in) return;
    const int q = cidx(G, i, k);
    const double *Hx = a.Hx, *Hz = a.Hz;
    const double gxw = gx[ty][tx], gxe = gx[ty][tx + 1], gzs = gz[ty][tx], gzn = gz[ty + 1][tx];
    const double Fw = i > 0 ? a.Dx[k * G.P + i] * (0.5 * (Hx[q - 1] + Hx[q]) - gxw) : 0.0;
    const double Fs = k > 0 ? a.Dz[k * G.P + i] * (0.5 * (Hz[q - G.P] + Hz[q]) - gzs) : 0.0;
    N.phix[k * G.P + i] = Fw * G.dz;
    N.phiz[k * G.P + i] = Fs * G.dx;
    if (i == G.nx - 1) N.phix[k * G.P + G.nx] = 0.0;
    if (k == G.nz - 1) N.phiz[G.nz * G.P + i] = 0.0;
    const double dtr1 = F.dt / a.rho1[q];
    N.u[q] = dtr1 * (Hx[q] - 0.5 * (gxw + gxe));
    N.w[q] = dtr1 * (Hz[q] - 0.5 * (gzs + gzn));
    const double pn = fma(-s2[y][x] * F.g, z, sx[y][x]);
    N.p[q] = pn;
    N.rho[q] = pn * a.psi[q];
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
    const int prd = a.F.nuh != a.F.mu;
    TRACED(tr, "enth_jacobi", ncell(a.G),
           (k_enth_jacobi<<<grid_of(a.G), kBlock, 0, st>>>(a, hin, hout, prd)));
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
               (k_mg_single<<<grid_of(L[0].G), kBlock, 0, st>>>(L[0], L[0].e2, a)));
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
               (k_mg_up<<<grid_of(L[l].G), kBlock, 0, st>>>(L[l], L[l + 1].e2, L[l + 1].G.P, L[l].e2,
                                                             l == 0, a)));
    return n;
}

int launch_cg_iter_tail(const StepArgs &a, const Level &L0, double *x, cudaStream_t st, Tracer *tr)
{
    TRACED(tr, "cg_pspmv", ncell(a.G), (k_cg_pspmv<<<grid_of(a.G), kBlock, 0, st>>>(a, L0)));
    TRACED(tr, "cg_update", ncell(a.G), (k_cg_update<<<grid_of(a.G), kBlock, 0, st>>>(a, L0, x)));
    return 2;
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
