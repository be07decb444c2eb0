// gea3d.cu -- the time step of the GEA pressure-based Euler solver
// (Girfoglio, Quaini & Rozza, arXiv 2303.10499, Section 3) on a uniform
// Cartesian x-y-z grid, FP64, and the C ABI of include/gea3d.h.
//
// One thread per cell on 32 x 8 x 1 blocks (grid z = the cell layer);
// neighbour values are read through the read-only cache with the one-layer
// wall ghosts applied on the fly (wall-normal velocity odd, tangential and
// scalars even, h with dh/dz = -g). The transport operator
// T(X) = (rho1/dt) X + C(X) - nu L(X) (fourth-order face values, 13-point
// cross stencil) is evaluated from the face fluxes in every sweep. The
// pressure equation is solved by CG preconditioned with a Galerkin V(1,1)
// cycle (piecewise-constant transfer over 2 x 2 x 2 cells, damped Jacobi
// smoothing), the loops as conditional WHILE nodes of a CUDA graph ended by
// a one-thread control kernel. Reductions are deterministic (block partials
// summed in a fixed order by the last block).
//
// Layout: every array (cells and faces) is indexed (k (ny+1) + j) P + i with
// P = nx + 1 rounded up to 32: x-face i lies between cells i-1 and i,
// y-face j between rows j-1 and j, z-face k between layers k-1 and k.
#include "gea_internal.cuh"
#include "../../include/gea3d.h"

#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <climits>
#include <vector>

namespace g3 {

constexpr int TX = 32, TY = 8, NT = TX * TY;
static_assert(NT == gea::NTHREADS, "block_sum reduces NTHREADS values");
constexpr int kMaxLev = 12;
constexpr int kCoarseSweeps = 2;
constexpr double kOmega = 0.8;
constexpr double kCoarsestRatio = 1.0;
constexpr double kRefT = 300.0;
enum { E3 = 0, U3 = 1, V3 = 2, W3 = 3, H3 = 4 };
enum { L_MOM = 0, L_ENTH = 1, L_CG = 2 };
enum { C_PRED = 0, C_MOM, C_ERHS, C_ENTH, C_HELM, C_RZ, C_PQ, C_UPD, C_DER, C_DIAG };

struct Geo {
    int nx, ny, nz, P;
    double dx, dy, dz;
    double idx, idy, idz, idx2, idy2, idz2, ivol;   // 1/dx, ..., 1/dx^2, ..., 1/(dx dy dz)
    double ax, ay, az;                              // face areas dy dz, dx dz, dx dy
};

__host__ __device__ inline int id3(const Geo &G, int i, int j, int k)
{
    return (k * (G.ny + 1) + j) * G.P + i;
}

struct Phy {
    double R, cp, g, mu, nuh, dt, idt, omega;
    double icp;      // 1/cp
    double les_d2;   // (cs Delta)^2 with Delta = (dx dy dz)^(1/3); 0: constant mu
};

struct St {
    double *rho, *u, *v, *w, *T, *h, *p, *pp, *pold, *phix, *phiy, *phiz;
};

// Helmholtz level: (A x)_i = c_i x_i + sum_f a_f (x_i - x_N), d = c + sum a,
// a on the x-, y- and z-faces (zero on walls).
struct Lev {
    Geo G;
    double *c, *d, *ax, *ay, *az, *r, *e2;   // e2: the preconditioned residual z
};

// FP32 level of the multigrid preconditioner (on the finest level the twin
// of the FP64 operator, r the FP32 copy of the FP64 step's CG residual and
// e2 unused): w = omega/d, e and e2 the smoothed corrections.
struct Lev32 {
    Geo G;
    float *c, *d, *ax, *ay, *az, *w, *r, *e, *e2;
};

// The transport operator T(X) = (rho1/dt) X + C(X) - mu L(X) of the step as
// a 13-point stencil (slot 0 the cell, then x-2, x-1, x+1, x+2, y-2, ...,
// z+2), the fourth-order face interpolation and the Laplacian folded into
// the weights; set once per step from the fluxes phi^n and rho1.
constexpr int NCF = 13;
struct Cf {
    double *c[NCF];
};

struct Sc {
    double bn2[4];
    double b2, r2, rz, pq, alpha, beta;
    int done[3], trips[3], sweeps[2], cg_it, corr, cg_iters[4];
    double cg_relres[4];
    int status, bad_cells;
    long long steps_done;
    int last_sweeps[2], last_cg_iters[4];
    double last_cg_relres[4];
    int last_status;
    long long launches;
    unsigned counters[16];
    double mass, energy;   // diagnostics (k_diag3)
};

struct Args {
    Geo G;
    Phy F;
    St S, N;
    double *rho1, *dinvu, *dinvh, *bu, *bv, *bw, *ua, *va, *wa, *ub, *vb, *wb, *bh, *ha, *hb;
    double *rho2, *psi, *Dx, *Dy, *Dz, *Hx, *Hy, *Hz, *b, *p0, *p1, *q;
    double *dtr1;   // dt / rho1
    double *kin;    // K1 = |u1|^2 / 2
    double *mueff;  // mu + mu_t (LES only)
    const double *gzc, *gzf;   // g z of the cell centres (layer k) and of the horizontal faces (k = 0..nz)
    Cf cf;
    Sc *sc;
    double *part;
    double jtol2, ctol2;
};

__device__ __forceinline__ double ld(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ldf(const float *p) { return __ldg(p); }

// Cell (i,j,k) of the thread, or false beyond the box.
__device__ __forceinline__ bool cell(const Geo &G, int &i, int &j, int &k)
{
    i = blockIdx.x * TX + threadIdx.x;
    j = blockIdx.y * TY + threadIdx.y;
    k = blockIdx.z;
    return i < G.nx && j < G.ny && k < G.nz;
}

// The CG kernels with a reduction (FP64 and FP32) and the finest
// prolongation walk kLayers consecutive cell layers of their column tile
// (one block reduction per kLayers cells a thread): (i, j) of the thread
// and its layer range [k0, k1). The layer loop stays rolled: unrolled, its
// interleaved loads took 56-79 registers a thread and the kernels ran
// 30-40 % slower at the lower occupancy.
constexpr int kLayers = 8;
__device__ __forceinline__ bool column(const Geo &G, int &i, int &j, int &k0, int &k1)
{
    i = blockIdx.x * TX + threadIdx.x;
    j = blockIdx.y * TY + threadIdx.y;
    k0 = blockIdx.z * kLayers;
    k1 = min(G.nz, k0 + kLayers);
    return i < G.nx && j < G.ny;
}

// X at (i,j,k) with at most one index one layer outside the box: the ghost
// of wall rule BC.
template <int BC>
__device__ __forceinline__ double at(const Geo &G, const Phy &F, const double *X, int i, int j, int k)
{
    if (i < 0) { const double v = ld(&X[id3(G, 0, j, k)]); return BC == U3 ? -v : v; }
    if (i >= G.nx) { const double v = ld(&X[id3(G, G.nx - 1, j, k)]); return BC == U3 ? -v : v; }
    if (j < 0) { const double v = ld(&X[id3(G, i, 0, k)]); return BC == V3 ? -v : v; }
    if (j >= G.ny) { const double v = ld(&X[id3(G, i, G.ny - 1, k)]); return BC == V3 ? -v : v; }
    if (k < 0) {
        const double v = ld(&X[id3(G, i, j, 0)]);
        return BC == W3 ? -v : (BC == H3 ? v + F.g * G.dz : v);
    }
    if (k >= G.nz) {
        const double v = ld(&X[id3(G, i, j, G.nz - 1)]);
        return BC == W3 ? -v : (BC == H3 ? v - F.g * G.dz : v);
    }
    return ld(&X[id3(G, i, j, k)]);
}

// X at the neighbour (i+di, j+dj, k+dk) of cell q: a fixed offset from q
// when the whole stencil of the cell lies inside the box (interior), the
// ghost rule otherwise.
template <int BC>
__device__ __forceinline__ double nbr(const Geo &G, const Phy &F, const double *X, int q, bool interior,
                                      int i, int j, int k, int di, int dj, int dk)
{
    if (interior) return ld(X + q + di + dj * G.P + dk * G.P * (G.ny + 1));
    return at<BC>(G, F, X, i + di, j + dj, k + dk);
}

__device__ __forceinline__ double i4(double xm, double xa, double xb, double xp)
{
    return (-xm + 7.0 * xa + 7.0 * xb - xp) * (1.0 / 12.0);
}

// Compact 7-point Laplacian through the ghosts.
template <int BC>
__device__ double lap(const Args &a, const double *X, int i, int j, int k)
{
    const Geo &G = a.G;
    const Phy &F = a.F;
    const double xc = at<BC>(G, F, X, i, j, k);
    return (at<BC>(G, F, X, i + 1, j, k) - xc + at<BC>(G, F, X, i - 1, j, k) - xc) * G.idx2 +
           (at<BC>(G, F, X, i, j + 1, k) - xc + at<BC>(G, F, X, i, j - 1, k) - xc) * G.idy2 +
           (at<BC>(G, F, X, i, j, k + 1) - xc + at<BC>(G, F, X, i, j, k - 1) - xc) * G.idz2;
}

__device__ double divg(const Args &a, int i, int j, int k)
{
    const Geo &G = a.G;
    return (ld(&a.S.phix[id3(G, i + 1, j, k)]) - ld(&a.S.phix[id3(G, i, j, k)]) +
            ld(&a.S.phiy[id3(G, i, j + 1, k)]) - ld(&a.S.phiy[id3(G, i, j, k)]) +
            ld(&a.S.phiz[id3(G, i, j, k + 1)]) - ld(&a.S.phiz[id3(G, i, j, k)])) *
           G.ivol;
}

// Deterministic grid sum of NV values per thread (3D grid of 32 x 8 blocks)
// in two levels: the last block of each group of kGroup blocks adds its
// group's block totals, the last group adds the group totals, each in a fixed
// order. True in thread 0 of the very last block, with the totals in tot.
// part holds kCntSlots doubles of group counters (zero between launches),
// then NV x blocks block totals, then NV x groups group totals. T is the
// type of the per-thread values and of the block sums (FP32 in the inner
// solves of the mixed step); block totals onward are FP64.
constexpr int kGroup = 1024;
constexpr int kCntSlots = 2048;   // 4096 group counters
template <int NV, class T = double>
__device__ bool gsum(const T (&v)[NV], double *red, double *part, unsigned *counter, double (&tot)[NV])
{
    __shared__ int flag;
    const int tid = threadIdx.x + threadIdx.y * TX;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    const int ng = (nb + kGroup - 1) / kGroup, grp = bid / kGroup, g0 = grp * kGroup;
    const int gn = min(kGroup, nb - g0);
    unsigned *gcnt = reinterpret_cast<unsigned *>(part);
    double *p1 = part + kCntSlots, *p2 = p1 + (size_t)NV * nb;
    T bt[NV];
    gea::block_sum<NV, T>(v, reinterpret_cast<T *>(red), bt);
    if (tid == 0) {
#pragma unroll
        for (int m = 0; m < NV; ++m) p1[(size_t)m * nb + bid] = (double)bt[m];
        __threadfence();
        flag = atomicAdd(&gcnt[grp], 1u) == (unsigned)gn - 1u;
    }
    __syncthreads();
    if (!flag) return false;
    __threadfence();
    double s[NV];
#pragma unroll
    for (int m = 0; m < NV; ++m) {
        s[m] = 0.0;
        for (int bb = tid; bb < gn; bb += NT) s[m] += __ldcg(&p1[(size_t)m * nb + g0 + bb]);
    }
    double gt[NV];
    gea::block_sum<NV>(s, red, gt);
    if (tid == 0) {
        gcnt[grp] = 0u;
#pragma unroll
        for (int m = 0; m < NV; ++m) p2[(size_t)m * ng + grp] = gt[m];
        __threadfence();
        flag = atomicAdd(counter, 1u) == (unsigned)ng - 1u;
    }
    __syncthreads();
    if (!flag) return false;
    __threadfence();
#pragma unroll
    for (int m = 0; m < NV; ++m) {
        s[m] = 0.0;
        for (int bb = tid; bb < ng; bb += NT) s[m] += __ldcg(&p2[(size_t)m * ng + bb]);
    }
    gea::block_sum<NV>(s, red, tot);
    if (tid == 0) *counter = 0u;
    return tid == 0;
}

__device__ __forceinline__ bool over(const Sc *sc, int which) { return sc->status || sc->done[which]; }

}  // namespace g3

namespace g3 {

// ---- set-up from conservative fields (dense nz x ny x nx arrays) ----

__global__ void k_derive(Geo G, Phy F, const double *rho, const double *ru, const double *rv,
                         const double *rw, const double *re, St S, Sc *sc)
{
    int i, j, k;
    if (!cell(G, i, j, k)) return;
    const int n = (k * G.ny + j) * G.nx + i, q = id3(G, i, j, k);
    const double z = (k + 0.5) * G.dz, cv = F.cp - F.R;
    const double r = rho[n], u = ru[n] / r, v = rv[n] / r, w = rw[n] / r;
    const double T = (re[n] / r - 0.5 * (u * u + v * v + w * w) - F.g * z) / cv;
    if (!(r > 0.0) || !(T > 0.0)) atomicAdd(&sc->bad_cells, 1);
    S.rho[q] = r; S.u[q] = u; S.v[q] = v; S.w[q] = w; S.T[q] = T; S.h[q] = F.cp * T;
    const double p = r * F.R * T;
    S.p[q] = p; S.pp[q] = p + r * F.g * z; S.pold[q] = p;
    const int sx = 1, sy = G.nx, sz = G.nx * G.ny;
    S.phix[q] = i > 0 ? 0.5 * (ru[n - sx] + ru[n]) * G.dy * G.dz : 0.0;
    S.phiy[q] = j > 0 ? 0.5 * (rv[n - sy] + rv[n]) * G.dx * G.dz : 0.0;
    S.phiz[q] = k > 0 ? 0.5 * (rw[n - sz] + rw[n]) * G.dx * G.dy : 0.0;
    if (i == G.nx - 1) S.phix[id3(G, G.nx, j, k)] = 0.0;
    if (j == G.ny - 1) S.phiy[id3(G, i, G.ny, k)] = 0.0;
    if (k == G.nz - 1) S.phiz[id3(G, i, j, G.nz)] = 0.0;
}

// Face force G_f = (p'_b - p'_a)/Delta - g z_f (rho_b - rho_a)/Delta of the
// face between cell q - s (a) and q (b) in direction d; zero on walls.
__device__ __forceinline__ double fforce(const double *pp, const double *rho, int q, int s,
                                         double inv, double gz)
{
    return fma(-gz, ld(&rho[q]) - ld(&rho[q - s]), ld(&pp[q]) - ld(&pp[q - s])) * inv;
}

// The face forces of cell (i,j,k): its west, south and bottom faces in fl
// (zero on walls) and the cell averages of the two faces per direction in g.
__device__ void cell_forces(const Args &a, const double *pp, const double *rho, int i, int j, int k,
                            double (&fl)[3], double (&g)[3])
{
    const Geo &G = a.G;
    const int q = id3(G, i, j, k), sx = 1, sy = G.P, sz = G.P * (G.ny + 1);
    const double gzc = ld(&a.gzc[k]);
    fl[0] = i > 0 ? fforce(pp, rho, q, sx, G.idx, gzc) : 0.0;
    const double fe = i + 1 < G.nx ? fforce(pp, rho, q + sx, sx, G.idx, gzc) : 0.0;
    fl[1] = j > 0 ? fforce(pp, rho, q, sy, G.idy, gzc) : 0.0;
    const double fn = j + 1 < G.ny ? fforce(pp, rho, q + sy, sy, G.idy, gzc) : 0.0;
    fl[2] = k > 0 ? fforce(pp, rho, q, sz, G.idz, ld(&a.gzf[k])) : 0.0;
    const double ft = k + 1 < G.nz ? fforce(pp, rho, q + sz, sz, G.idz, ld(&a.gzf[k + 1])) : 0.0;
    g[0] = 0.5 * (fl[0] + fe);
    g[1] = 0.5 * (fl[1] + fn);
    g[2] = 0.5 * (fl[2] + ft);
}

__device__ __forceinline__ void fin_pred(Sc *sc, const double (&t)[3])
{
    for (int m = 0; m < 3; ++m) sc->bn2[m] = t[m];
    sc->done[L_MOM] = 0;
    sc->trips[L_MOM] = 0;
    sc->sweeps[0] = 0;
}

// ---- Step 1 (eq. e1_d, eq. step2_sd first line) ----

// Smagorinsky LES: mu_eff = mu + rho^n (cs Delta)^2 |S|, |S| = sqrt(2 S_ij S_ij)
// from central differences of u^n (ghosts by the wall rules).
__global__ void k_les(Args a)
{
    if (a.sc->status) return;
    int i, j, k;
    if (!cell(a.G, i, j, k)) return;
    const Geo &G = a.G;
    const Phy &F = a.F;
    const double hx = 0.5 * G.idx, hy = 0.5 * G.idy, hz = 0.5 * G.idz;
    const double *u = a.S.u, *v = a.S.v, *w = a.S.w;
    const int q = id3(G, i, j, k);
    const bool in = i >= 1 && i + 1 < G.nx && j >= 1 && j + 1 < G.ny && k >= 1 && k + 1 < G.nz;
    auto U = [&](int di, int dj, int dk) { return nbr<U3>(G, F, u, q, in, i, j, k, di, dj, dk); };
    auto V = [&](int di, int dj, int dk) { return nbr<V3>(G, F, v, q, in, i, j, k, di, dj, dk); };
    auto Wv = [&](int di, int dj, int dk) { return nbr<W3>(G, F, w, q, in, i, j, k, di, dj, dk); };
    const double ux = (U(1, 0, 0) - U(-1, 0, 0)) * hx;
    const double uy = (U(0, 1, 0) - U(0, -1, 0)) * hy;
    const double uz = (U(0, 0, 1) - U(0, 0, -1)) * hz;
    const double vx = (V(1, 0, 0) - V(-1, 0, 0)) * hx;
    const double vy = (V(0, 1, 0) - V(0, -1, 0)) * hy;
    const double vz = (V(0, 0, 1) - V(0, 0, -1)) * hz;
    const double wx = (Wv(1, 0, 0) - Wv(-1, 0, 0)) * hx;
    const double wy = (Wv(0, 1, 0) - Wv(0, -1, 0)) * hy;
    const double wz = (Wv(0, 0, 1) - Wv(0, 0, -1)) * hz;
    const double sxy = uy + vx, sxz = uz + wx, syz = vz + wy;
    const double S = sqrt(2.0 * (ux * ux + vy * vy + wz * wz) + sxy * sxy + sxz * sxz + syz * syz);
    a.mueff[q] = F.mu + ld(&a.S.rho[q]) * F.les_d2 * S;
}

// rho1, the Jacobi reciprocals, b = rho^n u^n / dt - G_cell, initial guesses
// u^n; acc += |b|^2 per component.
__global__ void k_pred(Args a)
{
    if (a.sc->status) return;
    __shared__ double red[3 * NT];
    double acc[3] = {0.0, 0.0, 0.0}, tot[3];
    int i, j, k;
    if (cell(a.G, i, j, k)) {
        const Geo &G = a.G;
        const Phy &F = a.F;
        const int q = id3(G, i, j, k), sy = G.P, sz = G.P * (G.ny + 1);
        const double dv = divg(a, i, j, k), r = ld(&a.S.rho[q]);
        const double rho1 = r - F.dt * dv;
        a.rho1[q] = rho1;
        // diffusion weights per face: mu/Delta^2, or with LES the face mean of
        // mu_eff over Delta^2 (a wall face takes the cell's own, the even ghost)
        double mw, me, ms, mn, mb, mt;
        if (F.les_d2 > 0.0) {
            const double mc = ld(&a.mueff[q]);
            // (mu_c + mu_N)/2 / Delta^2, the halves folded into the factors
            const double hx = 0.5 * G.idx2, hy = 0.5 * G.idy2, hz = 0.5 * G.idz2;
            auto face = [&](int ii, int jj, int kk, double h) { return (mc + at<E3>(G, F, a.mueff, ii, jj, kk)) * h; };
            mw = face(i - 1, j, k, hx); me = face(i + 1, j, k, hx);
            ms = face(i, j - 1, k, hy); mn = face(i, j + 1, k, hy);
            mb = face(i, j, k - 1, hz); mt = face(i, j, k + 1, hz);
        } else {
            mw = me = F.mu * G.idx2;
            ms = mn = F.mu * G.idy2;
            mb = mt = F.mu * G.idz2;
        }
        const double cu = rho1 * F.idt + (7.0 / 12.0) * dv + ((mw + me) + (ms + mn) + (mb + mt));
        const double icu = 1.0 / cu;
        a.dinvu[q] = icu;
        // the enthalpy diagonal: the diffusion scaled by 1/Pr (LES requires Pr = 1)
        a.dinvh[q] = F.les_d2 > 0.0 ? icu
                                    : 1.0 / (rho1 * F.idt + (7.0 / 12.0) * dv +
                                             F.nuh * 2.0 * (G.idx2 + G.idy2 + G.idz2));
        // T as a stencil: the outgoing flux of a face times its fourth-order
        // value (-X_m + 7 X_a + 7 X_b - X_p)/12, minus the diffusion
        const double i12 = G.ivol * (1.0 / 12.0);
        const double pw = ld(&a.S.phix[q]), pe = ld(&a.S.phix[q + 1]);
        const double ps = ld(&a.S.phiy[q]), pn = ld(&a.S.phiy[q + sy]);
        const double pb = ld(&a.S.phiz[q]), pt = ld(&a.S.phiz[q + sz]);
        const Cf &cf = a.cf;
        cf.c[0][q] = cu;
        cf.c[1][q] = pw * i12;
        cf.c[2][q] = -(pe + 7.0 * pw) * i12 - mw;
        cf.c[3][q] = (7.0 * pe + pw) * i12 - me;
        cf.c[4][q] = -pe * i12;
        cf.c[5][q] = ps * i12;
        cf.c[6][q] = -(pn + 7.0 * ps) * i12 - ms;
        cf.c[7][q] = (7.0 * pn + ps) * i12 - mn;
        cf.c[8][q] = -pn * i12;
        cf.c[9][q] = pb * i12;
        cf.c[10][q] = -(pt + 7.0 * pb) * i12 - mb;
        cf.c[11][q] = (7.0 * pt + pb) * i12 - mt;
        cf.c[12][q] = -pt * i12;
        double fl[3], gc[3];
        cell_forces(a, a.S.pp, a.S.rho, i, j, k, fl, gc);
        const double gx = gc[0], gy = gc[1], gz = gc[2];
        a.dtr1[q] = F.dt / rho1;
        const double u = ld(&a.S.u[q]), v = ld(&a.S.v[q]), w = ld(&a.S.w[q]);
        const double bu = r * u * F.idt - gx, bv = r * v * F.idt - gy, bw = r * w * F.idt - gz;
        a.bu[q] = bu; a.bv[q] = bv; a.bw[q] = bw;
        a.ua[q] = u; a.va[q] = v; a.wa[q] = w;
        acc[0] = bu * bu; acc[1] = bv * bv; acc[2] = bw * bw;
    }
    if (gsum<3>(acc, red, a.part, &a.sc->counters[C_PRED], tot)) fin_pred(a.sc, tot);
}

// The 13 stencil weights of a cell.
struct W13 {
    double w[NCF];
};

__device__ __forceinline__ W13 weights(const Args &a, int q)
{
    W13 c;
#pragma unroll
    for (int m = 0; m < NCF; ++m) c.w[m] = ld(&a.cf.c[m][q]);
    return c;
}

// Off-centre part of T(X): sum over the 12 neighbour slots of weight times
// value (ghosts by rule BC; slots two cells beyond a wall carry weight 0).
template <int BC>
__device__ __forceinline__ double toff(const Args &a, const W13 &c, const double *X, int i, int j, int k)
{
    const Geo &G = a.G;
    const Phy &F = a.F;
    if (i >= 2 && i + 2 < G.nx && j >= 2 && j + 2 < G.ny && k >= 2 && k + 2 < G.nz) {
        // away from the walls: the neighbours at fixed offsets (same order)
        const int sy = G.P, sz = G.P * (G.ny + 1);
        const double *x = X + id3(G, i, j, k);
        double t = c.w[1] * ld(x - 2);
        t = fma(c.w[2], ld(x - 1), t);
        t = fma(c.w[3], ld(x + 1), t);
        t = fma(c.w[4], ld(x + 2), t);
        t = fma(c.w[5], ld(x - 2 * sy), t);
        t = fma(c.w[6], ld(x - sy), t);
        t = fma(c.w[7], ld(x + sy), t);
        t = fma(c.w[8], ld(x + 2 * sy), t);
        t = fma(c.w[9], ld(x - 2 * sz), t);
        t = fma(c.w[10], ld(x - sz), t);
        t = fma(c.w[11], ld(x + sz), t);
        t = fma(c.w[12], ld(x + 2 * sz), t);
        return t;
    }
    double t = c.w[1] * at<BC>(G, F, X, i - 2, j, k);
    t = fma(c.w[2], at<BC>(G, F, X, i - 1, j, k), t);
    t = fma(c.w[3], at<BC>(G, F, X, i + 1, j, k), t);
    t = fma(c.w[4], at<BC>(G, F, X, i + 2, j, k), t);
    t = fma(c.w[5], at<BC>(G, F, X, i, j - 2, k), t);
    t = fma(c.w[6], at<BC>(G, F, X, i, j - 1, k), t);
    t = fma(c.w[7], at<BC>(G, F, X, i, j + 1, k), t);
    t = fma(c.w[8], at<BC>(G, F, X, i, j + 2, k), t);
    t = fma(c.w[9], at<BC>(G, F, X, i, j, k - 2), t);
    t = fma(c.w[10], at<BC>(G, F, X, i, j, k - 1), t);
    t = fma(c.w[11], at<BC>(G, F, X, i, j, k + 1), t);
    t = fma(c.w[12], at<BC>(G, F, X, i, j, k + 2), t);
    return t;
}

__device__ __forceinline__ void copy_cell(const Geo &G, const double *x, double *y)
{
    int i, j, k;
    if (cell(G, i, j, k)) y[id3(G, i, j, k)] = ld(&x[id3(G, i, j, k)]);
}

// One Jacobi sweep of the three momentum components (pairs of sweeps; the
// second of a pair copies once the first met the tolerance). Five blocks per
// SM (48 registers, no spills) measured 3.5 % faster than four.
__global__ void __launch_bounds__(NT, 5) k_mom(Args a, const double *ui, const double *vi, const double *wi, double *uo, double *vo,
                      double *wo, int second)
{
    Sc *sc = a.sc;
    if (sc->status) return;
    if (second && sc->done[L_MOM]) {
        copy_cell(a.G, ui, uo);
        copy_cell(a.G, vi, vo);
        copy_cell(a.G, wi, wo);
        return;
    }
    __shared__ double red[3 * NT];
    double acc[3] = {0.0, 0.0, 0.0}, tot[3];
    int i, j, k;
    if (cell(a.G, i, j, k)) {
        const int q = id3(a.G, i, j, k);
        const double di = ld(&a.dinvu[q]);
        const W13 c = weights(a, q);
        // one component after the other (the empty asm keeps the compiler
        // from interleaving their loads, which would cost registers)
        const double u0 = ld(&ui[q]);
        const double ru = ld(&a.bu[q]) - fma(c.w[0], u0, toff<U3>(a, c, ui, i, j, k));
        uo[q] = fma(ru, di, u0);
        asm volatile("" ::: "memory");
        const double v0 = ld(&vi[q]);
        const double rv = ld(&a.bv[q]) - fma(c.w[0], v0, toff<V3>(a, c, vi, i, j, k));
        vo[q] = fma(rv, di, v0);
        asm volatile("" ::: "memory");
        const double w0 = ld(&wi[q]);
        const double rw = ld(&a.bw[q]) - fma(c.w[0], w0, toff<W3>(a, c, wi, i, j, k));
        wo[q] = fma(rw, di, w0);
        acc[0] = ru * ru; acc[1] = rv * rv; acc[2] = rw * rw;
    }
    if (gsum<3>(acc, red, a.part, &sc->counters[C_MOM], tot)) {
        sc->sweeps[0] += 1;
        if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) sc->status = GEA_ERR_NONFINITE;
        else if (tot[0] <= a.jtol2 * sc->bn2[0] && tot[1] <= a.jtol2 * sc->bn2[1] && tot[2] <= a.jtol2 * sc->bn2[2])
            sc->done[L_MOM] = 1;
    }
}

// ---- Step 2 (eq. step3_sd) ----

// K1 = |u1|^2/2 per cell (eq. step1_3sd); its wall ghosts are the mirrored
// cells' values (the squares of odd and even ghosts agree).
__global__ void k_kin(Args a, const double *u1, const double *v1, const double *w1)
{
    if (a.sc->status) return;
    int i, j, k;
    if (!cell(a.G, i, j, k)) return;
    const int q = id3(a.G, i, j, k);
    const double u = ld(&u1[q]), v = ld(&v1[q]), w = ld(&w1[q]);
    a.kin[q] = 0.5 * (u * u + v * v + w * w);
}

// Right-hand side of the enthalpy equation and its initial guess h^n:
// (rho h + rho K - p^{n-1})/dt - rho1 K1/dt - C(K1) + p^n/dt - rho1 g w1.
__global__ void k_enth_rhs(Args a, const double *w1)
{
    if (a.sc->status) return;
    __shared__ double red[NT];
    double acc[1] = {0.0}, tot[1];
    int i, j, k;
    if (cell(a.G, i, j, k)) {
        const Geo &G = a.G;
        const Phy &F = a.F;
        const int q = id3(G, i, j, k);
        // C(K1), fourth-order face values of K1 with even ghosts; the 1/12 of
        // the face values is applied once to the sum: 12 X_f = 7 (X_a + X_b) - (X_m + X_p)
        double s = 0.0;
        const double Kc = ld(&a.kin[q]);
        const bool in = i >= 2 && i + 2 < G.nx && j >= 2 && j + 2 < G.ny && k >= 2 && k + 2 < G.nz;
        auto K = [&](int ii, int jj, int kk) {
            return nbr<E3>(G, F, a.kin, q, in, i, j, k, ii - i, jj - j, kk - k);
        };
        auto f12 = [](double xm, double xa, double xb, double xp) { return fma(7.0, xa + xb, -(xm + xp)); };
        if (i + 1 < G.nx) s = fma(ld(&a.S.phix[id3(G, i + 1, j, k)]), f12(K(i - 1, j, k), Kc, K(i + 1, j, k), K(i + 2, j, k)), s);
        if (i > 0) s = fma(-ld(&a.S.phix[q]), f12(K(i - 2, j, k), K(i - 1, j, k), Kc, K(i + 1, j, k)), s);
        if (j + 1 < G.ny) s = fma(ld(&a.S.phiy[id3(G, i, j + 1, k)]), f12(K(i, j - 1, k), Kc, K(i, j + 1, k), K(i, j + 2, k)), s);
        if (j > 0) s = fma(-ld(&a.S.phiy[q]), f12(K(i, j - 2, k), K(i, j - 1, k), Kc, K(i, j + 1, k)), s);
        if (k + 1 < G.nz) s = fma(ld(&a.S.phiz[id3(G, i, j, k + 1)]), f12(K(i, j, k - 1), Kc, K(i, j, k + 1), K(i, j, k + 2)), s);
        if (k > 0) s = fma(-ld(&a.S.phiz[q]), f12(K(i, j, k - 2), K(i, j, k - 1), Kc, K(i, j, k + 1)), s);
        s *= G.ivol * (1.0 / 12.0);
        const double r = ld(&a.S.rho[q]), u = ld(&a.S.u[q]), v = ld(&a.S.v[q]), w = ld(&a.S.w[q]);
        const double h = ld(&a.S.h[q]), rho1 = ld(&a.rho1[q]);
        const double Kn = 0.5 * (u * u + v * v + w * w);
        const double be = (r * h + r * Kn - ld(&a.S.pold[q])) * F.idt;
        const double bh = be - rho1 * Kc * F.idt - s + ld(&a.S.p[q]) * F.idt - rho1 * F.g * ld(&w1[q]);
        a.bh[q] = bh;
        a.ha[q] = h;
        acc[0] = bh * bh;
    }
    if (gsum<1>(acc, red, a.part, &a.sc->counters[C_ERHS], tot)) {
        a.sc->bn2[3] = tot[0];
        a.sc->done[L_ENTH] = 0;
        a.sc->trips[L_ENTH] = 0;
        a.sc->sweeps[1] = 0;
    }
}

// One Jacobi sweep of h (pairs as for momentum); five blocks per SM (48
// registers) measured 8 % faster than four.
__global__ void __launch_bounds__(NT, 5) k_enth(Args a, const double *hi, double *ho, int second)
{
    Sc *sc = a.sc;
    if (sc->status) return;
    if (second && sc->done[L_ENTH]) {
        copy_cell(a.G, hi, ho);
        return;
    }
    __shared__ double red[NT];
    double acc[1] = {0.0}, tot[1];
    int i, j, k;
    if (cell(a.G, i, j, k)) {
        const int q = id3(a.G, i, j, k);
        const W13 c = weights(a, q);
        const double h0 = ld(&hi[q]);
        // T with nu_h = mu/Pr: the mu-stencil plus (mu - nu_h) L(h)
        double t = fma(c.w[0], h0, toff<H3>(a, c, hi, i, j, k));
        if (a.F.nuh != a.F.mu) t = fma(a.F.mu - a.F.nuh, lap<H3>(a, hi, i, j, k), t);
        const double r = ld(&a.bh[q]) - t;
        ho[q] = fma(r, ld(&a.dinvh[q]), h0);
        acc[0] = r * r;
    }
    if (gsum<1>(acc, red, a.part, &sc->counters[C_ENTH], tot)) {
        sc->sweeps[1] += 1;
        if (!isfinite(tot[0])) sc->status = GEA_ERR_NONFINITE;
        else if (tot[0] <= a.jtol2 * sc->bn2[3]) sc->done[L_ENTH] = 1;
    }
}

// EOS update (eqs. step3_2sd, step3_3sd): T^{n+1} = T^n + (h^{n+1} - h^n)/cp,
// psi = 1/(R T^{n+1}), rho2 = psi p^n, and c = psi/dt of the fine level.
__global__ void k_eos(Args a, Lev L, Lev32 m, const double *h1)
{
    if (a.sc->status) return;
    int i, j, k;
    if (!cell(a.G, i, j, k)) return;
    const Phy &F = a.F;
    const int q = id3(a.G, i, j, k);
    const double hq = ld(&h1[q]);
    const double T1 = fma(hq - ld(&a.S.h[q]), F.icp, ld(&a.S.T[q]));
    const double psi = 1.0 / (F.R * T1);
    a.N.T[q] = T1;
    a.N.h[q] = hq;
    a.rho2[q] = ld(&a.S.p[q]) * psi;
    a.psi[q] = psi;
    const double c = psi * F.idt;
    L.c[q] = c;
    m.c[q] = (float)c;
}

// Face coefficients of the fine level: D_f = dt rho2_f / rho1_f with face
// means of the two cells, on the cell's west, south and bottom faces (zero
// on walls; the last cells also zero the east, north and top wall faces),
// and a_f = D_f / Delta^2.
__global__ void k_faces(Args a, Lev L, Lev32 m)
{
    if (a.sc->status) return;
    int i, j, k;
    if (!cell(a.G, i, j, k)) return;
    const Geo &G = a.G;
    const int q = id3(G, i, j, k), sx = 1, sy = G.P, sz = G.P * (G.ny + 1);
    const double r2 = ld(&a.rho2[q]), r1 = ld(&a.rho1[q]), dt = a.F.dt;
    // the halves of the two face means cancel exactly
    auto D = [&](int qn) { return dt * (r2 + ld(&a.rho2[qn])) / (r1 + ld(&a.rho1[qn])); };
    const double Dw = i > 0 ? D(q - sx) : 0.0;
    const double Ds = j > 0 ? D(q - sy) : 0.0;
    const double Db = k > 0 ? D(q - sz) : 0.0;
    a.Dx[q] = Dw; a.Dy[q] = Ds; a.Dz[q] = Db;
    const double ax = Dw * G.idx2, ay = Ds * G.idy2, az = Db * G.idz2;
    L.ax[q] = ax; L.ay[q] = ay; L.az[q] = az;
    m.ax[q] = (float)ax; m.ay[q] = (float)ay; m.az[q] = (float)az;
    if (i == G.nx - 1) { a.Dx[q + sx] = 0.0; L.ax[q + sx] = 0.0; m.ax[q + sx] = 0.0f; }
    if (j == G.ny - 1) { a.Dy[q + sy] = 0.0; L.ay[q + sy] = 0.0; m.ay[q + sy] = 0.0f; }
    if (k == G.nz - 1) { a.Dz[q + sz] = 0.0; L.az[q + sz] = 0.0; m.az[q + sz] = 0.0f; }
}

// Diagonal d = c + the six face coefficients, and the Jacobi weight omega/d.
__global__ void k_diag(Lev L, Lev32 m, Sc *sc)
{
    if (sc->status) return;
    int i, j, k;
    if (!cell(L.G, i, j, k)) return;
    const Geo &G = L.G;
    const int q = id3(G, i, j, k), sy = G.P, sz = G.P * (G.ny + 1);
    const double d = ld(&L.c[q]) + (ld(&L.ax[q]) + ld(&L.ax[q + 1])) + (ld(&L.ay[q]) + ld(&L.ay[q + sy])) +
                     (ld(&L.az[q]) + ld(&L.az[q + sz]));
    L.d[q] = d;
    m.d[q] = (float)d;
    m.w[q] = (float)kOmega / (float)d;   // FP32 smoother weight: an FP32 division
}

}  // namespace g3

namespace g3 {

// ---- Step 3 (eq. step2_sd second line, eq. p_prime_sd, eq. step4_4sd) ----

// H(u) = rho^n u^n / dt - C(u) + mu L(u) at the newest velocity
__global__ void k_H(Args a, const double *U, const double *V, const double *W)
{
    if (a.sc->status) return;
    int i, j, k;
    if (!cell(a.G, i, j, k)) return;
    const int q = id3(a.G, i, j, k);
    const double r = ld(&a.S.rho[q]) * a.F.idt;
    // C(X) - mu L(X) = T(X) - (rho1/dt) X
    const W13 c = weights(a, q);
    const double c0 = c.w[0] - ld(&a.rho1[q]) * a.F.idt;
    a.Hx[q] = r * ld(&a.S.u[q]) - fma(c0, ld(&U[q]), toff<U3>(a, c, U, i, j, k));
    a.Hy[q] = r * ld(&a.S.v[q]) - fma(c0, ld(&V[q]), toff<V3>(a, c, V, i, j, k));
    a.Hz[q] = r * ld(&a.S.w[q]) - fma(c0, ld(&W[q]), toff<W3>(a, c, W, i, j, k));
}

// A x at cell (i,j,k) of level L for x given cellwise by xf(q, i, j, k) (interior
// neighbours only; wall faces have zero coefficients).
template <class XF>
__device__ __forceinline__ double helm(const Lev &L, XF xf, int i, int j, int k)
{
    const Geo &G = L.G;
    const int q = id3(G, i, j, k), sy = G.P, sz = G.P * (G.ny + 1);
    double t = ld(&L.d[q]) * xf(q, i, j, k);
    if (i > 0) t -= ld(&L.ax[q]) * xf(q - 1, i - 1, j, k);
    if (i + 1 < G.nx) t -= ld(&L.ax[q + 1]) * xf(q + 1, i + 1, j, k);
    if (j > 0) t -= ld(&L.ay[q]) * xf(q - sy, i, j - 1, k);
    if (j + 1 < G.ny) t -= ld(&L.ay[q + sy]) * xf(q + sy, i, j + 1, k);
    if (k > 0) t -= ld(&L.az[q]) * xf(q - sz, i, j, k - 1);
    if (k + 1 < G.nz) t -= ld(&L.az[q + sz]) * xf(q + sz, i, j, k + 1);
    return t;
}

__device__ __forceinline__ void fin_helm(Sc *sc, const double (&t)[2], double tol2, int corr)
{
    sc->b2 = t[0];
    sc->r2 = t[1];
    sc->cg_it = 0;
    sc->corr = corr;
    sc->trips[L_CG] = 0;
    sc->rz = 0.0;
    sc->beta = 0.0;
    sc->done[L_CG] = t[1] <= tol2 * t[0];
    sc->cg_iters[corr] = 0;
    sc->cg_relres[corr] = t[0] > 0.0 ? sqrt(t[1] / t[0]) : 0.0;
    if (!isfinite(t[0]) || !isfinite(t[1])) sc->status = GEA_ERR_NONFINITE;
}

// Mixed step: the inner FP32 solve's tolerance is relative to the initial
// residual r0 = b - A p'_prev (kept in b2); nothing to solve if r0 is already
// at the FP64 tolerance relative to b.
__device__ __forceinline__ void fin_helm_mixed(Sc *sc, const double (&t)[2], double tol2, int corr)
{
    sc->b2 = t[1];
    sc->r2 = t[1];
    sc->cg_it = 0;
    sc->corr = corr;
    sc->trips[L_CG] = 0;
    sc->rz = 0.0;
    sc->beta = 0.0;
    sc->done[L_CG] = t[1] <= tol2 * t[0];
    sc->cg_iters[corr] = 0;
    sc->cg_relres[corr] = 1.0;
    if (!isfinite(t[0]) || !isfinite(t[1])) sc->status = GEA_ERR_NONFINITE;
}

// b_i = (rho^n_i + psi_i rho2_i g z_i)/dt - sum_f D_f/Delta_f [H_f . n + g z_f (rho2_N - rho2_i)/Delta_f],
// r = b - A x with x = xin (copied to xout), p0 = 0; acc += (b^2, r^2).
// Mixed step (mr given): r0 rounded to FP32 into mr, and a zero FP32
// increment mx and first direction mp0.
__global__ void k_helm_rhs(Args a, Lev L, const double *xin, double *xout, int corr, float *mr = nullptr,
                           float *mx = nullptr, float *mp0 = nullptr, float *rf = nullptr)
{
    if (a.sc->status) return;
    __shared__ double red[2 * NT];
    double acc[2] = {0.0, 0.0}, tot[2];
    int i, j, k;
    if (cell(a.G, i, j, k)) {
        const Geo &G = a.G;
        const Phy &F = a.F;
        const int q = id3(G, i, j, k), sx = 1, sy = G.P, sz = G.P * (G.ny + 1);
        const double gc = ld(&a.gzc[k]), r2 = ld(&a.rho2[q]);
        // a face's D_f/Delta (s (H_c + H_N)/2 + g z_f (rho2_N - rho2_c)/Delta):
        // hs = s/2 with s the sign of the outward normal, gzi = g z_f/Delta
        auto face = [&](const double *D, const double *H, int fq, int nq, double hs, double gzi,
                        double idl) {
            return ld(&D[fq]) * idl * fma(gzi, ld(&a.rho2[nq]) - r2, hs * (ld(&H[q]) + ld(&H[nq])));
        };
        const double gx = gc * G.idx, gy = gc * G.idy;
        double fl = 0.0;
        if (i + 1 < G.nx) fl += face(a.Dx, a.Hx, q + sx, q + sx, 0.5, gx, G.idx);
        if (i > 0) fl += face(a.Dx, a.Hx, q, q - sx, -0.5, gx, G.idx);
        if (j + 1 < G.ny) fl += face(a.Dy, a.Hy, q + sy, q + sy, 0.5, gy, G.idy);
        if (j > 0) fl += face(a.Dy, a.Hy, q, q - sy, -0.5, gy, G.idy);
        if (k + 1 < G.nz) fl += face(a.Dz, a.Hz, q + sz, q + sz, 0.5, ld(&a.gzf[k + 1]) * G.idz, G.idz);
        if (k > 0) fl += face(a.Dz, a.Hz, q, q - sz, -0.5, ld(&a.gzf[k]) * G.idz, G.idz);
        const double b = fma(ld(&a.psi[q]) * r2, gc, ld(&a.S.rho[q])) * F.idt - fl;
        const double r = b - helm(L, [&](int qq, int, int, int) { return ld(&xin[qq]); }, i, j, k);
        a.b[q] = b;
        L.r[q] = r;
        xout[q] = ld(&xin[q]);
        a.p0[q] = 0.0;
        if (mr) {
            mr[q] = (float)r;
            mx[q] = 0.0f;
            mp0[q] = 0.0f;
        }
        if (rf) rf[q] = (float)r;
        acc[0] = b * b;
        acc[1] = r * r;
    }
    if (gsum<2>(acc, red, a.part, &a.sc->counters[C_HELM], tot)) {
        if (mr) fin_helm_mixed(a.sc, tot, a.ctol2, corr);
        else fin_helm(a.sc, tot, a.ctol2, corr);
    }
}

// ---- multigrid V(1,1) cycle in FP32 (the preconditioner of the FP64 CG) ----
//
// The preconditioner only shapes the search directions: the CG residual and
// its stopping test stay FP64, so the converged pressure is that of the FP64
// system. Every level's operator, weights and vectors are FP32 twins (Lev32);
// the finest level reads the FP64 residual and writes z in FP64.

template <class XF>
__device__ __forceinline__ float helm32(const Lev32 &L, XF xf, int i, int j, int k)
{
    const Geo &G = L.G;
    const int q = id3(G, i, j, k), sy = G.P, sz = G.P * (G.ny + 1);
    float t = ldf(&L.d[q]) * xf(q, i, j, k);
    if (i > 0) t -= ldf(&L.ax[q]) * xf(q - 1, i - 1, j, k);
    if (i + 1 < G.nx) t -= ldf(&L.ax[q + 1]) * xf(q + 1, i + 1, j, k);
    if (j > 0) t -= ldf(&L.ay[q]) * xf(q - sy, i, j - 1, k);
    if (j + 1 < G.ny) t -= ldf(&L.ay[q + sy]) * xf(q + sy, i, j + 1, k);
    if (k > 0) t -= ldf(&L.az[q]) * xf(q - sz, i, j, k - 1);
    if (k + 1 < G.nz) t -= ldf(&L.az[q + sz]) * xf(q + sz, i, j, k + 1);
    return t;
}

__device__ __forceinline__ float tof(double v) { return (float)v; }
__device__ __forceinline__ float tof(float v) { return v; }

// Galerkin coarsening (restriction = mean over the 8 children, piecewise-
// constant prolongation): c_C = mean of the children's c, a coarse face =
// (1/8) sum of its 4 fine faces, d_C = c_C + sum of its faces. One thread
// per coarse cell; sums in FP64, stored FP32.
__global__ void k_coarsen(Lev32 f, Lev32 c)
{
    int I, J, K;
    if (!cell(c.G, I, J, K)) return;
    const Geo &G = f.G, &H = c.G;
    const int Q = id3(H, I, J, K);
    double cs = 0.0, fx0 = 0.0, fx1 = 0.0, fy0 = 0.0, fy1 = 0.0, fz0 = 0.0, fz1 = 0.0;
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
                const int q = id3(G, i, j, k);
                cs += ldf(&f.c[q]);
                if (di == 0) fx0 += ldf(&f.ax[q]); else fx1 += ldf(&f.ax[q + 1]);
                if (dj == 0) fy0 += ldf(&f.ay[q]); else fy1 += ldf(&f.ay[q + G.P]);
                if (dk == 0) fz0 += ldf(&f.az[q]); else fz1 += ldf(&f.az[q + G.P * (G.ny + 1)]);
            }
    const double cc = 0.125 * cs;
    c.c[Q] = (float)cc;
    c.ax[Q] = (float)(0.125 * fx0); c.ay[Q] = (float)(0.125 * fy0); c.az[Q] = (float)(0.125 * fz0);
    if (I == H.nx - 1) c.ax[Q + 1] = (float)(0.125 * fx1);
    if (J == H.ny - 1) c.ay[Q + H.P] = (float)(0.125 * fy1);
    if (K == H.nz - 1) c.az[Q + H.P * (H.ny + 1)] = (float)(0.125 * fz1);
    const double d = cc + 0.125 * (fx0 + fx1 + fy0 + fy1 + fz0 + fz1);
    c.d[Q] = (float)d;
    c.w[Q] = (float)(kOmega / d);
}

// Pre-smoothing from zero, e = (omega/d) r, and restriction of r - A e to
// the coarse level (mean of the 8 children). One thread per coarse cell.
template <class RT>
__global__ void k_mg_down(Lev32 f, const RT *r, Lev32 c, Sc *sc)
{
    if (over(sc, L_CG)) return;
    int I, J, K;
    if (!cell(c.G, I, J, K)) return;
    const Geo &G = f.G;
    auto e = [&](int q, int, int, int) { return ldf(&f.w[q]) * tof(__ldg(&r[q])); };
    float s = 0.0f;
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
                const int q = id3(G, i, j, k);
                f.e[q] = e(q, i, j, k);
                s += tof(__ldg(&r[q])) - helm32(f, e, i, j, k);
            }
    c.r[id3(c.G, I, J, K)] = 0.125f * s;
}

// Coarsest level: damped Jacobi sweep (first: from zero).
__global__ void k_mg_coarse(Lev32 L, const float *ein, float *eout, int first, Sc *sc)
{
    if (over(sc, L_CG)) return;
    int i, j, k;
    if (!cell(L.G, i, j, k)) return;
    const int q = id3(L.G, i, j, k);
    const float w = ldf(&L.w[q]);
    if (first) {
        eout[q] = w * ldf(&L.r[q]);
        return;
    }
    eout[q] = ldf(&ein[q]) + w * (ldf(&L.r[q]) - helm32(L, [&](int qq, int, int, int) { return ldf(&ein[qq]); }, i, j, k));
}

__device__ __forceinline__ void fin_rz(Sc *sc, double t)
{
    sc->beta = (sc->cg_it == 0 || sc->rz == 0.0) ? 0.0 : t / sc->rz;
    sc->rz = t;
}

// z = e + w (r - A e) at cell (i,j,k) of level f, with e the cell's own
// smoothed correction plus its coarse parent's (prolongation and one
// damped-Jacobi post-smoothing sweep); the residual value in rq.
template <class RT>
__device__ __forceinline__ float mg_up_cell(const Lev32 &f, const RT *r, const float *ec, const Geo &cg, int i,
                                            int j, int k, RT &rq)
{
    const Geo &G = f.G;
    const int q = id3(G, i, j, k);
    // coarse parent of the cell, and of a neighbour one cell away: the
    // same parent or the adjacent one, by the parity of the cell's index
    const int Q = id3(cg, i >> 1, j >> 1, k >> 1), cy = cg.P, cz = cg.P * (cg.ny + 1);
    auto step = [](int d, int idx, int s) -> int {
        return d > 0 ? ((idx & 1) ? s : 0) : d < 0 ? ((idx & 1) ? 0 : -s) : 0;
    };
    auto ef = [&](int qq, int ii, int jj, int kk) {
        const int Qn = Q + step(ii - i, i, 1) + step(jj - j, j, cy) + step(kk - k, k, cz);
        return ldf(&f.e[qq]) + ldf(&ec[Qn]);
    };
    rq = __ldg(&r[q]);
    return ef(q, i, j, k) + ldf(&f.w[q]) * (tof(rq) - helm32(f, ef, i, j, k));
}

// Intermediate levels: one thread per cell, no reduction.
template <class RT, class OT>
__global__ void k_mg_up(Lev32 f, const RT *r, const float *ec, Geo cg, OT *out, Sc *sc)
{
    if (over(sc, L_CG)) return;
    int i, j, k;
    if (!cell(f.G, i, j, k)) return;
    RT rq;
    out[id3(f.G, i, j, k)] = (OT)mg_up_cell(f, r, ec, cg, i, j, k, rq);
}

// Finest level: column tiles of kLayers cells a thread (one block reduction
// per column), with the r.z reduction of CG in OT (FP64 for the FP64 CG,
// FP32 for the mixed step's).
template <class RT, class OT>
__global__ void k_mg_up_fin(Lev32 f, const RT *r, const float *ec, Geo cg, OT *out, Sc *sc, double *part)
{
    if (over(sc, L_CG)) return;
    __shared__ double red[NT];
    OT acc[1] = {(OT)0};
    double tot[1];
    int i, j, k0, k1;
    if (column(f.G, i, j, k0, k1))
#pragma unroll 1
        for (int k = k0; k < k1; ++k) {
            RT rq;
            const float z = mg_up_cell(f, r, ec, cg, i, j, k, rq);
            out[id3(f.G, i, j, k)] = (OT)z;
            acc[0] = fma((OT)rq, (OT)z, acc[0]);
        }
    if (gsum<1, OT>(acc, red, part, &sc->counters[C_RZ], tot)) fin_rz(sc, tot[0]);
}

// One level only: z = e + (omega/d)(r - A e), e = (omega/d) r; acc += r.z
// (T = double: the FP64 CG; T = float: the mixed step's FP32 CG).
template <class T>
__global__ void k_mg_single(Lev32 f, const T *r, T *out, Sc *sc, double *part)
{
    if (over(sc, L_CG)) return;
    __shared__ double red[NT];
    T acc[1] = {(T)0};
    double tot[1];
    int i, j, k;
    if (cell(f.G, i, j, k)) {
        const int q = id3(f.G, i, j, k);
        auto e = [&](int qq, int, int, int) { return ldf(&f.w[qq]) * (float)__ldg(&r[qq]); };
        const T rq = __ldg(&r[q]);
        const float z = e(q, i, j, k) + ldf(&f.w[q]) * ((float)rq - helm32(f, e, i, j, k));
        out[q] = (T)z;
        acc[0] = rq * (T)z;
    }
    if (gsum<1, T>(acc, red, part, &sc->counters[C_RZ], tot)) fin_rz(sc, tot[0]);
}

// ---- CG steps (directions alternate between p0 and p1 by parity) ----

// p = z + beta p_old (the new direction into the other buffer)
__global__ void k_pupd(Args a, Lev L)
{
    Sc *sc = a.sc;
    if (over(sc, L_CG)) return;
    int i, j, k;
    if (!cell(L.G, i, j, k)) return;
    const int it = sc->cg_it;
    const double *pold = (it & 1) ? a.p1 : a.p0;
    double *pnew = (it & 1) ? a.p0 : a.p1;
    const int q = id3(L.G, i, j, k);
    pnew[q] = fma(sc->beta, ld(&pold[q]), ld(&L.e2[q]));
}

// q = A p, acc += p.q; alpha = rz / p.q
__global__ void k_spmv(Args a, Lev L)
{
    Sc *sc = a.sc;
    if (over(sc, L_CG)) return;
    __shared__ double red[NT];
    double acc[1] = {0.0}, tot[1];
    const double *p = (sc->cg_it & 1) ? a.p0 : a.p1;
    int i, j, k0, k1;
    if (column(L.G, i, j, k0, k1))
#pragma unroll 1
        for (int k = k0; k < k1; ++k) {
            const int q = id3(L.G, i, j, k);
            const double pq = ld(&p[q]);
            const double Ap = helm(L, [&](int qq, int, int, int) { return ld(&p[qq]); }, i, j, k);
            a.q[q] = Ap;
            acc[0] = fma(pq, Ap, acc[0]);
        }
    if (gsum<1>(acc, red, a.part, &sc->counters[C_PQ], tot)) {
        sc->pq = tot[0];
        sc->alpha = tot[0] != 0.0 ? sc->rz / tot[0] : 0.0;
        if (!isfinite(tot[0])) sc->status = GEA_ERR_NONFINITE;
    }
}

// x += alpha p, r -= alpha q (in place, each cell its own) with an FP32 copy
// of r for the multigrid restriction; acc += r^2.
__global__ void k_update(Args a, Lev L, double *x, float *rf, int maxit)
{
    Sc *sc = a.sc;
    if (over(sc, L_CG)) return;
    __shared__ double red[NT];
    double acc[1] = {0.0}, tot[1];
    const int it = sc->cg_it;
    const double *p = (it & 1) ? a.p0 : a.p1;
    const double alpha = sc->alpha;
    int i, j, k0, k1;
    if (column(L.G, i, j, k0, k1))
#pragma unroll 1
        for (int k = k0; k < k1; ++k) {
            const int q = id3(L.G, i, j, k);
            x[q] = fma(alpha, ld(&p[q]), x[q]);
            const double rn = fma(-alpha, ld(&a.q[q]), L.r[q]);
            L.r[q] = rn;
            rf[q] = (float)rn;
            acc[0] = fma(rn, rn, acc[0]);
        }
    if (gsum<1>(acc, red, a.part, &sc->counters[C_UPD], tot)) {
        const int n = sc->cg_it + 1;
        sc->cg_it = n;
        sc->r2 = tot[0];
        sc->cg_iters[sc->corr] = n;
        sc->cg_relres[sc->corr] = sc->b2 > 0.0 ? sqrt(tot[0] / sc->b2) : 0.0;
        if (!isfinite(tot[0])) sc->status = GEA_ERR_NONFINITE;
        else if (tot[0] <= a.ctol2 * sc->b2) sc->done[L_CG] = 1;
    }
}

// Correction: face forces from the new p' and rho2, F_f = D_f (H_f - G_f),
// u = (dt/rho1)(H - G_cell), p = p' - rho2 g z, rho = p psi, phi = F |A|,
// p^{n-1} <- p^n. Each cell writes its west, south and bottom faces (and the
// walls beyond its east, north and top faces).
__global__ void k_correct(Args a)
{
    if (a.sc->status) return;
    int i, j, k;
    if (!cell(a.G, i, j, k)) return;
    const Geo &G = a.G;
    const int q = id3(G, i, j, k), sx = 1, sy = G.P, sz = G.P * (G.ny + 1);
    double fl[3], gc[3];
    cell_forces(a, a.N.pp, a.rho2, i, j, k, fl, gc);
    const double c1 = ld(&a.dtr1[q]);
    const double hx = ld(&a.Hx[q]), hy = ld(&a.Hy[q]), hz = ld(&a.Hz[q]);
    a.N.u[q] = c1 * (hx - gc[0]);
    a.N.v[q] = c1 * (hy - gc[1]);
    a.N.w[q] = c1 * (hz - gc[2]);
    const double pn = fma(-ld(&a.rho2[q]), ld(&a.gzc[k]), ld(&a.N.pp[q]));
    a.N.p[q] = pn;
    a.N.rho[q] = pn * ld(&a.psi[q]);
    a.N.pold[q] = ld(&a.S.p[q]);
    // F_f = D_f (H_f - G_f) |A_f| on the west, south and bottom faces
    a.N.phix[q] = i > 0 ? ld(&a.Dx[q]) * fma(0.5, hx + ld(&a.Hx[q - sx]), -fl[0]) * G.ax : 0.0;
    a.N.phiy[q] = j > 0 ? ld(&a.Dy[q]) * fma(0.5, hy + ld(&a.Hy[q - sy]), -fl[1]) * G.ay : 0.0;
    a.N.phiz[q] = k > 0 ? ld(&a.Dz[q]) * fma(0.5, hz + ld(&a.Hz[q - sz]), -fl[2]) * G.az : 0.0;
    if (i == G.nx - 1) a.N.phix[q + sx] = 0.0;
    if (j == G.ny - 1) a.N.phiy[q + sy] = 0.0;
    if (k == G.nz - 1) a.N.phiz[q + sz] = 0.0;
}

// ---- the mixed-precision step (GEA_FLAG_MIXED) ----
//
// Each implicit solve is one defect correction: an FP64 residual r0 of the
// FP64 operator at the previous value, an FP32 solve for the increment with
// FP32 copies of the operator to ||r|| <= mp_rtol ||r0||, and the FP64
// update. Increments take the homogeneous form of each wall rule (the h
// ghost offset cancels). FP32 reductions are summed in FP32 within a block
// and in FP64 across blocks.

// FP32 data of the mixed step: the stencil weights and reciprocals, the
// FP64 residuals rounded to FP32, the increments (Jacobi ping-pong), and the
// pressure increment with its CG vectors (r the FP32 residual, z the
// preconditioned residual).
struct Mx {
    float *c[NCF];
    float *dinvu, *dinvh, *r0u, *r0v, *r0w, *r0h;
    float *du[2], *dv[2], *dw[2], *dh[2];
    float *x, *p0, *p1, *q, *r, *z;
    double tol2;
};

// Increment at (i,j,k) with at most one index one layer outside the box: the
// homogeneous ghost of wall rule BC (odd for the wall-normal velocity, even
// otherwise).
template <int BC>
__device__ __forceinline__ float atf(const Geo &G, const float *X, int i, int j, int k)
{
    if (i < 0) { const float v = ldf(&X[id3(G, 0, j, k)]); return BC == U3 ? -v : v; }
    if (i >= G.nx) { const float v = ldf(&X[id3(G, G.nx - 1, j, k)]); return BC == U3 ? -v : v; }
    if (j < 0) { const float v = ldf(&X[id3(G, i, 0, k)]); return BC == V3 ? -v : v; }
    if (j >= G.ny) { const float v = ldf(&X[id3(G, i, G.ny - 1, k)]); return BC == V3 ? -v : v; }
    if (k < 0) { const float v = ldf(&X[id3(G, i, j, 0)]); return BC == W3 ? -v : v; }
    if (k >= G.nz) { const float v = ldf(&X[id3(G, i, j, G.nz - 1)]); return BC == W3 ? -v : v; }
    return ldf(&X[id3(G, i, j, k)]);
}

struct W13f {
    float w[NCF];
};

__device__ __forceinline__ W13f weightsf(const Mx &m, int q)
{
    W13f c;
#pragma unroll
    for (int s = 0; s < NCF; ++s) c.w[s] = ldf(&m.c[s][q]);
    return c;
}

// Off-centre part of the FP32 stencil applied to an increment.
template <int BC>
__device__ __forceinline__ float tofff(const Geo &G, const W13f &c, const float *X, int i, int j, int k)
{
    if (i >= 2 && i + 2 < G.nx && j >= 2 && j + 2 < G.ny && k >= 2 && k + 2 < G.nz) {
        const int sy = G.P, sz = G.P * (G.ny + 1);
        const float *x = X + id3(G, i, j, k);
        float t = c.w[1] * ldf(x - 2);
        t = fmaf(c.w[2], ldf(x - 1), t);
        t = fmaf(c.w[3], ldf(x + 1), t);
        t = fmaf(c.w[4], ldf(x + 2), t);
        t = fmaf(c.w[5], ldf(x - 2 * sy), t);
        t = fmaf(c.w[6], ldf(x - sy), t);
        t = fmaf(c.w[7], ldf(x + sy), t);
        t = fmaf(c.w[8], ldf(x + 2 * sy), t);
        t = fmaf(c.w[9], ldf(x - 2 * sz), t);
        t = fmaf(c.w[10], ldf(x - sz), t);
        t = fmaf(c.w[11], ldf(x + sz), t);
        t = fmaf(c.w[12], ldf(x + 2 * sz), t);
        return t;
    }
    float t = c.w[1] * atf<BC>(G, X, i - 2, j, k);
    t = fmaf(c.w[2], atf<BC>(G, X, i - 1, j, k), t);
    t = fmaf(c.w[3], atf<BC>(G, X, i + 1, j, k), t);
    t = fmaf(c.w[4], atf<BC>(G, X, i + 2, j, k), t);
    t = fmaf(c.w[5], atf<BC>(G, X, i, j - 2, k), t);
    t = fmaf(c.w[6], atf<BC>(G, X, i, j - 1, k), t);
    t = fmaf(c.w[7], atf<BC>(G, X, i, j + 1, k), t);
    t = fmaf(c.w[8], atf<BC>(G, X, i, j + 2, k), t);
    t = fmaf(c.w[9], atf<BC>(G, X, i, j, k - 2), t);
    t = fmaf(c.w[10], atf<BC>(G, X, i, j, k - 1), t);
    t = fmaf(c.w[11], atf<BC>(G, X, i, j, k + 1), t);
    t = fmaf(c.w[12], atf<BC>(G, X, i, j, k + 2), t);
    return t;
}

// Compact Laplacian of an increment with even ghosts (the enthalpy's Pr
// correction).
__device__ __forceinline__ float lapf(const Geo &G, const float *X, int i, int j, int k)
{
    const float xc = atf<E3>(G, X, i, j, k);
    return (atf<E3>(G, X, i + 1, j, k) - xc + atf<E3>(G, X, i - 1, j, k) - xc) * (float)G.idx2 +
           (atf<E3>(G, X, i, j + 1, k) - xc + atf<E3>(G, X, i, j - 1, k) - xc) * (float)G.idy2 +
           (atf<E3>(G, X, i, j, k + 1) - xc + atf<E3>(G, X, i, j, k - 1) - xc) * (float)G.idz2;
}

__device__ __forceinline__ void copy_cellf(const Geo &G, const float *x, float *y)
{
    int i, j, k;
    if (cell(G, i, j, k)) y[id3(G, i, j, k)] = ldf(&x[id3(G, i, j, k)]);
}

// FP64 residuals r0 = b - T(u^n) of the three momentum components, the FP32
// copies of the stencil and the reciprocals, and the first FP32 sweep from
// zero, du = r0 / T_CC; the loop's reference norms are ||r0||^2.
__global__ void k_mx_r0mom(Args a, Mx m)
{
    Sc *sc = a.sc;
    if (sc->status) return;
    __shared__ double red[3 * NT];
    double acc[3] = {0.0, 0.0, 0.0}, tot[3];
    int i, j, k;
    if (cell(a.G, i, j, k)) {
        const int q = id3(a.G, i, j, k);
        const W13 c = weights(a, q);
        const double u0 = ld(&a.S.u[q]);
        const double ru = ld(&a.bu[q]) - fma(c.w[0], u0, toff<U3>(a, c, a.S.u, i, j, k));
        asm volatile("" ::: "memory");
        const double v0 = ld(&a.S.v[q]);
        const double rv = ld(&a.bv[q]) - fma(c.w[0], v0, toff<V3>(a, c, a.S.v, i, j, k));
        asm volatile("" ::: "memory");
        const double w0 = ld(&a.S.w[q]);
        const double rw = ld(&a.bw[q]) - fma(c.w[0], w0, toff<W3>(a, c, a.S.w, i, j, k));
#pragma unroll
        for (int s = 0; s < NCF; ++s) m.c[s][q] = (float)c.w[s];
        const float di = (float)ld(&a.dinvu[q]);
        m.dinvu[q] = di;
        m.dinvh[q] = (float)ld(&a.dinvh[q]);
        const float fu = (float)ru, fv = (float)rv, fw = (float)rw;
        m.r0u[q] = fu; m.r0v[q] = fv; m.r0w[q] = fw;
        m.du[0][q] = fu * di; m.dv[0][q] = fv * di; m.dw[0][q] = fw * di;
        acc[0] = ru * ru; acc[1] = rv * rv; acc[2] = rw * rw;
    }
    if (gsum<3>(acc, red, a.part, &sc->counters[C_MOM], tot)) {
        for (int s = 0; s < 3; ++s) sc->bn2[s] = tot[s];
        sc->done[L_MOM] = 0;
        sc->trips[L_MOM] = 0;
        sc->sweeps[0] = 0;
        if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) sc->status = GEA_ERR_NONFINITE;
    }
}

// One FP32 Jacobi sweep of the momentum increments (pairs as in the FP64
// step: the second copies once the first met the tolerance).
__global__ void k_mx_mom(Args a, Mx m, const float *ui, const float *vi, const float *wi, float *uo, float *vo,
                         float *wo, int second)
{
    Sc *sc = a.sc;
    if (sc->status) return;
    if (second && sc->done[L_MOM]) {
        copy_cellf(a.G, ui, uo);
        copy_cellf(a.G, vi, vo);
        copy_cellf(a.G, wi, wo);
        return;
    }
    __shared__ double red[3 * NT];
    float acc[3] = {0.0f, 0.0f, 0.0f};
    double tot[3];
    int i, j, k;
    if (cell(a.G, i, j, k)) {
        const Geo &G = a.G;
        const int q = id3(G, i, j, k);
        const W13f c = weightsf(m, q);
        const float di = ldf(&m.dinvu[q]);
        const float u0 = ldf(&ui[q]), v0 = ldf(&vi[q]), w0 = ldf(&wi[q]);
        const float ru = ldf(&m.r0u[q]) - fmaf(c.w[0], u0, tofff<U3>(G, c, ui, i, j, k));
        const float rv = ldf(&m.r0v[q]) - fmaf(c.w[0], v0, tofff<V3>(G, c, vi, i, j, k));
        const float rw = ldf(&m.r0w[q]) - fmaf(c.w[0], w0, tofff<W3>(G, c, wi, i, j, k));
        uo[q] = fmaf(ru, di, u0);
        vo[q] = fmaf(rv, di, v0);
        wo[q] = fmaf(rw, di, w0);
        acc[0] = ru * ru; acc[1] = rv * rv; acc[2] = rw * rw;
    }
    if (gsum<3, float>(acc, red, a.part, &sc->counters[C_MOM], tot)) {
        sc->sweeps[0] += 1;
        if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) sc->status = GEA_ERR_NONFINITE;
        else if (tot[0] <= m.tol2 * sc->bn2[0] && tot[1] <= m.tol2 * sc->bn2[1] && tot[2] <= m.tol2 * sc->bn2[2])
            sc->done[L_MOM] = 1;
    }
}

// u^{n+1/3} = u^n + du (FP64).
__global__ void k_mx_u1(Args a, const float *du, const float *dv, const float *dw)
{
    if (a.sc->status) return;
    int i, j, k;
    if (!cell(a.G, i, j, k)) return;
    const int q = id3(a.G, i, j, k);
    a.ua[q] = ld(&a.S.u[q]) + (double)ldf(&du[q]);
    a.va[q] = ld(&a.S.v[q]) + (double)ldf(&dv[q]);
    a.wa[q] = ld(&a.S.w[q]) + (double)ldf(&dw[q]);
}

// FP64 residual r0 = b_h - T_h(h^n) (h^n with its wall rule), rounded to FP32,
// and the first FP32 sweep dh = r0 / T_h,CC; the loop's reference ||r0||^2.
__global__ void k_mx_r0h(Args a, Mx m)
{
    Sc *sc = a.sc;
    if (sc->status) return;
    __shared__ double red[NT];
    double acc[1] = {0.0}, tot[1];
    int i, j, k;
    if (cell(a.G, i, j, k)) {
        const int q = id3(a.G, i, j, k);
        const W13 c = weights(a, q);
        const double h0 = ld(&a.S.h[q]);
        double t = fma(c.w[0], h0, toff<H3>(a, c, a.S.h, i, j, k));
        if (a.F.nuh != a.F.mu) t = fma(a.F.mu - a.F.nuh, lap<H3>(a, a.S.h, i, j, k), t);
        const double r0 = ld(&a.bh[q]) - t;
        const float f = (float)r0;
        m.r0h[q] = f;
        m.dh[0][q] = f * ldf(&m.dinvh[q]);
        acc[0] = r0 * r0;
    }
    if (gsum<1>(acc, red, a.part, &sc->counters[C_ENTH], tot)) {
        sc->bn2[3] = tot[0];
        sc->done[L_ENTH] = 0;
        sc->trips[L_ENTH] = 0;
        sc->sweeps[1] = 0;
        if (!isfinite(tot[0])) sc->status = GEA_ERR_NONFINITE;
    }
}

// One FP32 Jacobi sweep of the enthalpy increment (even ghosts).
__global__ void k_mx_enth(Args a, Mx m, const float *hi, float *ho, int second)
{
    Sc *sc = a.sc;
    if (sc->status) return;
    if (second && sc->done[L_ENTH]) {
        copy_cellf(a.G, hi, ho);
        return;
    }
    __shared__ double red[NT];
    float acc[1] = {0.0f};
    double tot[1];
    int i, j, k;
    if (cell(a.G, i, j, k)) {
        const Geo &G = a.G;
        const int q = id3(G, i, j, k);
        const W13f c = weightsf(m, q);
        const float h0 = ldf(&hi[q]);
        float t = fmaf(c.w[0], h0, tofff<E3>(G, c, hi, i, j, k));
        if (a.F.nuh != a.F.mu) t = fmaf((float)(a.F.mu - a.F.nuh), lapf(G, hi, i, j, k), t);
        const float r = ldf(&m.r0h[q]) - t;
        ho[q] = fmaf(r, ldf(&m.dinvh[q]), h0);
        acc[0] = r * r;
    }
    if (gsum<1, float>(acc, red, a.part, &sc->counters[C_ENTH], tot)) {
        sc->sweeps[1] += 1;
        if (!isfinite(tot[0])) sc->status = GEA_ERR_NONFINITE;
        else if (tot[0] <= m.tol2 * sc->bn2[3]) sc->done[L_ENTH] = 1;
    }
}

// h^{n+1} = h^n + dh into ha (FP64).
__global__ void k_mx_h1(Args a, const float *dh)
{
    if (a.sc->status) return;
    int i, j, k;
    if (!cell(a.G, i, j, k)) return;
    const int q = id3(a.G, i, j, k);
    a.ha[q] = ld(&a.S.h[q]) + (double)ldf(&dh[q]);
}

// FP32 CG on the pressure increment with the FP32 finest operator M0.

// p = z + beta p_old
__global__ void k_mx_pupd(Args a, Mx m, Lev32 M0)
{
    Sc *sc = a.sc;
    if (over(sc, L_CG)) return;
    int i, j, k;
    if (!cell(M0.G, i, j, k)) return;
    const int it = sc->cg_it;
    const float *pold = (it & 1) ? m.p1 : m.p0;
    float *pnew = (it & 1) ? m.p0 : m.p1;
    const int q = id3(M0.G, i, j, k);
    pnew[q] = fmaf((float)sc->beta, ldf(&pold[q]), ldf(&m.z[q]));
}

// q = A p, acc += p.q; alpha = rz / p.q
__global__ void k_mx_spmv(Args a, Mx m, Lev32 M0)
{
    Sc *sc = a.sc;
    if (over(sc, L_CG)) return;
    __shared__ double red[NT];
    float acc[1] = {0.0f};
    double tot[1];
    const float *p = (sc->cg_it & 1) ? m.p0 : m.p1;
    int i, j, k0, k1;
    if (column(M0.G, i, j, k0, k1))
#pragma unroll 1
        for (int k = k0; k < k1; ++k) {
            const int q = id3(M0.G, i, j, k);
            const float Ap = helm32(M0, [&](int qq, int, int, int) { return ldf(&p[qq]); }, i, j, k);
            m.q[q] = Ap;
            acc[0] = fmaf(ldf(&p[q]), Ap, acc[0]);
        }
    if (gsum<1, float>(acc, red, a.part, &sc->counters[C_PQ], tot)) {
        sc->pq = tot[0];
        sc->alpha = tot[0] != 0.0 ? sc->rz / tot[0] : 0.0;
        if (!isfinite(tot[0])) sc->status = GEA_ERR_NONFINITE;
    }
}

// x += alpha p, r -= alpha q; acc += r^2, relative to ||r0||^2 with mp_rtol.
__global__ void k_mx_update(Args a, Mx m, Lev32 M0)
{
    Sc *sc = a.sc;
    if (over(sc, L_CG)) return;
    __shared__ double red[NT];
    float acc[1] = {0.0f};
    double tot[1];
    const float *p = (sc->cg_it & 1) ? m.p0 : m.p1;
    const float alpha = (float)sc->alpha;
    int i, j, k0, k1;
    if (column(M0.G, i, j, k0, k1))
#pragma unroll 1
        for (int k = k0; k < k1; ++k) {
            const int q = id3(M0.G, i, j, k);
            m.x[q] = fmaf(alpha, ldf(&p[q]), m.x[q]);
            const float rn = fmaf(-alpha, ldf(&m.q[q]), m.r[q]);
            m.r[q] = rn;
            acc[0] = fmaf(rn, rn, acc[0]);
        }
    if (gsum<1, float>(acc, red, a.part, &sc->counters[C_UPD], tot)) {
        const int n = sc->cg_it + 1;
        sc->cg_it = n;
        sc->r2 = tot[0];
        sc->cg_iters[sc->corr] = n;
        sc->cg_relres[sc->corr] = sc->b2 > 0.0 ? sqrt(tot[0] / sc->b2) : 0.0;
        if (!isfinite(tot[0])) sc->status = GEA_ERR_NONFINITE;
        else if (tot[0] <= m.tol2 * sc->b2) sc->done[L_CG] = 1;
    }
}

// p' += dp (FP64).
__global__ void k_mx_papply(Args a, Mx m)
{
    if (a.sc->status) return;
    int i, j, k;
    if (!cell(a.G, i, j, k)) return;
    const int q = id3(a.G, i, j, k);
    a.N.pp[q] = ld(&a.N.pp[q]) + (double)ldf(&m.x[q]);
}

// ---- loop control and step bookkeeping (one thread) ----

__global__ void k_ctl(Sc *sc, cudaGraphConditionalHandle h, int graph, int which, int maxtrips, int body)
{
    const int trips = ++sc->trips[which];
    const int done = sc->done[which];
    sc->launches += body;
    if (!done && !sc->status && trips >= maxtrips) sc->status = GEA_ERR_NOCONV;
    if (graph) cudaGraphSetConditional(h, (done || sc->status || trips >= maxtrips) ? 0u : 1u);
}

__global__ void k_begin(Sc *sc)
{
    for (int c = 0; c < 4; ++c) { sc->cg_iters[c] = 0; sc->cg_relres[c] = 0.0; }
}

__global__ void k_end(Sc *sc, int fixed)
{
    sc->launches += fixed;
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

}  // namespace g3

using namespace g3;

struct gea3d_ctx {
    Geo G;
    Phy F;
    gea_constants C;
    cudaStream_t stream = nullptr, cap = nullptr, cap2 = nullptr;
    std::vector<void *> allocs;
    St S[2];
    double *rho1, *dinvu, *dinvh, *bu, *bv, *bw, *ua, *va, *wa, *ub, *vb, *wb, *bh, *ha, *hb;
    double *rho2, *psi, *Dx, *Dy, *Dz, *Hx, *Hy, *Hz, *b, *p0, *p1, *q;
    double *dtr1;                         // dt / rho1
    double *kin;                          // K1
    double *mueff = nullptr;              // LES eddy viscosity field
    double *gz = nullptr;                 // g z: nz cell centres, then nz + 1 horizontal faces
    bool mixed = false;                   // GEA_FLAG_MIXED
    Mx mx{};                              // FP32 data of the mixed step
    Cf cf;                                // transport stencil weights
    double *stage = nullptr;              // dense conservative fields (5 arrays)
    std::vector<Lev> L;                   // the FP64 fine-level operator
    std::vector<Lev32> M;                 // the FP32 multigrid hierarchy
    Sc *sc = nullptr;
    double *part = nullptr;
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    bool have_state = false;
    long long steps_at_sync = 0;
    char err[256] = {0};
};

namespace {

int fail3(gea3d_ctx *c, int code, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CK3(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail3(ctx, GEA_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                         __LINE__);                                                                 \
    } while (0)

Geo make_geo(int nx, int ny, int nz, double lx, double ly, double lz)
{
    Geo G;
    G.nx = nx; G.ny = ny; G.nz = nz;
    G.P = (nx + 1 + 31) / 32 * 32;
    G.dx = lx / nx; G.dy = ly / ny; G.dz = lz / nz;
    G.idx = 1.0 / G.dx; G.idy = 1.0 / G.dy; G.idz = 1.0 / G.dz;
    G.idx2 = 1.0 / (G.dx * G.dx); G.idy2 = 1.0 / (G.dy * G.dy); G.idz2 = 1.0 / (G.dz * G.dz);
    G.ivol = 1.0 / (G.dx * G.dy * G.dz);
    G.ax = G.dy * G.dz; G.ay = G.dx * G.dz; G.az = G.dx * G.dy;
    return G;
}

// elements of one array (cells or faces) of a level
size_t elems(const Geo &G) { return (size_t)(G.nz + 1) * (G.ny + 1) * G.P; }

// Diagnostics (Remark 2) in three dimensions: theta' = T (p0/p)^(R/cp) -
// theta_bar(z) per cell into th (dense nz x ny x nx, x fastest; optional),
// mass = sum rho V and energy = sum rho (cv T + |u|^2/2 + g z) V (Section
// 2.1's total energy) into the scalars.
__global__ void k_diag3(Geo G, Phy F, double p0, St S, const double *thbar, const double *gzc, double *th, Sc *sc,
                        double *part)
{
    __shared__ double red[2 * NT];
    int i, j, k;
    double v[2] = {0.0, 0.0};
    if (cell(G, i, j, k)) {
        const int q = id3(G, i, j, k);
        const double T = ld(&S.T[q]), rho = ld(&S.rho[q]);
        if (th) th[((size_t)k * G.ny + j) * G.nx + i] = T / pow(ld(&S.p[q]) / p0, F.R / F.cp) - ld(&thbar[k]);
        const double u = ld(&S.u[q]), vv = ld(&S.v[q]), w = ld(&S.w[q]);
        const double V = G.dx * G.dy * G.dz;
        const double K = 0.5 * (u * u + vv * vv + w * w);
        v[0] = rho * V;
        v[1] = rho * ((F.cp - F.R) * T + K + ld(&gzc[k])) * V;
    }
    double tot[2];
    if (gsum<2>(v, red, part, &sc->counters[C_DIAG], tot)) {
        sc->mass = tot[0];
        sc->energy = tot[1];
    }
}

dim3 grid_of(const Geo &G) { return dim3((G.nx + TX - 1) / TX, (G.ny + TY - 1) / TY, G.nz); }
// the grid of the column kernels (kLayers cell layers per block)
dim3 gridc_of(const Geo &G) { return dim3((G.nx + TX - 1) / TX, (G.ny + TY - 1) / TY, (G.nz + kLayers - 1) / kLayers); }
const dim3 kBlk(TX, TY);
size_t nblocks(const Geo &G)
{
    const dim3 g = grid_of(G);
    return (size_t)g.x * g.y * g.z;
}

Args args_of(gea3d_ctx *c, int from)
{
    Args a;
    a.G = c->G; a.F = c->F;
    a.S = c->S[from]; a.N = c->S[from ^ 1];
    a.rho1 = c->rho1; a.dinvu = c->dinvu; a.dinvh = c->dinvh;
    a.bu = c->bu; a.bv = c->bv; a.bw = c->bw;
    a.ua = c->ua; a.va = c->va; a.wa = c->wa; a.ub = c->ub; a.vb = c->vb; a.wb = c->wb;
    a.bh = c->bh; a.ha = c->ha; a.hb = c->hb;
    a.rho2 = c->rho2; a.psi = c->psi; a.Dx = c->Dx; a.Dy = c->Dy; a.Dz = c->Dz;
    a.Hx = c->Hx; a.Hy = c->Hy; a.Hz = c->Hz; a.b = c->b; a.p0 = c->p0; a.p1 = c->p1; a.q = c->q;
    a.cf = c->cf;
    a.dtr1 = c->dtr1;
    a.kin = c->kin;
    a.mueff = c->mueff;
    a.gzc = c->gz;
    a.gzf = c->gz + c->G.nz;
    a.sc = c->sc; a.part = c->part;
    a.jtol2 = c->C.jac_rtol * c->C.jac_rtol;
    a.ctol2 = c->C.cg_rtol * c->C.cg_rtol;
    return a;
}

// WHILE node on the graph captured on s; body(stream, handle) captured into it
template <class Body>
int capture_while3(gea3d_ctx *ctx, cudaStream_t s, Body body)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edges = nullptr;
    size_t ndeps = 0;
    CK3(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &ndeps));
    if (cs != cudaStreamCaptureStatusActive) return fail3(ctx, GEA_ERR_CUDA, "capture not active");
    cudaGraphConditionalHandle h;
    CK3(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams prm = {cudaGraphNodeTypeConditional};
    prm.conditional.handle = h;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    cudaGraphNode_t node;
    CK3(cudaGraphAddNode(&node, g, deps, edges, ndeps, &prm));
    CK3(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    CK3(cudaStreamBeginCaptureToGraph(ctx->cap2, prm.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal));
    body(ctx->cap2, h);
    cudaGraph_t out = nullptr;
    CK3(cudaStreamEndCapture(ctx->cap2, &out));
    return GEA_OK;
}

// Event pairs around the launches of an eager step (per-kernel timing). A
// solver-loop kernel launched after its loop finished returns at once (a
// converged solve, or the second Jacobi sweep of a pair that copies): it is
// recorded with zero cells, the loop's flags read before the launch.
struct Trace3 {
    struct Rec {
        const char *name;
        long long cells;
        cudaEvent_t e0, e1;
    };
    std::vector<Rec> recs;
    const Sc *dsc = nullptr;
    // the loop whose finished flag makes the kernel return, or -1
    static int gate(const char *name)
    {
        static const char *cg[] = {"g3_mg_coarse", "g3_mg_down", "g3_mg_single", "g3_mg_up", "g3_pupd", "g3_spmv",
                                   "g3_update", "g3_mx_pupd", "g3_mx_spmv", "g3_mx_update"};
        for (const char *c : cg)
            if (!strcmp(name, c)) return L_CG;
        if (!strcmp(name, "g3_mom") || !strcmp(name, "g3_mx_mom")) return L_MOM;
        if (!strcmp(name, "g3_enth") || !strcmp(name, "g3_mx_enth")) return L_ENTH;
        return -1;
    }
    ~Trace3()
    {
        for (auto &r : recs) {
            cudaEventDestroy(r.e0);
            cudaEventDestroy(r.e1);
        }
    }
};

// Run go() (one launch on st), bracketed by an event pair when tracing.
template <class Go>
void traced(Trace3 *tr, const char *name, const Geo &G, cudaStream_t st, Go go)
{
    if (!tr) {
        go();
        return;
    }
    Trace3::Rec r{name, (long long)G.nx * G.ny * G.nz, nullptr, nullptr};
    const int g = Trace3::gate(name);
    if (g >= 0 && tr->dsc) {
        Sc h;
        if (cudaMemcpyAsync(&h, tr->dsc, sizeof(Sc), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess && (h.status || h.done[g]))
            r.cells = 0;
    }
    cudaEventCreate(&r.e0);
    cudaEventCreate(&r.e1);
    cudaEventRecord(r.e0, st);
    go();
    cudaEventRecord(r.e1, st);
    tr->recs.push_back(r);
}

// Run a loop body eagerly until its control kernel reports the loop over.
template <class Body>
int eager_while3(gea3d_ctx *ctx, cudaStream_t s, int which, int maxtrips, Body body)
{
    for (int t = 0; t < maxtrips + 1; ++t) {
        body(s, (cudaGraphConditionalHandle)0);
        Sc h;
        CK3(cudaMemcpyAsync(&h, ctx->sc, sizeof(Sc), cudaMemcpyDeviceToHost, s));
        CK3(cudaStreamSynchronize(s));
        if (h.done[which] || h.status || h.trips[which] >= maxtrips) break;
    }
    return GEA_OK;
}

// z = M^-1 r on the finest level (one FP32 V(1,1) cycle); returns launches
int vcycle(gea3d_ctx *ctx, const Args &a, cudaStream_t st, Trace3 *tr)
{
    Lev32 *M = ctx->M.data();
    Lev &F = ctx->L[0];
    const int nlev = (int)ctx->M.size();
    if (ctx->mixed) {
        // the mixed step's FP32 CG: from the FP32 residual r to z, both FP32
        const Mx &m = ctx->mx;
        if (nlev == 1) {
            traced(tr, "g3_mg_single", F.G, st, [&] {
                k_mg_single<float><<<grid_of(F.G), kBlk, 0, st>>>(M[0], m.r, m.z, a.sc, a.part);
            });
            return 1;
        }
        int n = 0;
        traced(tr, "g3_mg_down", M[1].G, st, [&] {
            k_mg_down<float><<<grid_of(M[1].G), kBlk, 0, st>>>(M[0], m.r, M[1], a.sc);
        });
        ++n;
        for (int l = 1; l + 1 < nlev; ++l, ++n)
            traced(tr, "g3_mg_down", M[l + 1].G, st, [&] {
                k_mg_down<float><<<grid_of(M[l + 1].G), kBlk, 0, st>>>(M[l], M[l].r, M[l + 1], a.sc);
            });
        Lev32 &C = M[nlev - 1];
        for (int s = 0; s < kCoarseSweeps; ++s, ++n) {
            float *out = ((kCoarseSweeps - 1 - s) % 2 == 0) ? C.e2 : C.e;
            const float *in = (out == C.e2) ? C.e : C.e2;
            traced(tr, "g3_mg_coarse", C.G, st, [&] {
                k_mg_coarse<<<grid_of(C.G), kBlk, 0, st>>>(C, in, out, s == 0, a.sc);
            });
        }
        for (int l = nlev - 2; l >= 1; --l, ++n)
            traced(tr, "g3_mg_up", M[l].G, st, [&] {
                k_mg_up<float, float><<<grid_of(M[l].G), kBlk, 0, st>>>(M[l], M[l].r, M[l + 1].e2, M[l + 1].G,
                                                                         M[l].e2, a.sc);
            });
        traced(tr, "g3_mg_up", F.G, st, [&] {
            k_mg_up_fin<float, float><<<gridc_of(F.G), kBlk, 0, st>>>(M[0], m.r, M[1].e2, M[1].G, m.z, a.sc,
                                                                      a.part);
        });
        return n + 1;
    }
    if (nlev == 1) {
        traced(tr, "g3_mg_single", F.G, st, [&] {
            k_mg_single<double><<<grid_of(F.G), kBlk, 0, st>>>(M[0], F.r, F.e2, a.sc, a.part);
        });
        return 1;
    }
    int n = 0;
    traced(tr, "g3_mg_down", M[1].G, st, [&] {
        k_mg_down<float><<<grid_of(M[1].G), kBlk, 0, st>>>(M[0], M[0].r, M[1], a.sc);
    });
    ++n;
    for (int l = 1; l + 1 < nlev; ++l, ++n)
        traced(tr, "g3_mg_down", M[l + 1].G, st, [&] {
            k_mg_down<float><<<grid_of(M[l + 1].G), kBlk, 0, st>>>(M[l], M[l].r, M[l + 1], a.sc);
        });
    Lev32 &C = M[nlev - 1];
    for (int s = 0; s < kCoarseSweeps; ++s, ++n) {
        float *out = ((kCoarseSweeps - 1 - s) % 2 == 0) ? C.e2 : C.e;
        const float *in = (out == C.e2) ? C.e : C.e2;
        traced(tr, "g3_mg_coarse", C.G, st, [&] {
            k_mg_coarse<<<grid_of(C.G), kBlk, 0, st>>>(C, in, out, s == 0, a.sc);
        });
    }
    for (int l = nlev - 2; l >= 1; --l, ++n)
        traced(tr, "g3_mg_up", M[l].G, st, [&] {
            k_mg_up<float, float><<<grid_of(M[l].G), kBlk, 0, st>>>(M[l], M[l].r, M[l + 1].e2, M[l + 1].G,
                                                                     M[l].e2, a.sc);
        });
    traced(tr, "g3_mg_up", F.G, st, [&] {
        k_mg_up_fin<double, double><<<gridc_of(F.G), kBlk, 0, st>>>(M[0], F.r, M[1].e2, M[1].G, F.e2, a.sc,
                                                                    a.part);
    });
    return n + 1;
}

// The kernel sequence of one step reading slot `from` (Section 3: Step 1,
// Step 2, n_corr PISO correctors). graph: captured on s, the loops as WHILE
// nodes; otherwise launched eagerly with host-checked loops, each launch
// bracketed by tr (if given).
int record3(gea3d_ctx *ctx, int from, cudaStream_t s, bool graph, Trace3 *tr)
{
    const Args a = args_of(ctx, from);
    Lev *L = ctx->L.data();
    Lev32 *M = ctx->M.data();
    const int nlev = (int)ctx->M.size();
    const Geo &G = ctx->G;
    const dim3 grid = grid_of(G);
    const dim3 gridc(grid.x, grid.y, (G.nz + kLayers - 1) / kLayers);   // column kernels
    const int jtrips = (ctx->C.jac_maxit + 1) / 2;
    const int gr = graph ? 1 : 0;
    int fixed = 0, rc;
    auto loop = [&](int which, int maxtrips, auto body) {
        return graph ? capture_while3(ctx, s, body) : eager_while3(ctx, s, which, maxtrips, body);
    };
    k_begin<<<1, 1, 0, s>>>(a.sc); ++fixed;
    if (ctx->mueff) { traced(tr, "g3_les", G, s, [&] { k_les<<<grid, kBlk, 0, s>>>(a); }); ++fixed; }
    traced(tr, "g3_pred", G, s, [&] { k_pred<<<grid, kBlk, 0, s>>>(a); }); ++fixed;
    const Mx &m = ctx->mx;
    if (ctx->mixed) {
        // FP64 residuals, FP32 Jacobi on the increments (pairs end in du[0]), FP64 update
        traced(tr, "g3_mx_r0mom", G, s, [&] { k_mx_r0mom<<<grid, kBlk, 0, s>>>(a, m); }); ++fixed;
        rc = loop(L_MOM, jtrips, [&](cudaStream_t bs, cudaGraphConditionalHandle h) {
            traced(tr, "g3_mx_mom", G, bs, [&] {
                k_mx_mom<<<grid, kBlk, 0, bs>>>(a, m, m.du[0], m.dv[0], m.dw[0], m.du[1], m.dv[1], m.dw[1], 0);
            });
            traced(tr, "g3_mx_mom", G, bs, [&] {
                k_mx_mom<<<grid, kBlk, 0, bs>>>(a, m, m.du[1], m.dv[1], m.dw[1], m.du[0], m.dv[0], m.dw[0], 1);
            });
            k_ctl<<<1, 1, 0, bs>>>(a.sc, h, gr, L_MOM, jtrips, 3);
        });
        if (rc) return rc;
        traced(tr, "g3_mx_u1", G, s, [&] { k_mx_u1<<<grid, kBlk, 0, s>>>(a, m.du[0], m.dv[0], m.dw[0]); }); ++fixed;
    } else {
        rc = loop(L_MOM, jtrips, [&](cudaStream_t bs, cudaGraphConditionalHandle h) {
            traced(tr, "g3_mom", G, bs, [&] { k_mom<<<grid, kBlk, 0, bs>>>(a, a.ua, a.va, a.wa, a.ub, a.vb, a.wb, 0); });
            traced(tr, "g3_mom", G, bs, [&] { k_mom<<<grid, kBlk, 0, bs>>>(a, a.ub, a.vb, a.wb, a.ua, a.va, a.wa, 1); });
            k_ctl<<<1, 1, 0, bs>>>(a.sc, h, gr, L_MOM, jtrips, 3);
        });
        if (rc) return rc;
    }
    traced(tr, "g3_kin", G, s, [&] { k_kin<<<grid, kBlk, 0, s>>>(a, a.ua, a.va, a.wa); }); ++fixed;
    traced(tr, "g3_enth_rhs", G, s, [&] { k_enth_rhs<<<grid, kBlk, 0, s>>>(a, a.wa); }); ++fixed;
    if (ctx->mixed) {
        traced(tr, "g3_mx_r0h", G, s, [&] { k_mx_r0h<<<grid, kBlk, 0, s>>>(a, m); }); ++fixed;
        rc = loop(L_ENTH, jtrips, [&](cudaStream_t bs, cudaGraphConditionalHandle h) {
            traced(tr, "g3_mx_enth", G, bs, [&] { k_mx_enth<<<grid, kBlk, 0, bs>>>(a, m, m.dh[0], m.dh[1], 0); });
            traced(tr, "g3_mx_enth", G, bs, [&] { k_mx_enth<<<grid, kBlk, 0, bs>>>(a, m, m.dh[1], m.dh[0], 1); });
            k_ctl<<<1, 1, 0, bs>>>(a.sc, h, gr, L_ENTH, jtrips, 3);
        });
        if (rc) return rc;
        traced(tr, "g3_mx_h1", G, s, [&] { k_mx_h1<<<grid, kBlk, 0, s>>>(a, m.dh[0]); }); ++fixed;
    } else {
        rc = loop(L_ENTH, jtrips, [&](cudaStream_t bs, cudaGraphConditionalHandle h) {
            traced(tr, "g3_enth", G, bs, [&] { k_enth<<<grid, kBlk, 0, bs>>>(a, a.ha, a.hb, 0); });
            traced(tr, "g3_enth", G, bs, [&] { k_enth<<<grid, kBlk, 0, bs>>>(a, a.hb, a.ha, 1); });
            k_ctl<<<1, 1, 0, bs>>>(a.sc, h, gr, L_ENTH, jtrips, 3);
        });
        if (rc) return rc;
    }
    traced(tr, "g3_eos", G, s, [&] { k_eos<<<grid, kBlk, 0, s>>>(a, L[0], M[0], a.ha); }); ++fixed;
    traced(tr, "g3_faces", G, s, [&] { k_faces<<<grid, kBlk, 0, s>>>(a, L[0], M[0]); }); ++fixed;
    traced(tr, "g3_diag", G, s, [&] { k_diag<<<grid, kBlk, 0, s>>>(L[0], M[0], a.sc); }); ++fixed;
    for (int l = 0; l + 1 < nlev; ++l, ++fixed)
        traced(tr, "g3_coarsen", M[l + 1].G, s, [&] {
            k_coarsen<<<grid_of(M[l + 1].G), kBlk, 0, s>>>(M[l], M[l + 1]);
        });
    const int body_cg = (nlev == 1 ? 4 : 3 + (nlev - 1) + kCoarseSweeps + (nlev - 1)) + 1;
    for (int c = 0; c < ctx->C.n_corr; ++c) {
        const double *U = c == 0 ? a.ua : a.N.u, *V = c == 0 ? a.va : a.N.v, *W = c == 0 ? a.wa : a.N.w;
        traced(tr, "g3_H", G, s, [&] { k_H<<<grid, kBlk, 0, s>>>(a, U, V, W); }); ++fixed;
        traced(tr, "g3_helm_rhs", G, s, [&] {
            if (ctx->mixed)
                k_helm_rhs<<<grid, kBlk, 0, s>>>(a, L[0], c == 0 ? a.S.pp : a.N.pp, a.N.pp, c, m.r, m.x, m.p0);
            else
                k_helm_rhs<<<grid, kBlk, 0, s>>>(a, L[0], c == 0 ? a.S.pp : a.N.pp, a.N.pp, c, nullptr, nullptr,
                                                 nullptr, ctx->M[0].r);
        });
        ++fixed;
        fixed += vcycle(ctx, a, s, tr);
        rc = loop(L_CG, ctx->C.cg_maxit, [&](cudaStream_t bs, cudaGraphConditionalHandle h) {
            if (ctx->mixed) {
                traced(tr, "g3_mx_pupd", G, bs, [&] { k_mx_pupd<<<grid, kBlk, 0, bs>>>(a, m, M[0]); });
                traced(tr, "g3_mx_spmv", G, bs, [&] { k_mx_spmv<<<gridc, kBlk, 0, bs>>>(a, m, M[0]); });
                traced(tr, "g3_mx_update", G, bs, [&] { k_mx_update<<<gridc, kBlk, 0, bs>>>(a, m, M[0]); });
            } else {
                traced(tr, "g3_pupd", G, bs, [&] { k_pupd<<<grid, kBlk, 0, bs>>>(a, L[0]); });
                traced(tr, "g3_spmv", G, bs, [&] { k_spmv<<<gridc, kBlk, 0, bs>>>(a, L[0]); });
                traced(tr, "g3_update", G, bs, [&] { k_update<<<gridc, kBlk, 0, bs>>>(a, L[0], a.N.pp, ctx->M[0].r, ctx->C.cg_maxit); });
            }
            vcycle(ctx, a, bs, tr);
            k_ctl<<<1, 1, 0, bs>>>(a.sc, h, gr, L_CG, ctx->C.cg_maxit, body_cg);
        });
        if (rc) return rc;
        if (ctx->mixed) {
            traced(tr, "g3_mx_papply", G, s, [&] { k_mx_papply<<<grid, kBlk, 0, s>>>(a, m); });
            ++fixed;
        }
        traced(tr, "g3_correct", G, s, [&] { k_correct<<<grid, kBlk, 0, s>>>(a); }); ++fixed;
    }
    ++fixed;
    k_end<<<1, 1, 0, s>>>(a.sc, fixed);
    return cudaGetLastError() == cudaSuccess ? GEA_OK : fail3(ctx, GEA_ERR_CUDA, "kernel launch failed");
}

int build3(gea3d_ctx *ctx, int from)
{
    cudaStream_t s = ctx->cap;
    CK3(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const int rc = record3(ctx, from, s, true, nullptr);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail3(ctx, GEA_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    ctx->graph[from] = g;
    CK3(cudaGraphInstantiate(&ctx->exec[from], g, 0));
    return GEA_OK;
}

}  // namespace

extern "C" {

int gea3d_create(const gea3d_grid *grid, const gea_constants *c, gea3d_ctx **out)
{
    if (!grid || !c || !out) return GEA_ERR_INVAL;
    *out = nullptr;
    if (grid->nx < 4 || grid->ny < 4 || grid->nz < 4 || !(grid->lx > 0) || !(grid->ly > 0) || !(grid->lz > 0))
        return GEA_ERR_INVAL;
    if ((long long)grid->nx * grid->ny * grid->nz > (1LL << 31) / 4) return GEA_ERR_INVAL;
    // the kernels index a field (ghost layers and row padding included) with
    // 32-bit integers
    if ((long long)(grid->nz + 1) * (grid->ny + 1) * ((grid->nx + 1 + 31) / 32 * 32) > INT_MAX) return GEA_ERR_INVAL;
    if (!(c->R > 0) || !(c->cp > c->R) || !(c->g >= 0) || !(c->p0 > 0) || !(c->mu >= 0) || !(c->Pr > 0) ||
        !(c->dt > 0) || c->n_corr < 1 || c->n_corr > 4 || !(c->jac_rtol > 0) || c->jac_maxit < 1 ||
        !(c->cg_rtol > 0) || c->cg_maxit < 1 || c->mg_min_cells < 0 || (c->flags & ~GEA_FLAG_MIXED) != 0 ||
        c->reading_flags != 0 ||
        (!(c->flags & GEA_FLAG_MIXED) && c->mp_rtol != 0.0) ||
        ((c->flags & GEA_FLAG_MIXED) && c->mp_rtol != 0.0 && !(c->mp_rtol >= 1e-7 && c->mp_rtol < 1.0)) ||
        !(c->cs >= 0.0) || (c->cs > 0.0 && c->Pr != 1.0))
        return GEA_ERR_INVAL;
    gea3d_ctx *ctx = new gea3d_ctx();
    ctx->C = *c;
    ctx->G = make_geo(grid->nx, grid->ny, grid->nz, grid->lx, grid->ly, grid->lz);
    ctx->F.R = c->R; ctx->F.cp = c->cp; ctx->F.g = c->g; ctx->F.mu = c->mu; ctx->F.nuh = c->mu / c->Pr;
    ctx->F.dt = c->dt; ctx->F.idt = 1.0 / c->dt; ctx->F.omega = kOmega; ctx->F.icp = 1.0 / c->cp;
    {
        const double delta = cbrt(ctx->G.dx * ctx->G.dy * ctx->G.dz);
        ctx->F.les_d2 = c->cs * c->cs * delta * delta;
    }
    // multigrid levels: halve all three sizes while they are even and >= 8
    // and (unless mg_min_cells is given) the Laplacian-to-diagonal estimate
    // 2 dt^2 R T (1/dx^2 + 1/dy^2 + 1/dz^2) exceeds 1
    std::vector<Geo> lg{ctx->G};
    double ratio = 2.0 * c->dt * c->dt * c->R * kRefT *
                   (1.0 / (ctx->G.dx * ctx->G.dx) + 1.0 / (ctx->G.dy * ctx->G.dy) + 1.0 / (ctx->G.dz * ctx->G.dz));
    for (;;) {
        const Geo &f = lg.back();
        if (f.nx % 2 || f.ny % 2 || f.nz % 2 || f.nx < 8 || f.ny < 8 || f.nz < 8) break;
        if (c->mg_min_cells > 0 && (long long)f.nx * f.ny * f.nz <= c->mg_min_cells) break;
        if (c->mg_min_cells == 0 && ratio <= kCoarsestRatio) break;
        if ((int)lg.size() >= kMaxLev) break;
        lg.push_back(make_geo(f.nx / 2, f.ny / 2, f.nz / 2, f.nx * f.dx, f.ny * f.dy, f.nz * f.dz));
        ratio *= 0.25;
    }
    bool ok = true;
    auto take = [&](size_t n) -> double * {
        void *p = nullptr;
        if (!ok) return nullptr;
        if (cudaMalloc(&p, n * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
            return nullptr;
        }
        cudaMemset(p, 0, n * sizeof(double));
        ctx->allocs.push_back(p);
        return static_cast<double *>(p);
    };
    const size_t E = elems(ctx->G);
    for (int s = 0; s < 2; ++s) {
        St &S = ctx->S[s];
        double **f[12] = {&S.rho, &S.u, &S.v, &S.w, &S.T, &S.h, &S.p, &S.pp, &S.pold, &S.phix, &S.phiy, &S.phiz};
        for (auto pp : f) *pp = take(E);
    }
    double **sc[] = {&ctx->rho1, &ctx->dinvu, &ctx->dinvh, &ctx->bu, &ctx->bv, &ctx->bw, &ctx->ua, &ctx->va,
                     &ctx->wa, &ctx->ub, &ctx->vb, &ctx->wb, &ctx->bh, &ctx->ha, &ctx->hb, &ctx->rho2,
                     &ctx->psi, &ctx->Dx, &ctx->Dy, &ctx->Dz, &ctx->Hx, &ctx->Hy, &ctx->Hz, &ctx->b, &ctx->p0,
                     &ctx->p1, &ctx->q};
    for (auto pp : sc) *pp = take(E);
    for (int m = 0; m < NCF; ++m) ctx->cf.c[m] = take(E);
    ctx->dtr1 = take(E);
    ctx->kin = take(E);
    if (c->cs > 0.0) ctx->mueff = take(E);
    {
        // the heights g z of the cell centres and of the horizontal faces,
        // rounded as the expressions g ((k + 1/2) dz) and g (k dz)
        const int nz = ctx->G.nz;
        std::vector<double> h(2 * (size_t)nz + 1);
        for (int k = 0; k < nz; ++k) h[k] = c->g * ((k + 0.5) * ctx->G.dz);
        for (int k = 0; k <= nz; ++k) h[nz + k] = c->g * (k * ctx->G.dz);
        ctx->gz = take(h.size());
        if (ctx->gz && cudaMemcpy(ctx->gz, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
            ok = false;
    }
    ctx->mixed = (c->flags & GEA_FLAG_MIXED) != 0;
    if (ctx->mixed) {
        Mx &m = ctx->mx;
        auto tf = [&]() { return reinterpret_cast<float *>(take((E + 1) / 2)); };
        for (int s = 0; s < NCF; ++s) m.c[s] = tf();
        m.dinvu = tf(); m.dinvh = tf(); m.r0u = tf(); m.r0v = tf(); m.r0w = tf(); m.r0h = tf();
        for (int b = 0; b < 2; ++b) { m.du[b] = tf(); m.dv[b] = tf(); m.dw[b] = tf(); m.dh[b] = tf(); }
        m.x = tf(); m.p0 = tf(); m.p1 = tf(); m.q = tf(); m.r = tf(); m.z = tf();
        const double rt = c->mp_rtol != 0.0 ? c->mp_rtol : 1e-5;
        m.tol2 = rt * rt;
    }
    ctx->stage = take(5 * (size_t)grid->nx * grid->ny * grid->nz);
    {
        Lev l;
        l.G = ctx->G;
        l.c = take(E); l.d = take(E); l.ax = take(E); l.ay = take(E); l.az = take(E);
        l.r = take(E); l.e2 = take(E);
        ctx->L.push_back(l);
    }
    auto takef = [&](size_t n) -> float * {
        // FP32 arrays: half as many doubles, rounded up
        return reinterpret_cast<float *>(take((n + 1) / 2));
    };
    for (size_t lv = 0; lv < lg.size(); ++lv) {
        Lev32 m;
        m.G = lg[lv];
        const size_t e = elems(lg[lv]);
        m.c = takef(e); m.d = takef(e); m.ax = takef(e); m.ay = takef(e); m.az = takef(e);
        m.w = takef(e); m.e = takef(e);
        // the FP64 step keeps an FP32 copy of the CG residual on the finest
        // level for the restriction (the mixed step's residual is FP32)
        m.r = (lv || !ctx->mixed) ? takef(e) : nullptr;
        m.e2 = lv ? takef(e) : nullptr;
        ctx->M.push_back(m);
    }
    {
        const size_t nb = nblocks(ctx->G), ng = (nb + kGroup - 1) / kGroup;
        if (ng > 2 * (size_t)kCntSlots) {
            gea3d_destroy(ctx);
            return GEA_ERR_INVAL;
        }
        ctx->part = take(kCntSlots + 3 * nb + 3 * ng + 64);
    }
    ctx->sc = reinterpret_cast<Sc *>(take((sizeof(Sc) + 7) / 8));
    if (!ok) {
        gea3d_destroy(ctx);
        return GEA_ERR_NOMEM;
    }
    if (cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->cap2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        gea3d_destroy(ctx);
        return GEA_ERR_CUDA;
    }
    *out = ctx;
    return GEA_OK;
}

int gea3d_set_stream(gea3d_ctx *ctx, void *stream)
{
    if (!ctx) return GEA_ERR_INVAL;
    ctx->stream = (cudaStream_t)stream;
    return GEA_OK;
}

int gea3d_set_conservative(gea3d_ctx *ctx, const double *rho, const double *rhou, const double *rhov,
                           const double *rhow, const double *rhoe, int32_t mem)
{
    if (!ctx || !rho || !rhou || !rhov || !rhow || !rhoe || (mem != GEA_MEM_HOST && mem != GEA_MEM_DEVICE))
        return GEA_ERR_INVAL;
    const Geo &G = ctx->G;
    const size_t n = (size_t)G.nx * G.ny * G.nz;
    // the old state is being replaced: until this call succeeds the context
    // holds none
    ctx->have_state = false;
    CK3(cudaMemsetAsync(ctx->sc, 0, sizeof(Sc), ctx->stream));
    const double *src[5] = {rho, rhou, rhov, rhow, rhoe};
    for (int f = 0; f < 5; ++f)
        CK3(cudaMemcpyAsync(ctx->stage + f * n, src[f], n * sizeof(double), cudaMemcpyDefault, ctx->stream));
    k_derive<<<grid_of(G), kBlk, 0, ctx->stream>>>(G, ctx->F, ctx->stage, ctx->stage + n, ctx->stage + 2 * n,
                                                   ctx->stage + 3 * n, ctx->stage + 4 * n, ctx->S[0], ctx->sc);
    CK3(cudaGetLastError());
    Sc h;
    CK3(cudaMemcpyAsync(&h, ctx->sc, sizeof(Sc), cudaMemcpyDeviceToHost, ctx->stream));
    CK3(cudaStreamSynchronize(ctx->stream));
    if (h.bad_cells) {
        ctx->have_state = false;
        return fail3(ctx, GEA_ERR_INVAL, "%d cells with rho <= 0 or T <= 0", h.bad_cells);
    }
    ctx->steps_at_sync = 0;
    ctx->have_state = true;
    return GEA_OK;
}

int gea3d_step_async(gea3d_ctx *ctx, int32_t n)
{
    if (!ctx || n < 0) return GEA_ERR_INVAL;
    if (!ctx->have_state) return fail3(ctx, GEA_ERR_STATE, "no state set");
    for (int f = 0; f < 2; ++f)
        if (!ctx->exec[f]) {
            const int rc = build3(ctx, f);
            if (rc) return rc;
        }
    for (int s = 0; s < n; ++s) {
        CK3(cudaGraphLaunch(ctx->exec[ctx->steps_at_sync & 1], ctx->stream));
        ctx->steps_at_sync += 1;
    }
    return GEA_OK;
}

int gea3d_sync(gea3d_ctx *ctx)
{
    if (!ctx) return GEA_ERR_INVAL;
    Sc h;
    CK3(cudaMemcpyAsync(&h, ctx->sc, sizeof(Sc), cudaMemcpyDeviceToHost, ctx->stream));
    CK3(cudaStreamSynchronize(ctx->stream));
    ctx->steps_at_sync = h.steps_done;
    if (h.last_status == GEA_ERR_NOCONV) return fail3(ctx, GEA_ERR_NOCONV, "a linear solve reached its iteration cap");
    if (h.last_status) return fail3(ctx, h.last_status, "device status %d", h.last_status);
    return GEA_OK;
}

int gea3d_step(gea3d_ctx *ctx, int32_t n)
{
    const int rc = gea3d_step_async(ctx, n);
    return rc ? rc : gea3d_sync(ctx);
}

int gea3d_get_state(gea3d_ctx *ctx, double *rho, double *u, double *v, double *w, double *T, double *p,
                    double *pp, int32_t mem)
{
    if (!ctx || (mem != GEA_MEM_HOST && mem != GEA_MEM_DEVICE)) return GEA_ERR_INVAL;
    if (!ctx->have_state) return fail3(ctx, GEA_ERR_STATE, "no state set");
    Sc h;
    CK3(cudaMemcpyAsync(&h, ctx->sc, sizeof(Sc), cudaMemcpyDeviceToHost, ctx->stream));
    CK3(cudaStreamSynchronize(ctx->stream));
    const St &S = ctx->S[h.steps_done & 1];
    const Geo &G = ctx->G;
    double *dst[7] = {rho, u, v, w, T, p, pp};
    const double *src[7] = {S.rho, S.u, S.v, S.w, S.T, S.p, S.pp};
    for (int f = 0; f < 7; ++f) {
        if (!dst[f]) continue;
        // (k (ny+1) + j) P + i -> (k ny + j) nx + i: one 3D copy per field (rows
        // of nx values, ny rows a layer out of the source's ny + 1, nz layers)
        cudaMemcpy3DParms c = {};
        c.srcPtr = make_cudaPitchedPtr(const_cast<double *>(src[f]), (size_t)G.P * sizeof(double),
                                       (size_t)G.nx * sizeof(double), (size_t)G.ny + 1);
        c.dstPtr = make_cudaPitchedPtr(dst[f], (size_t)G.nx * sizeof(double), (size_t)G.nx * sizeof(double),
                                       (size_t)G.ny);
        c.extent = make_cudaExtent((size_t)G.nx * sizeof(double), (size_t)G.ny, (size_t)G.nz);
        c.kind = cudaMemcpyDefault;
        CK3(cudaMemcpy3DAsync(&c, ctx->stream));
    }
    CK3(cudaStreamSynchronize(ctx->stream));
    return GEA_OK;
}

int gea3d_get_diag(gea3d_ctx *ctx, const double *theta_bar, double *theta_prime, double *mass, double *energy)
{
    if (!ctx) return GEA_ERR_INVAL;
    if (!ctx->have_state) return fail3(ctx, GEA_ERR_STATE, "no state set");
    if (theta_prime && !theta_bar) return fail3(ctx, GEA_ERR_INVAL, "theta_prime needs theta_bar");
    Sc h;
    CK3(cudaMemcpyAsync(&h, ctx->sc, sizeof(Sc), cudaMemcpyDeviceToHost, ctx->stream));
    CK3(cudaStreamSynchronize(ctx->stream));
    const St &S = ctx->S[h.steps_done & 1];
    const Geo &G = ctx->G;
    const size_t cells = (size_t)G.nx * G.ny * G.nz;
    // the staging area (5 dense fields) holds theta_bar, then theta'
    double *thb = ctx->stage, *tho = ctx->stage + cells;
    if (theta_bar) CK3(cudaMemcpyAsync(thb, theta_bar, G.nz * sizeof(double), cudaMemcpyDefault, ctx->stream));
    k_diag3<<<grid_of(G), kBlk, 0, ctx->stream>>>(G, ctx->F, ctx->C.p0, S, thb, ctx->gz,
                                                  theta_prime ? tho : nullptr, ctx->sc, ctx->part);
    CK3(cudaGetLastError());
    if (theta_prime)
        CK3(cudaMemcpyAsync(theta_prime, tho, cells * sizeof(double), cudaMemcpyDefault, ctx->stream));
    CK3(cudaMemcpyAsync(&h, ctx->sc, sizeof(Sc), cudaMemcpyDeviceToHost, ctx->stream));
    CK3(cudaStreamSynchronize(ctx->stream));
    if (mass) *mass = h.mass;
    if (energy) *energy = h.energy;
    return GEA_OK;
}

int gea3d_get_stats(gea3d_ctx *ctx, gea_stats *s)
{
    if (!ctx || !s) return GEA_ERR_INVAL;
    Sc h;
    CK3(cudaMemcpyAsync(&h, ctx->sc, sizeof(Sc), cudaMemcpyDeviceToHost, ctx->stream));
    CK3(cudaStreamSynchronize(ctx->stream));
    memset(s, 0, sizeof(*s));
    s->steps_done = h.steps_done;
    s->jac_u = h.last_sweeps[0];
    s->jac_h = h.last_sweeps[1];
    for (int c = 0; c < 4; ++c) { s->cg_iters[c] = h.last_cg_iters[c]; s->cg_relres[c] = h.last_cg_relres[c]; }
    s->status = h.last_status;
    s->mg_levels = (int)ctx->M.size();
    s->launches = h.launches;
    s->driver = ctx->mixed ? 2 : 0;
    return GEA_OK;
}

int gea3d_profile_step(gea3d_ctx *ctx, gea_kernel_time *out, int32_t max_entries, int32_t *n_entries)
{
    if (!ctx || max_entries < 0 || (!out && max_entries > 0) || !n_entries) return GEA_ERR_INVAL;
    if (!ctx->have_state) return fail3(ctx, GEA_ERR_STATE, "no state set");
    Sc h;
    CK3(cudaMemcpyAsync(&h, ctx->sc, sizeof(Sc), cudaMemcpyDeviceToHost, ctx->stream));
    CK3(cudaStreamSynchronize(ctx->stream));
    if (h.status) return fail3(ctx, h.status, "device status %d", h.status);
    {
        Trace3 tr;
        tr.dsc = ctx->sc;
        const int rc = record3(ctx, (int)(h.steps_done & 1), ctx->stream, false, &tr);
        if (rc) return rc;
        CK3(cudaStreamSynchronize(ctx->stream));
        std::vector<gea_kernel_time> agg;
        for (auto &r : tr.recs) {
            float ms = 0.f;
            CK3(cudaEventElapsedTime(&ms, r.e0, r.e1));
            size_t j = 0;
            while (j < agg.size() && strcmp(agg[j].name, r.name)) ++j;
            if (j == agg.size()) {
                gea_kernel_time k;
                memset(&k, 0, sizeof(k));
                snprintf(k.name, sizeof(k.name), "%s", r.name);
                agg.push_back(k);
            }
            agg[j].launches += 1;
            agg[j].cells += r.cells;
            agg[j].ms += ms;
        }
        *n_entries = (int32_t)agg.size();
        for (size_t j = 0; j < agg.size() && (int32_t)j < max_entries; ++j) out[j] = agg[j];
    }
    return gea3d_sync(ctx);
}

const char *gea3d_last_error(const gea3d_ctx *ctx) { return ctx ? ctx->err : "null context"; }

void gea3d_destroy(gea3d_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    for (int f = 0; f < 2; ++f) {
        if (ctx->exec[f]) cudaGraphExecDestroy(ctx->exec[f]);
        if (ctx->graph[f]) cudaGraphDestroy(ctx->graph[f]);
    }
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->cap2) cudaStreamDestroy(ctx->cap2);
    for (void *p : ctx->allocs) cudaFree(p);
    delete ctx;
}

}  // extern "C"
