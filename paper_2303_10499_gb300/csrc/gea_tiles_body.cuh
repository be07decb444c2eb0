// gea_tiles_body.cuh -- the phases of one time step of the GEA
// pressure-based Euler solver (Girfoglio, Quaini & Rozza, arXiv 2303.10499,
// Section 3) as tile-level device functions. A tile is BX x BZ cells, one
// per thread of a BX x BZ block of NTHREADS = 256 threads; (bx, bz) are the
// tile's coordinates. Both the per-phase kernels (gea_kernels.cu) and the
// persistent step kernels (gea_persistent_body.cuh) run these functions; the
// persistent kernel walks the tiles of a phase in a block-stride loop and
// separates phases with grid barriers.
//
// This file has no include guard and no namespace of its own: it is
// included inside one namespace per tile shape, where BX and BZ name the
// shape (gea_tiles.cuh: namespace gea::tiles, the 32 x 8 tile of the
// per-phase kernels; gea_persistent_*.cu: one namespace per shape of the
// persistent kernels, whose shape the tile-shape autotuner picks).
//
// GB300 executes FP64 at 1/64 of its FP32 rate (two FP64 lanes per SM per
// clock, about 1.2 TFLOP/s) while HBM delivers about 6.8 TB/s, so every phase
// is FP64-issue-bound. The functions execute as few FP64 instructions as
// possible and spend loads, integer and shared-memory work instead:
//  - neighbour values come from a shared-memory tile with a halo, wall ghosts
//    filled while loading, so the arithmetic has no boundary branches;
//  - the implicit transport operator of Steps 1-2 is assembled once per step
//    as a 9-point stencil; a Jacobi sweep and H(u) are 9 FMAs per component;
//  - the Helmholtz operator is kept as d x - sum a x_N with omega/d stored;
//    values needed at neighbours are computed once per tile cell;
//  - divisions are done once per step into stored reciprocals.
// Global reads go through L2 (ld.global.cg): within one persistent launch a
// buffer is rewritten by other blocks between phases, and L1 is not coherent
// across SMs.
//
// Shared memory: each function takes `sm`, a block-wide scratch area of at
// least kTileSmem doubles, and ends with a __syncthreads() so the next tile
// can reuse it. Reduction contributions are added to the caller's per-thread
// accumulators.
static_assert(BX * BZ == NTHREADS && BX % 2 == 0 && BZ % 2 == 0,
              "a tile is NTHREADS cells with even sides (2 x 2 restriction within a tile)");

template <int H, class R = double>
using Tile = R[BZ + 2 * H][BX + 2 * H];

constexpr int kT1 = (BZ + 2) * (BX + 2);   // doubles of a halo-1 tile
constexpr int kT2 = (BZ + 4) * (BX + 4);   // doubles of a halo-2 tile
constexpr int cmax(int a, int b) { return a > b ? a : b; }
// the largest phase footprint: four halo-1 tiles (pressure right-hand
// side), three halo-2 tiles (enthalpy right-hand side), two halo-1 tiles and
// the x- and z-face rows (EOS, correction) or a tile of residuals (restriction)
constexpr int kTileSmem =
    cmax(cmax(4 * kT1, 3 * kT2), 2 * kT1 + cmax(BZ * (BX + 1) + (BZ + 1) * BX, BZ * BX));

template <int H, class R = double>
__device__ __forceinline__ Tile<H, R> &tile_at(double *sm, int slot)
{
    return *reinterpret_cast<Tile<H, R> *>(reinterpret_cast<R *>(sm) + slot * (BZ + 2 * H) * (BX + 2 * H));
}

__device__ __forceinline__ double ld(const double *p) { return __ldcg(p); }
__device__ __forceinline__ float ld(const float *p) { return __ldcg(p); }

__device__ __forceinline__ bool cell_of(const Geom &G, int bx, int bz, int &i, int &k)
{
    i = bx * BX + threadIdx.x;
    k = bz * BZ + threadIdx.y;
    return i < G.nx && k < G.nz;
}

// Cell value at (i,k) just outside the box: the one-layer wall ghost of rule
// BC (wall-normal velocity odd, tangential velocity and scalars even, h with
// dh/dz = -g at the horizontal walls).
template <int BC, class R>
__device__ __forceinline__ R ghost(const Geom &G, const Phys &F, const R *X, int i, int k)
{
    if (i < 0) {
        const R v = ld(&X[k * G.P]);
        return BC == BC_U ? -v : v;
    }
    if (i >= G.nx) {
        const R v = ld(&X[k * G.P + G.nx - 1]);
        return BC == BC_U ? -v : v;
    }
    if (k < 0) {
        const R v = ld(&X[i]);
        if (BC == BC_W) return -v;
        if (BC == BC_H) return v + (R)(F.g * G.dz);
        return v;
    }
    const R v = ld(&X[(G.nz - 1) * G.P + i]);
    if (BC == BC_W) return -v;
    if (BC == BC_H) return v - (R)(F.g * G.dz);
    return v;
}

// Fill the (BZ+2H) x (BX+2H) tile of X around tile (bx, bz): cells inside the
// box, the one-layer wall ghosts of rule BC, zero elsewhere (deeper ghosts and
// corners only ever meet zero coefficients).
template <int BC, int H, class R>
__device__ __forceinline__ void load_tile(Tile<H, R> &s, const Geom &G, const Phys &F, const R *X,
                                          int bx, int bz)
{
    const int i0 = bx * BX - H, k0 = bz * BZ - H;
    // h differs from an even field only in its ghost rows below and above
    // the box; a tile that reaches neither (block-uniform test) loads it as
    // even, without the ghost offset's FP64 arithmetic in the loop
    if constexpr (BC == BC_H) {
        if (k0 >= 0 && k0 + BZ + 2 * H <= G.nz) {
            load_tile<BC_EVEN, H, R>(s, G, F, X, bx, bz);
            return;
        }
    }
    const int tid = threadIdx.x + threadIdx.y * BX;
    constexpr int W = BX + 2 * H, NE = (BZ + 2 * H) * (BX + 2 * H);
    for (int e = tid; e < NE; e += NTHREADS) {
        const int tk = e / W, ti = e - tk * W;
        const int i = i0 + ti, k = k0 + tk;
        const bool xin = i >= 0 && i < G.nx, zin = k >= 0 && k < G.nz;
        R v = 0;
        if (xin && zin) v = ld(&X[k * G.P + i]);
        else if (zin && (i == -1 || i == G.nx)) v = ghost<BC>(G, F, X, i, k);
        else if (xin && (k == -1 || k == G.nz)) v = ghost<BC>(G, F, X, i, k);
        s[tk][ti] = v;
    }
}

// Tile of X + Y (FP64 field plus FP32 increment with the same wall rule).
template <int BC, int H>
__device__ __forceinline__ void load_tile_sum(Tile<H> &s, const Geom &G, const Phys &F, const double *X,
                                              const float *Y, int bx, int bz)
{
    const int i0 = bx * BX - H, k0 = bz * BZ - H;
    const int tid = threadIdx.x + threadIdx.y * BX;
    constexpr int W = BX + 2 * H, NE = (BZ + 2 * H) * (BX + 2 * H);
    for (int e = tid; e < NE; e += NTHREADS) {
        const int tk = e / W, ti = e - tk * W;
        const int i = i0 + ti, k = k0 + tk;
        const bool xin = i >= 0 && i < G.nx, zin = k >= 0 && k < G.nz;
        double v = 0.0;
        if (xin && zin) v = ld(&X[k * G.P + i]) + (double)ld(&Y[k * G.P + i]);
        else if ((zin && (i == -1 || i == G.nx)) || (xin && (k == -1 || k == G.nz)))
            v = ghost<BC>(G, F, X, i, k) + (double)ghost<BC == BC_H ? BC_EVEN : BC>(G, F, Y, i, k);
        s[tk][ti] = v;
    }
}

// Same for a field given by f(q, i, k) at cell (i, k), index q (zero outside
// the box).
template <int H, class R, class Fn>
__device__ __forceinline__ void load_tile_fn(Tile<H, R> &s, const Geom &G, int bx, int bz, Fn f)
{
    const int i0 = bx * BX - H, k0 = bz * BZ - H;
    const int tid = threadIdx.x + threadIdx.y * BX;
    constexpr int W = BX + 2 * H, NE = (BZ + 2 * H) * (BX + 2 * H);
    for (int e = tid; e < NE; e += NTHREADS) {
        const int tk = e / W, ti = e - tk * W;
        const int i = i0 + ti, k = k0 + tk;
        s[tk][ti] = (i >= 0 && i < G.nx && k >= 0 && k < G.nz) ? (R)f(k * G.P + i, i, k) : (R)0;
    }
}

// Y = X on the tile's cells.
template <class R>
__device__ __forceinline__ void ph_copy(const Geom &G, const R *X, R *Y, int bx, int bz)
{
    int i, k;
    if (cell_of(G, bx, bz, i, k)) Y[cidx(G, i, k)] = ld(&X[cidx(G, i, k)]);
}

// 9-point cross stencil sum_o c_o X_o at tile position (y, x).
template <int H, class R>
__device__ __forceinline__ R apply9(const Stencil9T<R> &T, int q, const Tile<H, R> &s, int y, int x)
{
    R acc = ld(&T.cC[q]) * s[y][x];
    acc = fma(ld(&T.cE1[q]), s[y][x + 1], acc);
    acc = fma(ld(&T.cW1[q]), s[y][x - 1], acc);
    acc = fma(ld(&T.cN1[q]), s[y + 1][x], acc);
    acc = fma(ld(&T.cS1[q]), s[y - 1][x], acc);
    acc = fma(ld(&T.cE2[q]), s[y][x + 2], acc);
    acc = fma(ld(&T.cW2[q]), s[y][x - 2], acc);
    acc = fma(ld(&T.cN2[q]), s[y + 2][x], acc);
    acc = fma(ld(&T.cS2[q]), s[y - 2][x], acc);
    return acc;
}

// 5-point Laplacian (X_E + X_W - 2 X_C)/dx^2 + (X_N + X_S - 2 X_C)/dz^2.
template <int H, class R>
__device__ __forceinline__ R lap5(const Geom &G, const Tile<H, R> &s, int y, int x)
{
    const R c2 = (R)2 * s[y][x];
    return (s[y][x + 1] + s[y][x - 1] - c2) * (R)(G.idx * G.idx) +
           (s[y + 1][x] + s[y - 1][x] - c2) * (R)(G.idz * G.idz);
}

// A x = d x - sum a x_N at tile position (y, x) of cell (i, k) (zero tile
// entries and zero wall coefficients beyond the box).
template <int H, class R>
__device__ __forceinline__ R helm_tile(const LevelT<R> &L, int q, int i, int k, const Tile<H, R> &s,
                                       int y, int x)
{
    const Geom &G = L.G;
    R t = ld(&L.d[q]) * s[y][x];
    t = fma(-ld(&L.ax[k * G.P + i]), s[y][x - 1], t);
    t = fma(-ld(&L.ax[k * G.P + i + 1]), s[y][x + 1], t);
    t = fma(-ld(&L.az[k * G.P + i]), s[y - 1][x], t);
    t = fma(-ld(&L.az[(k + 1) * G.P + i]), s[y + 1][x], t);
    return t;
}

// The coefficients of the Helmholtz operator at a cell. With kPrefetch (set
// by the includer: the persistent kernels, whose occupancy the register
// file already fixes at three blocks per SM) the phases load a cell's own
// coefficients and inputs ahead of the tile barrier (they do not depend on
// the tile), so that their L2 latency overlaps the halo loads; without it
// (the per-phase kernels, where the extra live registers would cost
// occupancy) after the barrier. Two phases load early in every instance:
// the single-field Jacobi sweep and the CG direction update with A p, which
// measured faster that way in the per-phase kernels too (the 4096 x 2048
// enthalpy sweep went from 0.47 to 0.80 of the FP64 peak), while the
// two-field sweep, the multigrid phases and the right-hand sides lost
// occupancy and speed.
constexpr bool kPrefetchSweep1 = true;
constexpr bool kPrefetchSpmv = true;
template <class R>
struct HelmCoef {
    R d, aw, ae, as, an;
};

template <class R>
__device__ __forceinline__ HelmCoef<R> helm_coef(const LevelT<R> &L, int q, int i, int k)
{
    const Geom &G = L.G;
    return HelmCoef<R>{ld(&L.d[q]), ld(&L.ax[k * G.P + i]), ld(&L.ax[k * G.P + i + 1]), ld(&L.az[k * G.P + i]),
                       ld(&L.az[(k + 1) * G.P + i])};
}

// A x = d x - sum a x_N from preloaded coefficients (helm_tile's order).
template <int H, class R>
__device__ __forceinline__ R helm_apply(const HelmCoef<R> &c, const Tile<H, R> &s, int y, int x)
{
    R t = c.d * s[y][x];
    t = fma(-c.aw, s[y][x - 1], t);
    t = fma(-c.ae, s[y][x + 1], t);
    t = fma(-c.as, s[y - 1][x], t);
    t = fma(-c.an, s[y + 1][x], t);
    return t;
}

// The nine stencil weights of the transport operator at a cell, likewise
// loaded ahead of the tile barrier.
template <class R>
struct Coef9 {
    R cC, cE1, cW1, cN1, cS1, cE2, cW2, cN2, cS2;
};

template <class R>
__device__ __forceinline__ Coef9<R> coef9(const Stencil9T<R> &T, int q)
{
    return Coef9<R>{ld(&T.cC[q]),  ld(&T.cE1[q]), ld(&T.cW1[q]), ld(&T.cN1[q]), ld(&T.cS1[q]),
                    ld(&T.cE2[q]), ld(&T.cW2[q]), ld(&T.cN2[q]), ld(&T.cS2[q])};
}

// sum_o c_o X_o in apply9's order.
template <int H, class R>
__device__ __forceinline__ R apply9c(const Coef9<R> &c, const Tile<H, R> &s, int y, int x)
{
    R acc = c.cC * s[y][x];
    acc = fma(c.cE1, s[y][x + 1], acc);
    acc = fma(c.cW1, s[y][x - 1], acc);
    acc = fma(c.cN1, s[y + 1][x], acc);
    acc = fma(c.cS1, s[y - 1][x], acc);
    acc = fma(c.cE2, s[y][x + 2], acc);
    acc = fma(c.cW2, s[y][x - 2], acc);
    acc = fma(c.cN2, s[y + 2][x], acc);
    acc = fma(c.cS2, s[y - 2][x], acc);
    return acc;
}

// ---------------------------------------------------------------------------
// Smagorinsky eddy viscosity (LES): mu_eff = mu + rho (cs Delta)^2 |S| from
// rho^n and u^n, |S|^2 = 2 (du/dx)^2 + 2 (dw/dz)^2 + (du/dz + dw/dx)^2 with
// central differences (ghosts by the wall rules)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ph_les(const StepArgs &a, double *sm, int bx, int bz)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    Tile<1> &su = tile_at<1>(sm, 0), &sw = tile_at<1>(sm, 1);
    load_tile<BC_U, 1>(su, G, F, a.S.u, bx, bz);
    load_tile<BC_W, 1>(sw, G, F, a.S.w, bx, bz);
    __syncthreads();
    int i, k;
    if (cell_of(G, bx, bz, i, k)) {
        const int q = cidx(G, i, k);
        const int y = threadIdx.y + 1, x = threadIdx.x + 1;
        const double hx = 0.5 * G.idx, hz = 0.5 * G.idz;
        const double dudx = (su[y][x + 1] - su[y][x - 1]) * hx, dudz = (su[y + 1][x] - su[y - 1][x]) * hz;
        const double dwdx = (sw[y][x + 1] - sw[y][x - 1]) * hx, dwdz = (sw[y + 1][x] - sw[y - 1][x]) * hz;
        const double sh = dudz + dwdx;
        const double S = sqrt(2.0 * dudx * dudx + 2.0 * dwdz * dwdz + sh * sh);
        a.mueff[q] = fma(ld(&a.S.rho[q]) * F.les_d2, S, F.mu);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Step 1 (eq. e1_d and eq. step2_sd, first line)
// ---------------------------------------------------------------------------

// rho^{n+1/3} = rho^n - dt sum_j phi_j / V; the transport operator
//   T(X) = (rho1/dt) X + C(X) - mu L(X)
// as a 9-point stencil: the east face contributes f_e (-X_W1 + 7 X_C + 7 X_E1
// - X_E2) with f_e = phi_e / (12 V), the west face -f_w (-X_W2 + 7 X_W1 + 7 X_C
// - X_E1), likewise in z, and -mu L adds 2 mu (1/dx^2 + 1/dz^2) at the centre
// and -mu/dx^2, -mu/dz^2 at the nearest neighbours; the Jacobi reciprocals of
// the momentum (mu) and enthalpy (mu/Pr) diagonals; b = rho^n u^n / dt - G_cell^n
// with G_cell the average of the two face forces grad p'^n - g z grad rho^n
// per direction (zero on wall faces); the initial guess u^n.
// acc += (b_u^2, b_w^2).
//
// MX (mixed-precision path): instead of b, the reciprocals and the initial
// guess, the FP64 residuals r0 = b - T(u^n) of both components, FP32 copies
// of the operator, the reciprocals and r0, and the first FP32 Jacobi sweep
// from zero, du = r0 / T_CC; acc += (r0_u^2, r0_w^2).
//
// SW1 (FP64): also the first Jacobi sweep of the momentum predictor from the
// guess u^n, r0 = b - T(u^n), u = u^n + r0 / T_CC into ua, wa (the stencil of
// the cell is at hand and u^n needs no barrier); acc += (b_u^2, b_w^2,
// r0_u^2, r0_w^2).
template <bool MX, bool SW1 = false>
__device__ __forceinline__ void ph_pred_t(const StepArgs &a, const MixedArgs &m, double *sm, int bx,
                                          int bz, double (&acc)[SW1 ? 4 : 2])
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    const State &S = a.S;
    if (MX || SW1) {
        load_tile<BC_U, 2>(tile_at<2>(sm, 0), G, F, S.u, bx, bz);
        load_tile<BC_W, 2>(tile_at<2>(sm, 1), G, F, S.w, bx, bz);
        __syncthreads();
    }
    int i, k;
    if (cell_of(G, bx, bz, i, k)) {
        const int q = cidx(G, i, k);
        const double pw = ld(&S.phix[q]), pe = ld(&S.phix[q + 1]), ps = ld(&S.phiz[q]), pn = ld(&S.phiz[q + G.P]);
        const double div = (pe - pw + pn - ps) * G.iV;
        const double rq = ld(&S.rho[q]);
        const double rho1 = rq - F.dt * div;
        const double s12 = G.iV * (1.0 / 12.0);
        const double fe = pe * s12, fw = pw * s12, fn = pn * s12, fs = ps * s12;
        // diffusion: mu/dx^2 per face, or with LES the face mean of mu_eff
        // (a wall face takes the cell's own)
        double me, mw, mn, ms;
        if (F.les) {
            const double mc = ld(&a.mueff[q]);
            const double ix2 = 0.5 * G.idx * G.idx, iz2 = 0.5 * G.idz * G.idz;
            me = (mc + (i + 1 < G.nx ? ld(&a.mueff[q + 1]) : mc)) * ix2;
            mw = (mc + (i > 0 ? ld(&a.mueff[q - 1]) : mc)) * ix2;
            mn = (mc + (k + 1 < G.nz ? ld(&a.mueff[q + G.P]) : mc)) * iz2;
            ms = (mc + (k > 0 ? ld(&a.mueff[q - G.P]) : mc)) * iz2;
        } else {
            me = mw = F.mu * G.idx * G.idx;
            mn = ms = F.mu * G.idz * G.idz;
        }
        const double cC = rho1 * F.idt + (7.0 / 12.0) * div + ((me + mw) + (mn + ms));
        const double cE1 = fma(7.0, fe, fw) - me, cW1 = -fma(7.0, fw, fe) - mw;
        const double cN1 = fma(7.0, fn, fs) - mn, cS1 = -fma(7.0, fs, fn) - ms;
        const double cE2 = -fe, cW2 = fw, cN2 = -fn, cS2 = fs;
        a.T.cC[q] = cC;
        a.T.cE1[q] = cE1;
        a.T.cW1[q] = cW1;
        a.T.cE2[q] = cE2;
        a.T.cW2[q] = cW2;
        a.T.cN1[q] = cN1;
        a.T.cS1[q] = cS1;
        a.T.cN2[q] = cN2;
        a.T.cS2[q] = cS2;
        const double diu = 1.0 / cC;
        const double dih =
            F.pr_ne1 ? 1.0 / (cC + 2.0 * (F.nuh - F.mu) * (G.idx * G.idx + G.idz * G.idz)) : diu;
        if (!MX) {
            a.dinvu[q] = diu;
            a.dinvh[q] = dih;
        }
        // face forces (p'_b - p'_a - g z_f (rho_b - rho_a)) / Delta; the cell
        // and face heights g z come from per-row tables
        const double gz = ld(&a.gzc[k]);
        const double pq = ld(&S.pp[q]);
        double gxw = 0.0, gxe = 0.0, gzs = 0.0, gzn = 0.0;
        if (i > 0) gxw = fma(-gz, rq - ld(&S.rho[q - 1]), pq - ld(&S.pp[q - 1])) * G.idx;
        if (i + 1 < G.nx) gxe = fma(-gz, ld(&S.rho[q + 1]) - rq, ld(&S.pp[q + 1]) - pq) * G.idx;
        if (k > 0) gzs = fma(-ld(&a.gzf[k]), rq - ld(&S.rho[q - G.P]), pq - ld(&S.pp[q - G.P])) * G.idz;
        if (k + 1 < G.nz)
            gzn = fma(-ld(&a.gzf[k + 1]), ld(&S.rho[q + G.P]) - rq, ld(&S.pp[q + G.P]) - pq) * G.idz;
        const double u = ld(&S.u[q]), w = ld(&S.w[q]);
        const double bu = rq * u * F.idt - 0.5 * (gxw + gxe);
        const double bw = rq * w * F.idt - 0.5 * (gzs + gzn);
        a.rho1[q] = rho1;
        a.dtr1[q] = F.dt / rho1;
        const int y = threadIdx.y + 2, x = threadIdx.x + 2;
        // T(X) at the cell from a halo-2 tile, in apply9's order
        auto t9 = [&](const Tile<2> &t) {
            double v = cC * t[y][x];
            v = fma(cE1, t[y][x + 1], v);
            v = fma(cW1, t[y][x - 1], v);
            v = fma(cN1, t[y + 1][x], v);
            v = fma(cS1, t[y - 1][x], v);
            v = fma(cE2, t[y][x + 2], v);
            v = fma(cW2, t[y][x - 2], v);
            v = fma(cN2, t[y + 2][x], v);
            v = fma(cS2, t[y - 2][x], v);
            return v;
        };
        if (!MX) {
            a.bu[q] = bu;
            a.bw[q] = bw;
            acc[0] = fma(bu, bu, acc[0]);
            acc[1] = fma(bw, bw, acc[1]);
            if (SW1) {
                const double r0u = bu - t9(tile_at<2>(sm, 0)), r0w = bw - t9(tile_at<2>(sm, 1));
                a.ua[q] = fma(r0u, diu, u);
                a.wa[q] = fma(r0w, diu, w);
                acc[SW1 ? 2 : 0] = fma(r0u, r0u, acc[SW1 ? 2 : 0]);
                acc[SW1 ? 3 : 1] = fma(r0w, r0w, acc[SW1 ? 3 : 1]);
            } else {
                a.ua[q] = u;
                a.wa[q] = w;
            }
        } else {
            const double r0u = bu - t9(tile_at<2>(sm, 0)), r0w = bw - t9(tile_at<2>(sm, 1));
            m.T.cC[q] = (float)cC;
            m.T.cE1[q] = (float)cE1;
            m.T.cW1[q] = (float)cW1;
            m.T.cE2[q] = (float)cE2;
            m.T.cW2[q] = (float)cW2;
            m.T.cN1[q] = (float)cN1;
            m.T.cS1[q] = (float)cS1;
            m.T.cN2[q] = (float)cN2;
            m.T.cS2[q] = (float)cS2;
            const float fdiu = (float)diu;
            m.dinvu[q] = fdiu;
            m.dinvh[q] = (float)dih;
            const float fru = (float)r0u, frw = (float)r0w;
            m.r0u[q] = fru;
            m.r0w[q] = frw;
            m.du[0][q] = fru * fdiu;
            m.dw[0][q] = frw * fdiu;
            acc[0] = fma(r0u, r0u, acc[0]);
            acc[1] = fma(r0w, r0w, acc[1]);
        }
    }
    if (MX || SW1) __syncthreads();
}

__device__ __forceinline__ void ph_pred(const StepArgs &a, int bx, int bz, double (&acc)[2])
{
    ph_pred_t<false>(a, MixedArgs{}, nullptr, bx, bz, acc);
}

__device__ __forceinline__ void ph_pred_sweep(const StepArgs &a, double *sm, int bx, int bz, double (&acc)[4])
{
    ph_pred_t<false, true>(a, MixedArgs{}, sm, bx, bz, acc);
}

// One Jacobi sweep of T(X) = b for two fields with wall rules BCA, BCB:
// r = b - T(X), X <- X + r / T_CC. acc += (r_a^2, r_b^2).
template <class R, int BCA, int BCB>
__device__ __forceinline__ void ph_sweep2(const Geom &G, const Phys &F, const Stencil9T<R> &T,
                                          const R *dinv, const R *ba, const R *bb, const R *xa,
                                          const R *xb, R *ya, R *yb, double *sm, int bx, int bz,
                                          R (&acc)[2])
{
    Tile<2, R> &sa = tile_at<2, R>(sm, 0), &sb = tile_at<2, R>(sm, 1);
    int i, k;
    const bool in = cell_of(G, bx, bz, i, k);
    const int q = in ? cidx(G, i, k) : 0;
    Coef9<R> c{};
    R di = 0, bva = 0, bvb = 0;
    auto fetch = [&] {
        c = coef9(T, q);
        di = ld(&dinv[q]);
        bva = ld(&ba[q]);
        bvb = ld(&bb[q]);
    };
    if (kPrefetch && in) fetch();
    load_tile<BCA, 2, R>(sa, G, F, xa, bx, bz);
    load_tile<BCB, 2, R>(sb, G, F, xb, bx, bz);
    __syncthreads();
    if (in) {
        if (!kPrefetch) fetch();
        const int y = threadIdx.y + 2, x = threadIdx.x + 2;
        const R ra = bva - apply9c<2, R>(c, sa, y, x);
        const R rb = bvb - apply9c<2, R>(c, sb, y, x);
        ya[q] = fma(ra, di, sa[y][x]);
        yb[q] = fma(rb, di, sb[y][x]);
        acc[0] = fma(ra, ra, acc[0]);
        acc[1] = fma(rb, rb, acc[1]);
    }
    __syncthreads();
}

// One Jacobi sweep of T(X) + lc L(X) = b for one field with wall rule BC
// (lc = mu - mu/Pr turns the momentum stencil into the enthalpy one).
// acc += r^2.
template <class R, int BC>
__device__ __forceinline__ void ph_sweep1(const Geom &G, const Phys &F, const Stencil9T<R> &T,
                                          const R *dinv, const R *bv, R lc, const R *xin, R *xout,
                                          double *sm, int bx, int bz, R (&acc)[1])
// (lc is used when F.pr_ne1, i.e. mu/Pr != mu)
{
    Tile<2, R> &sh = tile_at<2, R>(sm, 0);
    int i, k;
    const bool in = cell_of(G, bx, bz, i, k);
    const int q = in ? cidx(G, i, k) : 0;
    Coef9<R> c{};
    R di = 0, bq = 0;
    auto fetch = [&] {
        c = coef9(T, q);
        di = ld(&dinv[q]);
        bq = ld(&bv[q]);
    };
    if (kPrefetchSweep1 && in) fetch();
    load_tile<BC, 2, R>(sh, G, F, xin, bx, bz);
    __syncthreads();
    if (in) {
        if (!kPrefetchSweep1) fetch();
        const int y = threadIdx.y + 2, x = threadIdx.x + 2;
        R t = apply9c<2, R>(c, sh, y, x);
        if (F.pr_ne1) t = fma(lc, lap5<2, R>(G, sh, y, x), t);
        const R r = bq - t;
        xout[q] = fma(r, di, sh[y][x]);
        acc[0] = fma(r, r, acc[0]);
    }
    __syncthreads();
}

// Momentum predictor sweep: u odd in x, w odd in z.
__device__ __forceinline__ void ph_mom(const StepArgs &a, const double *uin, const double *win,
                                       double *uout, double *wout, double *sm, int bx, int bz,
                                       double (&acc)[2])
{
    ph_sweep2<double, BC_U, BC_W>(a.G, a.F, a.T, a.dinvu, a.bu, a.bw, uin, win, uout, wout, sm, bx,
                                  bz, acc);
}

// ---------------------------------------------------------------------------
// Step 2 (eq. step3_sd, step3_2sd, step3_3sd)
// ---------------------------------------------------------------------------

// Right-hand side of the enthalpy equation:
//   (rho^n h^n + rho^n K^n - p^{n-1})/dt - rho1 K1/dt - C(K1) + p^n/dt - rho1 g w1
// with K1 = |u^{n+1/3}|^2/2 (eq. step1_3sd); initial guess h^n (into h0).
// acc += b_h^2.
// MX: u^{n+1/3} = u^n + du (written to ua, wa), and instead of b_h and h0 the
// FP64 residual r0 = b_h - T_h(h^n) (h^n with its wall rule), its FP32 copy
// and the first FP32 sweep dh = r0 / T_h,CC; acc += r0^2 instead.
// SW1 (FP64): h0 receives the first Jacobi sweep from h^n instead of h^n,
// r0 = b_h - T_h(h^n), h = h^n + r0 / T_h,CC; acc += (b_h^2, r0^2).
template <bool MX, bool SW1 = false>
__device__ __forceinline__ void ph_enth_rhs_t(const StepArgs &a, const MixedArgs &m, const double *u1,
                                              const double *w1, double *h0, double *sm, int bx,
                                              int bz, double (&acc)[SW1 ? 2 : 1])
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    const State &S = a.S;
    Tile<2> &su = tile_at<2>(sm, 0), &sw = tile_at<2>(sm, 1);
    if (MX) {
        load_tile_sum<BC_U, 2>(su, G, F, S.u, m.du[0], bx, bz);
        load_tile_sum<BC_W, 2>(sw, G, F, S.w, m.dw[0], bx, bz);
        load_tile<BC_H, 2>(tile_at<2>(sm, 2), G, F, S.h, bx, bz);
    } else {
        load_tile<BC_U, 2>(su, G, F, u1, bx, bz);
        load_tile<BC_W, 2>(sw, G, F, w1, bx, bz);
        if (SW1) load_tile<BC_H, 2>(tile_at<2>(sm, 2), G, F, S.h, bx, bz);
    }
    __syncthreads();
    // K1 in place of u (ghost velocities give the mirrored cell's K); u1 and
    // w1 at the cell centre are kept aside first
    const double u1c = su[threadIdx.y + 2][threadIdx.x + 2], w1c = sw[threadIdx.y + 2][threadIdx.x + 2];
    __syncthreads();
    {
        const int tid = threadIdx.x + threadIdx.y * BX;
        for (int e = tid; e < kT2; e += NTHREADS) {
            const int tk = e / (BX + 4), ti = e - tk * (BX + 4);
            su[tk][ti] = 0.5 * (su[tk][ti] * su[tk][ti] + sw[tk][ti] * sw[tk][ti]);
        }
    }
    __syncthreads();
    int i, k;
    if (cell_of(G, bx, bz, i, k)) {
        const int q = cidx(G, i, k);
        const int y = threadIdx.y + 2, x = threadIdx.x + 2;
        const Tile<2> &K = su;
        // convective sum of K1 with the four-point face values (wall faces
        // carry phi = 0)
        double c = ld(&S.phix[q + 1]) * (7.0 * (K[y][x] + K[y][x + 1]) - (K[y][x - 1] + K[y][x + 2]));
        c -= ld(&S.phix[q]) * (7.0 * (K[y][x - 1] + K[y][x]) - (K[y][x - 2] + K[y][x + 1]));
        c += ld(&S.phiz[q + G.P]) * (7.0 * (K[y][x] + K[y + 1][x]) - (K[y - 1][x] + K[y + 2][x]));
        c -= ld(&S.phiz[q]) * (7.0 * (K[y - 1][x] + K[y][x]) - (K[y - 2][x] + K[y + 1][x]));
        c *= G.iV * (1.0 / 12.0);
        const double rq = ld(&S.rho[q]), u = ld(&S.u[q]), w = ld(&S.w[q]), h = ld(&S.h[q]);
        // b~_e carries rho^n K^n, or rho^n K^{n-1} in the literal reading
        const double Kn = F.k_lagged ? ld(&S.Kold[q]) : 0.5 * (u * u + w * w);
        const double rho1 = ld(&a.rho1[q]);
        const double be = (rq * h + rq * Kn - ld(&S.pold[q])) * F.idt;
        const double bh = be - rho1 * K[y][x] * F.idt - c + ld(&S.p[q]) * F.idt - rho1 * F.g * w1c;
        if (!MX) {
            a.bh[q] = bh;
            acc[0] = fma(bh, bh, acc[0]);
            if (SW1) {
                const Tile<2> &sh = tile_at<2>(sm, 2);
                double t = apply9<2>(a.T, q, sh, y, x);
                if (F.pr_ne1) t = fma(F.mu - F.nuh, lap5<2>(G, sh, y, x), t);
                const double r0 = bh - t;
                h0[q] = fma(r0, ld(&a.dinvh[q]), sh[y][x]);
                acc[SW1 ? 1 : 0] = fma(r0, r0, acc[SW1 ? 1 : 0]);
            } else {
                h0[q] = h;
            }
        } else {
            a.ua[q] = u1c;
            a.wa[q] = w1c;
            const Tile<2> &sh = tile_at<2>(sm, 2);
            double t = apply9<2>(a.T, q, sh, y, x);
            if (F.pr_ne1) t = fma(F.mu - F.nuh, lap5<2>(G, sh, y, x), t);
            const double r0 = bh - t;
            const float fr = (float)r0;
            m.r0h[q] = fr;
            m.dh[0][q] = fr * ld(&m.dinvh[q]);
            acc[0] = fma(r0, r0, acc[0]);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void ph_enth_rhs(const StepArgs &a, const double *u1, const double *w1,
                                            double *h0, double *sm, int bx, int bz, double (&acc)[1])
{
    ph_enth_rhs_t<false>(a, MixedArgs{}, u1, w1, h0, sm, bx, bz, acc);
}

__device__ __forceinline__ void ph_enth_rhs_sweep(const StepArgs &a, const double *u1, const double *w1,
                                                  double *h0, double *sm, int bx, int bz, double (&acc)[2])
{
    ph_enth_rhs_t<false, true>(a, MixedArgs{}, u1, w1, h0, sm, bx, bz, acc);
}

// One Jacobi sweep of (rho1/dt) h + C(h) - (mu/Pr) L(h) = b_h (dh/dz = -g on
// the horizontal walls): the momentum stencil plus (mu - mu/Pr) L(h).
// acc += r^2.
__device__ __forceinline__ void ph_enth(const StepArgs &a, const double *hin, double *hout,
                                        double *sm, int bx, int bz, double (&acc)[1])
{
    ph_sweep1<double, BC_H>(a.G, a.F, a.T, a.dinvh, a.bh, a.F.mu - a.F.nuh, hin, hout, sm, bx, bz, acc);
}

// T^{n+1} = T^n + (h^{n+1} - h^n)/cp; psi = 1/(R T^{n+1}); rho^{n+2/3} = p^n/(R T^{n+1})
// (eq. step3_3sd); face coefficients D_f = dt rho2_f / rho1_f (linear face
// averages); the fine Helmholtz operator c = psi/dt, a_f = D_f |A_f|/(V Delta_f),
// d = c + sum a_f and omega/d. h1 holds h^{n+1}.
// MX: h^{n+1} = h^n + dh, and FP32 copies of the fine operator into L32.
template <bool MX>
__device__ __forceinline__ void ph_eos_t(const StepArgs &a, const Level &L, const LevelF &L32,
                                         const double *h1, const float *dh, double *sm, int bx, int bz)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    Tile<1> &s2 = tile_at<1>(sm, 0), &s1 = tile_at<1>(sm, 1);
    double(*fx)[BX + 1] = reinterpret_cast<double(*)[BX + 1]>(sm + 2 * kT1);
    double(*fz)[BX] = reinterpret_cast<double(*)[BX]>(sm + 2 * kT1 + BZ * (BX + 1));
    const State &S = a.S;
    const double icp = 1.0 / F.cp;
    auto h1_of = [&](int q) { return MX ? ld(&S.h[q]) + (double)ld(&dh[q]) : ld(&h1[q]); };
    load_tile_fn<1>(s2, G, bx, bz, [&](int q, int, int) {
        const double T1 = fma(h1_of(q) - ld(&S.h[q]), icp, ld(&S.T[q]));
        return ld(&S.p[q]) / (F.R * T1);
    });
    load_tile_fn<1>(s1, G, bx, bz, [&](int q, int, int) { return ld(&a.rho1[q]); });
    __syncthreads();
    int i, k;
    const bool in = cell_of(G, bx, bz, i, k);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int y = ty + 1, x = tx + 1;
    const double ix2 = G.idx * G.idx, iz2 = G.idz * G.idz;
    // dt rho2_f / rho1_f with linear face averages (the two halves cancel
    // exactly in binary)
    auto dface = [&](int ya, int xa, int yb, int xb) {
        return F.dt * (s2[ya][xa] + s2[yb][xb]) / (s1[ya][xa] + s1[yb][xb]);
    };
    if (in) {
        fx[ty][tx] = i > 0 ? dface(y, x - 1, y, x) : 0.0;
        fz[ty][tx] = k > 0 ? dface(y - 1, x, y, x) : 0.0;
        if (tx == BX - 1 || i == G.nx - 1) fx[ty][tx + 1] = i + 1 < G.nx ? dface(y, x, y, x + 1) : 0.0;
        if (ty == BZ - 1 || k == G.nz - 1) fz[ty + 1][tx] = k + 1 < G.nz ? dface(y, x, y + 1, x) : 0.0;
    }
    __syncthreads();
    if (in) {
        const int q = cidx(G, i, k);
        const double h1q = h1_of(q);
        const double T1 = fma(h1q - ld(&S.h[q]), icp, ld(&S.T[q]));
        const double psi = 1.0 / (F.R * T1);
        a.N.T[q] = T1;
        a.N.h[q] = h1q;
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
        if (MX) {
            L32.c[q] = (float)c;
            L32.d[q] = (float)d;
            L32.wd[q] = (float)(F.omega / d);
            L32.ax[k * G.P + i] = (float)(Dw * ix2);
            L32.az[k * G.P + i] = (float)(Ds * iz2);
            if (i == G.nx - 1) L32.ax[k * G.P + G.nx] = 0.0f;
            if (k == G.nz - 1) L32.az[G.nz * G.P + i] = 0.0f;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void ph_eos(const StepArgs &a, const Level &L, const double *h1,
                                       double *sm, int bx, int bz)
{
    ph_eos_t<false>(a, L, LevelF{}, h1, nullptr, sm, bx, bz);
}

// Galerkin coarsening with piecewise-constant transfer: the coarse reaction
// term averages the four fine ones, a coarse face coefficient is a quarter
// of the sum of its two fine faces. (bx, bz) is a tile of the coarse level.
template <class R>
__device__ __forceinline__ void ph_coarsen(const LevelT<R> &f, const LevelT<R> &c, double omega, int bx,
                                           int bz)
{
    const Geom &G = c.G;
    int I, K;
    if (!cell_of(G, bx, bz, I, K)) return;
    const int Pf = f.G.P;
    const int q00 = (2 * K) * Pf + 2 * I;
    const int Q = cidx(G, I, K);
    const R q4 = (R)0.25;
    const R cc = q4 * (ld(&f.c[q00]) + ld(&f.c[q00 + 1]) + ld(&f.c[q00 + Pf]) + ld(&f.c[q00 + Pf + 1]));
    const R aw = q4 * (ld(&f.ax[q00]) + ld(&f.ax[q00 + Pf]));
    const R ae = q4 * (ld(&f.ax[q00 + 2]) + ld(&f.ax[q00 + Pf + 2]));
    const R as = q4 * (ld(&f.az[q00]) + ld(&f.az[q00 + 1]));
    const R an = q4 * (ld(&f.az[q00 + 2 * Pf]) + ld(&f.az[q00 + 2 * Pf + 1]));
    c.c[Q] = cc;
    c.ax[K * G.P + I] = aw;
    c.az[K * G.P + I] = as;
    if (I == G.nx - 1) c.ax[K * G.P + G.nx] = ae;
    if (K == G.nz - 1) c.az[G.nz * G.P + I] = an;
    const R d = cc + aw + ae + as + an;
    c.d[Q] = d;
    c.wd[Q] = (R)omega / d;
}

// ---------------------------------------------------------------------------
// Step 3: PISO corrector (eq. step2_sd second line, eq. p_prime_sd, step4_4sd)
// ---------------------------------------------------------------------------

// H(u) = rho^n u^n/dt - C(u) + mu L(u) = rho^n u^n/dt + (rho1/dt) u - T(u) at the
// newest velocity.
__device__ __forceinline__ void ph_H(const StepArgs &a, const double *U, const double *W, double *sm,
                                     int bx, int bz)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    Tile<2> &su = tile_at<2>(sm, 0), &sw = tile_at<2>(sm, 1);
    int i, k;
    const bool in = cell_of(G, bx, bz, i, k);
    const int q = in ? cidx(G, i, k) : 0;
    // the cell's stencil weights (shared by both components) and state,
    // loaded ahead of the tile barrier
    Coef9<double> c{};
    double ru = 0.0, rw = 0.0, r1dt = 0.0;
    auto fetch = [&] {
        c = coef9(a.T, q);
        const double rdt = ld(&a.S.rho[q]) * F.idt;
        ru = rdt * ld(&a.S.u[q]);
        rw = rdt * ld(&a.S.w[q]);
        r1dt = ld(&a.rho1[q]) * F.idt;
    };
    if (kPrefetch && in) fetch();
    load_tile<BC_U, 2>(su, G, F, U, bx, bz);
    load_tile<BC_W, 2>(sw, G, F, W, bx, bz);
    __syncthreads();
    if (in) {
        if (!kPrefetch) fetch();
        const int y = threadIdx.y + 2, x = threadIdx.x + 2;
        a.Hx[q] = fma(r1dt, su[y][x], ru - apply9c<2>(c, su, y, x));
        a.Hz[q] = fma(r1dt, sw[y][x], rw - apply9c<2>(c, sw, y, x));
    }
    __syncthreads();
}

// Right-hand side of the pressure equation,
//   b_i = (rho^n_i + psi_i rho2_i g z_i)/dt
//         - (1/V) sum_f D_f |A_f| [H_f . n + g z_f (rho2_N - rho2_i)/Delta_f],
// the initial residual r = b - A x (x = xin, copied to xout) and p0 = 0.
// acc += (b^2, r^2).
// MX: r0 rounded to FP32 into L32.r (instead of L.r), and a zero pressure
// increment and first CG direction of the FP32 solve.
template <bool MX>
__device__ __forceinline__ void ph_helm_rhs_t(const StepArgs &a, const Level &L, const LevelF &L32,
                                              const MixedArgs &m, const double *xin, double *xout,
                                              double *sm, int bx, int bz, double (&acc)[2])
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    Tile<1> &sx = tile_at<1>(sm, 0), &s2 = tile_at<1>(sm, 1), &shx = tile_at<1>(sm, 2),
            &shz = tile_at<1>(sm, 3);
    int i, k;
    const bool in = cell_of(G, bx, bz, i, k);
    const int q0 = in ? cidx(G, i, k) : 0;
    // the cell's face coefficients and operator, loaded ahead of the tile
    // barrier
    double Dw = 0.0, De = 0.0, Ds = 0.0, Dn = 0.0;
    HelmCoef<double> hc{};
    auto fetch = [&] {
        Dw = ld(&a.Dx[k * G.P + i]);
        De = ld(&a.Dx[k * G.P + i + 1]);
        Ds = ld(&a.Dz[k * G.P + i]);
        Dn = ld(&a.Dz[(k + 1) * G.P + i]);
        hc = helm_coef(L, q0, i, k);
    };
    if (kPrefetch && in) fetch();
    load_tile_fn<1>(sx, G, bx, bz, [&](int q, int, int) { return ld(&xin[q]); });
    load_tile_fn<1>(s2, G, bx, bz, [&](int q, int, int) { return ld(&a.rho2[q]); });
    load_tile_fn<1>(shx, G, bx, bz, [&](int q, int, int) { return ld(&a.Hx[q]); });
    load_tile_fn<1>(shz, G, bx, bz, [&](int q, int, int) { return ld(&a.Hz[q]); });
    __syncthreads();
    if (in) {
        if (!kPrefetch) fetch();
        const int q = q0;
        const int y = threadIdx.y + 1, x = threadIdx.x + 1;
        const double gz = ld(&a.gzc[k]);
        const double gzx = gz * G.idx, gzs = ld(&a.gzf[k]) * G.idz, gzn = ld(&a.gzf[k + 1]) * G.idz;
        const double r2q = s2[y][x];
        // wall faces have D = 0 and zero tile entries beyond the box
        double flux = De * G.dz * fma(0.5, shx[y][x] + shx[y][x + 1], gzx * (s2[y][x + 1] - r2q));
        flux += Dw * G.dz * fma(-0.5, shx[y][x] + shx[y][x - 1], gzx * (s2[y][x - 1] - r2q));
        flux += Dn * G.dx * fma(0.5, shz[y][x] + shz[y + 1][x], gzn * (s2[y + 1][x] - r2q));
        flux += Ds * G.dx * fma(-0.5, shz[y][x] + shz[y - 1][x], gzs * (s2[y - 1][x] - r2q));
        const double b = fma(ld(&a.psi[q]) * r2q, gz, ld(&a.S.rho[q])) * F.idt - flux * G.iV;
        const double r = b - helm_apply<1>(hc, sx, y, x);
        a.b[q] = b;
        xout[q] = sx[y][x];
        if (!MX) {
            L.r[q] = r;
            a.p0[q] = 0.0;
        } else {
            L32.r[q] = (float)r;
            m.x[q] = 0.0f;
            m.p0[q] = 0.0f;
        }
        acc[0] = fma(b, b, acc[0]);
        acc[1] = fma(r, r, acc[1]);
    }
    __syncthreads();
}

__device__ __forceinline__ void ph_helm_rhs(const StepArgs &a, const Level &L, const double *xin,
                                            double *xout, double *sm, int bx, int bz,
                                            double (&acc)[2])
{
    ph_helm_rhs_t<false>(a, L, LevelF{}, MixedArgs{}, xin, xout, sm, bx, bz, acc);
}

// p' <- p' + dp (mixed-precision path: the FP32 solve's increment).
__device__ __forceinline__ void ph_p_apply(const StepArgs &a, const MixedArgs &m, int bx, int bz)
{
    int i, k;
    if (!cell_of(a.G, bx, bz, i, k)) return;
    const int q = cidx(a.G, i, k);
    a.N.pp[q] = ld(&a.N.pp[q]) + (double)ld(&m.x[q]);
}

// ---- V-cycle ----

// Restriction step of a level: pre-smooth with one damped Jacobi sweep from
// zero, e = (omega/d) r, and restrict the new residual r - A e (= (1-omega) r +
// sum a e_N) by averaging the four fine cells of each coarse cell. (bx, bz)
// is a tile of the fine level, whose sizes are even.
template <class R>
__device__ __forceinline__ void ph_mg_down(const LevelT<R> &f, const LevelT<R> &c, double omega,
                                           double *sm, int bx, int bz)
{
    const Geom &G = f.G;
    Tile<1, R> &se = tile_at<1, R>(sm, 0);
    R(*sres)[BX] = reinterpret_cast<R(*)[BX]>(reinterpret_cast<R *>(sm) + kT1);
    int i, k;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const bool in = cell_of(G, bx, bz, i, k);
    const int q0 = in ? cidx(G, i, k) : 0;
    HelmCoef<R> hc{};
    R rq = 0;
    auto fetch = [&] {   // ahead of the tile barrier
        hc = helm_coef(f, q0, i, k);
        rq = ld(&f.r[q0]);
    };
    if (kPrefetch && in) fetch();
    load_tile_fn<1, R>(se, G, bx, bz, [&](int q, int, int) { return ld(&f.wd[q]) * ld(&f.r[q]); });
    __syncthreads();
    if (in) {
        if (!kPrefetch) fetch();
        const int y = ty + 1, x = tx + 1;
        R t = (R)(1.0 - omega) * rq;
        t = fma(hc.aw, se[y][x - 1], t);
        t = fma(hc.ae, se[y][x + 1], t);
        t = fma(hc.as, se[y - 1][x], t);
        t = fma(hc.an, se[y + 1][x], t);
        f.e[q0] = se[y][x];
        sres[ty][tx] = t;
    }
    __syncthreads();
    // one thread per coarse cell: all four of its fine cells are inside the
    // box or all outside
    if (tx < BX / 2 && ty < BZ / 2) {
        const int I = bx * (BX / 2) + tx, K = bz * (BZ / 2) + ty;
        if (I < c.G.nx && K < c.G.nz)
            c.r[cidx(c.G, I, K)] = (R)0.25 * ((sres[2 * ty][2 * tx] + sres[2 * ty][2 * tx + 1]) +
                                              (sres[2 * ty + 1][2 * tx] + sres[2 * ty + 1][2 * tx + 1]));
    }
    __syncthreads();
}

// Coarsest level: one damped Jacobi sweep (first = starts from zero).
template <class R>
__device__ __forceinline__ void ph_mg_coarse(const LevelT<R> &L, const R *ein, R *eout, int first,
                                             double *sm, int bx, int bz)
{
    const Geom &G = L.G;
    int i, k;
    if (first) {
        if (cell_of(G, bx, bz, i, k)) {
            const int q = cidx(G, i, k);
            eout[q] = ld(&L.wd[q]) * ld(&L.r[q]);
        }
        return;
    }
    Tile<1, R> &se = tile_at<1, R>(sm, 0);
    load_tile_fn<1, R>(se, G, bx, bz, [&](int q, int, int) { return ld(&ein[q]); });
    __syncthreads();
    if (cell_of(G, bx, bz, i, k)) {
        const int q = cidx(G, i, k);
        const int y = threadIdx.y + 1, x = threadIdx.x + 1;
        eout[q] = fma(ld(&L.wd[q]), ld(&L.r[q]) - helm_tile<1, R>(L, q, i, k, se, y, x), se[y][x]);
    }
    __syncthreads();
}

// Prolongation step of a level: e' = e + P e_c (piecewise constant), then one
// damped Jacobi post-smoothing sweep e'' = e' + (omega/d)(r - A e'). At the
// finest level the result is z = M^-1 r; acc += r.z.
template <class R>
__device__ __forceinline__ void ph_mg_up(const LevelT<R> &f, const R *res, const R *ec, int Pc, R *out,
                                         double *sm, int bx, int bz, R (&acc)[1])
{
    const Geom &G = f.G;
    Tile<1, R> &se = tile_at<1, R>(sm, 0);
    int i, k;
    const bool in = cell_of(G, bx, bz, i, k);
    const int q0 = in ? cidx(G, i, k) : 0;
    HelmCoef<R> hc{};
    R rq = 0, wq = 0;
    auto fetch = [&] {   // ahead of the tile barrier
        hc = helm_coef(f, q0, i, k);
        rq = ld(&res[q0]);
        wq = ld(&f.wd[q0]);
    };
    if (kPrefetch && in) fetch();
    load_tile_fn<1, R>(se, G, bx, bz, [&](int q, int ii, int kk) {
        return ld(&f.e[q]) + ld(&ec[(kk >> 1) * Pc + (ii >> 1)]);
    });
    __syncthreads();
    if (in) {
        if (!kPrefetch) fetch();
        const int y = threadIdx.y + 1, x = threadIdx.x + 1;
        const R z = fma(wq, rq - helm_apply<1, R>(hc, se, y, x), se[y][x]);
        out[q0] = z;
        acc[0] = fma(rq, z, acc[0]);
    }
    __syncthreads();
}

// Single-level preconditioner: two Jacobi sweeps from zero,
// z = e + (omega/d)(r - A e) with e = (omega/d) r (omega = 1 unless the
// caller set another weight: then M^-1 A has the eigenvalues l (2 - l) of
// the Chebyshev-optimal degree-2 form); acc += r.z.
template <class R>
__device__ __forceinline__ void ph_mg_single(const LevelT<R> &f, R *out, double *sm, int bx, int bz,
                                             R (&acc)[1])
{
    const Geom &G = f.G;
    Tile<1, R> &se = tile_at<1, R>(sm, 0);
    int i, k;
    const bool in = cell_of(G, bx, bz, i, k);
    const int q = in ? cidx(G, i, k) : 0;
    HelmCoef<R> c{};
    R rq = 0, wq = 0;
    auto fetch = [&] {
        c = helm_coef(f, q, i, k);
        rq = ld(&f.r[q]);
        wq = ld(&f.wd[q]);
    };
    if (kPrefetch && in) fetch();
    load_tile_fn<1, R>(se, G, bx, bz, [&](int qq, int, int) { return ld(&f.wd[qq]) * ld(&f.r[qq]); });
    __syncthreads();
    if (in) {
        if (!kPrefetch) fetch();
        const int y = threadIdx.y + 1, x = threadIdx.x + 1;
        const R z = fma(wq, rq - helm_apply<1, R>(c, se, y, x), se[y][x]);
        out[q] = z;
        acc[0] = fma(rq, z, acc[0]);
    }
    __syncthreads();
}

// ---- CG vector steps ----

// p_new = z + beta p_old (computed once per tile cell) and q = A p_new;
// acc += p.q.
template <class R>
__device__ __forceinline__ void ph_pspmv(const LevelT<R> &L, const R *pold, R *pnew, R *qv, double beta,
                                         double *sm, int bx, int bz, R (&acc)[1])
{
    const Geom &G = L.G;
    const R *z = L.e2;
    const R b = (R)beta;
    Tile<1, R> &sp = tile_at<1, R>(sm, 0);
    int i, k;
    const bool in = cell_of(G, bx, bz, i, k);
    const int q = in ? cidx(G, i, k) : 0;
    HelmCoef<R> c{};
    if (kPrefetchSpmv && in) c = helm_coef(L, q, i, k);
    load_tile_fn<1, R>(sp, G, bx, bz, [&](int qq, int, int) { return fma(b, ld(&pold[qq]), ld(&z[qq])); });
    __syncthreads();
    if (in) {
        if (!kPrefetchSpmv) c = helm_coef(L, q, i, k);
        const int y = threadIdx.y + 1, x = threadIdx.x + 1;
        const R pq = sp[y][x];
        const R Ap = helm_apply<1, R>(c, sp, y, x);
        pnew[q] = pq;
        qv[q] = Ap;
        acc[0] = fma(pq, Ap, acc[0]);
    }
    __syncthreads();
}

// x += alpha p and r -= alpha q, fused with the first step of the next
// V-cycle on the new residual (a CG iteration then needs one grid-wide
// synchronisation less): the new residual and e = (omega/d) r_new are formed
// on the tile and its halo from the old r and q in one pass.
template <class R>
__device__ __forceinline__ void update_tiles(const LevelT<R> &L, const R *qv, const R *rin, R alpha,
                                             Tile<1, R> &sr, Tile<1, R> &se, int bx, int bz)
{
    const Geom &G = L.G;
    const int i0 = bx * BX - 1, k0 = bz * BZ - 1;
    const int tid = threadIdx.x + threadIdx.y * BX;
    constexpr int W = BX + 2, NE = (BZ + 2) * (BX + 2);
    for (int e = tid; e < NE; e += NTHREADS) {
        const int tk = e / W, ti = e - tk * W;
        const int i = i0 + ti, k = k0 + tk;
        R rn = 0, ev = 0;
        if (i >= 0 && i < G.nx && k >= 0 && k < G.nz) {
            const int q = k * G.P + i;
            rn = fma(-alpha, ld(&qv[q]), ld(&rin[q]));
            ev = ld(&L.wd[q]) * rn;
        }
        sr[tk][ti] = rn;
        se[tk][ti] = ev;
    }
}

// The residual is read from rin (halo included) and written to rout: other
// blocks still read the old residual while this one writes the new.
// Single-level preconditioner: then z = e + (omega/d)(r_new - A e);
// acc += (r_new^2, r_new . z).
template <class R>
__device__ __forceinline__ void ph_update_single(const LevelT<R> &L, const R *qv, const R *rin, R *rout,
                                                 R *x, const R *p, double alpha_d, double *sm, int bx,
                                                 int bz, R (&acc)[2])
{
    const Geom &G = L.G;
    const R alpha = (R)alpha_d;
    Tile<1, R> &sr = tile_at<1, R>(sm, 0), &se = tile_at<1, R>(sm, 1);
    int i, k;
    const bool in = cell_of(G, bx, bz, i, k);
    const int q = in ? cidx(G, i, k) : 0;
    HelmCoef<R> c{};
    R wq = 0, xq = 0, pq = 0;
    auto fetch = [&] {
        c = helm_coef(L, q, i, k);
        wq = ld(&L.wd[q]);
        xq = ld(&x[q]);
        pq = ld(&p[q]);
    };
    if (kPrefetch && in) fetch();
    update_tiles<R>(L, qv, rin, alpha, sr, se, bx, bz);
    __syncthreads();
    if (in) {
        if (!kPrefetch) fetch();
        const int y = threadIdx.y + 1, xx = threadIdx.x + 1;
        const R rn = sr[y][xx];
        x[q] = fma(alpha, pq, xq);
        rout[q] = rn;
        const R z = fma(wq, rn - helm_apply<1, R>(c, se, y, xx), se[y][xx]);
        L.e2[q] = z;
        acc[0] = fma(rn, rn, acc[0]);
        acc[1] = fma(rn, z, acc[1]);
    }
    __syncthreads();
}

// Multigrid preconditioner: then the restriction step of the finest level
// (pre-smoothed e and the averaged residual (1-omega) r_new + sum a e_N into
// the next level); acc += r_new^2.
template <class R>
__device__ __forceinline__ void ph_update_down(const LevelT<R> &f, const LevelT<R> &c, const R *qv,
                                               const R *rin, R *rout, R *x, const R *p, double alpha_d,
                                               double omega, double *sm, int bx, int bz, R (&acc)[1])
{
    const Geom &G = f.G;
    const R alpha = (R)alpha_d;
    Tile<1, R> &sr = tile_at<1, R>(sm, 0), &se = tile_at<1, R>(sm, 1);
    R(*sres)[BX] = reinterpret_cast<R(*)[BX]>(reinterpret_cast<R *>(sm) + 2 * kT1);
    int i, k;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const bool in = cell_of(G, bx, bz, i, k);
    const int q0 = in ? cidx(G, i, k) : 0;
    R aw = 0, ae = 0, as = 0, an = 0, xq = 0, pq = 0;
    auto fetch = [&] {   // ahead of the tile barrier
        aw = ld(&f.ax[k * G.P + i]);
        ae = ld(&f.ax[k * G.P + i + 1]);
        as = ld(&f.az[k * G.P + i]);
        an = ld(&f.az[(k + 1) * G.P + i]);
        xq = ld(&x[q0]);
        pq = ld(&p[q0]);
    };
    if (kPrefetch && in) fetch();
    update_tiles<R>(f, qv, rin, alpha, sr, se, bx, bz);
    __syncthreads();
    if (in) {
        if (!kPrefetch) fetch();
        const int q = q0;
        const int y = ty + 1, xx = tx + 1;
        const R rn = sr[y][xx];
        x[q] = fma(alpha, pq, xq);
        rout[q] = rn;
        R t = (R)(1.0 - omega) * rn;
        t = fma(aw, se[y][xx - 1], t);
        t = fma(ae, se[y][xx + 1], t);
        t = fma(as, se[y - 1][xx], t);
        t = fma(an, se[y + 1][xx], t);
        f.e[q] = se[y][xx];
        sres[ty][tx] = t;
        acc[0] = fma(rn, rn, acc[0]);
    }
    __syncthreads();
    if (tx < BX / 2 && ty < BZ / 2) {
        const int I = bx * (BX / 2) + tx, K = bz * (BZ / 2) + ty;
        if (I < c.G.nx && K < c.G.nz)
            c.r[cidx(c.G, I, K)] = (R)0.25 * ((sres[2 * ty][2 * tx] + sres[2 * ty][2 * tx + 1]) +
                                              (sres[2 * ty + 1][2 * tx] + sres[2 * ty + 1][2 * tx + 1]));
    }
    __syncthreads();
}

// ---- learned initial guess of a pressure solve ----

// The network's proposal e (dense FP32, row k at k nx): q = A e and
// acc += (r . e, e . A e).
template <class R>
__device__ __forceinline__ void ph_guess_dots(const LevelT<R> &L, const float *e, const R *r, R *q, double *sm,
                                              int bx, int bz, R (&acc)[2])
{
    const Geom &G = L.G;
    Tile<1, R> &se = tile_at<1, R>(sm, 0);
    load_tile_fn<1, R>(se, G, bx, bz, [&](int, int i, int k) { return (R)ld(&e[(size_t)k * G.nx + i]); });
    __syncthreads();
    int i, k;
    if (cell_of(G, bx, bz, i, k)) {
        const int qi = cidx(G, i, k);
        const int y = threadIdx.y + 1, x = threadIdx.x + 1;
        const R Ae = helm_tile<1, R>(L, qi, i, k, se, y, x);
        q[qi] = Ae;
        acc[0] = fma(ld(&r[qi]), se[y][x], acc[0]);
        acc[1] = fma(se[y][x], Ae, acc[1]);
    }
    __syncthreads();
}

// x += alpha e, r -= alpha q; acc += r^2.
template <class R>
__device__ __forceinline__ void ph_guess_apply(const LevelT<R> &L, const float *e, const R *q, R *r, R *x,
                                               double alpha_d, int bx, int bz, R (&acc)[1])
{
    int i, k;
    if (!cell_of(L.G, bx, bz, i, k)) return;
    const int qi = cidx(L.G, i, k);
    const R alpha = (R)alpha_d;
    x[qi] = fma(alpha, (R)ld(&e[(size_t)k * L.G.nx + i]), ld(&x[qi]));
    const R rn = fma(-alpha, ld(&q[qi]), ld(&r[qi]));
    r[qi] = rn;
    acc[0] = fma(rn, rn, acc[0]);
}

// Flux and velocity correction: F_f = D_f (H_f - G_f) with
// G_f = (p'_b - p'_a)/Delta - g z_f (rho2_b - rho2_a)/Delta; u = (dt/rho1)(H - G_cell);
// p = p' - rho2 g z; rho = p / (R T^{n+1}) = p psi; phi = F |A|; p^{n-1} <- p^n
// (and K^{n-1} <- K^n in the literal reading of eq. step3_sd).
__device__ __forceinline__ void ph_correct(const StepArgs &a, double *sm, int bx, int bz)
{
    const Geom &G = a.G;
    const Phys &F = a.F;
    Tile<1> &sx = tile_at<1>(sm, 0), &s2 = tile_at<1>(sm, 1);
    double(*gx)[BX + 1] = reinterpret_cast<double(*)[BX + 1]>(sm + 2 * kT1);
    double(*gz)[BX] = reinterpret_cast<double(*)[BX]>(sm + 2 * kT1 + BZ * (BX + 1));
    const State &N = a.N;
    int i, k;
    const bool in = cell_of(G, bx, bz, i, k);
    const int q0 = in ? cidx(G, i, k) : 0;
    // the cell's own inputs, loaded ahead of the tile barrier: H(u) at the
    // cell and at its west and south neighbours (the face averages), D on
    // the west and south faces, dt/rho1, psi, p^n
    double hxq = 0.0, hzq = 0.0, hxw = 0.0, hzs = 0.0, Dw = 0.0, Ds = 0.0, dtr1 = 0.0, psq = 0.0, pnq = 0.0;
    auto fetch = [&] {
        hxq = ld(&a.Hx[q0]);
        hzq = ld(&a.Hz[q0]);
        if (i > 0) {
            hxw = ld(&a.Hx[q0 - 1]);
            Dw = ld(&a.Dx[k * G.P + i]);
        }
        if (k > 0) {
            hzs = ld(&a.Hz[q0 - G.P]);
            Ds = ld(&a.Dz[k * G.P + i]);
        }
        dtr1 = ld(&a.dtr1[q0]);
        psq = ld(&a.psi[q0]);
        pnq = ld(&a.S.p[q0]);
    };
    if (kPrefetch && in) fetch();
    load_tile_fn<1>(sx, G, bx, bz, [&](int q, int, int) { return ld(&N.pp[q]); });
    load_tile_fn<1>(s2, G, bx, bz, [&](int q, int, int) { return ld(&a.rho2[q]); });
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int y = ty + 1, x = tx + 1;
    const double gzk = in ? ld(&a.gzc[k]) : 0.0;
    auto gxf = [&](int xa) {   // x-face between tile columns xa and xa+1 of row y
        return fma(-gzk, s2[y][xa + 1] - s2[y][xa], sx[y][xa + 1] - sx[y][xa]) * G.idx;
    };
    auto gzf = [&](int ya, int kf) {   // z-face between tile rows ya and ya+1, face index kf
        return fma(-ld(&a.gzf[kf]), s2[ya + 1][x] - s2[ya][x], sx[ya + 1][x] - sx[ya][x]) * G.idz;
    };
    if (in) {
        gx[ty][tx] = i > 0 ? gxf(x - 1) : 0.0;
        gz[ty][tx] = k > 0 ? gzf(y - 1, k) : 0.0;
        if (tx == BX - 1 || i == G.nx - 1) gx[ty][tx + 1] = i + 1 < G.nx ? gxf(x) : 0.0;
        if (ty == BZ - 1 || k == G.nz - 1) gz[ty + 1][tx] = k + 1 < G.nz ? gzf(y, k + 1) : 0.0;
    }
    __syncthreads();
    if (in) {
        if (!kPrefetch) fetch();
        const int q = q0;
        const double gxw = gx[ty][tx], gxe = gx[ty][tx + 1], gzs = gz[ty][tx], gzn = gz[ty + 1][tx];
        const double Fw = i > 0 ? Dw * (0.5 * (hxw + hxq) - gxw) : 0.0;   // wall faces carry zero
        const double Fs = k > 0 ? Ds * (0.5 * (hzs + hzq) - gzs) : 0.0;
        N.phix[k * G.P + i] = Fw * G.dz;
        N.phiz[k * G.P + i] = Fs * G.dx;
        if (i == G.nx - 1) N.phix[k * G.P + G.nx] = 0.0;
        if (k == G.nz - 1) N.phiz[G.nz * G.P + i] = 0.0;
        N.u[q] = dtr1 * (hxq - 0.5 * (gxw + gxe));
        N.w[q] = dtr1 * (hzq - 0.5 * (gzs + gzn));
        const double pn = fma(-s2[y][x], gzk, sx[y][x]);
        N.p[q] = pn;
        N.rho[q] = pn * psq;
        N.pold[q] = pnq;
        if (F.k_lagged) {
            const double un = ld(&a.S.u[q]), wn = ld(&a.S.w[q]);
            N.Kold[q] = 0.5 * (un * un + wn * wn);   // K^{n-1} of the next step
        }
    }
    __syncthreads();
}

// ---- what the block that completes a reduction does with the totals ----

__device__ __forceinline__ void fin_pred(Scal *sc, const double (&t)[2])
{
    sc->bn2[0] = t[0];
    sc->bn2[1] = t[1];
    sc->done[LOOP_MOM] = 0;
    sc->trips[LOOP_MOM] = 0;
    sc->sweeps[0] = 0;
}

__device__ __forceinline__ void fin_mom(Scal *sc, const double (&t)[2], double tol2)
{
    sc->sweeps[0] += 1;
    if (!isfinite(t[0]) || !isfinite(t[1])) sc->status = 5;
    else if (t[0] <= tol2 * sc->bn2[0] && t[1] <= tol2 * sc->bn2[1]) sc->done[LOOP_MOM] = 1;
}

__device__ __forceinline__ void fin_enth_rhs(Scal *sc, const double (&t)[1])
{
    sc->bn2[2] = t[0];
    sc->done[LOOP_ENTH] = 0;
    sc->trips[LOOP_ENTH] = 0;
    sc->sweeps[1] = 0;
}

__device__ __forceinline__ void fin_enth(Scal *sc, const double (&t)[1], double tol2)
{
    sc->sweeps[1] += 1;
    if (!isfinite(t[0])) sc->status = 5;
    else if (t[0] <= tol2 * sc->bn2[2]) sc->done[LOOP_ENTH] = 1;
}

__device__ __forceinline__ void fin_helm(Scal *sc, const double (&t)[2], double tol2, int corr)
{
    sc->b2 = t[0];
    sc->r2 = t[1];
    sc->cg_it = 0;
    sc->corr = corr;
    sc->trips[LOOP_CG] = 0;
    sc->rz = 0.0;
    sc->beta = 0.0;
    sc->done[LOOP_CG] = t[1] <= tol2 * t[0];
    sc->cg_iters[corr] = 0;
    sc->cg_relres[corr] = t[0] > 0.0 ? sqrt(t[1] / t[0]) : 0.0;
    if (!isfinite(t[0]) || !isfinite(t[1])) sc->status = 5;
}

// Mixed precision: the inner FP32 solve's tolerance is relative to the
// initial residual r0 = b - A p'_prev (kept in b2); nothing to solve if r0 is
// already at the FP64 tolerance relative to b.
__device__ __forceinline__ void fin_helm_mixed(Scal *sc, const double (&t)[2], double tol2_fp64, int corr)
{
    sc->b2 = t[1];
    sc->r2 = t[1];
    sc->cg_it = 0;
    sc->corr = corr;
    sc->trips[LOOP_CG] = 0;
    sc->rz = 0.0;
    sc->beta = 0.0;
    sc->done[LOOP_CG] = t[1] <= tol2_fp64 * t[0];
    sc->cg_iters[corr] = 0;
    sc->cg_relres[corr] = 1.0;
    if (!isfinite(t[0]) || !isfinite(t[1])) sc->status = GEA_ERR_NONFINITE;
}

__device__ __forceinline__ void fin_rz(Scal *sc, const double (&t)[1])
{
    sc->beta = (sc->cg_it == 0 || sc->rz == 0.0) ? 0.0 : t[0] / sc->rz;
    sc->rz = t[0];
}

__device__ __forceinline__ void fin_pq(Scal *sc, const double (&t)[1])
{
    sc->pq = t[0];
    sc->alpha = t[0] != 0.0 ? sc->rz / t[0] : 0.0;
    if (!isfinite(t[0])) sc->status = 5;
}

__device__ __forceinline__ void fin_update(Scal *sc, const double (&t)[1], double tol2)
{
    const int it = sc->cg_it + 1;
    sc->cg_it = it;
    sc->r2 = t[0];
    const int c = sc->corr;
    sc->cg_iters[c] = it;
    sc->cg_relres[c] = sc->b2 > 0.0 ? sqrt(t[0] / sc->b2) : 0.0;
    if (!isfinite(t[0])) sc->status = 5;
    else if (t[0] <= tol2 * sc->b2) sc->done[LOOP_CG] = 1;
}

// the step length minimising the A-norm error along e: alpha = r.e / e.Ae
// (0 if e.Ae is not positive)
__device__ __forceinline__ void fin_guess_dots(Scal *sc, const double (&t)[2])
{
    sc->galpha = (t[1] > 0.0 && isfinite(t[0]) && isfinite(t[1])) ? t[0] / t[1] : 0.0;
}

__device__ __forceinline__ void fin_guess_apply(Scal *sc, const double (&t)[1], double tol2)
{
    sc->r2 = t[0];
    sc->cg_relres[sc->corr] = sc->b2 > 0.0 ? sqrt(t[0] / sc->b2) : 0.0;
    if (!isfinite(t[0])) sc->status = GEA_ERR_NONFINITE;
    else if (t[0] <= tol2 * sc->b2) sc->done[LOOP_CG] = 1;
}
