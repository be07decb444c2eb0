// gea_internal.cuh -- device-side data layout and stencil helpers of the GEA
// time step (Girfoglio, Quaini & Rozza, arXiv 2303.10499, Section 3).
//
// Layout in HBM: every field is row-major with one row per grid row k and a
// row pitch P (doubles) that is a multiple of 32 and >= nx+1, so rows start
// on 256-byte boundaries. Cell fields use columns 0..nx-1 of rows 0..nz-1;
// x-face arrays use columns 0..nx (face f between cells f-1 and f) of rows
// 0..nz-1; z-face arrays use columns 0..nx-1 of rows 0..nz (face f between
// rows f-1 and f). Wall faces are stored and hold zero.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gea.h"

struct gea_net;
// The network forward pass on stream st (gea_net.cu); returns the number of
// kernels launched or -1.
int gea_net_run(gea_net *net, cudaStream_t st, int n, int h, int w, const float *r, float *y);
// Kernels of one network forward pass.
int gea_net_launches();
// Whether a network can take n samples of h x w.
bool gea_net_fits(const gea_net *net, int n, int h, int w);

namespace gea {

constexpr int BX = 32;          // threads per block along x (one warp per row)
constexpr int BZ = 8;           // rows per block
constexpr int NTHREADS = BX * BZ;
constexpr int kMaxLevels = 16;  // multigrid levels (grids up to 2^16 cells a side)

enum Bc { BC_EVEN = 0, BC_U = 1, BC_W = 2, BC_H = 3 };

struct Geom {
    int nx, nz, P;              // cells in x and z, row pitch in doubles
    double dx, dz, idx, idz, iV; // spacings, their inverses, 1/(dx dz)
};

struct Phys {
    double R, cp, g, p0, mu, nuh, dt, idt;   // nuh = mu / Pr
    double omega;                            // damped-Jacobi weight of the smoother
    double les_d2;                           // Smagorinsky (cs Delta)^2; 0: constant viscosity
    int k_lagged;                            // GEA_READING_K_LAGGED: K^{n-1} in eq. step3_sd
    // uniform branch flags as integers (an FP64 compare issues on the FP64 pipe)
    int les;                                 // les_d2 > 0
    int pr_ne1;                              // nuh != mu (Pr != 1): the enthalpy stencil differs
};

// Persistent state of one time level (Section 3's solution tuple plus the
// face mass fluxes phi, p^{n-1} and, for the literal reading of eq.
// step3_sd, K^{n-1}).
struct State {
    double *rho, *u, *w, *T, *h, *p, *pp, *pold, *phix, *phiz, *Kold;
};

// One multigrid level of the Helmholtz operator
//   (A x)_i = c_i x_i + sum_f a_f (x_i - x_N) = d_i x_i - sum_f a_f x_N,
// d_i = c_i + sum_f a_f, kept as d and wd = omega / d.
// R is the value type: double on the FP64 path, float for the inner solves
// of the mixed-precision path.
template <class R>
struct LevelT {
    Geom G;
    R *c, *d, *wd, *ax, *az;  // reaction, diagonal, omega/diagonal, face coefficients
    R *r, *e, *e2;            // residual, pre-smoothed correction, post-smoothed
    R *r_alt;                 // finest level: second residual buffer (CG iterations
                              // alternate r and r_alt; the update reads one, writes the other)
};
using Level = LevelT<double>;
using LevelF = LevelT<float>;

// Finest-level residual after `it` CG updates.
template <class R>
__host__ __device__ __forceinline__ R *res_of(const LevelT<R> &L, int it)
{
    return (it & 1) ? L.r_alt : L.r;
}

// The implicit transport operator of Steps 1-2,
//   T(X)_i = (rho1/dt) X_i + C(X)_i - mu L(X)_i,
// assembled once per step as a 9-point cross stencil (offsets 0, +-1, +-2 in x
// and z) on the ghost-extended field.
template <class R>
struct Stencil9T {
    R *cC, *cE1, *cE2, *cW1, *cW2, *cN1, *cN2, *cS1, *cS2;
};
using Stencil9 = Stencil9T<double>;
using Stencil9F = Stencil9T<float>;

// Buffers of the mixed-precision path: FP32 copies of the operators and the
// increments its inner solves iterate on (u, w, h and p' each get an FP64
// residual, an FP32 solve for the increment, and an FP64 update).
struct MixedArgs {
    Stencil9F T;                   // transport operator (with mu)
    float *dinvu, *dinvh;          // Jacobi reciprocals
    float *r0u, *r0w, *r0h;        // FP64 residuals of the predictors, rounded to FP32
    float *du[2], *dw[2], *dh[2];  // increments (Jacobi ping-pong)
    float *x, *p0, *p1, *q;        // pressure increment, CG directions, A p
    double tol2;                   // inner tolerance^2, relative to the initial residual
};

// Loop bookkeeping slots.
enum { LOOP_MOM = 0, LOOP_ENTH = 1, LOOP_CG = 2, NLOOPS = 3 };

// Device-resident scalars of one context.
struct Scal {
    double bn2[3];              // ||b_u||^2, ||b_w||^2, ||b_h||^2
    double b2, r2, rz, rz_old, pq, alpha, beta;
    int done[NLOOPS];           // convergence flag of the running loop
    int trips[NLOOPS];          // trips of the running loop
    int sweeps[2];              // Jacobi sweeps of this step (momentum, enthalpy)
    int cg_it;                  // CG iterations of the running solve
    int corr;                   // running corrector
    int cg_iters[4];
    double cg_relres[4];
    int status;                 // first device-side error of the running step
    int bad_cells;              // set_state validation
    long long steps_done;
    // last completed step (copied by the end-of-step kernel)
    int last_sweeps[2];
    int last_cg_iters[4];
    double last_cg_relres[4];
    int last_status;
    double mass, energy;        // diagnostics
    long long launches;         // kernel launches of completed and running steps
    unsigned counters[32];      // reduction arrival counters, one per kernel kind
    // persistent step kernels: grid barrier (a monotone arrival counter,
    // zero at the start of every launch, and the count of blocks that left
    // the launch, each on a cache line of its own) and per-step results
    alignas(128) unsigned bar_count;
    alignas(128) unsigned bar_exit;
    alignas(128) int u1_slot;   // 1 if u^{n+1/3} / h^{n+1} ended in the b buffers
    int h1_slot;
    unsigned long long press_ns; // globaltimer nanoseconds of the pressure solves, last step
    double galpha;              // step length of the learned initial guess
};

// Optional per-launch hook (profiled eager steps only; never during graph
// capture): begin/end bracket every kernel launch on stream st.
struct Tracer {
    virtual void begin(const char *name, long long cells, cudaStream_t st) = 0;
    virtual void end(cudaStream_t st) = 0;
    virtual ~Tracer() {}
};

enum {
    CNT_PRED = 0, CNT_MOM = 1, CNT_ENTH_RHS = 2, CNT_ENTH = 3, CNT_HELM = 4,
    CNT_RZ = 5, CNT_PQ = 6, CNT_UPD = 7, CNT_DIAG = 8, CNT_GUESS = 9
};

// Everything one time step's kernels need: the state read (S) and written
// (N), per-step scratch and the device scalars.
struct StepArgs {
    Geom G;
    Phys F;
    State S, N;
    Stencil9 T;                                          // transport operator (with mu)
    double *mueff;                                       // mu + mu_t per cell (LES)
    double *rho1, *dinvu, *dinvh, *bu, *bw, *ua, *wa, *ub, *wb;   // Step 1
    double *bh, *ha, *hb;                                // Step 2
    double *rho2, *psi, *Dx, *Dz, *Hx, *Hz, *b;          // Step 3
    double *dtr1;                                        // dt / rho^{n+1/3} (Step 1, used by Step 3)
    const double *gzc, *gzf;   // g z of the cell centres of row k (nz values) and of z-face k (nz + 1)
    double *p0, *p1, *q;                                 // CG directions (ping-pong) and A p
    Scal *sc;
    double *partials;
    double jac_rtol2, cg_rtol2;
    int tiles_per_block;   // per-phase kernels with a reduction: tiles a block walks (0: the size rule)
    // phase trace of the persistent kernels (gea_set_trace; null: off):
    // per block its entry time and SM, then per grid barrier its arrival
    // and release times (%globaltimer), for at most trace_bars barriers
    unsigned long long *trace;
    int trace_bars;
};

__device__ __forceinline__ int cidx(const Geom &G, int i, int k) { return k * G.P + i; }

// Cell value at (i,k), i in [-1, nx] and k in [-1, nz]; outside the box the
// one-layer ghost of the wall condition: wall-normal velocity odd (zero on
// the wall), tangential velocity and scalars even (zero gradient), h with
// dh/dz = -g on the bottom and top walls.
template <int BC>
__device__ __forceinline__ double ldc(const Geom &G, const Phys &F, const double *__restrict__ X,
                                      int i, int k)
{
    if (i < 0) {
        double v = X[k * G.P];
        return BC == BC_U ? -v : v;
    }
    if (i >= G.nx) {
        double v = X[k * G.P + G.nx - 1];
        return BC == BC_U ? -v : v;
    }
    if (k < 0) {
        double v = X[i];
        if (BC == BC_W) return -v;
        if (BC == BC_H) return v + F.g * G.dz;
        return v;
    }
    if (k >= G.nz) {
        double v = X[(G.nz - 1) * G.P + i];
        if (BC == BC_W) return -v;
        if (BC == BC_H) return v - F.g * G.dz;
        return v;
    }
    return X[k * G.P + i];
}

template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block totals of NV per-thread values, valid in thread 0. The values pass
// through shared memory (red: NV * NTHREADS doubles) and one warp adds them,
// 8 per lane and then a shuffle tree: about 1.5 FP64 additions per value per
// thread instead of 5 for a full-block shuffle tree (FP64 issue is the
// scarce resource on this GPU).
template <int NV, class T = double>
__device__ __forceinline__ void block_sum(const T (&v)[NV], T *red, T (&out)[NV])
{
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
#pragma unroll
    for (int j = 0; j < NV; ++j) red[j * NTHREADS + tid] = v[j];
    __syncthreads();
    if (tid < 32) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            T s = red[j * NTHREADS + tid];
#pragma unroll
            for (int q = 1; q < NTHREADS / 32; ++q) s += red[j * NTHREADS + tid + 32 * q];
            s = warp_sum(s);
            if (tid == 0) out[j] = s;
        }
    }
    __syncthreads();
}

// The partials buffer of a context: kGcntDoubles doubles of group counters
// (unsigned, zero between launches; the two-level grid sums below), then the
// block partials (the grid sums' block and group totals, or the persistent
// kernels' two buffers of kRedVals x blocks values).
constexpr int kSumGroup = 1024;                 // blocks per group of a grid sum
constexpr int kGroupCounters = 4096;            // groups a grid sum may have
constexpr int kGcntDoubles = kGroupCounters / 2;

// Deterministic grid-wide sum of NV values per thread (one launch), in two
// levels: the last block of each group of kSumGroup blocks adds the group's
// block totals, the last group adds the group totals, each in a fixed order
// (the arrivals spread over one counter per group instead of all blocks on
// one). Returns true in thread 0 of the very last block, with the totals in
// tot[]. Every thread of every block must call it.
// T is the type of the per-thread values and of the block sums (FP32 for the
// inner solves of the mixed-precision path); block partials and the grid
// total are FP64. red holds NV * NTHREADS doubles.
template <int NV, class T = double>
__device__ bool grid_sum(const T (&v)[NV], double *red, double *partials, unsigned *counter,
                         double (&tot)[NV])
{
    __shared__ int flag;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int bid = blockIdx.x + blockIdx.y * gridDim.x;
    const int nb = gridDim.x * gridDim.y;
    const int ng = (nb + kSumGroup - 1) / kSumGroup, grp = bid / kSumGroup, g0 = grp * kSumGroup;
    const int gn = min(kSumGroup, nb - g0);
    unsigned *gcnt = reinterpret_cast<unsigned *>(partials);
    double *p1 = partials + kGcntDoubles, *p2 = p1 + (size_t)NV * nb;
    T bt[NV];
    block_sum<NV, T>(v, reinterpret_cast<T *>(red), bt);
    if (tid == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) p1[(size_t)j * nb + bid] = (double)bt[j];
        __threadfence();
        flag = atomicAdd(&gcnt[grp], 1u) == (unsigned)gn - 1u;
    }
    __syncthreads();
    if (!flag) return false;
    __threadfence();
    double s[NV], gt[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        s[j] = 0.0;
        for (int b = tid; b < gn; b += NTHREADS) s[j] += __ldcg(&p1[(size_t)j * nb + g0 + b]);
    }
    block_sum<NV>(s, red, gt);
    if (ng == 1) {
        // one group: its sum is the total
        if (tid == 0) {
            gcnt[0] = 0u;
#pragma unroll
            for (int j = 0; j < NV; ++j) tot[j] = gt[j];
        }
        return tid == 0;
    }
    if (tid == 0) {
        gcnt[grp] = 0u;
#pragma unroll
        for (int j = 0; j < NV; ++j) p2[(size_t)j * ng + grp] = gt[j];
        __threadfence();
        flag = atomicAdd(counter, 1u) == (unsigned)ng - 1u;
    }
    __syncthreads();
    if (!flag) return false;
    __threadfence();
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        s[j] = 0.0;
        for (int b = tid; b < ng; b += NTHREADS) s[j] += __ldcg(&p2[(size_t)j * ng + b]);
    }
    block_sum<NV>(s, red, tot);
    if (tid == 0) *counter = 0u;
    return tid == 0;
}

// The light per-phase kernels with a grid reduction (the CG and V-cycle
// steps, the Jacobi sweeps) walk the tiles of a column of tpb tiles per
// block: fewer blocks, so fewer block reductions and arrivals. By the size
// rule (tpb = 0) grids of at least kMultiTileMin tiles take kTilesPerBlock
// and smaller grids one tile per block (fewer blocks would leave SMs idle);
// gea_set_tiles_per_block fixes tpb (the tile-column autotuner times the
// candidates). The kernels read the count back from the launch shape.
constexpr int kTilesPerBlock = 4;
constexpr int kMultiTileMin = 16384;
constexpr int kMaxTilesPerBlock = 16;
inline dim3 grid_tiles(const Geom &G, int tpb)
{
    const int tx = (G.nx + BX - 1) / BX, tz = (G.nz + BZ - 1) / BZ;
    if (tpb <= 0) tpb = (long long)tx * tz >= kMultiTileMin ? kTilesPerBlock : 1;
    return dim3(tx, (tz + tpb - 1) / tpb);
}
// f(bx, bz) for the block's tiles (block-uniform loop; each f ends with a
// block barrier).
template <class F>
__device__ __forceinline__ void block_tiles(const Geom &G, F f)
{
    const int tz = (G.nz + BZ - 1) / BZ;
    const int tpb = (tz + gridDim.y - 1) / gridDim.y;
    for (int t = 0; t < tpb; ++t) {
        const int bz = blockIdx.y * tpb + t;
        if (bz >= tz) break;
        f((int)blockIdx.x, bz);
    }
}

// ---- host-side launchers (gea_kernels.cu); tr may be null ----
void launch_derive(const Geom &G, const Phys &F, const double *rho, const double *rhou,
                   const double *rhow, const double *rhoe, const State &S, Scal *sc,
                   cudaStream_t st);
// conservative variables rho, rho u, rho w, rho e of state S (pitched arrays)
void launch_conserve(const Geom &G, const Phys &F, const State &S, double *rho, double *rhou, double *rhow,
                     double *rhoe, cudaStream_t st);
void launch_les(const StepArgs &a, cudaStream_t st, Tracer *tr);
void launch_pred_setup(const StepArgs &a, cudaStream_t st, Tracer *tr);
// second = 1: the second sweep of a pair (copies instead once converged)
void launch_mom_jacobi(const StepArgs &a, const double *uin, const double *win, double *uout,
                       double *wout, int second, cudaStream_t st, Tracer *tr);
void launch_enth_rhs(const StepArgs &a, cudaStream_t st, Tracer *tr);
void launch_enth_jacobi(const StepArgs &a, const double *hin, double *hout, int second,
                        cudaStream_t st, Tracer *tr);
void launch_eos_coef(const StepArgs &a, const Level &L0, cudaStream_t st, Tracer *tr);
void launch_mg_coarsen(const Level &f, const Level &c, double omega, cudaStream_t st, Tracer *tr);
void launch_H(const StepArgs &a, const double *U, const double *W, cudaStream_t st, Tracer *tr);
void launch_helm_rhs(const StepArgs &a, const Level &L0, const double *xin, double *xout,
                     int corr, cudaStream_t st, Tracer *tr);
// returns the number of kernels launched
int launch_vcycle(const StepArgs &a, Level *levels, int nlev, int ncoarse, cudaStream_t st,
                  Tracer *tr);
int launch_cg_iter(const StepArgs &a, Level *levels, int nlev, int ncoarse, double *x,
                   cudaStream_t st, Tracer *tr);
void launch_correct(const StepArgs &a, cudaStream_t st, Tracer *tr);
// graph: set the WHILE condition through h; otherwise bookkeeping only
void launch_loop_ctl(Scal *sc, cudaGraphConditionalHandle h, bool graph, int which,
                     int maxtrips, int body_launches, cudaStream_t st, Tracer *tr);
// sets the condition of the WHILE node that follows from the loop's flags
void launch_loop_gate(Scal *sc, cudaGraphConditionalHandle h, int which, cudaStream_t st);
void launch_step_begin(Scal *sc, cudaStream_t st, Tracer *tr);
void launch_step_end(Scal *sc, int fixed_launches, cudaStream_t st, Tracer *tr);
void launch_diag(const Geom &G, const Phys &F, const State &S, const double *theta_bar,
                 double *theta_out, Scal *sc, double *partials, cudaStream_t st);
int max_blocks(const Geom &G);
// learned initial guess of the pressure solve (gea_kernels.cu): the network
// (gea_net.cu) proposes a correction e for the residual r of level L; the
// step x += alpha e, r -= alpha A e minimises the A-norm error along e.
// launch_guess_in converts r for the network and, in a graph, sets the IF
// condition h of the pass (skipped once the solve has converged);
// launch_net_guess runs the network and the step. Returns the number of
// kernels launched, or -1 if the network failed.
template <class R>
void launch_guess_in(const StepArgs &a, const LevelT<R> &L, const R *r, float *dense_r,
                     cudaGraphConditionalHandle h, bool graph, cudaStream_t st, Tracer *tr);
template <class R>
int launch_net_guess(const StepArgs &a, const LevelT<R> &L, R *r, R *q, R *x, double tol2, gea_net *net,
                     float *dense_r, float *dense_e, cudaStream_t st, Tracer *tr);
// One iteration of flexible CG with the two-stage preconditioner (FP64
// levels L): z = g N(r) + M(r - g A N(r)) with the network N and one
// V-cycle M (s_buf: a field for r - g A N(r)), the direction update, q = A p,
// x and r. Returns the number of launches, or -1.
int launch_fcg_iter(const StepArgs &a, Level *L, int nlev, int ncoarse, double *x, gea_net *net,
                    float *dense_r, float *dense_e, double *s_buf, cudaStream_t st, Tracer *tr);
// mixed-precision step (gea_mixed.cu)
void launch_mx_pred(const StepArgs &a, const MixedArgs &m, cudaStream_t st, Tracer *tr);
void launch_mx_mom(const StepArgs &a, const MixedArgs &m, const float *ui, const float *wi, float *uo,
                   float *wo, int second, cudaStream_t st, Tracer *tr);
void launch_mx_enth_rhs(const StepArgs &a, const MixedArgs &m, cudaStream_t st, Tracer *tr);
void launch_mx_enth(const StepArgs &a, const MixedArgs &m, const float *hi, float *ho, int second,
                    cudaStream_t st, Tracer *tr);
void launch_mx_eos(const StepArgs &a, const Level &L0, const LevelF &L32, const float *dh, cudaStream_t st,
                   Tracer *tr);
void launch_mx_coarsen(const LevelF &f, const LevelF &c, double omega, cudaStream_t st, Tracer *tr);
void launch_mx_helm_rhs(const StepArgs &a, const Level &L0, const LevelF &L32, const MixedArgs &m,
                        const double *xin, double *xout, int corr, cudaStream_t st, Tracer *tr);
int launch_mx_vcycle(const StepArgs &a, LevelF *L, int nlev, int ncoarse, cudaStream_t st, Tracer *tr);
int launch_mx_cg_iter(const StepArgs &a, const MixedArgs &m, LevelF *L, int nlev, int ncoarse,
                      cudaStream_t st, Tracer *tr);
void launch_mx_p_apply(const StepArgs &a, const MixedArgs &m, cudaStream_t st, Tracer *tr);
// ---- persistent cooperative step kernels (gea_persistent_body.cuh) ----

// Arguments of one context's persistent launch (or of one member of an
// ensemble launch): both state slots' step arguments and the FP64 hierarchy.
struct PersistArgs {
    StepArgs a[2];          // a[s] reads state slot s and writes slot s ^ 1
    Level L[kMaxLevels];
    int nlev, ncoarse, nsteps, first_slot, n_corr, jac_maxit, cg_maxit;
    unsigned long long spin_limit;   // polls of a grid barrier before giving up
};

// FP32 data of the mixed-precision step for the persistent kernels: the
// increments' operator, vectors and CG buffers, and the FP32 multigrid
// hierarchy (nlev levels).
struct MixedPersist {
    MixedArgs m;
    LevelF Lf[kMaxLevels];
    int nlev;
};

// Grid-barrier polls before a block gives up (GEA_ERR_TIMEOUT): a few
// seconds of ~0.7 us polls by default (wait_polls < 0); 0 makes every block
// that is not the last to arrive give up at once.
constexpr unsigned long long kSpinLimit = 1ull << 23;
inline unsigned long long spin_limit_of(long long wait_polls)
{
    return wait_polls < 0 ? kSpinLimit : (unsigned long long)wait_polls;
}

// The persistent kernels exist for several tile shapes of NTHREADS threads
// (BX x BZ cells, one per thread); the tile-shape autotuner picks one per
// context. Each shape's host entry points:
//  max_blocks / mixed_max_blocks / ensemble_max_blocks: co-resident blocks of
//      the FP64, mixed-precision and ensemble kernels on this GPU (0 on error);
//  launch / launch_mixed: n steps of one context (the FP64 finest-to-coarsest
//      hierarchy L, or the FP64 finest level L0 with the FP32 operator m and
//      hierarchy Lf), wait_polls as in spin_limit_of;
//  launch_ensemble: one argument block per member in device memory
//      (persist_args_fill, or persist_args_fill_mixed for mixed-precision
//      members: mixed != 0) and the group table of the blocks: ngroups + 1
//      first blocks, ngroups + 1 first entries of the member list, then the
//      member list (a group of several blocks runs one member, a group of one
//      block one or more members in turn).
struct PersistOps {
    int bx, bz;
    int (*max_blocks)();
    int (*mixed_max_blocks)();
    int (*ensemble_max_blocks)(int mixed);
    cudaError_t (*launch)(const StepArgs a[2], const Level *L, int nlev, int ncoarse, int n_corr, int jac_maxit,
                          int cg_maxit, int first_slot, int nsteps, int blocks, long long wait_polls,
                          cudaStream_t st);
    cudaError_t (*launch_mixed)(const StepArgs a[2], const Level &L0, const MixedArgs &m, const LevelF *Lf,
                                int nlev, int ncoarse, int n_corr, int jac_maxit, int cg_maxit, int first_slot,
                                int nsteps, int blocks, long long wait_polls, cudaStream_t st);
    cudaError_t (*launch_ensemble)(const void *Pm, int mixed, const int *groups, int ngroups, int blocks,
                                   cudaStream_t st);
};
enum { SHAPE_32x8 = 0, SHAPE_16x16 = 1, SHAPE_64x4 = 2, NSHAPES = 3 };
const PersistOps &persist_ops(int shape);
// tiles of a grid for a tile shape
inline long long shape_tiles(const Geom &G, int bx, int bz)
{
    return (long long)((G.nx + bx - 1) / bx) * ((G.nz + bz - 1) / bz);
}
// bytes of one member's argument block of an ensemble launch
size_t persist_args_bytes(int mixed);
void persist_args_fill(void *dst, const StepArgs a[2], const Level *L, int nlev, int ncoarse, int n_corr,
                       int jac_maxit, int cg_maxit, int first_slot, int nsteps, long long wait_polls);
// the mixed-precision member's block: PersistArgs (the FP64 finest level
// L0) followed by MixedPersist (m, the FP32 hierarchy Lf[0 .. nlev-1])
void persist_args_fill_mixed(void *dst, const StepArgs a[2], const Level &L0, const MixedArgs &m,
                             const LevelF *Lf, int nlev, int ncoarse, int n_corr, int jac_maxit, int cg_maxit,
                             int first_slot, int nsteps, long long wait_polls);

}  // namespace gea
